"""Parity of the warp-per-sample kernel (kad_options.samples_per_block > 0)
with the oracle, through the C ABI.

The kernel runs every sample with one warp and shares large rounds between
warps through a job board; none of that may change a result.  Records (pairs,
distances, sigma_st, paths, overflow flags and the BFS work counters) and full
runs (counts, tau, epochs, calibration counts, L table) must equal the
oracle's bit for bit, for every number of samples per block, slot count,
meeting-set capacity and trace or expansion method.
"""
import numpy as np
import pytest

import oracle as O
from paper_1903_09422_gb300 import gen

from test_gpu_parity import GRAPHS, compare_records, rejection_ladder

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kad():
    import torch
    torch.cuda.set_device(0)
    from paper_1903_09422_gb300 import build, kad as K
    build.build()
    return K


WARP = dict(samples_per_block=32)


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("domain", [0, 1])
def test_warp_records_match_oracle(kad, name, domain):
    g = GRAPHS[name]()
    count = 1500
    with kad.Graph.from_csr(g) as G:
        rec = G.sample_records(seed=7, i0=123, count=count, domain=domain, **WARP)
    orc = O.samples(g, 7, 123, count, domain=domain)
    compare_records(rec, orc)
    for k in ("expanded", "scanned", "labelled", "pred_arcs", "increments"):
        assert rec["counters"][k] == orc["counters"][k], k


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_warp_full_run_matches_oracle(kad, name):
    g = GRAPHS[name]()
    eps, delta, seed = 0.05, 0.1, 3
    ref = O.kadabra(g, eps, delta, seed)
    with kad.Graph.from_csr(g) as G:
        r = G.run(eps, delta, seed, c0=True, ltab=True, **WARP)
    assert r["samples_per_block_used"] > 0
    assert (r["tau"], r["epochs"], r["omega"], r["calib_samples"], r["vd_bound"]) == \
        (ref["tau"], ref["epochs"], ref["omega"], ref["calib_samples"], ref["vd"])
    np.testing.assert_array_equal(r["c0"], ref["c0"])
    np.testing.assert_array_equal(r["L"], ref["L"])
    np.testing.assert_array_equal(r["counts"], ref["counts"])
    np.testing.assert_array_equal(r["bc"], ref["bc"])
    assert r["overflow_samples"] == ref["overflow_samples"]
    assert r["stopped_by_omega"] == int(ref["stopped_by_omega"])


@pytest.mark.parametrize("opt", [dict(samples_per_block=1), dict(samples_per_block=2), dict(samples_per_block=8),
                                 dict(samples_per_block=31), dict(samples_per_block=32, slots=1),
                                 dict(samples_per_block=32, slots=7), dict(samples_per_block=32, slots=333),
                                 dict(samples_per_block=16, mcap=0), dict(samples_per_block=16, mcap=1),
                                 dict(samples_per_block=16, mcap=0, debug=128), dict(samples_per_block=16, debug=128),
                                 dict(samples_per_block=16, ring_epochs=2), dict(samples_per_block=4, slots=3, ring_epochs=2),
                                 dict(samples_per_block=24, epoch_size=250), dict(samples_per_block=24, debug=1),
                                 dict(samples_per_block=24, debug=4), dict(samples_per_block=24, debug=16),
                                 dict(samples_per_block=24, debug=32), dict(samples_per_block=24, debug=64 | 32)])
def test_warp_result_independent_of_configuration(kad, opt):
    g = gen.rmat(12, 8, seed=1)
    eps, delta, seed = 0.03, 0.1, 11
    N = opt.get("epoch_size", 1000)
    ref = O.kadabra(g, eps, delta, seed, epoch=N)
    with kad.Graph.from_csr(g) as G:
        r = G.run(eps, delta, seed, **opt)
        rec = G.sample_records(seed, 0, 700, **{k: v for k, v in opt.items() if k != "epoch_size"})
    assert r["tau"] == ref["tau"] and r["epochs"] == ref["epochs"]
    np.testing.assert_array_equal(r["counts"], ref["counts"])
    compare_records(rec, O.samples(g, seed, 0, 700))


@pytest.mark.parametrize("spb", [32, 6])
def test_warp_hub_graph_records(kad, spb):
    # R-MAT scale 15 with edge factor 16: hub rows far longer than one warp's
    # share, so rounds are posted as arc jobs, frontiers as frontier jobs and
    # meeting rounds as pairwise jobs; the full scan must agree with the tests.
    g = gen.rmat(15, 16, seed=4)
    orc = O.samples(g, 13, 0, 1500)
    with kad.Graph.from_csr(g) as G:
        compare_records(G.sample_records(13, 0, 1500, samples_per_block=spb), orc)
        compare_records(G.sample_records(13, 0, 1500, samples_per_block=spb, debug=4), orc)
        compare_records(G.sample_records(13, 0, 1500, samples_per_block=spb, debug=1), orc)


def test_warp_trace_draw_rejections(kad):
    g, aleaves, bleaves = rejection_ladder()
    orc = O.samples(g, 7, 0, 3000)
    with kad.Graph.from_csr(g) as G:
        compare_records(G.sample_records(7, 0, 3000, **WARP), orc)


def test_warp_large_grid_frontiers(kad):
    # a 160x160 grid: frontiers of hundreds of vertices go out as frontier jobs
    g = gen.grid(160, seed=5)
    orc = O.samples(g, 3, 0, 600)
    with kad.Graph.from_csr(g) as G:
        compare_records(G.sample_records(3, 0, 600, **WARP), orc)
        compare_records(G.sample_records(3, 0, 600, samples_per_block=3), orc)
    ref = O.kadabra(g, 0.05, 0.1, 2)
    with kad.Graph.from_csr(g) as G:
        r = G.run(0.05, 0.1, 2, **WARP)
    assert (r["tau"], r["epochs"]) == (ref["tau"], ref["epochs"])
    np.testing.assert_array_equal(r["counts"], ref["counts"])
