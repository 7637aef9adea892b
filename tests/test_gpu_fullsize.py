"""Parity at the full sizes of the configured workloads.

R-MAT scale 20 (the benchmarked query) is compared end to end.  The 2048^2 grid
and the 4M-vertex hyperbolic graph are compared (a) record by record on a range
of samples, (b) on a run truncated after the first epoch, and (c) end to end
until the stop rule holds: calibration counts, the L table, counts, tau, the
stop epoch and the overflow count, all bit for bit.  The oracle's full runs of
(c) take a minute or so each; they start in worker processes (spawned, so that
no CUDA state is inherited) when the module's first test runs, and overlap with
the GPU work of the other tests.
"""
import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest

import oracle as O
from paper_1903_09422_gb300 import gen

pytestmark = pytest.mark.gpu

_cache = {}


def workload(name):
    if name not in _cache:
        _cache[name] = gen.workload_graph(name)
    return _cache[name]


def _oracle_full_run(name):
    # runs in a spawned worker: regenerates the workload on this machine
    from paper_1903_09422_gb300 import gen as G
    import oracle as OR
    g = G.workload_graph(name)
    w = G.WORKLOADS[name]
    r = OR.kadabra(g, w["eps"], w["delta"], w["seed"])
    return {k: r[k] for k in ("counts", "c0", "L", "tau", "epochs", "omega", "calib_samples", "overflow_samples",
                              "tau_star", "stopped_by_omega")}


@pytest.fixture(scope="module")
def oracle_runs():
    pool = cf.ProcessPoolExecutor(max_workers=2, mp_context=mp.get_context("spawn"))
    futs = {name: pool.submit(_oracle_full_run, name) for name in ("grid2048", "hyp4m")}
    yield futs
    pool.shutdown(wait=True, cancel_futures=True)


@pytest.fixture(scope="module")
def kad():
    import torch
    torch.cuda.set_device(0)
    from paper_1903_09422_gb300 import build, kad as K
    build.build()
    return K


def compare_records(rec, orc):
    for k in ("s", "t", "D", "sigma_st", "overflow", "paths"):
        np.testing.assert_array_equal(rec[k], orc[k], err_msg=k)
    for k in ("expanded", "scanned", "labelled", "pred_arcs", "increments"):
        assert rec["counters"][k] == orc["counters"][k], k


# the two sampling kernels: block per sample, warp per sample
KERNELS = {"block": {}, "warp": dict(samples_per_block=32)}
_rmat20_ref = {}


@pytest.mark.parametrize("name,count", [("rmat20", 2000), ("grid2048", 400), ("hyp4m", 400)])
@pytest.mark.parametrize("kernel", sorted(KERNELS))
def test_records_at_full_size(kad, oracle_runs, name, count, kernel):
    g = workload(name)
    w = gen.WORKLOADS[name]
    with kad.Graph.from_csr(g) as G:
        assert G.vd_bound == O.vd_bound(g)
        rec = G.sample_records(w["seed"], 5000, count, **KERNELS[kernel])
        cal = G.sample_records(w["seed"], 0, count // 2, domain=1, **KERNELS[kernel])
    compare_records(rec, O.samples(g, w["seed"], 5000, count))
    compare_records(cal, O.samples(g, w["seed"], 0, count // 2, domain=1))


@pytest.mark.parametrize("kernel", sorted(KERNELS))
def test_benchmarked_query_end_to_end(kad, kernel):
    name = "rmat20"
    g = workload(name)
    w = gen.WORKLOADS[name]
    if name not in _rmat20_ref:
        _rmat20_ref[name] = O.kadabra(g, w["eps"], w["delta"], w["seed"])
    ref = _rmat20_ref[name]
    with kad.Graph.from_csr(g) as G:
        r = G.run(w["eps"], w["delta"], w["seed"], c0=True, ltab=True, **KERNELS[kernel])
    assert (r["tau"], r["epochs"], r["omega"], r["calib_samples"]) == \
        (ref["tau"], ref["epochs"], ref["omega"], ref["calib_samples"])
    np.testing.assert_array_equal(r["c0"], ref["c0"])
    np.testing.assert_array_equal(r["L"], ref["L"])
    np.testing.assert_array_equal(r["counts"], ref["counts"])
    np.testing.assert_array_equal(r["bc"], ref["bc"])
    assert r["overflow_samples"] == ref["overflow_samples"]


@pytest.mark.parametrize("name", ["grid2048", "hyp4m"])
def test_truncated_run_at_full_size(kad, name):
    g = workload(name)
    w = gen.WORKLOADS[name]
    ref = O.kadabra(g, w["eps"], w["delta"], w["seed"], max_epochs=1)
    with kad.Graph.from_csr(g) as G:
        r = G.run(w["eps"], w["delta"], w["seed"], c0=True, ltab=True, max_epochs=1)
    assert (r["tau"], r["epochs"], r["omega"], r["calib_samples"]) == \
        (ref["tau"], ref["epochs"], ref["omega"], ref["calib_samples"])
    assert r["tau_star"] == ref["tau_star"]
    np.testing.assert_array_equal(r["c0"], ref["c0"])
    np.testing.assert_array_equal(r["L"], ref["L"])
    np.testing.assert_array_equal(r["counts"], ref["counts"])


@pytest.mark.parametrize("name", ["grid2048", "hyp4m"])
@pytest.mark.parametrize("kernel", sorted(KERNELS))
def test_run_to_stop_at_full_size(kad, oracle_runs, name, kernel):
    g = workload(name)
    w = gen.WORKLOADS[name]
    with kad.Graph.from_csr(g) as G:
        r = G.run(w["eps"], w["delta"], w["seed"], c0=True, ltab=True, **KERNELS[kernel])
    ref = oracle_runs[name].result(timeout=900)
    assert (r["tau"], r["epochs"], r["omega"], r["calib_samples"]) == \
        (ref["tau"], ref["epochs"], ref["omega"], ref["calib_samples"])
    assert r["stopped_by_omega"] == int(ref["stopped_by_omega"])
    assert r["tau_star"] == ref["tau_star"]
    assert r["overflow_samples"] == ref["overflow_samples"]
    np.testing.assert_array_equal(r["c0"], ref["c0"])
    np.testing.assert_array_equal(r["L"], ref["L"])
    np.testing.assert_array_equal(r["counts"], ref["counts"])
