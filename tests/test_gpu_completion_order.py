"""The completion-order (non-deterministic) mode of the epoch-based framework.

Which samples a run counts depends on timing, so the result is checked against
the oracle through the run's own list of counted samples: the counts must be
exactly the oracle's increments of those samples, the calibration is the
deterministic one, and the stop rule (Appendix B, evaluated with the oracle's f
and g) must hold at the final tau and fail one epoch earlier.
"""
import numpy as np
import pytest

import oracle as O
from paper_1903_09422_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kad():
    import torch
    torch.cuda.set_device(0)
    from paper_1903_09422_gb300 import build, kad as K
    build.build()
    return K


def oracle_counts(recs, idx, n):
    paths = recs["paths"][idx]
    c = np.zeros(n, np.int64)
    np.add.at(c, paths[paths >= 0], 1)
    return c


def rule_holds(counts, c0, L, tau, omega, eps):
    # Appendix B: stop iff f <= eps and g <= eps for every vertex (or tau >= omega);
    # f and g depend on a vertex only through (count, calibration count)
    if tau >= omega:
        return True
    pairs = np.unique(np.stack([np.asarray(counts, np.int64), np.asarray(c0, np.int64)]), axis=1)
    for c, k in pairs.T:
        Lv = L[k]
        if not (O.f(int(c), Lv, tau, omega) <= eps and O.g(int(c), Lv, tau, omega) <= eps):
            return False
    return True


CASES = {
    "rmat12": (lambda: gen.rmat(12, 8, seed=1), 0.03, 11, {}),
    "rmat12_128x8": (lambda: gen.rmat(12, 8, seed=1), 0.03, 12, dict(block_threads=128, blocks_per_sm=8)),
    "rmat12_N250": (lambda: gen.rmat(12, 8, seed=1), 0.04, 5, dict(epoch_size=250)),
    "grid40": (lambda: gen.grid(40, seed=3), 0.05, 3, {}),
    "rmat12_warp": (lambda: gen.rmat(12, 8, seed=1), 0.03, 11, dict(samples_per_block=32)),
    "rmat12_warp5": (lambda: gen.rmat(12, 8, seed=1), 0.03, 12, dict(samples_per_block=5)),
    "grid40_warp": (lambda: gen.grid(40, seed=3), 0.05, 3, dict(samples_per_block=32)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_completion_order_counts_exactly_the_listed_samples(kad, name):
    make, eps, seed, opt = CASES[name]
    g = make()
    delta = 0.1
    N = opt.get("epoch_size", 1000)
    ref = O.kadabra(g, eps, delta, seed, epoch=N)
    with kad.Graph.from_csr(g) as G:
        r = G.run(eps, delta, seed, c0=True, ltab=True, flags=kad.KAD_RUN_COMPLETION_ORDER, **opt)
        tau = r["tau"]
        order = G.run_order(tau).astype(np.int64)
        with pytest.raises(RuntimeError):
            G.run_order(r["samples_computed"] - r["calib_samples"] + 1)
    # calibration, omega and the L table are the deterministic ones
    assert r["omega"] == ref["omega"] and r["calib_samples"] == ref["calib_samples"]
    np.testing.assert_array_equal(r["c0"], ref["c0"])
    np.testing.assert_array_equal(r["L"], ref["L"])
    assert tau % N == 0 and tau >= N and r["epochs"] == tau // N
    assert len(np.unique(order)) == tau and order.min() >= 0
    recs = O.samples(g, seed, 0, int(order.max()) + 1)
    counts = oracle_counts(recs, order, g.n)
    np.testing.assert_array_equal(r["counts"].astype(np.int64), counts)
    np.testing.assert_array_equal(r["bc"], counts / float(tau))
    assert r["overflow_samples"] == int(recs["overflow"][order].sum())
    if r["stopped_by_omega"] == 0:
        assert rule_holds(counts, ref["c0"], ref["L"], tau, ref["omega"], eps)
    if tau > N:
        prev = oracle_counts(recs, order[: tau - N], g.n)
        assert not rule_holds(prev, ref["c0"], ref["L"], tau - N, ref["omega"], eps)


@pytest.mark.parametrize("opt", [{}, dict(samples_per_block=8)])
def test_completion_order_across_launches(kad, opt):
    # a two-epoch ring and few slots: the run needs several launches, each
    # issuing only as many samples as the ring has free fold positions
    g = gen.rmat(12, 8, seed=1)
    eps, delta, seed = 0.03, 0.1, 7
    ref = O.kadabra(g, eps, delta, seed)
    with kad.Graph.from_csr(g) as G:
        r = G.run(eps, delta, seed, flags=kad.KAD_RUN_COMPLETION_ORDER, ring_epochs=2, slots=40, **opt)
        order = G.run_order(r["tau"]).astype(np.int64)
    tau = r["tau"]
    assert tau % 1000 == 0
    assert r["ads_launches"] >= (tau // 1000 + 1) // 2
    assert len(np.unique(order)) == tau
    recs = O.samples(g, seed, 0, int(order.max()) + 1)
    counts = oracle_counts(recs, order, g.n)
    np.testing.assert_array_equal(r["counts"].astype(np.int64), counts)
    if r["stopped_by_omega"] == 0:
        assert rule_holds(counts, ref["c0"], ref["L"], tau, ref["omega"], eps)


def test_completion_order_list_needs_such_a_run(kad):
    g = gen.rmat(12, 8, seed=1)
    with kad.Graph.from_csr(g) as G:
        G.run(0.05, 0.1, 1)
        with pytest.raises(RuntimeError):
            G.run_order(1)


def test_completion_order_at_full_size(kad):
    # the benchmarked query (R-MAT scale 20, eps = 0.01) in completion order:
    # every count against the oracle's increments of the listed samples
    name = "rmat20"
    g = gen.workload_graph(name)
    w = gen.WORKLOADS[name]
    ref = O.kadabra(g, w["eps"], w["delta"], w["seed"], max_epochs=1)  # calibration and L
    with kad.Graph.from_csr(g) as G:
        r = G.run(w["eps"], w["delta"], w["seed"], c0=True, flags=kad.KAD_RUN_COMPLETION_ORDER)
        order = G.run_order(r["tau"]).astype(np.int64)
    tau, N = r["tau"], 1000
    np.testing.assert_array_equal(r["c0"], ref["c0"])
    assert len(np.unique(order)) == tau
    recs = O.samples(g, w["seed"], 0, int(order.max()) + 1)
    counts = oracle_counts(recs, order, g.n)
    np.testing.assert_array_equal(r["counts"].astype(np.int64), counts)
    assert r["overflow_samples"] == int(recs["overflow"][order].sum())
    assert rule_holds(counts, ref["c0"], ref["L"], tau, ref["omega"], w["eps"])
    prev = oracle_counts(recs, order[: tau - N], g.n)
    assert not rule_holds(prev, ref["c0"], ref["L"], tau - N, ref["omega"], w["eps"])
