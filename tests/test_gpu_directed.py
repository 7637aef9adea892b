"""Directed graphs on the GPU (Section 5: KADABRA also covers directed graphs)
against the oracle, through the C ABI.

Graph set-up builds the in-arc rows, the weak components and the vertex-diameter
bound through the strongly connected components on the device; the sampling
kernels search forward from s along out-arcs and backward from t along in-arcs.
Per-sample records (pairs, distances, path counts, paths, overflow flags), work
counters, the VD bound, and full runs (calibration counts, L table, counts, tau,
stop epoch) must equal the oracle's bit for bit, for both sampling kernels and
across launch configurations.
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


def random_digraph(n, p, seed):
    rng = np.random.default_rng(seed)
    a = rng.random((n, n)) < p
    np.fill_diagonal(a, False)
    return gen.from_arcs(n, np.argwhere(a), f"dig{n}_{seed}")


def cycle(n, off=0):
    return [(off + i, off + (i + 1) % n) for i in range(n)]


def bidirected(g):
    """A symmetric graph read as directed (every edge both ways)."""
    return gen.CSR(g.row_ptr, g.col, g.name + "_bi", True)


DGRAPHS = {
    "rmat12d": lambda: gen.rmat_directed(12, 8, seed=1),
    "rmat10d_s5": lambda: gen.rmat_directed(10, 4, seed=5),
    "rmat11d_all": lambda: gen.rmat_directed(11, 4, seed=2, lcc=False),  # many weak components
    "dig60": lambda: random_digraph(60, 0.05, 1),
    "dig200": lambda: random_digraph(200, 0.02, 2),
    "street40": lambda: gen.grid_oneway(40, seed=2),
    "dpath30": lambda: gen.from_arcs(30, [(i, i + 1) for i in range(29)]),
    "cycles": lambda: gen.from_arcs(17, cycle(9) + cycle(8, 9) + [(3, 10)]),
    "tournament": lambda: gen.from_arcs(24, [(i, j) for i in range(24) for j in range(i + 1, 24)]),
    "bistar": lambda: gen.from_arcs(40, [(0, i) for i in range(1, 40)] + [(i, 0) for i in range(1, 40)]),
    "bi_rmat10": lambda: bidirected(gen.rmat(10, 8, seed=3)),
}


def compare_records(rec, orc):
    for k in ("s", "t", "D", "sigma_st", "overflow"):
        np.testing.assert_array_equal(rec[k], orc[k], err_msg=k)
    np.testing.assert_array_equal(rec["paths"], orc["paths"], err_msg="paths")


def compare_runs(r, ref):
    assert (r["tau"], r["epochs"], r["omega"], r["calib_samples"], r["vd_bound"]) == \
        (ref["tau"], ref["epochs"], ref["omega"], ref["calib_samples"], ref["vd"])
    np.testing.assert_array_equal(r["counts"], ref["counts"])
    assert r["overflow_samples"] == ref["overflow_samples"]
    assert r["stopped_by_omega"] == int(ref["stopped_by_omega"])


@pytest.mark.parametrize("name", sorted(DGRAPHS))
def test_setup_matches_oracle(kad, name):
    g = DGRAPHS[name]()
    with kad.Graph.from_csr(g) as G:
        assert G.directed
        assert G.vd_bound == O.vd_bound(g)
        assert G.components == O.components(g)[0]


@pytest.mark.parametrize("name", sorted(DGRAPHS))
@pytest.mark.parametrize("domain", [0, 1])
def test_sample_records_match_oracle(kad, name, domain):
    g = DGRAPHS[name]()
    count = 1500
    with kad.Graph.from_csr(g) as G:
        rec = G.sample_records(seed=7, i0=123, count=count, domain=domain)
    orc = O.samples(g, 7, 123, count, domain=domain)
    compare_records(rec, orc)
    for k in ("expanded", "scanned", "labelled", "pred_arcs", "increments"):
        assert rec["counters"][k] == orc["counters"][k], k


@pytest.mark.parametrize("name", sorted(DGRAPHS))
def test_full_run_matches_oracle(kad, name):
    g = DGRAPHS[name]()
    eps, delta, seed = 0.05, 0.1, 3
    ref = O.kadabra(g, eps, delta, seed)
    with kad.Graph.from_csr(g) as G:
        r = G.run(eps, delta, seed, c0=True, ltab=True)
    compare_runs(r, ref)
    np.testing.assert_array_equal(r["c0"], ref["c0"])
    np.testing.assert_array_equal(r["L"], ref["L"])
    assert r["tau_star"] == ref["tau_star"]
    np.testing.assert_array_equal(r["bc"], ref["bc"])


def test_symmetric_graph_as_directed_equals_undirected_run(kad):
    # the same arcs read both ways: identical samples, so identical counts; only
    # the VD bound (and with it omega and the calibration length) may differ
    g = gen.rmat(11, 8, seed=4)
    with kad.Graph.from_csr(g) as U, kad.Graph.from_csr(bidirected(g)) as D:
        a = U.sample_records(5, 0, 1000)
        b = D.sample_records(5, 0, 1000, cap=U.path_cap)
        assert D.vd_bound <= U.vd_bound
    compare_records(a, b)


@pytest.mark.parametrize("opt", [dict(block_threads=256, blocks_per_sm=4), dict(block_threads=512, blocks_per_sm=2),
                                 dict(block_threads=128, blocks_per_sm=8), dict(block_threads=1024, blocks_per_sm=1),
                                 dict(debug=1), dict(debug=4), dict(debug=8), dict(debug=16), dict(debug=64),
                                 dict(mcap=0), dict(mcap=0, debug=128), dict(slots=3, ring_epochs=2),
                                 dict(samples_per_block=8), dict(samples_per_block=32),
                                 dict(samples_per_block=32, debug=1), dict(samples_per_block=32, debug=4),
                                 dict(pair_cost=1), dict(pair_cost=1, samples_per_block=8)])
def test_directed_result_independent_of_launch_configuration(kad, opt):
    g = gen.rmat_directed(13, 8, seed=3)
    eps, delta, seed = 0.03, 0.1, 11
    ref = O.kadabra(g, eps, delta, seed)
    with kad.Graph.from_csr(g) as G:
        r = G.run(eps, delta, seed, **opt)
        rec = G.sample_records(seed, 0, 700, **opt)
    compare_runs(r, ref)
    compare_records(rec, O.samples(g, seed, 0, 700))


@pytest.mark.parametrize("kind", [{}, dict(samples_per_block=32)])
def test_hub_rows_and_long_in_rows(kad, kind):
    # in-rows beyond 4096 arcs (sorted through the bitmap path) and hub
    # frontiers: records and work counters of both kernels equal the oracle's
    g = gen.rmat_directed(16, 16, seed=1)
    orc = O.samples(g, 21, 0, 1500)
    with kad.Graph.from_csr(g) as G:
        assert G.vd_bound == O.vd_bound(g)
        rec = G.sample_records(21, 0, 1500, **kind)
        recs = G.sample_records(21, 0, 1500, debug=1, **kind)  # trace by scanning rows
    for x in (rec, recs):
        compare_records(x, orc)
        for k in ("expanded", "scanned", "labelled", "pred_arcs", "increments"):
            assert x["counters"][k] == orc["counters"][k], k


def test_full_run_on_directed_rmat15_both_kernels(kad):
    g = gen.rmat_directed(15, 16, seed=2)
    ref = O.kadabra(g, 0.02, 0.1, 5)
    with kad.Graph.from_csr(g) as G:
        for kind in ({}, dict(samples_per_block=32)):
            compare_runs(G.run(0.02, 0.1, 5, **kind), ref)


def test_directed_completion_order_counts_the_listed_samples(kad):
    # completion order: the counted samples are listed, and their oracle
    # increments must sum to the counts
    g = gen.rmat_directed(12, 8, seed=1)
    with kad.Graph.from_csr(g) as G:
        r = G.run(0.03, 0.1, 9, flags=kad.KAD_RUN_COMPLETION_ORDER)
        order = G.run_order(r["tau"])
    assert len(order) == r["tau"] and len(set(order.tolist())) == r["tau"]
    cap = O.path_cap(g)
    want = np.zeros(g.n, np.int64)
    idx = np.sort(order.astype(np.int64))
    # the listed indices in contiguous runs, each fetched from the oracle
    starts = np.flatnonzero(np.diff(idx, prepend=-2) != 1)
    ends = np.append(starts[1:], len(idx))
    for a, b in zip(starts, ends):
        rows = O.samples(g, 9, int(idx[a]), int(b - a), cap=cap)["paths"]
        v = rows[rows >= 0]
        np.add.at(want, v, 1)
    np.testing.assert_array_equal(r["counts"], want)


def test_directed_full_size_records_and_truncated_run(kad):
    # R-MAT scale 18 directed (174K vertices, 3.9M arcs): set-up, sampled
    # records and a three-epoch run equal the oracle's
    g = gen.rmat_directed(18, 16, seed=1)
    orc = O.samples(g, 1, 0, 400)
    ref = O.kadabra(g, 0.01, 0.1, 1, max_epochs=3)
    with kad.Graph.from_csr(g) as G:
        assert G.vd_bound == O.vd_bound(g)
        assert G.components == O.components(g)[0]
        compare_records(G.sample_records(1, 0, 400), orc)
        r = G.run(0.01, 0.1, 1, max_epochs=3, c0=True)
    assert (r["tau"], r["epochs"], r["omega"]) == (ref["tau"], ref["epochs"], ref["omega"])
    np.testing.assert_array_equal(r["c0"], ref["c0"])
    np.testing.assert_array_equal(r["counts"], ref["counts"])


def test_sharded_directed_run_equals_single_gpu_run(kad):
    from test_gpu_shard import run_ranks, same_as
    g = gen.rmat_directed(11, 8, seed=4)
    ref = O.kadabra(g, 0.04, 0.1, 6)
    for r in run_ranks(kad, g, 2, 0.04, 0.1, 6):
        same_as(r, ref)


def test_directed_csr_validation(kad):
    # directed rows must still be sorted, in range, without self-loops or
    # duplicates; asymmetry is fine
    ok = gen.from_arcs(4, [(0, 1), (1, 2), (2, 3)])
    with kad.Graph.from_csr(ok) as G:
        assert G.vd_bound == 4
    for rp, col in (([0, 2, 2, 2], [2, 1]), ([0, 1, 1, 1], [0]), ([0, 2, 2, 2], [1, 1]), ([0, 1, 1, 1], [5])):
        with pytest.raises(kad.KadError):
            kad.Graph(np.array(rp, np.int32), np.array(col, np.int32), directed=True)
    # the same asymmetric CSR is refused as undirected
    with pytest.raises(kad.KadError):
        kad.Graph(ok.row_ptr, ok.col)


def test_directed_rmat20_run_to_stop_matches_oracle(kad):
    # the directed R-MAT scale-20 workload (645K vertices, 16M arcs) at
    # eps = 0.01: set-up, stop epoch, tau, calibration counts and counts
    g = gen.workload_graph("rmat20d")
    w = gen.WORKLOADS["rmat20d"]
    ref = O.kadabra(g, w["eps"], w["delta"], w["seed"])
    with kad.Graph.from_csr(g) as G:
        assert (G.vd_bound, G.components) == (ref["vd"], O.components(g)[0])
        r = G.run(w["eps"], w["delta"], w["seed"], c0=True)
    compare_runs(r, ref)
    np.testing.assert_array_equal(r["c0"], ref["c0"])


def test_directed_graphs_served_beside_undirected_ones(kad):
    # the query server holds directed and undirected graphs at once; every
    # query's result equals the same query run alone, and the oracle's
    graphs = [gen.rmat_directed(11, 8, seed=3), gen.rmat(11, 8, seed=3), gen.grid_oneway(30, seed=5)]
    queries = [(i % 3, (0.05, 0.03)[i % 2], 40 + i) for i in range(12)]
    alone = {}
    for gi, g in enumerate(graphs):
        with kad.Graph.from_csr(g) as G:
            for qi, (qg, eps, seed) in enumerate(queries):
                if qg == gi:
                    alone[qi] = G.run(eps, 0.1, seed)
    with kad.Server(workers=4) as S:
        gids = [S.add_graph(g) for g in graphs]
        mixed = [S.wait(t) for t in [S.submit(gids[qg], eps, 0.1, seed) for qg, eps, seed in queries]]
    for qi, r in enumerate(mixed):
        a = alone[qi]
        assert (r["tau"], r["epochs"], r["omega"]) == (a["tau"], a["epochs"], a["omega"])
        np.testing.assert_array_equal(r["bc"], a["bc"])
    for qi in (0, 2):
        qg, eps, seed = queries[qi]
        np.testing.assert_array_equal(mixed[qi]["bc"], O.kadabra(graphs[qg], eps, 0.1, seed)["bc"])


def test_autotuner_on_a_directed_graph(kad):
    # the autotuner's candidates (block and warp variants) all run the directed
    # build; the tuned run and a second one equal the oracle's
    g = gen.rmat_directed(13, 8, seed=4)
    ref = O.kadabra(g, 0.03, 0.1, 8)
    with kad.Graph.from_csr(g) as G:
        r1 = G.run(0.03, 0.1, 8, flags=kad.KAD_RUN_AUTOTUNE)
        r2 = G.run(0.03, 0.1, 8, flags=kad.KAD_RUN_AUTOTUNE)
    for r in (r1, r2):
        compare_runs(r, ref)


def _digraph_case(seed):
    """Random digraphs of varied shape: density, reciprocity, a planted cycle
    chain, and isolated parts (weak components of several kinds)."""
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(30, 400))
    p = float(rng.uniform(0.3, 4.0)) / n
    a = rng.random((n, n)) < p
    recip = float(rng.uniform(0, 0.6))
    a |= a.T & (rng.random((n, n)) < recip)
    np.fill_diagonal(a, False)
    arcs = [tuple(x) for x in np.argwhere(a)]
    # a chain of three cycles (a long chain of components)
    k = int(rng.integers(3, 9))
    base = int(rng.integers(0, max(1, n - 3 * k)))
    for c in range(3):
        ids = [base + c * k + i for i in range(k)]
        arcs += [(ids[i], ids[(i + 1) % k]) for i in range(k)]
        if c:
            arcs.append((base + (c - 1) * k, ids[0]))
    return gen.from_arcs(n, arcs, f"case{seed}")


@pytest.mark.parametrize("seed", range(24))
def test_random_digraphs_match_oracle(kad, seed):
    g = _digraph_case(seed)
    with kad.Graph.from_csr(g) as G:
        assert (G.vd_bound, G.components) == (O.vd_bound(g), O.components(g)[0])
        rec = G.sample_records(seed, 0, 600, domain=seed % 2)
        r = G.run(0.08, 0.1, seed, samples_per_block=(8 if seed % 3 == 0 else None))
    compare_records(rec, O.samples(g, seed, 0, 600, domain=seed % 2))
    compare_runs(r, O.kadabra(g, 0.08, 0.1, seed))


@pytest.mark.parametrize("case", ["no_arcs", "one_arc", "path_up", "path_down"])
def test_directed_edge_cases(kad, case):
    # no arcs (every pair unreachable, VD 1); a single arc; directed paths of
    # 3,000 vertices with ids rising or falling along the path (a chain of 3,000
    # singleton components: long forward-backward BFSs, colour propagation one
    # vertex per pass when ids fall, 3,000 relaxations of the chain)
    n = 3000
    if case == "no_arcs":
        g = gen.from_arcs(50, np.zeros((0, 2), np.int64))
    elif case == "one_arc":
        g = gen.from_arcs(2, [(0, 1)])
    elif case == "path_up":
        g = gen.from_arcs(n, [(i, i + 1) for i in range(n - 1)])
    else:
        g = gen.from_arcs(n, [(i + 1, i) for i in range(n - 1)])
    want = O.vd_bound(g)
    assert want == {"no_arcs": 1, "one_arc": 2}.get(case, n)
    ref = O.kadabra(g, 0.1, 0.1, 5)
    with kad.Graph.from_csr(g) as G:
        assert (G.vd_bound, G.components) == (want, O.components(g)[0])
        r = G.run(0.1, 0.1, 5)
        rec = G.sample_records(5, 0, 300)
    compare_runs(r, ref)
    compare_records(rec, O.samples(g, 5, 0, 300))


def test_tight_bound_with_isolated_vertices(kad):
    # components of one vertex: a = b = m = v0, eccentricity 0
    g = gen.from_edges(9, [(0, 1), (1, 2), (5, 6)])
    with kad.Graph.from_csr(g, tight_vd=True) as G:
        assert G.vd_bound == O.vd_bound_tight(g) == 3
