"""Parity of the CUDA path (through the C ABI) with the oracle.

Integer results (pairs, distances, sigma_st, paths, counts, tau, epochs,
calibration counts, overflow flags, work counters) must match bit for bit; f, g
and the L table must agree within 1e-12 relative (expected: bit-exact, both
sides use the same correctly rounded operation order).
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


def diamond_chain(k, width=2):
    edges, nxt, prev = [], 1, 0
    for _ in range(k):
        for m in range(nxt, nxt + width):
            edges += [(prev, m), (m, nxt + width)]
        prev, nxt = nxt + width, nxt + width + 1
    return gen.from_edges(prev + 1, edges)


def rejection_ladder(la=200, lb=150, lc=200, k2=61):
    """A graph on which the s side's trace-back draws from a count in (2^63, 2^64)
    that is not a power of two, so Lemire's rule rejects a quarter of those draws.

    Hub A (la leaves) starts a ladder of k2 width-2 diamonds and one width-3
    diamond that ends at hub B (lc leaves); B reaches hub B' (lb leaves) through
    one more width-2 diamond (q1, q2).  For s a leaf of A and t a leaf of B', the
    balanced search takes t to B first (B' has the smaller degree sum), then s
    walks the ladder and meets t's side at B: sigma_s(B) = 3 * 2^61, sigma_t(B) = 2,
    sigma_st = 3 * 2^62.  The s side's first trace draw is U(3 * 2^61); the t side's
    first is U(2), a real choice between q1 and q2.
    Returns (graph, leaves of A, leaves of B')."""
    ed, nid = [], [0]

    def new():
        nid[0] += 1
        return nid[0] - 1

    A = new()
    aleaves = [new() for _ in range(la)]
    ed += [(A, x) for x in aleaves]
    prev = A
    for _ in range(k2):
        m1, m2, j = new(), new(), new()
        ed += [(prev, m1), (prev, m2), (m1, j), (m2, j)]
        prev = j
    xs = [new() for _ in range(3)]
    B = new()
    for x in xs:
        ed += [(prev, x), (x, B)]
    q1, q2, Bp = new(), new(), new()
    ed += [(B, q1), (B, q2), (q1, Bp), (q2, Bp)]
    ed += [(B, new()) for _ in range(lc)]
    bleaves = [new() for _ in range(lb)]
    ed += [(Bp, x) for x in bleaves]
    return gen.from_edges(nid[0], ed, name="rejection_ladder"), set(aleaves), set(bleaves)


def mixed_components(seed=9):
    # a large R-MAT component, a grid, small random pieces and isolated vertices,
    # with the vertex ids shuffled so that no component is a contiguous id range
    parts = [gen.rmat(13, 8, seed=2), gen.grid(25, seed=3)] + [gen.er(40, 0.12, seed=10 + i) for i in range(6)]
    edges, base = [], 0
    for g in parts:
        src = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
        up = g.col > src
        edges.append(np.stack([src[up] + base, g.col[up] + base], axis=1))
        base += g.n
    n = base + 700  # isolated vertices at the end
    perm = np.random.default_rng(seed).permutation(n)
    e = perm[np.concatenate(edges)]
    return gen.from_edges(n, e.tolist(), name="mixed_components")


GRAPHS = {
    "mixed_comp": mixed_components,
    "rmat12": lambda: gen.rmat(12, 8, seed=1),
    "rmat10_s5": lambda: gen.rmat(10, 4, seed=5),
    "er60": lambda: gen.er(60, 0.1, seed=2),
    "er200": lambda: gen.er(200, 0.1, seed=4),
    "grid9x13": lambda: gen.grid_plain(9, 13),
    "grid64": lambda: gen.grid(64, seed=3),
    "path40": lambda: gen.path_graph(40),
    "star50": lambda: gen.star_graph(50),
    "diamond70": lambda: diamond_chain(70),
    "two_comp": lambda: gen.from_edges(12, [(0, 1), (1, 2), (2, 3), (3, 0), (4, 5), (5, 6), (6, 7), (7, 8), (8, 9),
                                            (9, 10), (10, 11)]),
    "isolated": lambda: gen.from_edges(6, [(0, 1), (1, 2)]),
    "ladder": lambda: rejection_ladder()[0],
}


def compare_records(rec, orc):
    for k in ("s", "t", "D", "sigma_st", "overflow"):
        np.testing.assert_array_equal(rec[k], orc[k], err_msg=k)
    np.testing.assert_array_equal(rec["paths"], orc["paths"], err_msg="paths")


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("domain", [0, 1])
def test_sample_records_match_oracle(kad, name, domain):
    g = GRAPHS[name]()
    count = 1500
    with kad.Graph.from_csr(g) as G:
        assert G.vd_bound == O.vd_bound(g)
        rec = G.sample_records(seed=7, i0=123, count=count, domain=domain)
    orc = O.samples(g, 7, 123, count, domain=domain)
    compare_records(rec, orc)
    # the BFS work counters are properties of the samples; trace_arcs counts
    # what each implementation actually read during the trace-back
    for k in ("expanded", "scanned", "labelled", "pred_arcs", "increments"):
        assert rec["counters"][k] == orc["counters"][k], k


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_full_run_matches_oracle(kad, name):
    g = GRAPHS[name]()
    eps, delta, seed = 0.05, 0.1, 3
    ref = O.kadabra(g, eps, delta, seed)
    with kad.Graph.from_csr(g) as G:
        r = G.run(eps, delta, seed, c0=True, ltab=True)
    assert (r["tau"], r["epochs"], r["omega"], r["calib_samples"], r["vd_bound"]) == \
        (ref["tau"], ref["epochs"], ref["omega"], ref["calib_samples"], ref["vd"])
    np.testing.assert_array_equal(r["c0"], ref["c0"])
    np.testing.assert_array_equal(r["L"], ref["L"])
    assert r["tau_star"] == ref["tau_star"]
    np.testing.assert_array_equal(r["counts"], ref["counts"])
    np.testing.assert_array_equal(r["bc"], ref["bc"])
    assert r["overflow_samples"] == ref["overflow_samples"]
    assert r["stopped_by_omega"] == int(ref["stopped_by_omega"])
    assert r["samples_computed"] >= r["tau"]


@pytest.mark.parametrize("opt", [dict(block_threads=128), dict(block_threads=256), dict(block_threads=1024),
                                 dict(block_threads=512, blocks_per_sm=2), dict(block_threads=256, blocks_per_sm=4), dict(slots=1), dict(slots=7),
                                 dict(mcap=0), dict(mcap=1), dict(mcap=0, debug=128), dict(debug=128),
                                 dict(ring_epochs=2), dict(slots=3, ring_epochs=2),
                                 dict(epoch_size=250), dict(debug=1), dict(debug=2), dict(debug=4),
                                 dict(debug=2, block_threads=512, blocks_per_sm=2), dict(debug=8), dict(debug=16),
                                 dict(debug=16, block_threads=256, blocks_per_sm=4), dict(debug=64),
                                 dict(debug=64 | 32, block_threads=128, blocks_per_sm=8),
                                 dict(block_threads=128, blocks_per_sm=8),
                                 dict(block_threads=1024, blocks_per_sm=1)])
def test_result_independent_of_launch_configuration(kad, opt):
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


def test_meeting_round_methods_agree_on_hub_graph(kad):
    # The pairwise frontier test and the full scan of the expanding side's rows
    # must find the same meeting sets (hence the same records as the oracle).
    g = gen.rmat(15, 16, seed=4)
    orc = O.samples(g, 13, 0, 1500)
    with kad.Graph.from_csr(g) as G:
        a = G.sample_records(13, 0, 1500)
        b = G.sample_records(13, 0, 1500, debug=4)
    compare_records(a, orc)
    compare_records(b, orc)
    for k in ("expanded", "scanned", "labelled", "pred_arcs", "increments"):
        assert a["counters"][k] == orc["counters"][k] == b["counters"][k], k


@pytest.mark.parametrize("pair_cost", [1, 4, 64, 1 << 20])
def test_pair_cost_changes_speed_not_results(kad, pair_cost):
    # The pairwise test's cost factor decides how often the meeting round tests
    # frontier pairs instead of scanning the expanding side's rows (1: whenever
    # the frontiers' product is below the arcs; 2^20: practically never).  The
    # block- and warp-per-sample kernels' records, work counters and full runs
    # equal the oracle's at every factor.
    g = gen.rmat(15, 16, seed=4)
    orc = O.samples(g, 13, 0, 1500)
    ref = O.kadabra(g, 0.02, 0.1, 13)
    with kad.Graph.from_csr(g) as G:
        recs = [G.sample_records(13, 0, 1500, pair_cost=pair_cost),
                G.sample_records(13, 0, 1500, pair_cost=pair_cost, samples_per_block=8)]
        runs = [G.run(0.02, 0.1, 13, pair_cost=pair_cost),
                G.run(0.02, 0.1, 13, pair_cost=pair_cost, samples_per_block=24)]
    for rec in recs:
        compare_records(rec, orc)
        for k in ("expanded", "scanned", "labelled", "pred_arcs", "increments"):
            assert rec["counters"][k] == orc["counters"][k], k
    for r in runs:
        assert r["pair_cost_used"] == pair_cost
        assert (r["tau"], r["epochs"]) == (ref["tau"], ref["epochs"])
        np.testing.assert_array_equal(r["counts"], ref["counts"])


def test_hub_graph_records_and_runs_per_variant(kad):
    # A graph with hub rows (long levels, meetings found mid-level, samples
    # abandoned after the stop): records, work counters and full-run counts
    # equal the oracle's under several kernel variants.
    g = gen.rmat(15, 16, seed=5)
    orc = O.samples(g, 21, 0, 2000)
    ref = O.kadabra(g, 0.02, 0.1, 21)
    with kad.Graph.from_csr(g) as G:
        recs = [G.sample_records(21, 0, 2000, block_threads=bt, blocks_per_sm=bps) for bt, bps in ((512, 2), (256, 4))]
        runs = [G.run(0.02, 0.1, 21, block_threads=bt, blocks_per_sm=bps) for bt, bps in ((512, 2), (256, 4), (128, 8))]
    for rec in recs:
        compare_records(rec, orc)
        for k in ("expanded", "scanned", "labelled", "pred_arcs", "increments"):
            assert rec["counters"][k] == orc["counters"][k], k
    for r in runs:
        assert (r["tau"], r["epochs"]) == (ref["tau"], ref["epochs"])
        np.testing.assert_array_equal(r["counts"], ref["counts"])


def test_trace_methods_agree_on_hub_graph(kad):
    # Trace-back from the predecessor level's list (hub vertices) and by scanning
    # the adjacency (forced) must both give the oracle's paths.
    g = gen.rmat(15, 16, seed=3)
    orc = O.samples(g, 9, 0, 1500)
    with kad.Graph.from_csr(g) as G:
        a = G.sample_records(9, 0, 1500)
        b = G.sample_records(9, 0, 1500, debug=1)
    compare_records(a, orc)
    compare_records(b, orc)
    assert a["counters"]["trace_arcs"] < b["counters"]["trace_arcs"]


def test_meeting_selection_paths_agree_on_hub_graph(kad):
    # Many-member meeting sets: the rank selection over up to mcap members, the
    # digit-wise selection over the recorded members (mcap 0 and 16: all or most
    # in the global extension) and over the other side's frontier (no extension);
    # all must give the oracle's records.
    g = gen.rmat(14, 16, seed=2)
    orc = O.samples(g, 5, 0, 800)
    with kad.Graph.from_csr(g) as G:
        runs = [G.sample_records(5, 0, 800, mcap=0), G.sample_records(5, 0, 800, mcap=16),
                G.sample_records(5, 0, 800, mcap=256), G.sample_records(5, 0, 800, mcap=0, debug=128),
                G.sample_records(5, 0, 800, mcap=16, debug=128)]
        r = G.run(0.02, 0.1, 5, mcap=16)
    for a in runs:
        compare_records(a, orc)
    ref = O.kadabra(g, 0.02, 0.1, 5)
    assert r["tau"] == ref["tau"]
    np.testing.assert_array_equal(r["counts"], ref["counts"])


@pytest.mark.parametrize("k", [1, 2, 5])
def test_truncated_run_matches_oracle(kad, k):
    g = gen.rmat(12, 8, seed=1)
    ref = O.kadabra(g, 0.01, 0.1, 4, max_epochs=k)
    with kad.Graph.from_csr(g) as G:
        r = G.run(0.01, 0.1, 4, max_epochs=k)
    assert r["tau"] == ref["tau"] == 1000 * min(k, ref["epochs"])
    np.testing.assert_array_equal(r["counts"], ref["counts"])


def test_autotuner_keeps_results_and_choice(kad):
    g = gen.rmat(15, 8, seed=6)
    assert g.n >= 16384
    ref = O.kadabra(g, 0.05, 0.1, 8)
    with kad.Graph.from_csr(g) as G:
        r1 = G.run(0.05, 0.1, 8, flags=kad.KAD_RUN_AUTOTUNE)
        r2 = G.run(0.05, 0.1, 8, flags=kad.KAD_RUN_AUTOTUNE)
        r3 = G.run(0.05, 0.1, 8)  # without the flag: the average-degree rule
        # the caller's factor stands; the tuned variant is kept
        r4 = G.run(0.05, 0.1, 8, flags=kad.KAD_RUN_AUTOTUNE, pair_cost=32)
    pick = lambda r: (r["block_threads_used"], r["blocks_per_sm_used"], r["samples_per_block_used"])
    assert pick(r1) in {(512, 2, 0), (256, 4, 0), (256, 2, 0), (1024, 1, 0), (128, 8, 0), (1024, 1, 8), (1024, 1, 24)}
    assert pick(r1) == pick(r2) == pick(r4)
    assert r1["pair_cost_used"] in {4, 8, 16} and r2["pair_cost_used"] == r1["pair_cost_used"]
    assert r4["pair_cost_used"] == 32
    assert (r3["block_threads_used"], r3["blocks_per_sm_used"]) == ((256, 4) if g.m <= 8 * g.n else (512, 2))
    assert r3["pair_cost_used"] == 8
    for r in (r1, r2, r3, r4):
        assert r["tau"] == ref["tau"]
        np.testing.assert_array_equal(r["counts"], ref["counts"])


def test_autotuner_cost_stage_after_a_fixed_cost_run(kad):
    # The variant tuned under a caller's cost factor is kept; a later run that
    # leaves the factor open times all three factors on that variant.
    g = gen.rmat(15, 16, seed=7)
    assert g.n >= 16384
    ref = O.kadabra(g, 0.05, 0.1, 3)
    with kad.Graph.from_csr(g) as G:
        r1 = G.run(0.05, 0.1, 3, flags=kad.KAD_RUN_AUTOTUNE, pair_cost=2)
        r2 = G.run(0.05, 0.1, 3, flags=kad.KAD_RUN_AUTOTUNE)
        r3 = G.run(0.05, 0.1, 3, flags=kad.KAD_RUN_AUTOTUNE)
    pick = lambda r: (r["block_threads_used"], r["blocks_per_sm_used"], r["samples_per_block_used"])
    assert pick(r1) == pick(r2) == pick(r3)
    assert r1["pair_cost_used"] == 2
    assert r2["pair_cost_used"] in {4, 8, 16} and r3["pair_cost_used"] == r2["pair_cost_used"]
    for r in (r1, r2, r3):
        assert r["tau"] == ref["tau"]
        np.testing.assert_array_equal(r["counts"], ref["counts"])


def test_fg_kernel_matches_oracle(kad):
    g = gen.rmat(12, 8, seed=1)
    ref = O.kadabra(g, 0.05, 0.1, 1)
    tau, om = ref["tau"], ref["omega"]
    f, gg = kad.eval_fg(ref["counts"], ref["c0"], ref["L"], tau, om)
    fo = np.array([O.f(int(c), float(ref["L"][k]), tau, om) for c, k in zip(ref["counts"], ref["c0"])])
    go = np.array([O.g(int(c), float(ref["L"][k]), tau, om) for c, k in zip(ref["counts"], ref["c0"])])
    np.testing.assert_allclose(f, fo, rtol=1e-12, atol=0)
    np.testing.assert_allclose(gg, go, rtol=1e-12, atol=0)
    assert np.array_equal(f, fo) and np.array_equal(gg, go)  # expected bit-exact


def test_repeated_runs_and_graph_reuse(kad):
    g = gen.rmat(11, 8, seed=9)
    with kad.Graph.from_csr(g) as G:
        r1 = G.run(0.05, 0.1, 5)
        r2 = G.run(0.02, 0.1, 6)
        r3 = G.run(0.05, 0.1, 5)
    np.testing.assert_array_equal(r1["counts"], r3["counts"])
    ref = O.kadabra(g, 0.02, 0.1, 6)
    np.testing.assert_array_equal(r2["counts"], ref["counts"])


def test_device_outputs_and_device_graph(kad):
    import torch
    g = gen.rmat(12, 8, seed=1)
    ref = O.kadabra(g, 0.05, 0.1, 2)
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    with kad.Graph.from_device(rp, col) as G:
        d_bc = torch.empty(g.n, dtype=torch.float64, device="cuda")
        d_cnt = torch.empty(g.n, dtype=torch.int32, device="cuda")
        r = G.run_device(0.05, 0.1, 2, d_bc=d_bc, d_counts=d_cnt)
        torch.cuda.synchronize()
    assert r["tau"] == ref["tau"]
    np.testing.assert_array_equal(d_cnt.cpu().numpy().view(np.uint32), ref["counts"])
    np.testing.assert_array_equal(d_bc.cpu().numpy(), ref["bc"])


def test_bad_csr_is_rejected(kad):
    g = gen.er(30, 0.2, seed=1)
    col = g.col.copy()
    col[0], col[1] = col[1], col[0]  # unsorted row
    with pytest.raises(kad.KadError) as e:
        kad.Graph(g.row_ptr, col)
    assert e.value.status == 2
    # asymmetric: drop one arc's reverse by pointing it elsewhere
    h = gen.path_graph(10)
    col = h.col.copy()
    col[-1] = 7  # last row (vertex 9) now points to 7 instead of 8
    with pytest.raises(kad.KadError):
        kad.Graph(h.row_ptr, col)
    # asymmetric through an extra downward arc whose reverse is missing: every
    # upward arc has its reverse, only the arc counts differ
    rp = np.array(list(h.row_ptr[:-1]) + [h.row_ptr[-1] + 1], np.int32)
    col = np.concatenate([h.col[:-1], np.array([7, 8], np.int32)])  # row 9 = [7, 8]
    with pytest.raises(kad.KadError) as e:
        kad.Graph(rp, col)
    assert e.value.status == 2
    with pytest.raises(kad.KadError):
        kad.Graph(np.array([0, 1], np.int32), np.array([0], np.int32))  # n = 1


def test_single_arc_asymmetry_is_found_anywhere(kad):
    # one arc moved to another target inside its sorted row (hub rows and short
    # rows, every position within a thread's group of arcs): the moved arc has no
    # reverse, so the graph is rejected
    g = gen.rmat(13, 8, seed=2)
    rp, col = g.row_ptr, g.col
    rng = np.random.default_rng(5)
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(rp))
    done = 0
    for e in rng.permutation(g.m):
        u, lo, hi = rows[e], rp[rows[e]], rp[rows[e] + 1]
        left = col[e - 1] if e > lo else -1
        right = col[e + 1] if e + 1 < hi else g.n
        cand = [x for x in range(left + 1, right) if x != col[e] and x != u]
        if not cand:
            continue
        bad = col.copy()
        bad[e] = cand[len(cand) // 2]
        with pytest.raises(kad.KadError) as ex:
            kad.Graph(rp, bad)
        assert ex.value.status == 2
        done += 1
        if done == 12:
            break
    assert done == 12


def test_invalid_run_arguments(kad):
    g = gen.path_graph(10)
    with kad.Graph.from_csr(g) as G:
        for eps, delta in [(0, 0.1), (1.0, 0.1), (0.1, 0), (0.1, 1.5)]:
            with pytest.raises(kad.KadError) as e:
                G.run(eps, delta, 1)
            assert e.value.status == 1
        for pc in (-1, (1 << 20) + 1):
            with pytest.raises(kad.KadError) as e:
                G.run(0.1, 0.1, 1, pair_cost=pc)
            assert e.value.status == 1
            with pytest.raises(kad.KadError) as e:
                G.sample_records(1, 0, 10, pair_cost=pc)
            assert e.value.status == 1
        r = G.run(0.1, 0.1, 1)  # the handle stays usable
        assert r["tau"] > 0 and r["pair_cost_used"] == 8


def test_workspace_kept_across_graphs(kad):
    # A freed graph's workspace serves the next graph (larger and smaller n,
    # records and full runs), and kad_trim releases it.
    graphs = [gen.rmat(12, 8, seed=1), gen.grid(30, seed=2), gen.rmat(13, 8, seed=3), gen.er(120, 0.1, seed=4)]
    for i, g in enumerate(graphs):
        ref = O.kadabra(g, 0.05, 0.1, 5 + i)
        with kad.Graph.from_csr(g) as G:
            rec = G.sample_records(5 + i, 0, 300)
            r = G.run(0.05, 0.1, 5 + i)
        compare_records(rec, O.samples(g, 5 + i, 0, 300))
        assert r["tau"] == ref["tau"]
        np.testing.assert_array_equal(r["counts"], ref["counts"])
        if i == 1:
            kad.trim()
    kad.trim()


def test_default_variant_follows_average_degree(kad):
    # without a named variant: 256x4 on graphs of average degree up to 8,
    # 512x2 on denser ones; the results are those of the oracle either way
    for g, want in ((gen.grid(48, seed=7), (256, 4)), (gen.rmat(12, 8, seed=1), (512, 2)),
                    (gen.er(300, 0.25, seed=2), (512, 2))):
        assert (g.m <= 8 * g.n) == (want == (256, 4))
        ref = O.kadabra(g, 0.05, 0.1, 3)
        with kad.Graph.from_csr(g) as G:
            r = G.run(0.05, 0.1, 3)
        assert (r["block_threads_used"], r["blocks_per_sm_used"]) == want
        np.testing.assert_array_equal(r["counts"], ref["counts"])


def test_trace_draw_rejections_match_oracle(kad):
    # Samples whose s-side trace-back draw is rejected by Lemire's rule (the
    # count is 3 * 2^61): every later draw of the sample, including the t side's,
    # comes from a later stream position.  The oracle shows that the range below
    # holds such samples; the CUDA path must give the same records.
    g, aleaves, bleaves = rejection_ladder()
    seed, count = 7, 3000
    orc = O.samples(g, seed, 0, count)
    rejected = 0
    for i in range(count):
        s, t = int(orc["s"][i]), int(orc["t"][i])
        if s in aleaves and t in bleaves:
            assert int(orc["sigma_st"][i]) == 3 * 2**62
            # stream words used by the pair, meeting and first s-side trace draws
            # against those used without the trace draw: more than one word apart
            # means the trace draw was rejected at least once
            _, u3 = O.stream_draws(seed, i, 0, [g.n, g.n - 1, 3 * 2**62])
            _, u4 = O.stream_draws(seed, i, 0, [g.n, g.n - 1, 3 * 2**62, 3 * 2**61])
            rejected += (u4 - u3) > 1
    assert rejected >= 10, rejected
    assert not orc["overflow"].any()
    with kad.Graph.from_csr(g) as G:
        for opt in (dict(), dict(block_threads=256, blocks_per_sm=4), dict(block_threads=1024)):
            compare_records(G.sample_records(seed, 0, count, **opt), orc)


def test_smallest_workload_exact_triple(kad):
    # R-MAT scale 12, eps = 0.05, delta = 0.1, seed 1: the smallest configured
    # workload, end to end, at its own seed.
    w = gen.WORKLOADS["rmat12"]
    g = gen.workload_graph("rmat12")
    ref = O.kadabra(g, w["eps"], w["delta"], w["seed"])
    with kad.Graph.from_csr(g) as G:
        r = G.run(w["eps"], w["delta"], w["seed"], c0=True, ltab=True)
    assert (r["tau"], r["epochs"], r["omega"], r["calib_samples"], r["vd_bound"]) == \
        (ref["tau"], ref["epochs"], ref["omega"], ref["calib_samples"], ref["vd"])
    np.testing.assert_array_equal(r["c0"], ref["c0"])
    np.testing.assert_array_equal(r["L"], ref["L"])
    np.testing.assert_array_equal(r["counts"], ref["counts"])
    np.testing.assert_array_equal(r["bc"], ref["bc"])
    assert r["overflow_samples"] == ref["overflow_samples"]


def test_graph_without_edges(kad):
    # n isolated vertices: VD 1, every pair unreachable, counts all zero
    g = gen.from_edges(40, [])
    assert g.m == 0
    ref = O.kadabra(g, 0.1, 0.1, 2)
    for tight in (False, True):
        with kad.Graph.from_csr(g, tight_vd=tight) as G:
            assert (G.vd_bound, G.components) == (1, 40)
            r = G.run(0.1, 0.1, 2)
            rec = G.sample_records(2, 0, 200)
        assert (r["tau"], r["epochs"], r["omega"]) == (ref["tau"], ref["epochs"], ref["omega"])
        assert not r["counts"].any()
        compare_records(rec, O.samples(g, 2, 0, 200))
