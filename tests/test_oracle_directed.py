"""Pins of the oracle on directed graphs (Section 5: KADABRA also covers
directed graphs).

The s side searches along out-arcs and the t side along in-arcs, so a sample's
D must be the directed distance s -> t (0 when t cannot be reached), sigma_st
the number of shortest directed paths, and the drawn path one of them, drawn
uniformly.  The in-arc rows are the transpose, the components the weak ones,
and the vertex-diameter bound goes through the strongly connected components.
Everything here is checked against brute force, scipy's routines, closed forms
and exact directed betweenness (Brandes over out-arcs).
"""
import itertools
from collections import Counter

import numpy as np
import pytest

import oracle as O
from paper_1903_09422_gb300 import gen
from test_oracle_paths import adj_lists, all_shortest_paths_bruteforce, bfs_dist, interior
from test_oracle_stop import brandes_ordered

sp = pytest.importorskip("scipy.sparse")
csgraph = pytest.importorskip("scipy.sparse.csgraph")


def random_digraph(n, p, seed):
    rng = np.random.default_rng(seed)
    a = rng.random((n, n)) < p
    np.fill_diagonal(a, False)
    return gen.from_arcs(n, np.argwhere(a), f"dig{n}_{seed}")


def as_scipy(g):
    return sp.csr_matrix((np.ones(g.m), g.col, g.row_ptr), shape=(g.n, g.n))


def canon(labels):
    """Relabel a partition by first appearance in id order."""
    first, out = {}, np.empty(len(labels), np.int64)
    for v, c in enumerate(labels):
        out[v] = first.setdefault(int(c), len(first))
    return out


def directed_path(n):
    return gen.from_arcs(n, [(i, i + 1) for i in range(n - 1)], f"dpath{n}")


def directed_cycle(n, off=0):
    return [(off + i, off + (i + 1) % n) for i in range(n)]


def true_vd(g):
    d = csgraph.shortest_path(as_scipy(g), method="D", directed=True, unweighted=True)
    return int(np.max(d[np.isfinite(d)])) + 1


GRAPHS = [random_digraph(n, p, sd) for n, p, sd in ((12, 0.2, 1), (20, 0.12, 2), (30, 0.08, 3), (40, 0.05, 4))]


# ------------------------------------------------------------------ structure
@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_transpose_components_and_scc_match_scipy(gi):
    g = GRAPHS[gi]
    rpT, colT = O.transpose(g)
    T = as_scipy(g).T.tocsr()
    T.sort_indices()
    np.testing.assert_array_equal(rpT, T.indptr)
    np.testing.assert_array_equal(colT, T.indices)
    nc, comp = O.components(g)
    k, ref = csgraph.connected_components(as_scipy(g), directed=True, connection="weak")
    assert nc == k
    np.testing.assert_array_equal(comp, canon(ref))  # numbered by smallest member
    ns, scc = O.scc(g)
    k, ref = csgraph.connected_components(as_scipy(g), directed=True, connection="strong")
    assert ns == k
    np.testing.assert_array_equal(canon(scc), canon(ref))


def test_transpose_of_rmat_matches_scipy():
    g = gen.rmat_directed(12, 8, seed=2)
    rpT, colT = O.transpose(g)
    T = as_scipy(g).T.tocsr()
    T.sort_indices()
    np.testing.assert_array_equal(rpT, T.indptr)
    np.testing.assert_array_equal(colT, T.indices)
    k, ref = csgraph.connected_components(as_scipy(g), directed=True, connection="strong")
    ns, scc = O.scc(g)
    assert ns == k
    np.testing.assert_array_equal(canon(scc), canon(ref))


# ------------------------------------------------------ vertex-diameter bound
def test_vd_closed_forms():
    # directed path: every vertex its own component, the chain holds all n
    for n in (2, 3, 10):
        assert O.vd_bound(directed_path(n)) == n
    # directed cycle: one component, ecc_in = ecc_out = n-1, capped at |S| = n
    for n in (3, 7):
        assert O.vd_bound(gen.from_arcs(n, directed_cycle(n))) == n
    # two cycles joined by one arc: a shortest path can run around both
    a, b = 5, 4
    g = gen.from_arcs(a + b, directed_cycle(a) + directed_cycle(b, a) + [(2, a + 1)])
    assert O.vd_bound(g) == a + b == true_vd(g)
    # transitive tournament: all singletons, chain of k (true VD is 2)
    k = 6
    g = gen.from_arcs(k, [(i, j) for i in range(k) for j in range(i + 1, k)])
    assert O.vd_bound(g) == k and true_vd(g) == 2
    # bidirected star: centre root, ecc_in = ecc_out = 1, so 3 (only ecc_out
    # would give 2 < 3, a leaf root 5)
    n = 9
    g = gen.from_arcs(n, [(0, i) for i in range(1, n)] + [(i, 0) for i in range(1, n)])
    assert O.vd_bound(g) == 3 == true_vd(g)


def test_vd_on_symmetric_graphs_is_the_undirected_rule_capped_by_size():
    # a symmetric graph read as directed: each component is one strongly
    # connected component, its root the largest-degree vertex, and
    # ecc_in = ecc_out = ecc, so the bound is max over components of
    # min(|C|, 2 ecc + 1)
    gs = [gen.er(60, 0.05, seed=s, lcc=False) for s in (1, 2, 3)] + [gen.grid_plain(5, 7), gen.path_graph(9)]
    # a degree tie between vertices 1 and 4 (degree 4) with different
    # eccentricities: the smallest id gives min(11, 2*5 + 1) = 11, vertex 4 would give 9
    tie = gen.from_edges(11, [(i, i + 1) for i in range(6)] + [(1, 7), (1, 8), (4, 9), (4, 10)])
    gs.append(tie)
    assert O.vd_bound(tie, directed=True) == 11
    for g in gs:
        nc, comp = O.components(g)
        deg = np.diff(g.row_ptr)
        want = 1
        for c in range(nc):
            members = np.flatnonzero(comp == c)
            root = members[np.argmax(deg[members])]  # first maximum: smallest id
            d = bfs_dist(adj_lists(g), int(root))
            ecc = max(d[v] for v in members)
            want = max(want, min(len(members), 2 * ecc + 1))
        assert O.vd_bound(g, directed=True) == want
        assert O.vd_bound(g, directed=True) <= O.vd_bound(g)


@pytest.mark.parametrize("seed", range(12))
def test_vd_bound_holds_on_random_digraphs(seed):
    g = random_digraph(25 + seed, 0.06 + 0.01 * (seed % 4), seed)
    vd = O.vd_bound(g)
    assert true_vd(g) <= vd <= g.n
    assert vd <= max(np.bincount(O.components(g)[1]))


def test_vd_bound_holds_on_directed_rmat_and_street_grid():
    for g in (gen.rmat_directed(10, 8, seed=3), gen.grid_oneway(12, seed=4)):
        assert true_vd(g) <= O.vd_bound(g) <= g.n


# ------------------------------------------------------------------- samples
@pytest.mark.parametrize("gi", range(len(GRAPHS)))
def test_sigma_distance_and_paths_match_bruteforce(gi):
    g = GRAPHS[gi]
    adj = adj_lists(g)  # out-arcs
    rng = np.random.default_rng(gi)
    pairs = [(s, t) for s in range(g.n) for t in range(g.n) if s != t]
    pairs = [pairs[i] for i in rng.choice(len(pairs), min(80, len(pairs)), replace=False)]
    reached = 0
    for s, t in pairs:
        D, paths = all_shortest_paths_bruteforce(adj, s, t)
        rows, sst = O.pair_paths(g, s, t, 3, seed=5)
        if D is None:  # t cannot be reached from s
            assert sst == 0 and (rows < 0).all()
            continue
        reached += 1
        assert sst == len(paths)
        for row in rows:
            p = [s] + interior(row) + [t]
            assert len(p) - 1 == D
            assert tuple(p) in set(paths)
    assert reached > 0


def test_samples_report_directed_distance_or_zero():
    g = gen.rmat_directed(10, 8, seed=1)
    r = O.samples(g, 7, 0, 400)
    d = csgraph.shortest_path(as_scipy(g), method="D", directed=True, unweighted=True)
    for s, t, D, row in zip(r["s"], r["t"], r["D"], r["paths"]):
        if np.isfinite(d[s, t]):
            assert D == int(d[s, t])
            p = [int(s)] + interior(row) + [int(t)]
            assert len(p) == D + 1
            for u, w in zip(p, p[1:]):  # every step is an arc u -> w
                assert w in g.col[g.row_ptr[u]:g.row_ptr[u + 1]]
        else:
            assert D == 0 and (row < 0).all()
    assert (r["D"] == 0).any() and (r["D"] > 1).any()
    assert r["counters"]["increments"] == int(np.maximum(r["D"] - 1, 0).sum())


def test_path_uniform_chi_square_directed_pair():
    g = random_digraph(40, 0.1, 7)
    adj = adj_lists(g)
    best = None
    for s, t in itertools.permutations(range(g.n), 2):
        D, paths = all_shortest_paths_bruteforce(adj, s, t)
        if D is not None and len(paths) >= 6:
            best = (s, t, paths)
            break
    assert best is not None
    s, t, paths = best
    n = 500 * len(paths)
    rows, sst = O.pair_paths(g, s, t, n, seed=9)
    assert sst == len(paths)
    c = Counter(tuple([s] + interior(r) + [t]) for r in rows)
    assert set(c) == set(paths)
    exp = n / len(paths)
    chi2 = sum((v - exp) ** 2 / exp for v in c.values())
    dof = len(paths) - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof)


def test_symmetric_graph_read_as_directed_draws_the_same_samples():
    # with in-arc rows equal to the out-arc rows, every draw, distance and path
    # is the undirected one
    g = gen.rmat(11, 8, seed=4)
    gd = gen.CSR(g.row_ptr, g.col, g.name, True)
    a, b = O.samples(g, 3, 0, 500, cap=40), O.samples(gd, 3, 0, 500, cap=40)
    for k in ("s", "t", "D", "sigma_st", "paths"):
        np.testing.assert_array_equal(a[k], b[k])
    assert a["counters"] == b["counters"]


# ----------------------------------------------------------------- estimator
def test_eps_delta_guarantee_against_directed_brandes():
    # Brandes' algorithm over out-arcs gives directed betweenness over ordered
    # pairs; with probability >= 1 - delta every |b~(v) - b(v)/(n(n-1))| <= eps
    graphs = [random_digraph(50, 0.08, 11), gen.rmat_directed(7, 8, seed=2), gen.grid_oneway(8, seed=3)]
    runs, fails = 0, 0
    for g in graphs:
        exact = brandes_ordered(g) / (g.n * (g.n - 1))
        for seed in range(1, 41):
            r = O.kadabra(g, 0.05, 0.1, seed=seed)
            runs += 1
            fails += int(np.max(np.abs(r["bc"] - exact)) > 0.05)
            assert r["counts"].sum() == r["counters"]["increments"]
    assert fails <= 0.1 * runs
    assert runs == 120


def test_brandes_directed_matches_networkx():
    nx = pytest.importorskip("networkx")
    g = random_digraph(35, 0.1, 5)
    G = nx.DiGraph()
    G.add_nodes_from(range(g.n))
    G.add_edges_from((v, int(w)) for v in range(g.n) for w in g.col[g.row_ptr[v]:g.row_ptr[v + 1]])
    ref = nx.betweenness_centrality(G, normalized=False)  # ordered pairs when directed
    assert np.allclose(brandes_ordered(g), [ref[v] for v in range(g.n)])


def test_balance_counts_degrees_in_the_expanding_direction():
    # s = 0 -> a1, a2, a3 -> t = 4.  Degree sums: out(s) = 3 = in(t), a tie, so
    # the s side expands first; its next frontier {a1, a2, a3} has out-degree
    # sum 3 <= in(t) = 3, so s expands again and meets t.  Hand count: 4
    # vertices expanded, 6 arcs scanned, 3 labelled, 6 arcs into the next level
    # or M.  (Counting the t side's out-degree instead would expand t first:
    # 2 vertices expanded.)
    g = gen.from_arcs(5, [(0, 1), (0, 2), (0, 3), (1, 4), (2, 4), (3, 4)])
    seen = 0
    for i in range(400):
        r = O.samples(g, 2, i, 1)
        if (r["s"][0], r["t"][0]) != (0, 4):
            continue
        seen += 1
        assert r["D"][0] == 2 and r["sigma_st"][0] == 3
        c = r["counters"]
        assert (c["expanded"], c["scanned"], c["labelled"], c["pred_arcs"]) == (4, 6, 3, 6)
    assert seen > 0


def test_vd_root_is_largest_out_plus_in_degree():
    # a strongly connected random digraph on which the root rule matters: the
    # bound for one component is min(|S|, ecc_in(r) + ecc_out(r) + 1) at r =
    # the vertex of largest out- plus in-degree (smallest id on ties), here 14,
    # where the largest out-degree alone would give 13; the eccentricities are
    # computed by scipy's BFS on the graph and its transpose
    g = random_digraph(30, 0.07, 1143)
    A = as_scipy(g)
    assert csgraph.connected_components(A, directed=True, connection="strong")[0] == 1
    out, inn = np.diff(g.row_ptr), np.bincount(g.col, minlength=g.n)

    def w(r):
        e_out = csgraph.shortest_path(A, directed=True, unweighted=True, indices=r).max()
        e_in = csgraph.shortest_path(A.T.tocsr(), directed=True, unweighted=True, indices=r).max()
        return min(g.n, int(e_out) + int(e_in) + 1)

    r = int(np.argmax(out + inn))  # first maximum: smallest id
    assert (w(r), w(int(np.argmax(out)))) == (14, 13)
    assert O.vd_bound(g) == w(r)
