"""Pins of the oracle's sample(): shortest-path counts, distances, path validity
and uniformity, increments (Section 2.3: a uniform pair, then a uniform shortest
path; x_i(v) = 1 for the path's interior vertices)."""
import itertools
from collections import Counter, deque

import numpy as np
import pytest

import oracle as O
from paper_1903_09422_gb300 import gen

U64MAX = 2**64 - 1


def adj_lists(g):
    return [list(g.col[g.row_ptr[v]:g.row_ptr[v + 1]]) for v in range(g.n)]


def bfs_dist(adj, s):
    d = [-1] * len(adj)
    d[s] = 0
    q = deque([s])
    while q:
        u = q.popleft()
        for w in adj[u]:
            if d[w] < 0:
                d[w] = d[u] + 1
                q.append(w)
    return d


def all_shortest_paths_bruteforce(adj, s, t):
    """Enumerate every simple s-t path of minimum length by depth-first search
    with no pruning beyond simplicity and the length of the best path found."""
    best = [None]
    found = []

    def dfs(u, path, seen):
        if best[0] is not None and len(path) - 1 > best[0]:
            return
        if u == t:
            L = len(path) - 1
            if best[0] is None or L < best[0]:
                best[0] = L
                found.clear()
            if L == best[0]:
                found.append(tuple(path))
            return
        for w in adj[u]:
            if w not in seen:
                seen.add(w)
                path.append(w)
                dfs(w, path, seen)
                path.pop()
                seen.discard(w)

    dfs(s, [s], {s})
    return best[0], found


def interior(row):
    return [int(x) for x in row if x >= 0]


def small_graphs():
    gs = [gen.er(n, 0.15, seed=sd) for n, sd in ((14, 1), (18, 2), (22, 3))]
    gs += [gen.grid_plain(3, 4), gen.grid_plain(4, 4)]
    return gs


@pytest.mark.parametrize("gi", range(5))
def test_sigma_and_distance_match_bruteforce(gi):
    g = small_graphs()[gi]
    adj = adj_lists(g)
    pairs = [(s, t) for s in range(g.n) for t in range(g.n) if s != t]
    rng = np.random.default_rng(gi)
    if len(pairs) > 60:
        pairs = [pairs[i] for i in rng.choice(len(pairs), 60, replace=False)]
    for s, t in pairs:
        D, paths = all_shortest_paths_bruteforce(adj, s, t)
        rows, sst = O.pair_paths(g, s, t, 3, seed=5)
        assert sst == len(paths)
        for row in rows:
            p = [s] + interior(row) + [t]
            assert len(p) - 1 == D
            assert tuple(p) in set(paths)


def test_sigma_against_networkx_er():
    nx = pytest.importorskip("networkx")
    for sd in range(3):
        g = gen.er(45, 0.1, seed=10 + sd)
        G = nx.Graph()
        G.add_nodes_from(range(g.n))
        for v in range(g.n):
            for w in g.col[g.row_ptr[v]:g.row_ptr[v + 1]]:
                G.add_edge(v, int(w))
        rng = np.random.default_rng(sd)
        for _ in range(40):
            s, t = (int(x) for x in rng.choice(g.n, 2, replace=False))
            rows, sst = O.pair_paths(g, s, t, 1, seed=1)
            assert sst == sum(1 for _ in nx.all_shortest_paths(G, s, t))
            assert len(interior(rows[0])) + 1 == nx.shortest_path_length(G, s, t)


def test_path_uniform_chi_square_grid_corner():
    # 4x4 grid, corner to corner: C(6,3) = 20 shortest paths, each equally likely.
    g = gen.grid_plain(4, 4)
    n = 20000
    rows, sst = O.pair_paths(g, 0, 15, n, seed=3)
    assert sst == 20
    c = Counter(tuple(interior(r)) for r in rows)
    assert len(c) == 20
    exp = n / 20
    chi2 = sum((v - exp) ** 2 / exp for v in c.values())
    assert chi2 < 50.0  # 19 dof; p ~ 1e-4


def test_path_uniform_chi_square_er_pair():
    g = gen.er(40, 0.12, seed=7)
    adj = adj_lists(g)
    best = None
    for s, t in itertools.combinations(range(g.n), 2):
        D, paths = all_shortest_paths_bruteforce(adj, s, t)
        if len(paths) >= 6:
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


def test_path_graph_paths_are_the_unique_segment():
    g = gen.path_graph(30)
    r = O.samples(g, seed=4, i0=0, count=300)
    for s, t, D, row in zip(r["s"], r["t"], r["D"], r["paths"]):
        assert D == abs(int(s) - int(t))
        step = 1 if t > s else -1
        assert interior(row) == list(range(int(s) + step, int(t), step))
        assert r["sigma_st"][0] >= 1


def test_star_graph_centre_on_every_leaf_pair():
    g = gen.star_graph(25)
    r = O.samples(g, seed=2, i0=0, count=500)
    for s, t, D, row in zip(r["s"], r["t"], r["D"], r["paths"]):
        if s != 0 and t != 0:
            assert D == 2 and interior(row) == [0]
        else:
            assert D == 1 and interior(row) == []


def test_pairs_uniform_over_ordered_pairs():
    # Section 2.3: (s, t) uniform over the n(n-1) ordered pairs with s != t.
    g = gen.grid_plain(2, 3)
    n = 60000
    r = O.samples(g, seed=8, i0=0, count=n)
    assert (r["s"] != r["t"]).all()
    c = Counter(zip(r["s"].tolist(), r["t"].tolist()))
    assert len(c) == 30
    exp = n / 30
    chi2 = sum((v - exp) ** 2 / exp for v in c.values())
    assert chi2 < 29 + 6 * np.sqrt(58)


def test_increments_equal_path_length_minus_one():
    g = gen.rmat(10, 8, seed=3)
    r = O.samples(g, seed=1, i0=0, count=2000)
    adj = [set(a) for a in adj_lists(g)]
    tot = 0
    for s, t, D, row in zip(r["s"], r["t"], r["D"], r["paths"]):
        p = [int(s)] + interior(row) + [int(t)]
        assert len(p) - 1 == D
        assert all(p[i + 1] in adj[p[i]] for i in range(len(p) - 1))
        assert len(set(p)) == len(p)
        tot += D - 1
    assert r["counters"]["increments"] == tot


def test_different_components_give_no_path():
    # Appendix C.1: pairs in different components are skipped (no increments).
    g = gen.from_edges(8, [(0, 1), (1, 2), (2, 3), (4, 5), (5, 6), (6, 7)])
    r = O.samples(g, seed=1, i0=0, count=400)
    comp = np.array([0, 0, 0, 0, 1, 1, 1, 1])
    cross = comp[r["s"]] != comp[r["t"]]
    assert cross.any() and (~cross).any()
    assert (r["D"][cross] == 0).all()
    assert (r["D"][~cross] > 0).all()
    assert (r["paths"][cross] == -1).all()


def diamond_chain(k, width=2):
    """k diamonds in series: sigma between the ends is width^k."""
    edges, nxt, prev = [], 1, 0
    for _ in range(k):
        mids = list(range(nxt, nxt + width))
        end = nxt + width
        for m in mids:
            edges += [(prev, m), (m, end)]
        prev, nxt = end, end + 1
    return gen.from_edges(prev + 1, edges), prev


def test_sigma_closed_form_and_saturation():
    g, end = diamond_chain(40)
    _, sst = O.pair_paths(g, 0, end, 1)
    assert sst == 2**40
    g, end = diamond_chain(63)
    _, sst = O.pair_paths(g, 0, end, 1)
    assert sst == 2**63
    g, end = diamond_chain(70)  # 2^70 > 2^64 - 1: saturates
    rows, sst = O.pair_paths(g, 0, end, 200)
    assert sst == U64MAX
    # the draw proceeds on saturated values and still returns a valid shortest path
    for row in rows[:20]:
        assert len(interior(row)) == 2 * 70 - 1
    g3, end3 = diamond_chain(44, width=3)  # 3^44 > 2^64
    _, sst = O.pair_paths(g3, 0, end3, 1)
    assert sst == U64MAX
    g3, end3 = diamond_chain(40, width=3)  # 3^40 < 2^64
    _, sst = O.pair_paths(g3, 0, end3, 1)
    assert sst == 3**40


def test_overflow_flag_on_samples():
    g, end = diamond_chain(70)
    r = O.samples(g, seed=1, i0=0, count=3000)
    far = (np.abs(r["s"] // 3 - r["t"] // 3) >= 68)
    assert (r["overflow"][r["sigma_st"] == U64MAX] == 1).all()
    assert (r["overflow"][r["sigma_st"] < U64MAX] == 0).all()
    assert r["overflow"][far].all() if far.any() else True
