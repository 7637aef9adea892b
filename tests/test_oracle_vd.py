"""Pins of the oracle's preprocessing: connected components and the
vertex-diameter bound behind omega (Section 2.3: the maximal number of samples
comes mostly from an upper bound on the diameter; Appendix C.1: pairs in
different components are skipped).

The reading under test: in every component, a BFS from the component's vertex of
largest degree (smallest id on ties) gives ecc(v0); the diameter is at most
2 ecc(v0), and VD = max over components of 2 ecc(v0) + 1.  Each pin below is a
value fixed by the mathematics of a graph family, or an independent library
computation, chosen so that the plausible mistakes fail one of them: ecc instead
of 2 ecc, the highest id on degree ties, the first component instead of the
largest bound, a bound that is not an upper bound on the diameter.
"""
import numpy as np
import pytest

import oracle as O
from paper_1903_09422_gb300 import gen


def union(*graphs):
    """Disjoint union, vertex ids of each graph shifted past the previous ones."""
    edges, off = [], 0
    for g in graphs:
        for u in range(g.n):
            for w in g.col[g.row_ptr[u]:g.row_ptr[u + 1]]:
                if u < w:
                    edges.append((u + off, int(w) + off))
        off += g.n
    return gen.from_edges(off, edges)


def cycle_graph(n):
    return gen.from_edges(n, [(i, (i + 1) % n) for i in range(n)])


@pytest.mark.parametrize("n", [3, 4, 5, 10, 33])
def test_path_bound(n):
    # P_n: vertex 1 is the lowest id of the largest degree (2); ecc(1) = n - 2
    assert O.vd_bound(gen.path_graph(n)) == 2 * (n - 2) + 1


def test_two_vertex_path():
    # both vertices have degree 1: v0 = 0, ecc = 1
    assert O.vd_bound(gen.path_graph(2)) == 3


@pytest.mark.parametrize("n", [3, 5, 50])
def test_star_bound(n):
    # the centre (degree n-1) reaches every leaf in one step
    assert O.vd_bound(gen.star_graph(n)) == 3


@pytest.mark.parametrize("n", [3, 4, 7, 8, 21])
def test_cycle_bound(n):
    # every vertex has degree 2: v0 = 0, ecc = floor(n/2)
    assert O.vd_bound(cycle_graph(n)) == 2 * (n // 2) + 1


@pytest.mark.parametrize("a,b", [(3, 3), (3, 7), (6, 4), (10, 10)])
def test_grid_bound(a, b):
    # interior vertices have degree 4; the lowest-id one is (1, 1), whose
    # farthest vertex is the corner (a-1, b-1) at distance (a-2) + (b-2)
    assert O.vd_bound(gen.grid_plain(a, b)) == 2 * ((a - 2) + (b - 2)) + 1


def test_degree_tie_goes_to_the_smallest_id():
    # path 0..7 with a leaf 8 on vertex 1 and a leaf 9 on vertex 4: vertices 1
    # and 4 both have degree 3.  ecc(1) = 6 (to 7), ecc(4) = 4 (to 0 and 8).
    g = gen.from_edges(10, [(i, i + 1) for i in range(7)] + [(1, 8), (4, 9)])
    deg = np.diff(g.row_ptr)
    assert deg[1] == deg[4] == deg.max() == 3
    assert O.vd_bound(g) == 13  # 2 * ecc(1) + 1; the highest id would give 9


def test_largest_component_bound_wins():
    # component 0 (ids 0..2) is P_3 with bound 3; component 1 is P_10 with 17
    g = union(gen.path_graph(3), gen.path_graph(10))
    assert O.vd_bound(g) == 17
    g2 = union(gen.path_graph(10), gen.path_graph(3))
    assert O.vd_bound(g2) == 17
    g3 = union(gen.star_graph(6), cycle_graph(9), gen.path_graph(4))
    assert O.vd_bound(g3) == max(3, 9, 5)


def test_isolated_vertices():
    # every component is a single vertex: ecc = 0, VD = 1
    g = gen.from_edges(5, [])
    assert O.vd_bound(g) == 1
    nc, comp = O.components(g)
    assert nc == 5 and list(comp) == [0, 1, 2, 3, 4]


def test_components_numbered_by_smallest_vertex():
    g = gen.from_edges(8, [(0, 5), (5, 7), (1, 2), (3, 4), (4, 6)])
    nc, comp = O.components(g)
    assert nc == 3
    assert list(comp) == [0, 1, 1, 2, 2, 0, 2, 0]


def _brute_force_reference(g):
    """Independent computation with scipy's components and BFS distances."""
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    A = sp.csr_matrix((np.ones(g.m), g.col, g.row_ptr), shape=(g.n, g.n))
    nc, lab = csg.connected_components(A, directed=False)
    deg = np.diff(g.row_ptr)
    vd, diam = 1, 0
    for c in range(nc):
        members = np.flatnonzero(lab == c)
        v0 = members[np.argmax(deg[members])]  # argmax takes the first (smallest id) maximum
        d = csg.shortest_path(A, unweighted=True, indices=[v0])[0]
        ecc = int(d[members].max())
        vd = max(vd, 2 * ecc + 1)
        D = csg.shortest_path(A, unweighted=True, indices=members)[:, members]
        diam = max(diam, int(D.max()))
    return nc, lab, vd, diam


@pytest.mark.parametrize("seed", range(12))
def test_random_graphs_against_scipy(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(20, 120))
    p = float(rng.uniform(0.01, 0.08))
    iu = np.triu_indices(n, 1)
    keep = rng.random(iu[0].size) < p
    g = gen.from_edges(n, zip(iu[0][keep], iu[1][keep]))
    nc, lab, vd_ref, diam = _brute_force_reference(g)
    onc, ocomp = O.components(g)
    assert onc == nc
    # same partition (scipy numbers components in its own order)
    for c in range(nc):
        members = np.flatnonzero(ocomp == c)
        assert members.size and len(set(lab[members])) == 1
        assert members[0] == np.flatnonzero(lab == lab[members[0]])[0]
    assert O.vd_bound(g) == vd_ref
    # it is an upper bound on the vertex diameter (longest shortest path + 1)
    assert O.vd_bound(g) >= diam + 1


def test_bound_is_upper_bound_on_workload_sized_graphs():
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    for g in (gen.rmat(9, 8, seed=3), gen.grid(24, seed=2), gen.er(150, 0.03, seed=4)):
        A = sp.csr_matrix((np.ones(g.m), g.col, g.row_ptr), shape=(g.n, g.n))
        D = csg.shortest_path(A, unweighted=True)
        diam = int(D[np.isfinite(D)].max())
        vd = O.vd_bound(g)
        assert diam + 1 <= vd <= 2 * diam + 1


# ---------------------------------------------------------------- double sweep
# The opt-in bound: a = farthest from v0, b = farthest from a, m = the midpoint
# of an a-b shortest path nearest v0 (d(a, m) = ceil(d(a, b)/2), then smallest
# d(v0, m), then smallest id); per component 2 min(ecc(v0), ecc(m)) + 1.

@pytest.mark.parametrize("n", [2, 3, 4, 5, 10, 33])
def test_tight_path(n):
    # P_n: v0 = 1, a = n-1, b = 0, d = n-1; the midpoint at distance ceil((n-1)/2)
    # from a has eccentricity ceil((n-1)/2) (n = 2: v0 = 0, m = 0, ecc 1)
    assert O.vd_bound_tight(gen.path_graph(n)) == 2 * (-(-(n - 1) // 2)) + 1


def _grid_tight(r, c):
    """Closed form on the plain r x c grid (r, c >= 3): v0 = (1,1), a = (r-1,c-1),
    b = (0,0), d = r+c-2; the midpoints are the (i,j) with i+j = k = d - ceil(d/2);
    those with i, j >= 1 are nearest v0 (distance k-2, the others k), and of them
    the smallest id has the smallest i."""
    d = r + c - 2
    k = d - (-(-d // 2))
    i = max(1, k - (c - 1))
    j = k - i
    ecc_m = max(i + j, i + (c - 1 - j), (r - 1 - i) + j, (r - 1 - i) + (c - 1 - j))
    ecc_0 = (r - 2) + (c - 2)
    return 2 * min(ecc_0, ecc_m) + 1


@pytest.mark.parametrize("r,c", [(3, 3), (5, 7), (5, 8), (7, 5), (4, 9), (9, 9), (6, 13)])
def test_tight_grid(r, c):
    # 5x7: 15 (the smallest-id midpoint (0,5) alone would give 17); 5x8: 15
    # (a midpoint at floor(d/2) from a would give 17)
    assert O.vd_bound_tight(gen.grid_plain(r, c)) == _grid_tight(r, c)
    assert _grid_tight(5, 7) == 15 and _grid_tight(5, 8) == 15


def test_tight_star_cycle_and_components():
    assert O.vd_bound_tight(gen.star_graph(9)) == 3
    for n in (5, 8, 11):  # every vertex has eccentricity floor(n/2)
        assert O.vd_bound_tight(cycle_graph(n)) == 2 * (n // 2) + 1
    # the maximum over components
    g = union(gen.path_graph(4), gen.grid_plain(5, 7), gen.star_graph(5))
    assert O.vd_bound_tight(g) == 15


def _tight_reference(g):
    """The double-sweep rule with scipy's components and BFS distances; ties
    broken explicitly (np.lexsort / first maximum = smallest id)."""
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    A = sp.csr_matrix((np.ones(g.m), g.col, g.row_ptr), shape=(g.n, g.n))
    nc, lab = csg.connected_components(A, directed=False)
    deg = np.diff(g.row_ptr)
    vd = 1
    for c in range(nc):
        mem = np.flatnonzero(lab == c)
        bfs = lambda src: csg.shortest_path(A, unweighted=True, indices=[src])[0][mem].astype(int)
        v0 = mem[np.argmax(deg[mem])]
        d0 = bfs(v0)
        a = mem[np.argmax(d0)]  # farthest, smallest id
        da = bfs(a)
        b = mem[np.argmax(da)]
        db = bfs(b)
        d = int(da.max())
        cand = np.flatnonzero((da + db == d) & (da == (d + 1) // 2))
        m = mem[cand[np.lexsort((mem[cand], d0[cand]))[0]]]  # nearest v0, then smallest id
        vd = max(vd, 2 * min(int(d0.max()), int(bfs(m).max())) + 1)
    return vd


@pytest.mark.parametrize("seed", range(12))
def test_tight_bound_between_diameter_and_standard_bound(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(20, 120))
    p = float(rng.uniform(0.01, 0.08))
    iu = np.triu_indices(n, 1)
    keep = rng.random(iu[0].size) < p
    g = gen.from_edges(n, zip(iu[0][keep], iu[1][keep]))
    _, _, vd_ref, diam = _brute_force_reference(g)
    assert diam + 1 <= O.vd_bound_tight(g) <= vd_ref
    assert O.vd_bound_tight(g) == _tight_reference(g)


@pytest.mark.parametrize("seed", range(20))
def test_tight_bound_against_scipy_on_grids_with_holes(seed):
    # grids with removed edges and shortcuts: many distance ties and vertices at
    # the midpoint distance that are off every a-b shortest path
    g = gen.grid(6 + seed % 7, p_remove=0.15, shortcut_frac=0.02, seed=seed, lcc=False)
    assert O.vd_bound_tight(g) == _tight_reference(g)


def test_tight_bound_on_workload_sized_graphs():
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    for g in (gen.rmat(9, 8, seed=3), gen.grid(24, seed=2), gen.er(150, 0.03, seed=4), gen.grid(40, seed=5)):
        A = sp.csr_matrix((np.ones(g.m), g.col, g.row_ptr), shape=(g.n, g.n))
        D = csg.shortest_path(A, unweighted=True)
        diam = int(D[np.isfinite(D)].max())
        assert diam + 1 <= O.vd_bound_tight(g) <= O.vd_bound(g)
