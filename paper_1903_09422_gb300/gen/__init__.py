"""Seeded synthetic graph inputs for the KADABRA workloads.

The paper measures on 27 real-world undirected graphs (social, hyperlink and road
networks; Section 4 and Appendix E).  Those are not available here, so these
generators stand in for them.  Each returns the canonical symmetric CSR
(``row_ptr`` int32[n+1], ``col`` int32[m], rows sorted, no self-loops, no
duplicates), optionally reduced to the largest connected component.  The
directed generators (KADABRA also covers directed graphs, Section 5) return the
out-arc CSR with ``directed`` set, reduced to the largest weakly connected
component.

This module is the only code shared by the CUDA path's tests and the oracle's:
it produces inputs and holds none of the sampling method's arithmetic.
"""
import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_SO = os.path.join(_HERE, "libkadgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator library in-tree (plain C, a few seconds)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            vp = ctypes.c_void_p
            lib.gg_rmat.restype = vp
            lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, ctypes.c_int]
            lib.gg_rmat_directed.restype = vp
            lib.gg_rmat_directed.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_uint64, ctypes.c_int]
            lib.gg_grid.restype = vp
            lib.gg_grid.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_uint64, ctypes.c_int]
            lib.gg_er.restype = vp
            lib.gg_er.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_uint64, ctypes.c_int]
            lib.gg_hyperbolic.restype = vp
            lib.gg_hyperbolic.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                          ctypes.c_int]
            lib.gg_hyperbolic_radius.restype = ctypes.c_double
            lib.gg_hyperbolic_radius.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double]
            lib.gg_n.restype = ctypes.c_int32
            lib.gg_n.argtypes = [vp]
            lib.gg_m.restype = ctypes.c_int64
            lib.gg_m.argtypes = [vp]
            lib.gg_copy.restype = None
            lib.gg_copy.argtypes = [vp, vp, vp]
            lib.gg_destroy.restype = None
            lib.gg_destroy.argtypes = [vp]
            _lib = lib
    return _lib


@dataclass
class CSR:
    """Graph as a CSR with int32 indices: symmetric when undirected, the out-arc
    rows when ``directed``."""
    row_ptr: np.ndarray
    col: np.ndarray
    name: str = ""
    directed: bool = False

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def m(self) -> int:
        return int(self.col.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def _take(h, name, directed=False):
    if not h:
        raise MemoryError("graph generator failed (invalid parameters or out of memory)")
    lib = _load()
    try:
        n, m = lib.gg_n(h), lib.gg_m(h)
        rp = np.empty(n + 1, dtype=np.int32)
        col = np.empty(max(m, 1), dtype=np.int32)
        lib.gg_copy(h, rp.ctypes.data, col.ctypes.data)
    finally:
        lib.gg_destroy(h)
    return CSR(rp, col[:m], name, directed)


def rmat(scale: int, edge_factor: int, a=0.57, b=0.19, c=0.19, seed: int = 1, lcc: bool = True) -> CSR:
    """R-MAT with edge_factor * 2^scale edge draws, made undirected and simple."""
    h = _load().gg_rmat(scale, edge_factor, a, b, c, seed, int(lcc))
    return _take(h, f"rmat{scale}_ef{edge_factor}_s{seed}")


def rmat_directed(scale: int, edge_factor: int, a=0.57, b=0.19, c=0.19, seed: int = 1, lcc: bool = True) -> CSR:
    """Directed R-MAT: each of edge_factor * 2^scale draws (u, w) gives the arc u -> w."""
    h = _load().gg_rmat_directed(scale, edge_factor, a, b, c, seed, int(lcc))
    return _take(h, f"rmat{scale}d_ef{edge_factor}_s{seed}", True)


def grid(side: int, p_remove=0.05, shortcut_frac=0.001, seed: int = 1, lcc: bool = True) -> CSR:
    """side x side 4-neighbour grid, edges removed w.p. p_remove, plus shortcuts."""
    h = _load().gg_grid(side, p_remove, shortcut_frac, seed, int(lcc))
    return _take(h, f"grid{side}_s{seed}")


def er(n: int, p: float, seed: int = 1, lcc: bool = True) -> CSR:
    """Erdos-Renyi G(n, p)."""
    h = _load().gg_er(n, p, seed, int(lcc))
    return _take(h, f"er{n}_p{p}_s{seed}")


def hyperbolic(n: int, avg_deg=20.0, gamma=2.5, seed: int = 1, lcc: bool = True) -> CSR:
    """Threshold (temperature 0) random hyperbolic graph."""
    h = _load().gg_hyperbolic(n, avg_deg, gamma, seed, int(lcc))
    return _take(h, f"hyp{n}_s{seed}")


def hyperbolic_radius(n: int, avg_deg=20.0, gamma=2.5) -> float:
    return float(_load().gg_hyperbolic_radius(n, avg_deg, gamma))


def from_edges(n: int, edges, name: str = "custom") -> CSR:
    """Symmetric simple CSR from an undirected edge list (self-loops and duplicates dropped)."""
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    e = e[e[:, 0] != e[:, 1]]
    both = np.concatenate([e, e[:, ::-1]], axis=0)
    key = np.unique(both[:, 0] * n + both[:, 1])
    u, v = key // n, key % n
    rp = np.zeros(n + 1, dtype=np.int32)
    np.add.at(rp, u + 1, 1)
    rp = np.cumsum(rp).astype(np.int32)
    return CSR(rp, v.astype(np.int32), name)


def from_arcs(n: int, arcs, name: str = "custom_d") -> CSR:
    """Directed simple CSR from an arc list (self-loops and duplicates dropped)."""
    e = np.asarray(arcs if isinstance(arcs, np.ndarray) else list(arcs), dtype=np.int64).reshape(-1, 2)
    e = e[e[:, 0] != e[:, 1]]
    key = np.unique(e[:, 0] * n + e[:, 1])
    u, v = key // n, key % n
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, u + 1, 1)
    rp = np.cumsum(rp).astype(np.int32)
    return CSR(rp, v.astype(np.int32), name, True)


def largest_weak_component(g: CSR) -> CSR:
    """The directed graph induced by its largest weakly connected component
    (ties: the one holding the smallest id), ids renumbered in order."""
    n = g.n
    lab = np.arange(n)
    src = np.repeat(np.arange(n), np.diff(g.row_ptr))
    dst = g.col.astype(np.int64)
    while True:  # propagate the smallest id along arcs both ways, then jump
        new = lab.copy()
        np.minimum.at(new, dst, new[src])
        np.minimum.at(new, src, new[dst])
        new = new[new]
        if np.array_equal(new, lab):
            break
        lab = new
    best = int(np.argmax(np.bincount(lab, minlength=n)))
    keep = lab == best
    newid = np.cumsum(keep) - 1
    m = keep[src] & keep[dst]
    arcs = np.stack([newid[src[m]], newid[dst[m]]], axis=1)
    return from_arcs(int(keep.sum()), arcs, g.name + "_lwcc")


def grid_oneway(side: int, p_oneway=0.3, seed: int = 1, lcc: bool = True) -> CSR:
    """Directed side x side 4-neighbour grid (a street map): each edge is a
    one-way arc, in a random direction, with probability p_oneway, else both arcs."""
    rng = np.random.default_rng(seed)
    ids = np.arange(side * side).reshape(side, side)
    e = np.concatenate([np.stack([ids[:, :-1].ravel(), ids[:, 1:].ravel()], 1),
                        np.stack([ids[:-1, :].ravel(), ids[1:, :].ravel()], 1)])
    one = rng.random(len(e)) < p_oneway
    flip = rng.random(len(e)) < 0.5
    fwd = np.where((one & flip)[:, None], e[:, ::-1], e)
    arcs = np.concatenate([fwd, e[~one][:, ::-1]])
    g = from_arcs(side * side, arcs, f"grid{side}d_s{seed}")
    return largest_weak_component(g) if lcc else g


def path_graph(n: int) -> CSR:
    return from_edges(n, [(i, i + 1) for i in range(n - 1)], f"path{n}")


def star_graph(n: int) -> CSR:
    return from_edges(n, [(0, i) for i in range(1, n)], f"star{n}")


def grid_plain(rows: int, cols: int) -> CSR:
    ed = []
    for r in range(rows):
        for c in range(cols):
            v = r * cols + c
            if c + 1 < cols:
                ed.append((v, v + 1))
            if r + 1 < rows:
                ed.append((v, v + cols))
    return from_edges(rows * cols, ed, f"grid{rows}x{cols}")


# Named workloads: graph recipe plus the (eps, delta, seed) each is run at.
WORKLOADS = {
    "rmat12": dict(kind="rmat", scale=12, edge_factor=8, eps=0.05, delta=0.1, seed=1),
    "rmat15": dict(kind="rmat", scale=15, edge_factor=16, eps=0.01, delta=0.1, seed=1),
    "rmat18": dict(kind="rmat", scale=18, edge_factor=16, eps=0.01, delta=0.1, seed=1),
    "rmat20": dict(kind="rmat", scale=20, edge_factor=16, eps=0.01, delta=0.1, seed=1),
    "grid2048": dict(kind="grid", side=2048, eps=0.01, delta=0.1, seed=1),
    "rmat18d": dict(kind="rmat_directed", scale=18, edge_factor=16, eps=0.01, delta=0.1, seed=1),
    "rmat20d": dict(kind="rmat_directed", scale=20, edge_factor=16, eps=0.01, delta=0.1, seed=1),
    "hyp4m": dict(kind="hyperbolic", n=4 * (1 << 20), eps=0.005, delta=0.1, seed=1),
}


def describe(name: str) -> str:
    w = WORKLOADS[name]
    if w["kind"] == "rmat":
        g = f"R-MAT scale {w['scale']} ef {w['edge_factor']} (a,b,c=.57,.19,.19) undirected LCC"
    elif w["kind"] == "rmat_directed":
        g = f"R-MAT scale {w['scale']} ef {w['edge_factor']} (a,b,c=.57,.19,.19) directed, largest weak component"
    elif w["kind"] == "grid":
        g = f"{w['side']}x{w['side']} grid, 5% edges removed, 0.1% shortcuts, LCC"
    else:
        g = f"threshold hyperbolic n={w['n']} avg deg 20 gamma 2.5, LCC"
    return f"{g}; eps={w['eps']} delta={w['delta']} seed={w['seed']}"


def workload_graph(name: str, graph_seed: int = 1) -> CSR:
    w = WORKLOADS[name]
    if w["kind"] == "rmat":
        return rmat(w["scale"], w["edge_factor"], seed=graph_seed)
    if w["kind"] == "rmat_directed":
        return rmat_directed(w["scale"], w["edge_factor"], seed=graph_seed)
    if w["kind"] == "grid":
        return grid(w["side"], seed=graph_seed)
    if w["kind"] == "hyperbolic":
        return hyperbolic(w["n"], seed=graph_seed)
    raise KeyError(name)
