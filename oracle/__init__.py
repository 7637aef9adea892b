"""ctypes wrapper of the KADABRA oracle (kadabra_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  The
CUDA library and its Python binding never do, and the oracle never imports them.

Every function here marshals arguments; the arithmetic is in the C file, which
cites the paper (arXiv 1903.09422) section by section.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kadabra_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# -ffp-contract=off: no fused multiply-add may change the rounding of f, g, L, omega.
CFLAGS = ["-O2", "-std=gnu99", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile the oracle in-tree with gcc (a second or two)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Result(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_uint64), ("omega", ctypes.c_uint64), ("calib_samples", ctypes.c_uint64),
                ("overflow_samples", ctypes.c_uint64), ("epochs", ctypes.c_uint64), ("samples", ctypes.c_uint64),
                ("vd", ctypes.c_int32), ("stopped_by_omega", ctypes.c_int32), ("tau_star", ctypes.c_double),
                ("counters", ctypes.c_uint64 * 6)]


COUNTER_NAMES = ("expanded", "scanned", "labelled", "pred_arcs", "trace_arcs", "increments")


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            vp, i32, i64, u32, u64, dbl = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                           ctypes.c_uint64, ctypes.c_double)
            lib.orc_philox4x32_10.argtypes = [vp, vp, vp]
            lib.orc_philox4x32_10.restype = None
            lib.orc_stream_draws.argtypes = [u64, u64, u32, vp, i64, vp, vp]
            lib.orc_stream_draws.restype = None
            lib.orc_stream_words.argtypes = [u64, u64, u32, i64, vp]
            lib.orc_stream_words.restype = None
            lib.orc_transpose.argtypes = [i32, vp, vp, vp, vp]
            lib.orc_transpose.restype = None
            lib.orc_components.argtypes = [i32, vp, vp, vp, vp, vp]
            lib.orc_components.restype = i32
            lib.orc_scc.argtypes = [i32, vp, vp, vp, vp, vp]
            lib.orc_scc.restype = i32
            lib.orc_vd_bound.argtypes = [i32, vp, vp, vp, vp]
            lib.orc_vd_bound.restype = i32
            lib.orc_vd_bound_tight.argtypes = [i32, vp, vp]
            lib.orc_vd_bound_tight.restype = i32
            lib.orc_omega.argtypes = [i32, dbl, dbl]
            lib.orc_omega.restype = u64
            lib.orc_calib_samples.argtypes = [u64, u32, u32]
            lib.orc_calib_samples.restype = u64
            for fn in (lib.orc_f, lib.orc_g):
                fn.argtypes = [u64, dbl, u64, u64]
                fn.restype = dbl
            lib.orc_L.argtypes = [dbl, dbl, dbl, u64]
            lib.orc_L.restype = dbl
            lib.orc_tau_star.argtypes = [vp, u64, dbl, dbl, u64]
            lib.orc_tau_star.restype = dbl
            lib.orc_samples.argtypes = [i32, vp, vp, vp, vp, u64, u32, u64, i64, vp, vp, vp, vp, vp, vp, i32, vp]
            lib.orc_samples.restype = ctypes.c_int
            lib.orc_pair_paths.argtypes = [i32, vp, vp, vp, vp, i32, i32, u64, u32, i64, vp, i32, vp]
            lib.orc_pair_paths.restype = ctypes.c_int
            lib.orc_kadabra.argtypes = [i32, vp, vp, vp, vp, i32, dbl, dbl, u64, u32, u32, u64, vp, vp, vp, vp, i64,
                                        ctypes.POINTER(_Result)]
            lib.orc_kadabra.restype = ctypes.c_int
            _lib = lib
    return _lib


def _arr(x):
    a = np.ascontiguousarray(x, dtype=np.int32)
    return a if a.size else np.zeros(1, dtype=np.int32)


class _Rows:
    """A graph's CSR arrays as the C functions take them: the out-arc rows, and
    for a directed graph (``g.directed``) the in-arc rows too (else NULL).  The
    arrays stay referenced by this object for the duration of a call."""

    def __init__(self, g, force_directed=False):
        self.n = g.n
        self.rp = _arr(g.row_ptr)
        self.col = _arr(g.col)
        self.rpT = self.colT = None
        if getattr(g, "directed", False):
            rpT, colT = transpose(g)
            self.rpT, self.colT = _arr(rpT), _arr(colT)
        elif force_directed:
            self.rpT, self.colT = self.rp, self.col

    def args(self):
        rpT = self.rpT.ctypes.data if self.rpT is not None else None
        colT = self.colT.ctypes.data if self.colT is not None else None
        return (self.n, self.rp.ctypes.data, self.col.ctypes.data, rpT, colT)


def transpose(g):
    """The in-arc CSR (row_ptr, col) of a directed graph, rows ascending."""
    rp, col = _arr(g.row_ptr), _arr(g.col)
    m = int(np.asarray(g.col).size)
    rpT = np.zeros(g.n + 1, np.int32)
    colT = np.zeros(max(m, 1), np.int32)
    _load().orc_transpose(g.n, rp.ctypes.data, col.ctypes.data, rpT.ctypes.data, colT.ctypes.data)
    return rpT, colT[:m]


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def stream_words(seed, index, domain, count):
    out = np.zeros(count, dtype=np.uint64)
    _load().orc_stream_words(seed, index, domain, count, out.ctypes.data)
    return out


def stream_draws(seed, index, domain, ms):
    ms = np.ascontiguousarray(ms, dtype=np.uint64)
    out = np.zeros(ms.size, dtype=np.uint64)
    used = ctypes.c_uint64(0)
    _load().orc_stream_draws(seed, index, domain, ms.ctypes.data, ms.size, out.ctypes.data, ctypes.byref(used))
    return out, int(used.value)


def components(g):
    """(count, labels): connected components, the weak ones of a directed graph."""
    r = _Rows(g)
    comp = np.zeros(g.n, dtype=np.int32)
    nc = _load().orc_components(*r.args(), comp.ctypes.data)
    return int(nc), comp


def scc(g):
    """(count, labels): strongly connected components (labels in the order found)."""
    r = _Rows(g, force_directed=True)
    out = np.zeros(g.n, dtype=np.int32)
    ns = _load().orc_scc(*r.args(), out.ctypes.data)
    return int(ns), out


def vd_bound(g, directed=None):
    """The vertex-diameter bound: the undirected rule, or the directed one for
    a directed graph (or for any graph with directed=True)."""
    r = _Rows(g, force_directed=bool(directed))
    return int(_load().orc_vd_bound(*r.args()))


def vd_bound_tight(g):
    """The opt-in double-sweep bound of an undirected graph (see the C source)."""
    r = _Rows(g)
    if r.rpT is not None:
        raise ValueError("the double-sweep bound is defined for undirected graphs")
    return int(_load().orc_vd_bound_tight(r.n, r.rp.ctypes.data, r.col.ctypes.data))


def omega(vd, eps, delta):
    return int(_load().orc_omega(vd, eps, delta))


def calib_samples(omega_, epoch=1000, calib_div=100):
    return int(_load().orc_calib_samples(omega_, epoch, calib_div))


def f(c, L, tau, omega_):
    return float(_load().orc_f(c, L, tau, omega_))


def g(c, L, tau, omega_):
    return float(_load().orc_g(c, L, tau, omega_))


def L_of(b0, tstar, eps, omega_):
    return float(_load().orc_L(b0, tstar, eps, omega_))


def tau_star(hist, eps, delta, omega_):
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    return float(_load().orc_tau_star(h.ctypes.data, h.size - 1, eps, delta, omega_))


def path_cap(g):
    return max(vd_bound(g) - 2, 1)


def samples(g, seed, i0, count, domain=0, cap=None):
    """Per-sample records of samples [i0, i0+count): dict of arrays."""
    r = _Rows(g)
    cap = path_cap(g) if cap is None else cap
    s = np.zeros(count, np.int32)
    t = np.zeros(count, np.int32)
    D = np.zeros(count, np.int32)
    sst = np.zeros(count, np.uint64)
    ovf = np.zeros(count, np.int32)
    paths = np.full((count, cap), -1, np.int32)
    ctr = np.zeros(6, np.uint64)
    rc = _load().orc_samples(*r.args(), seed, domain, i0, count, s.ctypes.data,
                             t.ctypes.data, D.ctypes.data, sst.ctypes.data, ovf.ctypes.data, paths.ctypes.data, cap,
                             ctr.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"oracle samples failed: {rc}")
    return dict(s=s, t=t, D=D, sigma_st=sst, overflow=ovf, paths=paths, cap=cap,
                counters=dict(zip(COUNTER_NAMES, (int(x) for x in ctr))))


def pair_paths(g, s, t, count, seed=1, domain=0, cap=None):
    """`count` uniform shortest s-t path draws; returns (paths[count, cap], sigma_st)."""
    r = _Rows(g)
    cap = path_cap(g) if cap is None else cap
    paths = np.full((count, cap), -1, np.int32)
    sst = ctypes.c_uint64(0)
    rc = _load().orc_pair_paths(*r.args(), s, t, seed, domain, count, paths.ctypes.data, cap, ctypes.byref(sst))
    if rc != 0:
        raise RuntimeError(f"oracle pair_paths failed: {rc}")
    return paths, int(sst.value)


def kadabra(g, eps, delta, seed, epoch=1000, calib_div=100, max_epochs=0, tight_vd=False):
    """Full KADABRA run.  max_epochs > 0 truncates the adaptive phase (timing samples);
    tight_vd: omega from the double-sweep bound (undirected graphs)."""
    r = _Rows(g)
    lib = _load()
    vd = vd_bound_tight(g) if tight_vd else lib.orc_vd_bound(*r.args())
    om = lib.orc_omega(vd, eps, delta)
    t0 = lib.orc_calib_samples(om, epoch, calib_div)
    counts = np.zeros(g.n, np.uint32)
    bc = np.zeros(g.n, np.float64)
    c0 = np.zeros(g.n, np.uint32)
    Ltab = np.zeros(t0 + 1, np.float64)
    res = _Result()
    rc = lib.orc_kadabra(*r.args(), vd, eps, delta, seed, epoch, calib_div, max_epochs,
                         counts.ctypes.data, bc.ctypes.data, c0.ctypes.data, Ltab.ctypes.data, Ltab.size,
                         ctypes.byref(res))
    if rc != 0:
        raise RuntimeError(f"oracle kadabra failed: {rc}")
    return dict(counts=counts, bc=bc, c0=c0, L=Ltab, tau=int(res.tau), omega=int(res.omega),
                calib_samples=int(res.calib_samples), overflow_samples=int(res.overflow_samples),
                epochs=int(res.epochs), vd=int(res.vd), stopped_by_omega=bool(res.stopped_by_omega),
                tau_star=float(res.tau_star), counters=dict(zip(COUNTER_NAMES, (int(x) for x in res.counters))))
