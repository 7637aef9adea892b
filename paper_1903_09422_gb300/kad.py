"""Python binding of libkad (include/kad.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module
converts arrays, passes the CUDA stream (PyTorch's current stream by default)
and turns status codes into exceptions.  It has no CPU fallback: if
libkad.so is missing, importing the binding fails.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkad.so")

KAD_GRAPH_TRUSTED = 1
KAD_GRAPH_DIRECTED = 2
KAD_GRAPH_TIGHT_VD = 4
KAD_RUN_TIMING = 1
KAD_RUN_AUTOTUNE = 2
KAD_RUN_COMPLETION_ORDER = 4
WORK_NAMES = ("expanded", "scanned", "labelled", "pred_arcs", "trace_arcs", "increments")


class KadError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} (status {status})" if what else status_string(status))


class Options(ctypes.Structure):
    _fields_ = [("epoch_size", ctypes.c_uint32), ("calib_div", ctypes.c_uint32), ("ring_epochs", ctypes.c_uint32),
                ("slots", ctypes.c_int32), ("mcap", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("flags", ctypes.c_uint32), ("debug", ctypes.c_uint32),
                ("max_epochs", ctypes.c_uint32), ("samples_per_block", ctypes.c_int32), ("pair_cost", ctypes.c_int32)]


class Result(ctypes.Structure):
    _fields_ = [("bc", ctypes.c_void_p), ("counts", ctypes.c_void_p), ("c0", ctypes.c_void_p),
                ("ltab", ctypes.c_void_p), ("ltab_cap", ctypes.c_int64),
                ("tau", ctypes.c_uint64), ("omega", ctypes.c_uint64), ("calib_samples", ctypes.c_uint64),
                ("samples_computed", ctypes.c_uint64), ("overflow_samples", ctypes.c_uint64),
                ("epochs", ctypes.c_uint32), ("vd_bound", ctypes.c_int32), ("sigma_overflow", ctypes.c_int32),
                ("stopped_by_omega", ctypes.c_int32), ("tau_star", ctypes.c_double),
                ("work", ctypes.c_uint64 * 6),
                ("t_total_ms", ctypes.c_double), ("t_calib_ms", ctypes.c_double), ("t_ads_ms", ctypes.c_double),
                ("t_ads_kernel_ms", ctypes.c_double), ("ads_launches", ctypes.c_uint32),
                ("slots_used", ctypes.c_int32), ("kernel_launches", ctypes.c_uint32),
                ("block_threads_used", ctypes.c_int32), ("blocks_per_sm_used", ctypes.c_int32),
                ("phase_cycles", ctypes.c_uint64 * 6), ("t_host_ms", ctypes.c_double), ("t_setup_ms", ctypes.c_double),
                ("t_table_ms", ctypes.c_double), ("t_dev_calib_ms", ctypes.c_double),
                ("t_dev_first_close_ms", ctypes.c_double), ("t_dev_stop_ms", ctypes.c_double),
                ("t_dev_end_ms", ctypes.c_double), ("issued_at_stop", ctypes.c_uint64),
                ("samples_per_block_used", ctypes.c_int32), ("pair_cost_used", ctypes.c_int32),
                ("bfs_split_cycles", ctypes.c_uint64 * 2)]

PHASE_NAMES = ("draw", "bfs", "meet", "trace", "reset", "close")


class ServerOptions(ctypes.Structure):
    _fields_ = [("workers", ctypes.c_int32), ("slots_per_query", ctypes.c_int32), ("hbm_budget", ctypes.c_int64),
                ("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32), ("policy", ctypes.c_int32)]


EXPORTS = ("kad_graph_create", "kad_graph_create_device", "kad_graph_free", "kad_graph_info", "kad_options_default",
           "kad_run", "kad_run_device", "kad_sample_records", "kad_sample_records_noalloc", "kad_eval_fg",
           "kad_server_create", "kad_server_add_graph", "kad_submit", "kad_poll", "kad_wait", "kad_server_free",
           "kad_status_string", "kad_version", "kad_trim", "kad_run_order", "kad_run_sharded", "kad_shard_range")

_lib = None


def load():
    """Load libkad.so (raises ImportError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u32, u64, dbl = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64,
                                   ctypes.c_double)
    st = ctypes.c_int
    lib.kad_graph_create.argtypes = [i32, vp, vp, u32, vp, ctypes.POINTER(vp)]
    lib.kad_graph_create.restype = st
    lib.kad_graph_create_device.argtypes = [i32, i64, vp, vp, u32, vp, ctypes.POINTER(vp)]
    lib.kad_graph_create_device.restype = st
    lib.kad_graph_free.argtypes = [vp]
    lib.kad_graph_free.restype = None
    lib.kad_graph_info.argtypes = [vp, vp, vp, vp, vp]
    lib.kad_graph_info.restype = st
    lib.kad_options_default.argtypes = [ctypes.POINTER(Options)]
    lib.kad_options_default.restype = None
    lib.kad_run.argtypes = [vp, dbl, dbl, u64, vp, ctypes.POINTER(Options), ctypes.POINTER(Result)]
    lib.kad_run.restype = st
    lib.kad_run_device.argtypes = [vp, dbl, dbl, u64, vp, ctypes.POINTER(Options), vp, vp, ctypes.POINTER(Result)]
    lib.kad_run_device.restype = st
    lib.kad_sample_records.argtypes = [vp, u64, u32, u64, i64, vp, ctypes.POINTER(Options), vp, vp, vp, vp, vp, vp,
                                       i32, vp]
    lib.kad_sample_records.restype = st
    lib.kad_sample_records_noalloc.argtypes = [i32, vp, vp, vp, u64, u32, u64, i64, vp, vp, vp, vp, vp, vp, vp,
                                               i32]
    lib.kad_sample_records_noalloc.restype = st
    lib.kad_eval_fg.argtypes = [i32, vp, vp, vp, i32, u64, u64, vp, vp]
    lib.kad_eval_fg.restype = st
    lib.kad_server_create.argtypes = [ctypes.POINTER(ServerOptions), ctypes.POINTER(vp)]
    lib.kad_server_create.restype = st
    lib.kad_server_add_graph.argtypes = [vp, i32, vp, vp, u32, ctypes.POINTER(ctypes.c_int32)]
    lib.kad_server_add_graph.restype = st
    lib.kad_submit.argtypes = [vp, i32, dbl, dbl, u64, vp, ctypes.POINTER(ctypes.c_uint64)]
    lib.kad_submit.restype = st
    lib.kad_poll.argtypes = [vp, u64, ctypes.POINTER(ctypes.c_int)]
    lib.kad_poll.restype = st
    lib.kad_wait.argtypes = [vp, u64, i64, ctypes.POINTER(Result), ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
    lib.kad_wait.restype = st
    lib.kad_server_free.argtypes = [vp]
    lib.kad_server_free.restype = None
    lib.kad_status_string.argtypes = [st]
    lib.kad_status_string.restype = ctypes.c_char_p
    lib.kad_version.argtypes = []
    lib.kad_version.restype = u32
    lib.kad_trim.argtypes = []
    lib.kad_trim.restype = None
    lib.kad_run_order.argtypes = [vp, vp, u64]
    lib.kad_run_order.restype = st
    lib.kad_run_sharded.argtypes = [vp, dbl, dbl, u64, i32, i32, ALLGATHER_FN, vp, vp, ctypes.POINTER(Options),
                                    ctypes.POINTER(Result)]
    lib.kad_run_sharded.restype = st
    lib.kad_shard_range.argtypes = [i64, i32, i32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.kad_shard_range.restype = None
    _lib = lib
    return lib


# int allgather(void *user, const void *send, size_t bytes, void *recv)
ALLGATHER_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


def shard_range(count, rank, world):
    """kad_shard_range: the chunk [lo, hi) of `count` items that `rank` of `world` takes."""
    lo, hi = ctypes.c_int64(0), ctypes.c_int64(0)
    load().kad_shard_range(count, rank, world, ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def make_allgather(fn):
    """Wrap fn(send: bytes) -> bytes (all ranks' sends concatenated in rank order)
    as the C callback of kad_run_sharded.  Keep the returned object alive for the
    duration of the call."""
    def cb(user, send, nbytes, recv):
        try:
            out = fn(ctypes.string_at(send, nbytes))
            ctypes.memmove(recv, out, len(out))
            return 0
        except Exception:
            return 1
    return ALLGATHER_FN(cb)


def torch_allgather(group=None):
    """An allgather over a torch.distributed process group (host bytes in, host
    bytes out; device tensors when the group's backend is NCCL)."""
    import torch
    import torch.distributed as dist

    def fn(payload):
        world = dist.get_world_size(group)
        dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
        src = torch.frombuffer(bytearray(payload), dtype=torch.uint8).to(dev)
        dst = torch.empty(world * src.numel(), dtype=torch.uint8, device=dev)
        dist.all_gather_into_tensor(dst, src, group=group)
        return dst.cpu().numpy().tobytes()
    return fn


def status_string(s):
    return load().kad_status_string(s).decode()


def _check(s, what):
    if s != 0:
        raise KadError(s, what)


def _stream_handle(stream):
    """cudaStream_t of `stream` (a torch.cuda.Stream, an int handle, or None =
    PyTorch's current stream)."""
    if isinstance(stream, int):
        return stream
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def options(**kw):
    o = Options()
    load().kad_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if v is None:
            continue
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


class Graph:
    """A graph resident on the current CUDA device (kad_graph)."""

    def __init__(self, row_ptr, col, trusted=False, stream=None, directed=False, tight_vd=False, _handle=None):
        """directed: row_ptr/col list the out-arcs of a directed graph; tight_vd: the
        double-sweep vertex-diameter bound (undirected graphs)."""
        lib = load()
        self._h = None
        self.directed = bool(directed)
        flags = ((KAD_GRAPH_TRUSTED if trusted else 0) | (KAD_GRAPH_DIRECTED if directed else 0) |
                 (KAD_GRAPH_TIGHT_VD if tight_vd else 0))
        if _handle is not None:
            self._h = _handle
        else:
            rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
            cl = np.ascontiguousarray(col, dtype=np.int32)
            if cl.size == 0:
                cl = np.zeros(1, np.int32)
            h = ctypes.c_void_p()
            _check(lib.kad_graph_create(rp.size - 1, rp.ctypes.data, cl.ctypes.data, flags, _stream_handle(stream),
                                        ctypes.byref(h)), "kad_graph_create")
            self._h = h
        n, m, vd, nc = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib.kad_graph_info(self._h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(vd), ctypes.byref(nc)),
               "kad_graph_info")
        self.n, self.m, self.vd_bound, self.components = n.value, m.value, vd.value, nc.value

    @classmethod
    def from_csr(cls, csr, **kw):
        kw.setdefault("directed", bool(getattr(csr, "directed", False)))
        return cls(csr.row_ptr, csr.col, **kw)

    @classmethod
    def from_device(cls, d_row_ptr, d_col, trusted=False, stream=None, directed=False, tight_vd=False):
        """From device tensors (torch, int32, contiguous); copied device-to-device."""
        lib = load()
        h = ctypes.c_void_p()
        n = d_row_ptr.numel() - 1
        flags = ((KAD_GRAPH_TRUSTED if trusted else 0) | (KAD_GRAPH_DIRECTED if directed else 0) |
                 (KAD_GRAPH_TIGHT_VD if tight_vd else 0))
        _check(lib.kad_graph_create_device(n, d_col.numel(), d_row_ptr.data_ptr(), d_col.data_ptr(), flags,
                                           _stream_handle(stream), ctypes.byref(h)), "kad_graph_create_device")
        g = cls(None, None, _handle=h)
        g.directed = bool(directed)
        return g

    @property
    def path_cap(self):
        return max(self.vd_bound - 2, 1)

    def close(self):
        if self._h:
            load().kad_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------- runs
    def run(self, eps, delta, seed, stream=None, bc=True, counts=True, c0=False, ltab=False, timing=False, **opt):
        """kad_run: returns a dict with the scalars of kad_result and the requested arrays."""
        lib = load()
        o = options(**opt)
        if timing:
            o.flags |= KAD_RUN_TIMING
        r = Result()
        out = {}
        if bc:
            out["bc"] = np.zeros(self.n, np.float64)
            r.bc = out["bc"].ctypes.data
        if counts:
            out["counts"] = np.zeros(self.n, np.uint32)
            r.counts = out["counts"].ctypes.data
        if c0:
            out["c0"] = np.zeros(self.n, np.uint32)
            r.c0 = out["c0"].ctypes.data
        if ltab:
            cap = 1 << 22
            out["L"] = np.zeros(cap, np.float64)
            r.ltab = out["L"].ctypes.data
            r.ltab_cap = cap
        _check(lib.kad_run(self._h, eps, delta, seed, _stream_handle(stream), ctypes.byref(o), ctypes.byref(r)),
               "kad_run")
        out.update(_result_scalars(r))
        if ltab:
            out["L"] = out["L"][: r.calib_samples + 1].copy()
        return out

    def run_device(self, eps, delta, seed, d_bc=None, d_counts=None, stream=None, timing=False, **opt):
        """kad_run_device: per-vertex outputs into device tensors (float64 / int32-sized)."""
        lib = load()
        o = options(**opt)
        if timing:
            o.flags |= KAD_RUN_TIMING
        r = Result()
        _check(lib.kad_run_device(self._h, eps, delta, seed, _stream_handle(stream), ctypes.byref(o),
                                  d_bc.data_ptr() if d_bc is not None else None,
                                  d_counts.data_ptr() if d_counts is not None else None, ctypes.byref(r)),
               "kad_run_device")
        return _result_scalars(r)

    def run_sharded(self, eps, delta, seed, rank, world, allgather, stream=None, counts=True, c0=False, ltab=False,
                    **opt):
        """kad_run_sharded: this rank's part of a run split among `world` ranks.
        allgather: fn(send: bytes) -> bytes, all ranks' sends in rank order."""
        lib = load()
        o = options(**opt)
        r = Result()
        out = {}
        bc = np.zeros(self.n, dtype=np.float64)
        r.bc = bc.ctypes.data
        if counts:
            out["counts"] = np.zeros(self.n, dtype=np.uint32)
            r.counts = out["counts"].ctypes.data
        if c0:
            out["c0"] = np.zeros(self.n, dtype=np.uint32)
            r.c0 = out["c0"].ctypes.data
        if ltab:
            out["L"] = np.zeros(1 << 22, dtype=np.float64)
            r.ltab = out["L"].ctypes.data
            r.ltab_cap = out["L"].size
        cb = make_allgather(allgather)
        _check(lib.kad_run_sharded(self._h, eps, delta, seed, rank, world, cb, None, _stream_handle(stream),
                                   ctypes.byref(o), ctypes.byref(r)), "kad_run_sharded")
        out["bc"] = bc
        out.update(_result_scalars(r))
        if ltab:
            out["L"] = out["L"][: r.calib_samples + 1].copy()
        return out

    def run_order(self, count):
        """kad_run_order: the adaptive sample indices at fold positions [0, count)
        of the last completion-order run on this graph."""
        out = np.zeros(count, np.uint64)
        _check(load().kad_run_order(self._h, out.ctypes.data, count), "kad_run_order")
        return out

    def sample_records(self, seed, i0, count, domain=0, cap=None, stream=None, **opt):
        """Per-sample records of samples [i0, i0+count) (same layout as the oracle's)."""
        lib = load()
        cap = self.path_cap if cap is None else cap
        o = options(**opt)
        s = np.zeros(count, np.int32)
        t = np.zeros(count, np.int32)
        D = np.zeros(count, np.int32)
        sst = np.zeros(count, np.uint64)
        ovf = np.zeros(count, np.int32)
        paths = np.zeros((count, cap), np.int32)
        work = np.zeros(6, np.uint64)
        _check(lib.kad_sample_records(self._h, seed, domain, i0, count, _stream_handle(stream), ctypes.byref(o),
                                      s.ctypes.data, t.ctypes.data, D.ctypes.data, sst.ctypes.data, ovf.ctypes.data,
                                      paths.ctypes.data, cap, work.ctypes.data), "kad_sample_records")
        return dict(s=s, t=t, D=D, sigma_st=sst, overflow=ovf, paths=paths, cap=cap,
                    counters=dict(zip(WORK_NAMES, (int(x) for x in work))))


def _result_scalars(r):
    d = {k: getattr(r, k) for k in ("tau", "omega", "calib_samples", "samples_computed", "overflow_samples", "epochs",
                                    "vd_bound", "sigma_overflow", "stopped_by_omega", "tau_star", "t_total_ms",
                                    "t_calib_ms", "t_ads_ms", "t_ads_kernel_ms", "ads_launches", "slots_used",
                                    "kernel_launches", "block_threads_used", "blocks_per_sm_used", "t_host_ms",
                                    "t_setup_ms", "t_table_ms", "t_dev_calib_ms", "t_dev_first_close_ms",
                                    "t_dev_stop_ms", "t_dev_end_ms", "issued_at_stop", "samples_per_block_used",
                                    "pair_cost_used")}
    d["counters"] = dict(zip(WORK_NAMES, (int(x) for x in r.work)))
    d["phase_cycles"] = dict(zip(PHASE_NAMES, (int(x) for x in r.phase_cycles)))
    d["bfs_split_cycles"] = dict(passes=int(r.bfs_split_cycles[0]), close=int(r.bfs_split_cycles[1]))
    return d


def sample_records_noalloc(d_row_ptr, d_col, seed, i0, count, out, cap, domain=0, d_comp=None, stream=None):
    """kad_sample_records_noalloc: every array is a caller-owned device tensor.

    `out` holds device tensors s, t, D (int32), sigma_st (int64/uint64),
    overflow (uint8) with `count` entries and paths (int32, count x cap).
    The library allocates nothing; its scratch is a fixed device array.
    """
    lib = load()
    n = d_row_ptr.numel() - 1
    _check(lib.kad_sample_records_noalloc(n, d_row_ptr.data_ptr(), d_col.data_ptr(),
                                          d_comp.data_ptr() if d_comp is not None else None, seed, domain, i0,
                                          count, _stream_handle(stream), out["s"].data_ptr(), out["t"].data_ptr(),
                                          out["D"].data_ptr(), out["sigma_st"].data_ptr(),
                                          out["overflow"].data_ptr(), out["paths"].data_ptr(), cap),
           "kad_sample_records_noalloc")


class Server:
    """Query server (kad_server): resident graphs, concurrent queries.

    ctypes releases the GIL during every call, so a Python thread can submit
    while another waits."""

    def __init__(self, workers=0, slots_per_query=0, hbm_budget=0, block_threads=0, blocks_per_sm=0, policy=0):
        lib = load()
        o = ServerOptions(workers, slots_per_query, hbm_budget, block_threads, blocks_per_sm, policy)
        h = ctypes.c_void_p()
        _check(lib.kad_server_create(ctypes.byref(o), ctypes.byref(h)), "kad_server_create")
        self._h = h
        self._n = []
        self._bufs = {}

    def add_graph(self, csr, trusted=False):
        directed = bool(getattr(csr, "directed", False))
        rp = np.ascontiguousarray(csr.row_ptr, dtype=np.int32)
        cl = np.ascontiguousarray(csr.col, dtype=np.int32)
        if cl.size == 0:
            cl = np.zeros(1, np.int32)
        gid = ctypes.c_int32()
        _check(load().kad_server_add_graph(self._h, rp.size - 1, rp.ctypes.data, cl.ctypes.data,
                                           (KAD_GRAPH_TRUSTED if trusted else 0) |
                                           (KAD_GRAPH_DIRECTED if directed else 0), ctypes.byref(gid)),
               "kad_server_add_graph")
        self._n.append(rp.size - 1)
        return gid.value

    def submit(self, gid, eps, delta, seed, want_bc=True):
        n = self._n[gid] if 0 <= gid < len(self._n) else 0  # an unknown gid is rejected by kad_submit
        bc = np.zeros(max(n, 1), np.float64) if want_bc else None
        t = ctypes.c_uint64()
        _check(load().kad_submit(self._h, gid, eps, delta, seed, bc.ctypes.data if bc is not None else None,
                                 ctypes.byref(t)), "kad_submit")
        self._bufs[t.value] = bc
        return t.value

    def poll(self, ticket):
        d = ctypes.c_int()
        _check(load().kad_poll(self._h, ticket, ctypes.byref(d)), "kad_poll")
        return bool(d.value)

    def wait(self, ticket, timeout_s=None):
        r = Result()
        qm, lm = ctypes.c_double(), ctypes.c_double()
        tn = -1 if timeout_s is None else int(timeout_s * 1e9)
        st = load().kad_wait(self._h, ticket, tn, ctypes.byref(r), ctypes.byref(qm), ctypes.byref(lm))
        if st == 5 and timeout_s is not None:
            raise TimeoutError(f"query {ticket} still running")
        bc = self._bufs.pop(ticket, None)
        _check(st, "kad_wait")
        d = _result_scalars(r)
        d["bc"] = bc
        d["queue_ms"] = qm.value
        d["latency_ms"] = lm.value
        return d

    def close(self):
        if self._h:
            load().kad_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def eval_fg(counts, c0, ltab, tau, omega):
    """The device stop-check arithmetic (Appendix B f and g) for every vertex."""
    lib = load()
    counts = np.ascontiguousarray(counts, np.uint32)
    c0 = np.ascontiguousarray(c0, np.uint32)
    ltab = np.ascontiguousarray(ltab, np.float64)
    f = np.zeros(counts.size, np.float64)
    g = np.zeros(counts.size, np.float64)
    _check(lib.kad_eval_fg(counts.size, counts.ctypes.data, c0.ctypes.data, ltab.ctypes.data, ltab.size, tau, omega,
                           f.ctypes.data, g.ctypes.data), "kad_eval_fg")
    return f, g


def trim():
    """kad_trim: free the workspace kept from freed graphs."""
    load().kad_trim()


def version():
    v = load().kad_version()
    return (v >> 16, v & 0xffff)
