"""kad_sample_records_noalloc: the records entry point for callers that may not
allocate device memory (they own every device buffer through their own pool, so
the library must not call cudaMalloc/cudaFree; its scratch is a fixed device
array instead).  Its output must equal the allocating entry point's,
kad_sample_records, record for record, on consecutive calls, and the oracle's.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kad():
    import torch
    torch.cuda.set_device(0)
    from paper_1903_09422_gb300 import build, kad as K
    build.build()
    K.load()
    return K


def _noalloc(kad, g, seed, i0, count, cap, d_comp=None):
    import torch
    d_rp = torch.from_numpy(g.row_ptr).cuda()
    d_col = torch.from_numpy(g.col).cuda()
    out = dict(s=torch.empty(count, dtype=torch.int32, device="cuda"),
               t=torch.empty(count, dtype=torch.int32, device="cuda"),
               D=torch.empty(count, dtype=torch.int32, device="cuda"),
               sigma_st=torch.empty(count, dtype=torch.int64, device="cuda"),
               overflow=torch.empty(count, dtype=torch.uint8, device="cuda"),
               paths=torch.empty((count, cap), dtype=torch.int32, device="cuda"))
    kad.sample_records_noalloc(d_rp, d_col, seed, i0, count, out, cap, d_comp=d_comp)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["sigma_st"] = res["sigma_st"].view(np.uint64)
    res["overflow"] = res["overflow"].astype(np.int32)
    return res


def _same(a, b):
    for k in ("s", "t", "D", "sigma_st", "overflow", "paths"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls(kad):
    from paper_1903_09422_gb300 import gen
    g = gen.rmat(12, 8, seed=1)
    with kad.Graph.from_csr(g) as G:
        cap = G.path_cap
        for i0, count in ((0, 700), (700, 1300)):  # two calls in a row share the scratch
            ref = G.sample_records(5, i0, count)
            _same(_noalloc(kad, g, 5, i0, count, cap), ref)


def test_noalloc_without_component_labels_on_a_disconnected_graph(kad):
    from paper_1903_09422_gb300 import gen
    g = gen.from_edges(12, [(0, 1), (1, 2), (2, 3), (3, 0), (4, 5), (5, 6), (6, 7), (7, 8), (8, 9), (9, 10),
                            (10, 11)])
    with kad.Graph.from_csr(g) as G:
        ref1 = G.sample_records(3, 0, 400)
        ref2 = G.sample_records(3, 400, 400)
        cap = G.path_cap
    _same(_noalloc(kad, g, 3, 0, 400, cap), ref1)
    _same(_noalloc(kad, g, 3, 400, 400, cap), ref2)


def _slots_for(n):
    """Sampling slots the fixed scratch holds for n vertices (same sizing as the
    entry point: 48 MiB minus a 4 KiB head and 4 MiB of path lengths; per slot a
    16-byte record, sigma2 and a list entry per vertex, and a bitmap word per 32
    vertices; a shared component array; every part 256-byte aligned)."""
    a = lambda x: (x + 255) & ~255
    area = (48 << 20) - 4096 - (1 << 20) * 4
    for slots in range(64, 0, -1):
        need = a(n * 4) + a(slots * n * 16) + a(slots * n * 8) + a(slots * n * 4) + a(slots * ((n + 31) // 32) * 4)
        if need <= area:
            return slots
    return 0


def test_noalloc_with_fewer_slots_matches_the_oracle(kad):
    # R-MAT scale 18 (n = 173,790) leaves room for only a few sampling slots in
    # the fixed scratch, so the entry point runs with fewer than its 64 slots.
    import oracle as O
    from paper_1903_09422_gb300 import gen
    g = gen.rmat(18, 16, seed=1)
    assert 1 < _slots_for(g.n) < 64
    cap = O.path_cap(g)
    for i0, count in ((0, 240), (240, 160)):  # two calls in a row share the scratch
        got = _noalloc(kad, g, 9, i0, count, cap)
        ref = O.samples(g, 9, i0, count)
        ref["overflow"] = ref["overflow"].astype(np.int32)
        _same(got, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch(kad):
    lib = kad.load()
    big = 2_000_000  # above the scratch's 1.44M-vertex limit; rejected before any device work
    assert lib.kad_sample_records_noalloc(big, 8, 8, None, 1, 0, 0, 10, None, 8, 8, 8, 8, 8, 8, 4) == 1
    assert lib.kad_sample_records_noalloc(100, 8, 8, None, 1, 0, 0, (1 << 20) + 1, None, 8, 8, 8, 8, 8, 8, 4) == 1
