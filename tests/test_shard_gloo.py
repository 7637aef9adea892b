"""Host logic of the sharded run on two gloo ranks (CPU, no GPU).

kad_run_sharded splits the calibration range and every epoch's sample indices
into contiguous chunks (kad_shard_range), exchanges each phase's path rows with
an allgather, and folds all rows on every rank before the stop check.  Here the
oracle stands in for the GPU sampler of each rank's chunk, the rows travel in
the library's block layout through kad.torch_allgather over gloo, and the fold
and the stop rule (Appendix B, with the oracle's f, g, L and tau*) applied to the
gathered rows must reproduce the single-rank oracle run: same calibration
counts, counts, tau and stop epoch on both ranks.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1903_09422_gb300 import build
    build.build()


def test_shard_range_partitions():
    from paper_1903_09422_gb300 import kad
    for count in (0, 1, 7, 1000, 1001, 12345):
        for world in (1, 2, 3, 7, 8):
            spans = [kad.shard_range(count, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == count
            for (lo, hi), (lo2, _) in zip(spans, spans[1:]):
                assert hi == lo2
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
    assert kad.shard_range(10, 3, 2) == (0, 0)  # rank out of range: empty


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def pack(rows, maxc, cap):
    """[maxc lengths][maxc flags][maxc x cap vertices], int32, absent rows -1."""
    blk = np.zeros(2 * maxc + maxc * cap, np.int32)
    blk[:maxc] = -1
    c = rows["D"].size
    blk[:c] = np.maximum(rows["D"] - 1, 0)
    blk[maxc:maxc + c] = rows["overflow"]
    blk[2 * maxc:2 * maxc + c * cap] = rows["paths"].reshape(-1)
    return blk.tobytes()


def fold(blob, world, maxc, cap, into):
    blocks = np.frombuffer(blob, np.int32).reshape(world, 2 * maxc + maxc * cap)
    ovf = 0
    for b in blocks:
        lens, flags, paths = b[:maxc], b[maxc:2 * maxc], b[2 * maxc:].reshape(maxc, cap)
        for j in range(maxc):
            if lens[j] < 0:
                continue
            ovf += int(flags[j])
            np.add.at(into, paths[j, :lens[j]], 1)
    return ovf


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    import oracle as O
    from paper_1903_09422_gb300 import gen, kad
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        g = gen.rmat(10, 8, seed=3)
        eps, delta, seed, N = 0.06, 0.1, 9, 250
        omega = O.omega(O.vd_bound(g), eps, delta)
        tau0 = O.calib_samples(omega, N, 100)
        cap = O.path_cap(g)
        maxc = -(-max(tau0, N) // world)
        allgather = kad.torch_allgather()
        # calibration
        lo, hi = kad.shard_range(tau0, rank, world)
        rows = O.samples(g, seed, lo, hi - lo, domain=1, cap=cap)
        c0 = np.zeros(g.n, np.int64)
        fold(allgather(pack(rows, maxc, cap)), world, maxc, cap, c0)
        hist = np.bincount(c0, minlength=tau0 + 1)
        ts = O.tau_star(hist, eps, delta, omega)
        L = np.array([O.L_of(c / tau0, ts, eps, omega) for c in range(tau0 + 1)])
        # adaptive epochs until the stop rule holds
        cnt = np.zeros(g.n, np.int64)
        ovf, k = 0, 0
        while True:
            lo, hi = kad.shard_range(N, rank, world)
            rows = O.samples(g, seed, k * N + lo, hi - lo, domain=0, cap=cap)
            ovf += fold(allgather(pack(rows, maxc, cap)), world, maxc, cap, cnt)
            k += 1
            tau = k * N
            if tau >= omega:
                break
            pairs = np.unique(np.stack([cnt, c0]), axis=1)
            if all(O.f(int(c), L[j], tau, omega) <= eps and O.g(int(c), L[j], tau, omega) <= eps for c, j in pairs.T):
                break
        q.put((rank, dict(c0=c0, cnt=cnt, tau=tau, epochs=k, ovf=ovf, L=L, ts=ts)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_fold_and_stop_like_one():
    import oracle as O
    from paper_1903_09422_gb300 import gen
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = O.kadabra(gen.rmat(10, 8, seed=3), 0.06, 0.1, 9, epoch=250)
    for r in (0, 1):
        o = out[r]
        assert (o["tau"], o["epochs"], o["ovf"]) == (ref["tau"], ref["epochs"], ref["overflow_samples"])
        np.testing.assert_array_equal(o["c0"], ref["c0"])
        np.testing.assert_array_equal(o["cnt"], ref["counts"])
        np.testing.assert_array_equal(o["L"], ref["L"])
        assert o["ts"] == ref["tau_star"]
