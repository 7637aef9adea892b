"""The sharded run (kad_run_sharded): each epoch's sample indices split among
ranks, every rank folding all ranks' path rows and taking the same stop
decision (Section 6's distributed reduction, with Appendix D.2's fixed
sample-to-epoch assignment).

One GPU is available, so several ranks are emulated by host threads, each with
its own graph handle and stream on the same device.  The ranks wait for each
other only on the host, inside the allgather; no kernel waits for another.
Every rank's counts, tau, epochs, calibration counts and L table must equal the
single-GPU kad_run's, and the oracle's, bit for bit.
"""
import threading

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


class ThreadAllgather:
    """An allgather among `world` host threads: each deposits its bytes, waits
    for the others, and takes all of them in rank order."""

    def __init__(self, world):
        self.world = world
        self.slots = [None] * world
        self.barrier = threading.Barrier(world, timeout=600)

    def for_rank(self, r):
        def fn(payload):
            self.slots[r] = payload
            self.barrier.wait()
            out = b"".join(self.slots)
            self.barrier.wait()  # nobody overwrites a slot before all have read
            return out
        return fn


def run_ranks(kad, g, world, eps, delta, seed, **opt):
    import torch
    ag = ThreadAllgather(world)
    results, errors = [None] * world, []

    def body(r):
        try:
            torch.cuda.set_device(0)
            stream = torch.cuda.Stream()
            with kad.Graph.from_csr(g) as G:
                results[r] = G.run_sharded(eps, delta, seed, r, world, ag.for_rank(r), stream=stream, c0=True,
                                           ltab=True, **opt)
        except Exception as ex:  # reported below
            errors.append(ex)
            ag.barrier.abort()

    threads = [threading.Thread(target=body, args=(r,)) for r in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=900)
    assert not errors, errors
    return results


def same_as(r, ref, cut=False):
    assert (r["tau"], r["epochs"], r["omega"], r["calib_samples"]) == \
        (ref["tau"], ref["epochs"], ref["omega"], ref["calib_samples"])
    np.testing.assert_array_equal(r["counts"], ref["counts"])
    np.testing.assert_array_equal(r["c0"], ref["c0"])
    np.testing.assert_array_equal(r["L"], ref["L"])
    np.testing.assert_array_equal(r["bc"], ref["bc"])
    assert r["tau_star"] == ref["tau_star"]
    assert r["overflow_samples"] == ref["overflow_samples"]
    # 2: the run was cut by max_epochs (the oracle's binding reports a bool)
    assert r["stopped_by_omega"] == (2 if cut else int(ref["stopped_by_omega"]))


@pytest.mark.parametrize("world", [1, 2, 3])
def test_sharded_run_equals_single_gpu_run(kad, world):
    g = gen.rmat(12, 8, seed=1)
    eps, delta, seed = 0.03, 0.1, 11
    ref = O.kadabra(g, eps, delta, seed)
    with kad.Graph.from_csr(g) as G:
        single = G.run(eps, delta, seed, c0=True, ltab=True)
    same_as(single, ref)
    for r in run_ranks(kad, g, world, eps, delta, seed):
        same_as(r, ref)


def test_sharded_run_ragged_chunks_and_kernels(kad):
    # an epoch size that 3 ranks cannot split evenly, a disconnected graph, the
    # warp-per-sample kernel on one configuration, a hub graph whose meeting
    # rounds take the pairwise test at every chance, and a diamond chain whose
    # path counts saturate (overflowed samples are counted alike)
    cases = [(gen.grid(40, seed=3), 0.05, 3, dict(epoch_size=250)),
             (GRAPHS_MIXED(), 0.05, 4, {}),
             (gen.rmat(11, 8, seed=2), 0.04, 5, dict(samples_per_block=8)),
             (gen.rmat(12, 16, seed=4), 0.04, 7, dict(pair_cost=1)),
             (diamond(70), 0.05, 6, {})]
    for g, eps, seed, opt in cases:
        ref = O.kadabra(g, eps, 0.1, seed, epoch=opt.get("epoch_size", 1000))
        for r in run_ranks(kad, g, 3, eps, 0.1, seed, **opt):
            same_as(r, ref)
            assert r["pair_cost_used"] == opt.get("pair_cost", 8)


def test_sharded_truncated_run_at_full_size(kad):
    # the benchmarked R-MAT scale-20 query split between two ranks, cut after
    # three epochs on both sides
    g = gen.workload_graph("rmat20")
    w = gen.WORKLOADS["rmat20"]
    ref = O.kadabra(g, w["eps"], w["delta"], w["seed"], max_epochs=3)
    for r in run_ranks(kad, g, 2, w["eps"], w["delta"], w["seed"], max_epochs=3):
        same_as(r, ref, cut=True)


def test_sharded_run_rejects_bad_arguments(kad):
    g = gen.rmat(10, 8, seed=1)
    with kad.Graph.from_csr(g) as G:
        with pytest.raises(RuntimeError):
            G.run_sharded(0.05, 0.1, 1, 2, 2, lambda b: b)  # rank out of range
        with pytest.raises(RuntimeError):
            G.run_sharded(0.05, 0.1, 1, 0, 1, lambda b: b, flags=kad.KAD_RUN_COMPLETION_ORDER)
        with pytest.raises(RuntimeError):
            G.run_sharded(0.05, 0.1, 1, 0, 1, lambda b: b, pair_cost=-1)
        with pytest.raises(RuntimeError):
            G.run_sharded(0.05, 0.1, 1, 0, 1, lambda b: None)  # a failing collective


def GRAPHS_MIXED():
    from test_gpu_parity import mixed_components
    return mixed_components()


def diamond(k):
    from test_gpu_parity import diamond_chain
    return diamond_chain(k)
