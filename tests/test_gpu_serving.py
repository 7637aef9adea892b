"""The query server: queries that run concurrently on the device (continuous
batching) give exactly the results each gives alone."""
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


def mixed_graphs():
    return [gen.rmat(12, 8, seed=1), gen.rmat(11, 16, seed=2), gen.grid(40, seed=3), gen.er(150, 0.1, seed=4),
            gen.hyperbolic(6000, seed=5), gen.path_graph(60)]


def test_results_alone_equal_results_in_the_mix(kad):
    graphs = mixed_graphs()
    queries = [(i % len(graphs), (0.05, 0.03, 0.02)[i % 3], 100 + i) for i in range(30)]
    alone = {}
    for gi, g in enumerate(graphs):
        with kad.Graph.from_csr(g) as G:
            for qi, (qg, eps, seed) in enumerate(queries):
                if qg == gi:
                    alone[qi] = G.run(eps, 0.1, seed)
    with kad.Server(workers=6) as S:
        gids = [S.add_graph(g) for g in graphs]
        tickets = [S.submit(gids[qg], eps, 0.1, seed) for qg, eps, seed in queries]
        mixed = [S.wait(t) for t in tickets]
    for qi, r in enumerate(mixed):
        a = alone[qi]
        assert (r["tau"], r["epochs"], r["omega"]) == (a["tau"], a["epochs"], a["omega"])
        np.testing.assert_array_equal(r["bc"], a["bc"])
        assert r["latency_ms"] >= r["queue_ms"] >= 0
    # and against the oracle for a few of them
    for qi in (0, 3, 5):
        qg, eps, seed = queries[qi]
        ref = O.kadabra(graphs[qg], eps, 0.1, seed)
        np.testing.assert_array_equal(mixed[qi]["bc"], ref["bc"])


def test_scheduling_policy_does_not_change_results(kad):
    graphs = mixed_graphs()[:4]
    queries = [(i % 4, (0.05, 0.03)[i % 2], 300 + i) for i in range(16)]
    out = {}
    for policy in (0, 1):
        with kad.Server(workers=3, policy=policy) as S:
            gids = [S.add_graph(g) for g in graphs]
            tickets = [S.submit(gids[qg], eps, 0.1, seed) for qg, eps, seed in queries]
            out[policy] = [S.wait(t) for t in tickets]
    for a, b in zip(out[0], out[1]):
        assert a["tau"] == b["tau"]
        np.testing.assert_array_equal(a["bc"], b["bc"])


def test_admission_by_footprint_still_answers_everything(kad):
    graphs = mixed_graphs()[:3]
    with kad.Server(workers=4, hbm_budget=1) as S:  # every query exceeds the budget: one at a time
        gids = [S.add_graph(g) for g in graphs]
        tickets = [S.submit(gids[i % 3], 0.05, 0.1, 7 + i) for i in range(9)]
        res = [S.wait(t) for t in tickets]
    for i, r in enumerate(res):
        ref = O.kadabra(graphs[i % 3], 0.05, 0.1, 7 + i)
        assert r["tau"] == ref["tau"]
        np.testing.assert_array_equal(r["bc"], ref["bc"])


def test_server_frees_with_queued_queries(kad):
    S = kad.Server(workers=2)
    gid = S.add_graph(gen.rmat(12, 8, seed=1))
    for i in range(20):
        S.submit(gid, 0.02, 0.1, i)
    S.close()  # queued queries are cancelled; running ones finish first


def test_server_rejects_bad_queries(kad):
    with kad.Server(workers=1) as S:
        gid = S.add_graph(gen.rmat(10, 8, seed=1))
        with pytest.raises(kad.KadError):
            S.submit(gid + 5, 0.05, 0.1, 1)
        with pytest.raises(kad.KadError):
            S.submit(gid, 1.5, 0.1, 1)
        t = S.submit(gid, 0.05, 0.1, 1)
        assert S.wait(t)["tau"] > 0


def test_serving_stream_graphs_against_the_oracle(kad):
    # graphs of the serving stream itself (the bench's recipe: R-MAT, grid with
    # shortcuts and hyperbolic graphs of 10^4..10^6 vertices), queried
    # concurrently through the server at the stream's accuracies: every result
    # equals the oracle's full run, bit for bit
    import bench
    specs = {i: (i, k, n) for i, k, n in bench.serve_specs(64)}
    picks = [6, 5, 16, 36, 8, 10]  # R-MAT, hyperbolic, grid at ~1.1e4 and ~1e5 vertices
    graphs = [bench._serve_graph(specs[i]) for i in picks]
    queries = [(j, (0.05, 0.02, 0.01)[j % 3], 500 + j) for j in range(len(picks))]
    queries += [(j, 0.05, 600 + j) for j in range(len(picks))]
    with kad.Server(workers=4) as S:
        gids = [S.add_graph(g, trusted=True) for g in graphs]
        res = [S.wait(t) for t in [S.submit(gids[qg], eps, 0.1, seed) for qg, eps, seed in queries]]
    for (qg, eps, seed), r in zip(queries, res):
        ref = O.kadabra(graphs[qg], eps, 0.1, seed)
        assert (r["tau"], r["epochs"], r["omega"]) == (ref["tau"], ref["epochs"], ref["omega"]), (qg, eps)
        np.testing.assert_array_equal(r["bc"], ref["bc"])
