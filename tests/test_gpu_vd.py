"""The opt-in double-sweep vertex-diameter bound (KAD_GRAPH_TIGHT_VD) on the GPU
against the oracle: the bound itself on small and full-size graphs, and full
runs whose omega comes from it (Section 2.3: omega from an upper bound on the
diameter; any vertex x gives diam <= 2 ecc(x))."""
import numpy as np
import pytest

import oracle as O
from paper_1903_09422_gb300 import gen
from test_gpu_parity import GRAPHS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kad():
    import torch
    torch.cuda.set_device(0)
    from paper_1903_09422_gb300 import build, kad as K
    build.build()
    return K


EXTRA = {
    "grid5x7": lambda: gen.grid_plain(5, 7),
    "grid5x8": lambda: gen.grid_plain(5, 8),
    "holes": lambda: gen.grid(30, p_remove=0.15, shortcut_frac=0.02, seed=4, lcc=False),
    "grid300": lambda: gen.grid(300, seed=7),
    "hyp20k": lambda: gen.hyperbolic(20000, seed=3),
    "rmat16": lambda: gen.rmat(16, 16, seed=2),
}


@pytest.mark.parametrize("name", sorted(GRAPHS) + sorted(EXTRA))
def test_tight_bound_matches_oracle(kad, name):
    g = (GRAPHS.get(name) or EXTRA[name])()
    want = O.vd_bound_tight(g)
    with kad.Graph.from_csr(g, tight_vd=True) as G:
        assert G.vd_bound == want
    with kad.Graph.from_csr(g) as G:
        assert G.vd_bound == O.vd_bound(g) >= want


@pytest.mark.parametrize("name", ["grid9x13", "grid64", "path40", "mixed_comp", "rmat12"])
def test_full_run_with_tight_bound_matches_oracle(kad, name):
    g = GRAPHS[name]()
    ref = O.kadabra(g, 0.05, 0.1, 3, tight_vd=True)
    with kad.Graph.from_csr(g, tight_vd=True) as G:
        r = G.run(0.05, 0.1, 3, c0=True, ltab=True)
    assert (r["tau"], r["epochs"], r["omega"], r["calib_samples"], r["vd_bound"]) == \
        (ref["tau"], ref["epochs"], ref["omega"], ref["calib_samples"], ref["vd"])
    np.testing.assert_array_equal(r["c0"], ref["c0"])
    np.testing.assert_array_equal(r["L"], ref["L"])
    np.testing.assert_array_equal(r["counts"], ref["counts"])


def test_tight_bound_on_full_size_workloads(kad):
    # the C2, C3 and C4 graphs: the bound and its omega
    for name in ("rmat20", "grid2048", "hyp4m"):
        g = gen.workload_graph(name)
        w = gen.WORKLOADS[name]
        want = O.vd_bound_tight(g)
        with kad.Graph.from_csr(g, tight_vd=True) as G:
            assert G.vd_bound == want, name
            r = G.run(w["eps"], w["delta"], w["seed"], max_epochs=1)
        assert r["omega"] == O.omega(want, w["eps"], w["delta"])


def test_tight_flag_is_ignored_for_directed_graphs(kad):
    g = gen.rmat_directed(11, 8, seed=2)
    with kad.Graph.from_csr(g, tight_vd=True) as G:
        assert G.vd_bound == O.vd_bound(g)
