"""Pins of the oracle's stopping condition (Appendix B: f, g; Section 2.3: omega,
delta_L/delta_U with sum <= delta) and of the full run's estimator against exact
betweenness (Section 2.2 definition; the (eps, delta) guarantee of Section 2.3)."""
import math
from collections import deque

import numpy as np
import pytest

import oracle as O
from paper_1903_09422_gb300 import gen

sympy = pytest.importorskip("sympy")


def f_exact(c, L, tau, omega, digits=60):
    """Appendix B's f evaluated in exact rational arithmetic plus a 60-digit sqrt."""
    S = sympy
    b = S.Rational(c, tau)
    Lr = S.Rational(L)  # exact value of the binary64 input
    a = S.Rational(1, 3) - S.Rational(omega, tau)
    return (Lr / tau * (a + S.sqrt(a * a + 2 * b * omega / Lr))).evalf(digits)


def g_exact(c, L, tau, omega, digits=60):
    S = sympy
    b = S.Rational(c, tau)
    Lr = S.Rational(L)
    a = S.Rational(1, 3) + S.Rational(omega, tau)
    return (Lr / tau * (a + S.sqrt(a * a + 2 * b * omega / Lr))).evalf(digits)


@pytest.mark.parametrize("c,L,tau,omega", [
    (0, 17.25, 1000, 1200), (37, 12.5, 4000, 35000), (950, 3.0, 1000, 1200), (5, 20.0, 30000, 35000),
    (12345, 9.75, 40000, 35000)])
def test_f_g_match_appendix_b_closed_form(c, L, tau, omega):
    f = O.f(c, L, tau, omega)
    g = O.g(c, L, tau, omega)
    fe, ge = f_exact(c, L, tau, omega), g_exact(c, L, tau, omega)
    assert abs(g - float(ge)) <= 4e-16 * abs(float(ge))
    if abs(float(fe)) > 1e-300:
        # f = (L/T)(a + sqrt(a^2 + x)) cancels when a < 0; allow a few ulps of |a|.
        tol = 8e-16 * (abs(float(fe)) + L / tau * abs(1 / 3 - omega / tau))
        assert abs(f - float(fe)) <= tol
    else:
        assert abs(f) <= 1e-15 * L / tau


def test_f_is_zero_at_b0_when_omega_over_tau_exceeds_a_third():
    # a = 1/3 - omega/tau < 0 and b = 0 give f = (L/T)(a + |a|) = 0.
    for tau, omega in [(1000, 1200), (1000, 400), (2000, 100000)]:
        assert O.f(0, 15.0, tau, omega) == 0.0


def test_monotone_in_b_and_tau():
    # Appendix B: f and g grow with b~; g decreases with tau.
    om = 35000
    for L in (5.0, 15.0, 25.0):
        fs = [O.f(c, L, 10000, om) for c in range(0, 5000, 37)]
        gs = [O.g(c, L, 10000, om) for c in range(0, 5000, 37)]
        assert all(x <= y for x, y in zip(fs, fs[1:]))
        assert all(x <= y for x, y in zip(gs, gs[1:]))
        assert all(f <= g for f, g in zip(fs, gs))
        # g at fixed b~ (c/tau fixed) decreases with tau
        g_tau = [O.g(tau // 10, L, tau, om) for tau in range(1000, 100000, 1000)]
        assert all(x >= y for x, y in zip(g_tau, g_tau[1:]))


def test_omega_hand_values():
    # omega = ceil((0.5/eps^2)(floor(log2(max(VD-2,1))) + 1 + ln(2/delta)))
    assert O.omega(9, 0.05, 0.1) == math.ceil(200 * (2 + 1 + math.log(20)))  # = 1200
    assert O.omega(9, 0.05, 0.1) == 1200
    assert O.omega(3, 0.1, 0.1) == math.ceil(50 * (0 + 1 + math.log(20)))
    assert O.omega(1, 0.1, 0.1) == O.omega(3, 0.1, 0.1)
    assert O.omega(34, 0.01, 0.1) == math.ceil(5000 * (5 + 1 + math.log(20)))


def test_calib_samples_rule():
    assert O.calib_samples(1200, 1000, 100) == 1000
    assert O.calib_samples(35000, 1000, 100) == 1000
    assert O.calib_samples(150000, 1000, 100) == 2000
    assert O.calib_samples(5, 1000, 100) == 1000
    assert O.calib_samples(250001, 500, 100) == 2500 + 500


def test_L_solves_g_equals_eps_at_tau_star():
    # L(b0, tau*) is the log(1/delta) that makes g(b0, e^-L, omega, tau*) = eps.
    S = sympy
    for b0, ts, eps, om in [(0.0, 9000.5, 0.01, 35000), (0.02, 15000.25, 0.01, 35000), (0.3, 800.0, 0.05, 1200)]:
        L = O.L_of(b0, ts, eps, om)
        Lr, T = S.Rational(L), S.Rational(ts)
        a = S.Rational(1, 3) + om / T
        g = (Lr / T * (a + S.sqrt(a * a + 2 * S.Rational(b0) * om / Lr))).evalf(40)
        assert abs(float(g) - eps) <= 1e-13 * eps


def test_tau_star_bisection_is_tight():
    hist = np.zeros(1001, np.uint64)
    hist[0], hist[1], hist[3], hist[40] = 3000, 500, 20, 1
    eps, delta, om = 0.05, 0.1, 1200
    ts = O.tau_star(hist, eps, delta, om)

    def mass(t):
        return sum(int(h) * 2 * math.exp(-O.L_of(c / 1000, t, eps, om)) for c, h in enumerate(hist) if h)

    assert mass(ts) <= delta / 2
    assert mass(ts * (1 - 1e-9)) > delta / 2


# ----------------------------------------------------------------- estimator


def brandes_ordered(g):
    """Brandes' algorithm (J. Math. Sociol. 2001), unweighted; betweenness over
    ordered pairs s != t, i.e. b(v) = sum_{s != t != v} sigma_st(v)/sigma_st."""
    n = g.n
    adj = [g.col[g.row_ptr[v]:g.row_ptr[v + 1]] for v in range(n)]
    bc = np.zeros(n)
    for s in range(n):
        S, P = [], [[] for _ in range(n)]
        sigma = np.zeros(n)
        sigma[s] = 1
        d = [-1] * n
        d[s] = 0
        q = deque([s])
        while q:
            v = q.popleft()
            S.append(v)
            for w in adj[v]:
                if d[w] < 0:
                    d[w] = d[v] + 1
                    q.append(w)
                if d[w] == d[v] + 1:
                    sigma[w] += sigma[v]
                    P[w].append(v)
        delta = np.zeros(n)
        while S:
            w = S.pop()
            for v in P[w]:
                delta[v] += sigma[v] / sigma[w] * (1 + delta[w])
            if w != s:
                bc[w] += delta[w]
    return bc


def test_brandes_matches_networkx():
    nx = pytest.importorskip("networkx")
    g = gen.er(60, 0.1, seed=4)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    G.add_edges_from((v, int(w)) for v in range(g.n) for w in g.col[g.row_ptr[v]:g.row_ptr[v + 1]])
    ref = nx.betweenness_centrality(G, normalized=False)  # unordered pairs
    bc = brandes_ordered(g)
    assert np.allclose(bc, [2 * ref[v] for v in range(g.n)])


def test_path_and_star_closed_forms_via_full_run():
    # Path P_n: b(i) = 2 i (n-1-i) over ordered pairs.  Star: centre (n-1)(n-2).
    n = 21
    r = O.kadabra(gen.path_graph(n), 0.05, 0.1, seed=3)
    exact = np.array([2 * i * (n - 1 - i) for i in range(n)]) / (n * (n - 1))
    assert np.max(np.abs(r["bc"] - exact)) <= 0.05
    assert r["bc"][0] == 0 and r["bc"][-1] == 0
    r = O.kadabra(gen.star_graph(n), 0.05, 0.1, seed=3)
    assert abs(r["bc"][0] - (n - 2) / n) <= 0.05
    assert (r["bc"][1:] == 0).all()


def test_eps_delta_guarantee_against_brandes():
    # Section 2.3: with probability >= 1 - delta every |b~(v) - b(v)/(n(n-1))| <= eps.
    graphs = [gen.er(n, 0.1, seed=sd) for n, sd in ((40, 1), (80, 2), (150, 3))]
    runs, fails = 0, 0
    for g in graphs:
        exact = brandes_ordered(g) / (g.n * (g.n - 1))
        for seed in range(1, 121):
            for eps in (0.05, 0.1):
                r = O.kadabra(g, eps, 0.1, seed=seed)
                assert r["counts"].sum() > 0
                runs += 1
                fails += int(np.max(np.abs(r["bc"] - exact)) > eps)
    # one-sided binomial bound: far below delta * runs in practice
    assert fails <= 0.1 * runs
    assert runs == 720


def test_full_run_invariants():
    g = gen.rmat(12, 8, seed=1)
    r = O.kadabra(g, 0.05, 0.1, seed=1)
    assert r["tau"] % 1000 == 0 and r["epochs"] == r["tau"] // 1000
    assert (r["counts"] <= r["tau"]).all()
    assert r["counts"].sum() == r["counters"]["increments"]
    assert r["tau"] <= ((r["omega"] + 999) // 1000) * 1000
    np.testing.assert_array_equal(r["bc"], r["counts"] / r["tau"])
    # truncated run: same prefix of samples, so counts of epoch 1 agree
    r1 = O.kadabra(g, 0.05, 0.1, seed=1, max_epochs=1)
    assert r1["tau"] == 1000
