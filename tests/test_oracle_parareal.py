"""Pins of the oracle's parareal driver (Algorithm 2, eq. (formula4)) and its parameter
derivation (no GPU)."""
import numpy as np
import pytest

import oracle as O
import pr_inputs as pi
from oracle.parareal import derive_params, steps_for


def test_parameter_derivation_of_the_paper_setup():
    # Sec. 4.1: dt = 1e-2, DeltaT = T0 = 5, dT = 0.5, delta_M = 5, N = 200 (T = 1000 after
    # the [0, T0] window): 500 fine and 10 coarse steps per subinterval, and
    # n_s = floor(T0 / (dt dM)) + 1 = 101 snapshots per window (Case I).
    w = pi.Workload("paper", 8, pi.Flow("paper_kolmogorov"), 0.5, 1000.0, 200, 1e-2)
    p = derive_params(w)
    assert (p.S, p.Lc, p.dM, p.n_s, p.n_s0) == (500, 10, 5, 101, 101)
    assert p.T0 == 5.0 and p.dT == 0.5
    assert p.gamma1 == 1.0 - 5e-6 and abs(p.gamma3 - (1.0 - 2e-8)) < 1e-17


def test_parameter_derivation_of_the_workloads():
    c1 = derive_params(pi.ABC_16)
    assert (c1.S, c1.dM, c1.n_s, c1.Lc) == (125, 5, 26, 10)
    c2 = derive_params(pi.KOL_64)
    assert (c2.S, c2.dM, c2.n_s) == (157, 5, 32)
    assert abs(c2.dt - 10.0 / 64 / 157) < 1e-18
    c3 = derive_params(pi.ABC_128)
    assert (c3.S, c3.dM, c3.n_s) == (391, 6, 64)


def test_steps_for_rounds_near_integers():
    assert steps_for(0.125, 1e-3) == 125
    assert steps_for(0.15625, 1e-3) == 157
    assert steps_for(1.0, 0.3) == 4


@pytest.fixture(scope="module")
def tiny_run():
    w = pi.tiny(n=8, n_sub=4, T=0.08, dt=2e-3, f_seed=7)
    prm = derive_params(w)
    ref = O.sequential_fine(w, prm)
    hist = O.parareal(w, prm, k_max=prm.N, reference=ref)
    return w, prm, ref, hist


def test_finite_termination(tiny_run):
    # U^k_n is the sequential fine solution for n <= k (Sec. 3.3), so k = N is exact.
    w, prm, ref, hist = tiny_run
    for k in range(1, prm.N + 1):
        U = hist["U"][k]
        for n in range(k + 1):
            assert O.rel_l2(U[n], ref[n]) < 1e-12, (k, n)
    assert max(hist["err"][prm.N]) < 1e-12


def test_interfaces_left_of_k_are_frozen(tiny_run):
    w, prm, ref, hist = tiny_run
    for k in range(1, prm.N + 1):
        for n in range(k):
            assert np.array_equal(hist["U"][k][n], hist["U"][k - 1][n])
        assert np.array_equal(hist["U"][k][k], hist["F"][k - 1][k - 1])


def test_error_decreases_over_iterations(tiny_run):
    w, prm, ref, hist = tiny_run
    errs = [max(e) for e in hist["err"]]
    for a, b in zip(errs[:-1], errs[1:]):
        assert b <= a * 1.0001


def test_iteration0_is_coarse_propagation_in_V0(tiny_run):
    w, prm, ref, hist = tiny_run
    V0 = hist["V0"]
    U0 = hist["U"][0]
    assert np.array_equal(U0[0], ref[0])      # U^0_0 = u_hat0 = F(0, T0, u0)
    for n in range(1, prm.N + 1):             # U^0_n, n >= 1, lie in span V0
        u = U0[n].reshape(-1)
        assert np.linalg.norm(u - V0 @ (V0.T @ u)) < 1e-12 * np.linalg.norm(u)


def test_update_formula_with_augmented_space():
    # One iteration by hand from the building blocks equals the driver's U^1.
    w = pi.tiny(n=8, n_sub=3, T=0.06, dt=2e-3, m_l=1, p=1)
    prm = derive_params(w)
    op = O.make_operator(w)
    hist = O.parareal(w, prm, k_max=1)
    U0, V0 = hist["U"][0], hist["V0"]
    F, R1 = {}, {}
    for n in range(prm.N):
        F[n], Wn = O.fine_propagate(op, U0[n], prm.T0 + n * prm.DeltaT, prm.S, prm.dt,
                                    prm.dM, prm.n_s, tol=prm.lin_tol)
        R1[n], _, _ = O.pod_mode(Wn, prm.gamma2, prm.m_cap)
    U = [U0[0], F[0]]
    for n in range(1, prm.N):
        W = np.concatenate([R1[n - 1], R1[n], V0], axis=1)
        R2, _, _ = O.pod_mode(W, prm.gamma3, prm.m_cap)
        V, _ = O.augment(R2, U[n])
        t = prm.T0 + n * prm.DeltaT
        a, _ = O.coarse_propagate(op, V, U[n], t, prm.Lc, prm.dT)
        b, _ = O.coarse_propagate(op, V, U0[n], t, prm.Lc, prm.dT)
        U.append((a + F[n].reshape(-1) - b).reshape(U0[0].shape))
    for n in range(prm.N + 1):
        assert np.array_equal(U[n], hist["U"][1][n])


def test_variants_converge_and_11_is_at_least_as_fast_as_00():
    # Sec. 4.1: more neighbouring data in the coarse space speeds convergence up.
    errs = {}
    for ml, p in ((0, 0), (1, 1)):
        w = pi.tiny(n=8, n_sub=5, T=0.25, dt=5e-3, m_l=ml, p=p, m_cap=0)
        prm = derive_params(w)
        ref = O.sequential_fine(w, prm)
        h = O.parareal(w, prm, k_max=2, reference=ref, record=False)
        errs[(ml, p)] = max(h["err"][-1])
    assert errs[(1, 1)] <= errs[(0, 0)] * 1.0001


def test_exact_coarse_space_converges_in_one_iteration(monkeypatch):
    # With G = F (complete coarse space V = I and dT = dt) the update of eq. (formula4)
    # gives U^1_{n+1} = F(U^1_n) + F(U^0_n) - F(U^0_n): the sequential fine solution after
    # one iteration whatever U^0 was.  Iteration 0 gets a poor 3-dimensional V0 so
    # that U^0 is far from exact; a dropped or mis-signed term in the update fails here.
    import sys
    P = sys.modules["oracle.parareal"]
    w = pi.tiny(n=5, n_sub=4, T=0.04, dt=2e-3, f_seed=3)
    prm = derive_params(w, dT=2e-3)
    assert prm.Lc == prm.S
    Ng = w.Ng
    eye = np.eye(Ng)
    poor = np.linalg.qr(np.random.default_rng(0).standard_normal((Ng, 3)))[0]

    def fake_pod(W, gamma, cap=0, tau=1e-13, reorth=True):
        if gamma == prm.gamma1 and W.shape[1] == prm.n_s0 and fake_pod.first:
            fake_pod.first = False
            return poor, 3, None
        return eye, Ng, None
    fake_pod.first = True
    monkeypatch.setattr(P, "pod_mode", fake_pod)
    monkeypatch.setattr(P, "augment", lambda R, U, tol=0: (R, False))
    ref = O.sequential_fine(w, prm)
    hist = O.parareal(w, prm, k_max=1, reference=ref)
    assert max(hist["err"][0]) > 1e-3
    assert max(hist["err"][1]) < 1e-12


def test_parareal_I_reaches_the_sequential_solution_at_k_equals_N():
    # plain parareal with the fixed coarse space V0 (Sec. 4, "Parareal-I"): after k = N
    # iterations every U^N_n is the sequential fine solution, whatever G is
    w = pi.tiny(n=6, n_sub=4, T=0.04, dt=2e-3, f_seed=3)
    prm = derive_params(w, method="parareal_I")
    ref = O.sequential_fine(w, prm)
    hist = O.parareal(w, prm, reference=ref)
    assert hist["k"] == w.n_sub
    assert max(hist["err"][0]) > 1e-4
    assert max(hist["err"][-1]) < 1e-13


def test_parareal_I_with_an_exact_coarse_propagator_converges_in_one_iteration(monkeypatch):
    # V0 = I and dT = dt make G = F: U^1 is exact after one iteration.  A poor V0 would
    # not; the coarse space of every later iteration must be V0 itself.
    import sys
    P = sys.modules["oracle.parareal"]
    w = pi.tiny(n=5, n_sub=4, T=0.04, dt=2e-3, f_seed=3)
    prm = derive_params(w, dT=2e-3, method="parareal_I")
    Ng = w.Ng
    monkeypatch.setattr(P, "pod_mode", lambda W, gamma, cap=0, tau=1e-13, reorth=True:
                        (np.eye(Ng), Ng, None))
    ref = O.sequential_fine(w, prm)
    hist = O.parareal(w, prm, k_max=1, reference=ref)
    assert max(hist["err"][1]) < 1e-12


def test_parareal_I_differs_from_the_adaptive_method_and_keeps_v0():
    # the comparator must not build level-1/2 bases (its iterates use V0 only): with a
    # poor V0 its first iterate is worse than the adaptive one on the same inputs
    w = pi.tiny(n=6, n_sub=4, T=0.04, dt=2e-3, f_seed=3, m_cap=2)
    ref = O.sequential_fine(w, derive_params(w))
    ha = O.parareal(w, derive_params(w), k_max=1, reference=ref)
    hp = O.parareal(w, derive_params(w, method="parareal_I"), k_max=1, reference=ref)
    assert hp["m1"][0] == {} and hp["m2"][0] == {}
    assert max(hp["err"][1]) > 2 * max(ha["err"][1])
