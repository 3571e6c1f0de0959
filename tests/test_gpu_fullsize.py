"""Full-size parity on the 64^3 Kolmogorov workload (64 subintervals x 157 fine steps, the
launch configuration bench.py times), on outputs the oracle can recompute one at a time:
sampled fine end states and snapshots from the GPU's own U^0_n, the level-1 POD of the
GPU's own snapshots, and one augmented coarse update from the GPU's own basis and states.
"""
import numpy as np
import pytest

import oracle as O
import pr_inputs as pi
from test_gpu_parity import davis_kahan_tol, rel, span_dist

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", params=[0, 1], ids=["fp64", "fp32"])
def kol64(request, gpu):
    bd, torch = gpu
    w = pi.KOL_64
    s = bd.Parareal.from_workload(w, precision=request.param)
    s.set_initial(w.u0(), w.f())
    s.iteration0()
    U0 = s.interfaces()
    s.fine_sweep(1)
    s.pod_update(1)
    s.coarse_sweep(1)
    s.check(1)
    U1 = s.interfaces()
    yield request.param, w, s, U0, U1
    s.close()


def test_fine_end_states_and_snapshots(kol64):
    prec, w, s, U0, U1 = kol64
    prm = O.derive_params(w)
    op = O.make_operator(w)
    tol = 1e-12 if prec == 0 else 1e-5
    for n in ((0, 63) if prec == 0 else (37,)):
        Fo, Wo = O.fine_propagate(op, U0[n], prm.T0 + n * prm.DeltaT, prm.S, prm.dt, prm.dM,
                                  prm.n_s, tol=prm.lin_tol)
        assert rel(s.fine_end(n), Fo) < tol, n
        Wg = s.snapshots(n)
        for j in (0, prm.n_s // 2, prm.n_s - 1):
            assert rel(Wg[j], Wo[:, j]) < tol, (n, j)


def test_level1_pod_of_gpu_snapshots(kol64):
    prec, w, s, U0, U1 = kol64
    prm = O.derive_params(w)
    for n in (5, 50):
        Wg = s.snapshots(n).T                      # the GPU's own FP64 snapshots
        Ro, mo, lam = O.pod_mode(Wg, prm.gamma2, prm.m_cap, 1e-13)
        Rg = s.basis(1, n).T.astype(np.float64)
        assert Rg.shape[1] == mo, (n, Rg.shape, mo)
        tol = davis_kahan_tol(lam, mo, 1.1e-16)
        assert span_dist(Rg, Ro) < tol, (n, span_dist(Rg, Ro), tol)


def test_coarse_update_from_gpu_basis(kol64):
    prec, w, s, U0, U1 = kol64
    prm = O.derive_params(w)
    op = O.make_operator(w)
    n = 40
    R = s.basis(2, n).T.astype(np.float64)
    F = s.fine_end(n)

    def update(U, Up):
        V, _ = O.augment(R, U)
        t_n = prm.T0 + n * prm.DeltaT
        g1, _ = O.coarse_propagate(op, V, U, t_n, prm.Lc, prm.dT)
        g2, _ = O.coarse_propagate(op, V, Up, t_n, prm.Lc, prm.dT)
        return g1 + F.reshape(-1) - g2

    ref = update(U1[n], U0[n])
    pert = update(U1[n] * (1 + 1e-13 * np.random.default_rng(3).standard_normal(U1[n].shape)), U0[n])
    env = rel(pert, ref)
    e = rel(U1[n + 1], ref)
    assert e < max(1e-12, 10 * env), (e, env)
