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


# ---------------------------------------------------------------------------------------
# The grid sizes of the other two configurations: 128^3 ABC (eps 0.005, dt 5e-4) and 256^3
# Kolmogorov sin(8y) (eps 0.002, dt 2.5e-4).  The fine kernel tiles them differently
# from 64^3 (8 and 4 grid rows per CTA pass); a few steps are compared point for point.
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_fine_steps_at_128(gpu, prec):
    bd, torch = gpu
    from test_gpu_parity import dev
    w = pi.Workload("abc128", 128, pi.Flow("abc"), 0.005, 1.0, 8, 5e-4, m_cap=8, f_seed=7)
    s = bd.Parareal.from_workload(w, precision=prec)
    op = O.make_operator(w)
    u = np.stack([pi.initial_state(128, seed=50 + b) for b in range(2)])
    s.set_initial(u[0], w.f())
    out, snap = s.op_fine(dev(torch, u), 3, 3, 2)
    out, snap = out.cpu().numpy(), snap.cpu().numpy()
    tol = 1e-12 if prec == 0 else 1e-5
    for b in range(2):
        ue, W = O.fine_propagate(op, u[b], 0.0, 3, s.dt_eff, 3, 2, tol=1e-14)
        assert rel(out[b], ue) < tol
        assert rel(snap[b, 1], W[:, 1]) < tol
    s.close()


@pytest.mark.parametrize("prec", [1, 0], ids=["fp32", "fp64"])
def test_fine_steps_at_256(gpu, prec):
    # the 256^3 case: Kolmogorov sin(8y) plus the seeded divergence-free perturbation of
    # amplitude 0.05 (stored per point, FINE_MODE_IMPLICIT_PERT)
    bd, torch = gpu
    from test_gpu_parity import dev
    w = pi.Workload("kol256", 256, pi.Flow("kolmogorov", k=8, pert_seed=4, pert_amp=0.05), 0.002, 1.0,
                    8, 2.5e-4, n_snap=16, m_cap=8)
    s = bd.Parareal.from_workload(w, precision=prec)
    op = O.make_operator(w)
    u = pi.initial_state(256, seed=60)[None]
    s.set_initial(u[0], None)
    out, _ = s.op_fine(dev(torch, u), 2)
    out = out.cpu().numpy()
    ue, _ = O.fine_propagate(op, u[0], 0.0, 2, s.dt_eff, tol=1e-14)
    assert rel(out[0], ue) < (1e-12 if prec == 0 else 1e-5)
    s.close()


def test_parareal_iteration_at_128(gpu):
    # iteration 0 and one iteration of the method on a 128^3 ABC problem (N = 4, two fine
    # steps per subinterval), within the method's own rounding envelope
    bd, torch = gpu
    from test_gpu_parity import oracle_envelope
    w = pi.Workload("abc128_short", 128, pi.Flow("abc"), 0.005, 0.004, 4, 5e-4, n_snap=0,
                    m_cap=4)
    prm = O.derive_params(w)
    hist, env = oracle_envelope(w, prm, 1, 1e-13)
    s = bd.Parareal.from_workload(w)
    s.set_initial(w.u0(), w.f())
    s.iteration0()
    U0 = s.interfaces()
    s.iterate(1)
    U1 = s.interfaces()
    for k, U in ((0, U0), (1, U1)):
        for n in range(w.n_sub + 1):
            e = rel(U[n], hist["U"][k][n])
            assert e < max(1e-12, 10 * env[k][n]), (k, n, e, env[k][n])
    s.close()
