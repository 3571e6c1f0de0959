"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same seeded
inputs.  Tolerances (relative L2 per grid function): FP64 mode 1e-12, FP32 mode 1e-5.
"""
import numpy as np
import pytest

import oracle as O
import pr_inputs as pi
from oracle.discretisation import Operator

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-5


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def span_dist(A, B):
    """|| P_A - P_B ||_2 for orthonormal column blocks (N x m)."""
    if A.shape[1] != B.shape[1]:
        return np.inf
    M = A.T @ B
    s = np.linalg.svd(M, compute_uv=False)
    return float(np.sqrt(max(0.0, 1.0 - min(s) ** 2)))


def solver(bd, w, precision=0, **kw):
    return bd.Parareal.from_workload(w, precision=precision, **kw)


# ---------------------------------------------------------------------- operator
@pytest.mark.parametrize("flow", [pi.Flow("abc", A=1.0, B=0.7, C=1.3), pi.Flow("kolmogorov", k=3),
                                  pi.Flow("const", b0=0.3, b1=-0.8, b2=1.1)])
@pytest.mark.parametrize("n", [8, 12, 16])
def test_apply_L_matches_oracle(gpu, flow, n):
    bd, torch = gpu
    w = pi.Workload("op", n, flow, 0.037, 1.0, 2, 1e-3, n_snap=8, m_cap=8)
    s = solver(bd, w)
    us = np.stack([pi.initial_state(n, seed=3), pi.forcing(n, seed=4)])
    op = Operator(O.Grid(n), flow, 0.037)
    for transpose in (False, True):
        out = s.op_apply_L(torch.tensor(us, device="cuda"), transpose=transpose).cpu().numpy()
        for i in range(2):
            ref = op.LT(us[i], 0.0) if transpose else op.L(us[i], 0.0)
            assert rel(out[i], ref) < 1e-13


# ---------------------------------------------------------------------- fine propagator
@pytest.mark.parametrize("n,B,steps,dM,nsnap", [(8, 3, 12, 4, 4), (12, 2, 9, 3, 4), (16, 5, 7, 7, 2)])
def test_fine_propagator_fp64(gpu, n, B, steps, dM, nsnap):
    bd, torch = gpu
    w = pi.Workload("fine", n, pi.Flow("abc"), 0.05, 1.0, 8, 1e-3, f_seed=5, m_cap=8)
    s = solver(bd, w)
    op = O.make_operator(w)
    u = np.stack([pi.initial_state(n, seed=10 + b) for b in range(B)])
    out, snap = s.op_fine(torch.tensor(u, device="cuda"), steps, dM, nsnap)
    out, snap = out.cpu().numpy(), snap.cpu().numpy()
    for b in range(B):
        ue, W = O.fine_propagate(op, u[b], 0.0, steps, s.dt_eff, dM, nsnap, tol=1e-14)
        assert rel(out[b], ue) < TOL64
        for j in range(nsnap):
            assert rel(snap[b, j], W[:, j]) < TOL64


def test_fine_propagator_fp32(gpu):
    bd, torch = gpu
    n, B, steps = 16, 3, 40
    w = pi.Workload("fine32", n, pi.Flow("kolmogorov", k=2), 0.02, 1.0, 8, 1e-3, f_seed=6, m_cap=8)
    s = solver(bd, w, precision=bd.PR_FP32)
    op = O.make_operator(w)
    u = np.stack([pi.initial_state(n, seed=20 + b) for b in range(B)])
    out, snap = s.op_fine(torch.tensor(u, device="cuda"), steps, 10, 5, fp32=True)
    out, snap = out.cpu().numpy(), snap.cpu().numpy()
    for b in range(B):
        ue, W = O.fine_propagate(op, u[b], 0.0, steps, s.dt_eff, 10, 5, tol=1e-14)
        assert rel(out[b], ue) < TOL32
        for j in range(5):
            assert rel(snap[b, j], W[:, j]) < TOL32


def test_fine_propagator_ragged_groups(gpu):
    # B not a multiple of the group count, explicit odd group size, non-power-of-two grid
    bd, torch = gpu
    n, B = 12, 7
    w = pi.Workload("rag", n, pi.Flow("abc"), 0.05, 1.0, 8, 1e-3, m_cap=8)
    op = O.make_operator(w)
    u = np.stack([pi.initial_state(n, seed=40 + b) for b in range(B)])
    for G in (1, 3, 7):
        s = solver(bd, w, group_ctas=G)
        out, _ = s.op_fine(torch.tensor(u, device="cuda"), 5)
        out = out.cpu().numpy()
        for b in (0, B - 1):
            ue, _ = O.fine_propagate(op, u[b], 0.0, 5, s.dt_eff, tol=1e-14)
            assert rel(out[b], ue) < TOL64


# ---------------------------------------------------------------------- POD
def _trajectory_snapshots(w, steps, dM, nsnap, seed):
    op = O.make_operator(w)
    _, W = O.fine_propagate(op, pi.initial_state(w.n, seed=seed), 0.0, steps, 2e-3, dM, nsnap,
                            tol=1e-14)
    return W


@pytest.mark.parametrize("precision", [0, 1])
def test_pod_mode_matches_oracle(gpu, precision):
    bd, torch = gpu
    n = 10
    w = pi.Workload("pod", n, pi.Flow("abc"), 0.05, 1.0, 4, 1e-3, n_snap=0, m_cap=13)
    s = solver(bd, w, precision=precision)
    rng = np.random.default_rng(0)
    Ws = [_trajectory_snapshots(w, 60, 5, 13, seed=50 + b) for b in range(2)]
    # a random matrix with a prescribed geometric spectrum
    Q1, _ = np.linalg.qr(rng.standard_normal((w.Ng, 13)))
    Q2, _ = np.linalg.qr(rng.standard_normal((13, 13)))
    Ws.append(Q1 @ np.diag(np.logspace(0, -4, 13)) @ Q2)
    Wt = np.stack([W.T for W in Ws])           # (B, n_cols, Ng)
    dt = np.float32 if precision else np.float64
    tt = torch.float32 if precision else torch.float64
    for gamma in (0.99, 0.999999):
        R, m = s.op_pod(torch.tensor(Wt.astype(dt).reshape(3, 13, n, n, n), dtype=tt, device="cuda"),
                        gamma, cap=0)
        R = R.cpu().numpy().reshape(3, -1, w.Ng)
        for b, W in enumerate(Ws):
            tau = 1e-6 if precision else 1e-13
            Ro, mo, lam = O.pod_mode(W.astype(dt).astype(np.float64), gamma, 0, tau)
            assert m[b] == mo, (b, gamma, m[b], mo)
            Rg = R[b, :m[b]].T.astype(np.float64)
            assert np.max(np.abs(Rg.T @ Rg - np.eye(m[b]))) < (1e-6 if precision else 1e-13)
            # leading modes are well separated: the spans agree
            assert span_dist(Rg, Ro) < (1e-3 if precision else 1e-8)


# ---------------------------------------------------------------------- coarse update
@pytest.mark.parametrize("m", [0, 3, 7])
def test_coarse_update_matches_oracle(gpu, m):
    bd, torch = gpu
    n = 10
    w = pi.Workload("cu", n, pi.Flow("kolmogorov", k=2), 0.03, 1.0, 4, 1e-3, m_cap=8, f_seed=3)
    s = solver(bd, w)
    op = O.make_operator(w)
    rng = np.random.default_rng(m)
    R = np.linalg.qr(rng.standard_normal((w.Ng, max(m, 1))))[0][:, :m]
    U = pi.initial_state(n, seed=7).reshape(-1)
    Up = U + 0.05 * pi.forcing(n, seed=8).reshape(-1)
    F = pi.initial_state(n, seed=9).reshape(-1)
    t = lambda a: torch.tensor(a, device="cuda")
    Rt = t(np.ascontiguousarray(R.T)) if m > 0 else t(np.zeros((1, w.Ng)))
    out = s.op_coarse_update(Rt, m, t(U), t(Up), t(F)).cpu().numpy()
    V, _ = O.augment(R, U)
    g1, _ = O.coarse_propagate(op, V, U, 0.0, s.Lc, s.DeltaT / s.Lc)
    g2, _ = O.coarse_propagate(op, V, Up, 0.0, s.Lc, s.DeltaT / s.Lc)
    ref = g1 + F - g2
    assert rel(out, ref) < TOL64


# ---------------------------------------------------------------------- whole iterations
def _run_gpu_iterations(bd, w, k_max, precision=0, **kw):
    s = solver(bd, w, precision=precision, **kw)
    s.set_initial(w.u0(), w.f())
    s.iteration0()
    Us = [s.interfaces()]
    for k in range(1, k_max + 1):
        s.iterate(k)
        Us.append(s.interfaces())
    return s, Us


@pytest.mark.parametrize("wl", ["tiny", "tiny_forced", "tiny_00"])
def test_parareal_iterates_fp64(gpu, wl):
    bd, torch = gpu
    w = {"tiny": pi.tiny(n=8, n_sub=4, T=0.08, dt=2e-3),
         "tiny_forced": pi.tiny(n=10, n_sub=5, T=0.1, dt=2e-3, f_seed=2, flow=pi.Flow("kolmogorov", k=2)),
         "tiny_00": pi.tiny(n=8, n_sub=4, T=0.08, dt=2e-3, m_l=0, p=0)}[wl]
    prm = O.derive_params(w)
    hist = O.parareal(w, prm, k_max=w.n_sub)
    s, Us = _run_gpu_iterations(bd, w, w.n_sub)
    for k in range(w.n_sub + 1):
        for n in range(w.n_sub + 1):
            assert rel(Us[k][n], hist["U"][k][n]) < TOL64, (k, n)


def test_parareal_abc16_fp64_and_fp32(gpu):
    bd, torch = gpu
    w = pi.ABC_16
    prm = O.derive_params(w)
    hist = O.parareal(w, prm, k_max=3)
    _, U64 = _run_gpu_iterations(bd, w, 3)
    _, U32 = _run_gpu_iterations(bd, w, 3, precision=bd.PR_FP32)
    worst64 = max(rel(U64[k][n], hist["U"][k][n]) for k in range(4) for n in range(w.n_sub + 1))
    worst32 = max(rel(U32[k][n], hist["U"][k][n]) for k in range(4) for n in range(w.n_sub + 1))
    print(f"abc16: worst rel L2 vs oracle fp64 {worst64:.3e} fp32 {worst32:.3e}")
    assert worst64 < TOL64
    assert worst32 < TOL32


def test_finite_termination_and_reference(gpu):
    bd, torch = gpu
    w = pi.tiny(n=8, n_sub=5, T=0.1, dt=2e-3, f_seed=1)
    prm = O.derive_params(w)
    ref = O.sequential_fine(w, prm)
    s = solver(bd, w)
    s.set_initial(w.u0(), w.f())
    s.compute_reference()
    rep = s.solve(0.0, k_max=w.n_sub)
    assert rep["k"] == w.n_sub
    U = s.interfaces()
    for n in range(w.n_sub + 1):
        assert rel(U[n], ref[n]) < TOL64
    assert rep["max_err"] < TOL64


# ---------------------------------------------------------------------- failure paths
def test_failure_paths_leave_context_usable(gpu):
    bd, torch = gpu
    w = pi.tiny(n=8, n_sub=3, T=0.06, dt=2e-3)
    # barrier time-out: spin limit 0 with several CTAs per subinterval
    s = solver(bd, w, spin_limit=0, group_ctas=4)
    s.set_initial(w.u0(), w.f())
    with pytest.raises(bd.PRError) as ei:
        s.iteration0()
        s.sync()
    assert ei.value.status == 6
    # the device is still usable: a normal solver runs afterwards
    s2 = solver(bd, w)
    s2.set_initial(w.u0(), w.f())
    s2.iteration0()
    s2.iterate(1)
    # BiCGStab cap
    s3 = solver(bd, w, lin_maxit=1)
    s3.set_initial(w.u0(), w.f())
    with pytest.raises(bd.PRError) as ei:
        s3.iteration0()
        s3.sync()
    assert ei.value.status == 4
    # non-finite input
    u0 = w.u0().copy()
    u0[1, 2, 3] = np.nan
    with pytest.raises(bd.PRError) as ei:
        s2.set_initial(u0, None)
    assert ei.value.status == 7
    # out-of-order phases
    s4 = solver(bd, w)
    s4.set_initial(w.u0(), w.f())
    with pytest.raises(bd.PRError) as ei:
        s4.fine_sweep(1)
    assert ei.value.status == 8


def test_rewind_repeats_iteration_exactly(gpu):
    bd, torch = gpu
    w = pi.tiny(n=8, n_sub=4, T=0.08, dt=2e-3)
    s = solver(bd, w)
    s.set_initial(w.u0(), w.f())
    s.iteration0()
    s.iterate(1)
    a = s.interfaces()
    s.rewind()
    s.iterate(1)
    b = s.interfaces()
    assert np.array_equal(a, b)
    s.iterate(2)
