"""The explicit fine integrator (classical RK4, pr_opts.fine = PR_FINE_RK4) on the GPU
against the oracle's rk4 mode: single propagations (steady and time-dependent flows,
both precisions) and whole parareal iterations with it as F."""
import numpy as np
import pytest

import oracle as O
import pr_inputs as pi
from oracle.fine import fine_propagate_rk4
from test_gpu_parity import TOL32, TOL64, dev, oracle_envelope, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("flow", [pi.Flow("abc"), pi.Flow("paper_abc", w=1.3)], ids=["abc", "paper_abc"])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_rk4_propagation(gpu, flow, prec):
    bd, torch = gpu
    w = pi.Workload("rk", 16, flow, 0.05, 1.0, 8, 2e-3, f_seed=4, m_cap=8)
    s = bd.Parareal.from_workload(w, precision=prec, fine=bd.PR_FINE_RK4)
    op = O.make_operator(w)
    B, steps, t0 = 3, 20, 0.4
    u = np.stack([pi.initial_state(16, seed=70 + b) for b in range(B)])
    s.set_initial(u[0], w.f())
    out, snap = s.op_fine(dev(torch, u), steps, 5, 4, t0=t0)
    out, snap = out.cpu().numpy(), snap.cpu().numpy()
    tol = TOL64 if prec == 0 else TOL32
    for b in range(B):
        ue, W = fine_propagate_rk4(op, u[b], t0, steps, s.dt_eff, 5, 4)
        assert rel(out[b], ue) < tol, (b, rel(out[b], ue))
        for j in range(4):
            assert rel(snap[b, j], W[:, j]) < tol
    # the explicit result is not the implicit one
    ie, _ = O.fine_propagate(op, u[0], t0, steps, s.dt_eff, tol=1e-14)
    assert rel(out[0], ie) > max(1e-6, 10 * tol)
    s.close()


@pytest.mark.parametrize("wl", ["tiny", "tiny_kol"])
def test_parareal_with_rk4_fine(gpu, wl):
    bd, torch = gpu
    w = (pi.tiny(n=8, n_sub=4, T=0.08, dt=2e-3) if wl == "tiny" else
         pi.tiny(n=10, n_sub=4, T=0.08, dt=2e-3, f_seed=2, flow=pi.Flow("paper_kolmogorov")))
    prm = O.derive_params(w, fine="rk4")
    K = 3
    hist, env = oracle_envelope(w, prm, K, 1e-13)
    s = bd.Parareal.from_workload(w, fine=bd.PR_FINE_RK4)
    s.set_initial(w.u0(), w.f())
    s.iteration0()
    Us = [s.interfaces()]
    for k in range(1, K + 1):
        s.iterate(k)
        Us.append(s.interfaces())
    for k in range(K + 1):
        for n in range(w.n_sub + 1):
            e = rel(Us[k][n], hist["U"][k][n])
            assert e < max(TOL64, 10 * env[k][n]), (k, n, e, env[k][n])
    # finite termination on the RK4 sequential solution
    ref = O.sequential_fine(w, prm)
    for k in range(K + 1, w.n_sub + 1):
        s.iterate(k)
    U = s.interfaces()
    for n in range(w.n_sub + 1):
        assert rel(U[n], ref[n]) < TOL64, n
    s.close()
