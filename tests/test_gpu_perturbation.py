"""Flows with a stored divergence-free velocity perturbation (pr_flow.pert, the 256^3
Kolmogorov case's "seeded random divergence-free perturbation") on the GPU against the
oracle: the operator and its transpose, the fine propagator in both precision modes,
whole parareal iterations (adaptive and Parareal-II), and the refused combinations."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
import pr_inputs as pi
from oracle.discretisation import apply_L, apply_LT
from test_gpu_parity import TOL32, TOL64, dev, oracle_envelope, rel

pytestmark = pytest.mark.gpu

KOLP = pi.Flow("kolmogorov", k=2, pert_seed=4, pert_amp=0.3)
ABCP = pi.Flow("abc", pert_seed=2, pert_amp=0.2)


def workload(flow, n=8, n_sub=4, T=0.2, dt=0.01, f_seed=3, eps=0.03, name="pert"):
    return pi.tiny(n=n, n_sub=n_sub, T=T, dt=dt, flow=flow, f_seed=f_seed, eps=eps, name=name)


@pytest.mark.parametrize("transpose", [False, True])
def test_operator_and_transpose(gpu, transpose):
    bd, torch = gpu
    w = workload(ABCP, n=12)
    s = bd.Parareal.from_workload(w)
    s.set_initial(w.u0(), w.f())
    op = O.make_operator(w)
    vel = op.vel(0.0)
    u = np.stack([pi.initial_state(12, seed=40 + b) for b in range(3)])
    out = s.op_apply_L(dev(torch, u), transpose=transpose).cpu().numpy()
    f = apply_LT if transpose else apply_L
    for b in range(3):
        ref = f(u[b], vel, w.eps, op.grid.h)
        assert rel(out[b], ref) < 1e-13, (b, rel(out[b], ref))
    # the no-allocation entry point reads the same stored field from the workspace
    ut = dev(torch, u)
    o2 = torch.empty_like(ut)
    s._check(s._lib.pr_op_apply_L_noalloc(s.ctx, C.c_void_p(ut.data_ptr()), C.c_void_p(o2.data_ptr()),
                                          3, int(transpose)))
    assert np.array_equal(o2.cpu().numpy(), out)
    # the perturbation is seen: the plain field gives a different result
    plain = O.make_operator(workload(pi.Flow("abc"), n=12))
    assert rel(out[0], f(u[0], plain.vel(0.0), w.eps, op.grid.h)) > 1e-3
    s.close()


@pytest.mark.parametrize("flow", [KOLP, ABCP], ids=["kol", "abc"])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_fine_propagator(gpu, flow, prec):
    bd, torch = gpu
    w = workload(flow, n=12)
    s = bd.Parareal.from_workload(w, precision=prec)
    op = O.make_operator(w)
    B, steps = 3, 25
    u = np.stack([pi.initial_state(12, seed=30 + b) for b in range(B)])
    s.set_initial(u[0], w.f())
    out, snap = s.op_fine(dev(torch, u), steps, 5, 4)
    out, snap = out.cpu().numpy(), snap.cpu().numpy()
    tol = TOL64 if prec == 0 else TOL32
    for b in range(B):
        ue, W = O.fine_propagate(op, u[b], 0.0, steps, s.dt_eff, 5, 4, tol=1e-14)
        assert rel(out[b], ue) < tol, (b, rel(out[b], ue))
        for j in range(4):
            assert rel(snap[b, j], W[:, j]) < tol
    s.close()


@pytest.mark.parametrize("method", ["adaptive", "parareal_II"])
def test_parareal_iterates_fp64(gpu, method):
    bd, torch = gpu
    w = workload(KOLP)
    prm = O.derive_params(w, method=method)
    K = 3
    hist, env = oracle_envelope(w, prm, K, 1e-13)
    code = bd.PR_METHOD_ADAPTIVE if method == "adaptive" else bd.PR_METHOD_PARAREAL_II
    s = bd.Parareal.from_workload(w, method=code)
    s.set_initial(w.u0(), w.f())
    s.iteration0()
    Us = [s.interfaces()]
    for k in range(1, K + 1):
        s.iterate(k)
        Us.append(s.interfaces())
    worst = 0.0
    for k in range(K + 1):
        for n in range(w.n_sub + 1):
            e = rel(Us[k][n], hist["U"][k][n])
            tol = max(TOL64, 10 * env[k][n])
            worst = max(worst, e / tol)
            assert e < tol, (k, n, e, env[k][n])
    # finite termination on the sequential fine solution of the perturbed problem
    ref = O.sequential_fine(w, prm)
    for k in range(K + 1, w.n_sub + 1):
        s.iterate(k)
    U = s.interfaces()
    for n in range(w.n_sub + 1):
        assert rel(U[n], ref[n]) < TOL64, n
    s.close()
    print(f"perturbed {method}: worst error / tolerance {worst:.3f}")


def test_parareal_iterates_fp32(gpu):
    bd, torch = gpu
    w = workload(ABCP)
    prm = O.derive_params(w)
    K = 3
    hist, env = oracle_envelope(w, prm, K, 1e-8, where="fine")
    s = bd.Parareal.from_workload(w, precision=bd.PR_FP32)
    s.set_initial(w.u0(), w.f())
    s.iteration0()
    for k in range(1, K + 1):
        s.iterate(k)
        U = s.interfaces()
        for n in range(w.n_sub + 1):
            e = rel(U[n], hist["U"][k][n])
            assert e < max(TOL32, 10 * env[k][n]), (k, n, e)
    s.close()


def test_refused_combinations(gpu):
    bd, torch = gpu
    # a perturbation on a time-dependent flow, or with the explicit fine integrator
    with pytest.raises(bd.PRError):
        bd.Parareal.from_workload(workload(pi.Flow("paper_abc", pert_seed=1)))
    with pytest.raises(bd.PRError):
        bd.Parareal.from_workload(workload(KOLP), fine=bd.PR_FINE_RK4)
    # one fine launch runs one stencil kind: perturbed and plain contexts do not batch
    a, b = workload(KOLP, name="a"), workload(pi.Flow("kolmogorov", k=2), name="b")
    sa, sb = (bd.Parareal.from_workload(x, group_ctas=4) for x in (a, b))
    for s, x in ((sa, a), (sb, b)):
        s.set_initial(x.u0(), x.f())
        s.iteration0()
    with pytest.raises(bd.PRError):
        bd.fine_sweep_batch([sa, sb], [1, 1])
    sa.close()
    sb.close()


def test_server_batches_perturbed_requests_apart(gpu):
    bd, torch = gpu
    reqs = [workload(KOLP, name="p"), workload(pi.Flow("kolmogorov", k=2), name="q"),
            workload(ABCP, name="r")]
    srv = bd.Server()
    ids = [srv.submit(w, w.u0(), w.f(), tol=1e-9, precision=bd.PR_FP64, group_ctas=4) for w in reqs]
    for _ in range(200):
        act, pend = srv.step()
        if act == 0 and pend == 0:
            break
    for w, i in zip(reqs, ids):
        st, k, inc = srv.query(i)
        assert st == bd.PR_REQ_DONE, srv.request_error(i)
        prm = O.derive_params(w)
        h = O.parareal(w, prm, k_max=k)
        assert rel(srv.result(i), h["U"][k][w.n_sub]) < 1e-10, w.name
    srv.close()
