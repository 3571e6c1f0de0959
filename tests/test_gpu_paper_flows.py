"""The paper's own time-dependent flows (eq. (koleq) and the phase-shifted ABC field of
Sec. 4.2) on the GPU against the oracle: the fine propagator from a nonzero start time,
the sequential fine reference, whole parareal iterations of the adaptive method and of
Parareal-I, and finite termination."""
import numpy as np
import pytest

import oracle as O
import pr_inputs as pi
from test_gpu_parity import TOL32, TOL64, dev, oracle_envelope, rel

pytestmark = pytest.mark.gpu

FLOWS = {"kol": pi.Flow("paper_kolmogorov"), "abc": pi.Flow("paper_abc", w=1.3)}


def workload(name, n=8, n_sub=4, T=0.4, dt=0.01, f_seed=None, eps=0.05):
    return pi.tiny(n=n, n_sub=n_sub, T=T, dt=dt, flow=FLOWS[name], f_seed=f_seed, eps=eps,
                   name=f"paper_{name}")


@pytest.mark.parametrize("name", list(FLOWS))
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "fp32"])
def test_fine_propagator_from_a_nonzero_time(gpu, name, prec):
    bd, torch = gpu
    w = workload(name, n=12, f_seed=5)
    s = bd.Parareal.from_workload(w, precision=prec)
    op = O.make_operator(w)
    B, steps, t0 = 3, 25, 0.7
    u = np.stack([pi.initial_state(12, seed=30 + b) for b in range(B)])
    s.set_initial(u[0], w.f())
    out, snap = s.op_fine(dev(torch, u), steps, 5, 4, t0=t0)
    out, snap = out.cpu().numpy(), snap.cpu().numpy()
    tol = TOL64 if prec == 0 else TOL32
    for b in range(B):
        ue, W = O.fine_propagate(op, u[b], t0, steps, s.dt_eff, 5, 4, tol=1e-14)
        assert rel(out[b], ue) < tol, (b, rel(out[b], ue))
        for j in range(4):
            assert rel(snap[b, j], W[:, j]) < tol
    # a frozen field would differ: the test sees the time dependence
    ue0, _ = O.fine_propagate(op, u[0], 0.0, steps, s.dt_eff, tol=1e-14)
    assert rel(out[0], ue0) > 1e3 * tol
    s.close()


@pytest.mark.parametrize("name", list(FLOWS))
def test_sequential_reference(gpu, name):
    bd, torch = gpu
    w = workload(name)
    prm = O.derive_params(w)
    s = bd.Parareal.from_workload(w)
    s.set_initial(w.u0(), w.f())
    s.compute_reference(True)
    s.iteration0()
    ref = O.sequential_fine(w, prm)
    rep = s.solve(1e-14, k_max=w.n_sub, ref=None)
    U = s.interfaces()
    for n in range(w.n_sub + 1):
        assert rel(U[n], ref[n]) < TOL64, n        # finite termination: k = N is exact
    assert rep["k"] == w.n_sub or rep["converged"]
    s.close()


@pytest.mark.parametrize("name", list(FLOWS))
@pytest.mark.parametrize("method", ["adaptive", "parareal_I"])
def test_parareal_iterates(gpu, name, method):
    bd, torch = gpu
    w = workload(name, f_seed=3)
    prm = O.derive_params(w, method=method)
    K = 3
    hist, env = oracle_envelope(w, prm, K, 1e-13)
    code = bd.PR_METHOD_ADAPTIVE if method == "adaptive" else bd.PR_METHOD_PARAREAL_I
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
    s.close()
    print(f"paper {name} {method}: worst error / tolerance {worst:.3f}")


@pytest.mark.parametrize("name", list(FLOWS))
def test_parareal_iterates_fp32(gpu, name):
    bd, torch = gpu
    w = workload(name, f_seed=3)
    prm = O.derive_params(w)
    K = 3
    hist, env = oracle_envelope(w, prm, K, 1e-8, where="fine")
    s = bd.Parareal.from_workload(w, precision=bd.PR_FP32)
    s.set_initial(w.u0(), w.f())
    s.iteration0()
    Us = [s.interfaces()]
    for k in range(1, K + 1):
        s.iterate(k)
        Us.append(s.interfaces())
    for k in range(K + 1):
        for n in range(w.n_sub + 1):
            e = rel(Us[k][n], hist["U"][k][n])
            assert e < max(TOL32, 10 * env[k][n]), (k, n, e)
    s.close()


def test_time_less_operators_are_refused_for_time_dependent_flows(gpu):
    bd, torch = gpu
    w = workload("kol")
    s = bd.Parareal.from_workload(w)
    s.set_initial(w.u0(), w.f())
    u = dev(torch, w.u0()[None])
    with pytest.raises(bd.PRError):
        s.op_apply_L(u)
    s.close()
