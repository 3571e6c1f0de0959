"""The comparator "Parareal-I" of Sec. 4 (plain parareal on the fixed iteration-0 POD
space V0) on the GPU against the oracle's parareal_I mode: whole iterations and finite
termination at k = N."""
import numpy as np
import pytest

import oracle as O
import pr_inputs as pi
from test_gpu_parity import TOL32, TOL64, WORKLOADS, oracle_envelope, rel

pytestmark = pytest.mark.gpu


def run(bd, w, k_max, precision, T0=None):
    kw = dict(method=bd.PR_METHOD_PARAREAL_I)
    if T0 is not None:
        kw["T0"] = T0
    s = bd.Parareal.from_workload(w, precision=precision, **kw)
    s.set_initial(w.u0(), w.f())
    s.iteration0()
    Us = [s.interfaces()]
    for k in range(1, k_max + 1):
        s.iterate(k)
        Us.append(s.interfaces())
    return s, Us


@pytest.mark.parametrize("wl,prec", [("tiny", 0), ("tiny_forced", 0), ("abc16", 0),
                                     ("tiny", 1), ("tiny_forced", 1)])
def test_parareal_I_iterates(gpu, wl, prec):
    bd, torch = gpu
    w = WORKLOADS[wl]()
    prm = O.derive_params(w, method="parareal_I")
    K = min(w.n_sub, 3)
    if prec == 0:
        hist, env = oracle_envelope(w, prm, K, 1e-13)
        base, scale = TOL64, 10
    else:
        hist, env = oracle_envelope(w, prm, K, 1e-8, where="fine")
        base, scale = TOL32, 10
    s, Us = run(bd, w, K, prec)
    worst = 0.0
    for k in range(K + 1):
        for n in range(w.n_sub + 1):
            e = rel(Us[k][n], hist["U"][k][n])
            tol = max(base, scale * env[k][n])
            worst = max(worst, e / tol)
            assert e < tol, (k, n, e, env[k][n])
    d = s.diagnostics()
    assert d["m0"] == hist["m0"] and not d["m2"].any()    # V0 only, no level-2 bases
    s.close()
    print(f"parareal_I {wl} prec {prec}: worst error / tolerance {worst:.3f}")


def test_parareal_I_finite_termination_with_a_long_window(gpu):
    # the paper's comparator uses a longer Case-I window; at k = N the iterate is the
    # sequential fine solution whatever the coarse space
    bd, torch = gpu
    w = pi.tiny(n=8, n_sub=4, T=0.08, dt=2e-3, f_seed=3)
    T0 = 0.06
    prm = O.derive_params(w, T0=T0, method="parareal_I")
    ref = O.sequential_fine(w, prm)
    s, Us = run(bd, w, w.n_sub, 0, T0=T0)
    for n in range(w.n_sub + 1):
        assert rel(Us[-1][n], ref[n]) < TOL64, n
    assert rel(Us[0][w.n_sub], ref[w.n_sub]) > 1e-6
    s.close()


# ---------------------------------------------------------------------------------------
# Parareal-II: the coarse propagator is implicit Euler on the grid coarsened by 2.
@pytest.mark.parametrize("wl,prec", [("tiny", 0), ("tiny_forced", 0), ("tiny", 1),
                                     ("paper_abc", 0)])
def test_parareal_II_iterates(gpu, wl, prec):
    bd, torch = gpu
    if wl == "paper_abc":
        w = pi.tiny(n=8, n_sub=4, T=0.4, dt=0.01, flow=pi.Flow("paper_abc", w=1.3), f_seed=3)
    else:
        w = WORKLOADS[wl]()
    prm = O.derive_params(w, method="parareal_II")
    K = 3
    if prec == 0:
        hist, env = oracle_envelope(w, prm, K, 1e-13)
        base = TOL64
    else:
        hist, env = oracle_envelope(w, prm, K, 1e-8, where="fine")
        base = TOL32
    s = bd.Parareal.from_workload(w, precision=prec, method=bd.PR_METHOD_PARAREAL_II)
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
            tol = max(base, 10 * env[k][n])
            worst = max(worst, e / tol)
            assert e < tol, (k, n, e, env[k][n])
    # finite termination on the sequential fine solution
    ref = O.sequential_fine(w, prm)
    for k in range(K + 1, w.n_sub + 1):
        s.iterate(k)
    U = s.interfaces()
    for n in range(w.n_sub + 1):
        assert rel(U[n], ref[n]) < base, n
    s.close()
    print(f"parareal_II {wl} prec {prec}: worst error / tolerance {worst:.3f}")


def test_parareal_II_needs_an_even_grid(gpu):
    bd, torch = gpu
    w = pi.tiny(n=9, n_sub=2)
    with pytest.raises(bd.PRError):
        bd.Parareal.from_workload(w, method=bd.PR_METHOD_PARAREAL_II)
