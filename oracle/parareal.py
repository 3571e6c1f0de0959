"""Algorithm 2 (the adaptive parareal framework) with the update of eq. (formula4).

Time layout (Sec. 2.3, Case II): the fine propagator first runs on [0, T0] (Case I);
parareal then runs on [T0, T0 + T] split into N subintervals [t_n, t_{n+1}],
t_n = T0 + n DeltaT, DeltaT = T / N.

Iteration 0 (Algorithm 2, lines for Case I):
    u_hat0, W = F(0, T0, u0) with snapshots;  V0 = POD_Mode(W, gamma1);
    U^0_0 = u_hat0,  U^0_{n+1} = G_0(t_n, t_{n+1}, P_{V0} U^0_n).
Iteration k >= 1:
    F_n, W^k_{n,0} = F(t_n, t_{n+1}, U^{k-1}_n)          n = k-1 .. N-1
    R^k_{n,0} = POD_Mode(W^k_{n,0}, gamma2)               n = k-1 .. N-1
    R^k_n = POD_Mode(W^k_n, gamma3), eq. (W^k_n)          n = k .. N-1   (reading R9)
    U^k_n = U^{k-1}_n for n < k, U^k_k = F_{k-1}                         (reading R10)
    for n = k .. N-1 in order:
        V = [R^k_n, d^k_n] (augmentation with U^k_n, eqs. (eqaug)/(eq12))
        U^k_{n+1} = G_V(U^k_n) + F_n - G_V(P_V U^{k-1}_n)         eq. (formula4)
Stop when max_n ||U^k_n - U^{k-1}_n|| / ||U^k_n|| <= tol, or k = N, or k = k_max
(reading R12).

The comparator "Parareal-I" of Sec. 4 (method = "parareal_I") is plain parareal with
the POD space of iteration 0 as the coarse space for every subinterval and iteration:
no level-1 or level-2 POD and no augmentation, U^k_{n+1} = G_{V0}(U^k_n) + F_n -
G_{V0}(U^{k-1}_n); the paper gives it a longer Case-I window (T0 = 10).

The comparator "Parareal-II" (method = "parareal_II") is plain parareal whose coarse
propagator is implicit Euler with step dT on a grid coarsened by coarse_factor (2):
G(x) = P G_c(R x), restriction by injection, prolongation by trilinear interpolation
(reading R18).  Iteration 0 keeps the Case-I window [0, T0] of the other methods
(u_hat0 = F(0, T0, u0)) and then U^0_{n+1} = G(U^0_n).  The error of eq. (error) is measured against the sequential fine
solution U_n = F(0, t_n, u0).

Parameter readings (R3, R4, R15, R16): S = fine steps per subinterval is DeltaT/dt
rounded up to an integer and the step is DeltaT/S; T0 = DeltaT; dT = DeltaT/10;
delta_M = 5 unless a snapshot count is prescribed, in which case delta_M =
floor(S/(n_snap-1)); n_s = floor(S/delta_M) + 1 (the paper's n_s formula), at most n_snap.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

from .coarse import augment, coarse_grid_propagate, coarse_propagate, restrict
from .discretisation import Grid, Operator
from .discretisation import make_operator
from .fine import fine_propagate as _fine_implicit_euler, fine_propagate_rk4
from .pod import level2_blocks, pod_mode


def steps_for(span: float, dt: float) -> int:
    """Smallest integer S with span / S <= dt (ratios within 1e-9 of an integer round)."""
    q = span / dt
    r = round(q)
    return int(r) if abs(q - r) < 1e-9 * max(1.0, q) else int(math.ceil(q))


@dataclasses.dataclass
class Params:
    N: int
    DeltaT: float
    S: int              # fine steps per subinterval
    dt: float           # effective fine step DeltaT / S
    T0: float
    S0: int             # fine steps on [0, T0]
    dT: float           # coarse step
    Lc: int             # coarse steps per subinterval
    dM: int
    n_s: int            # snapshots per subinterval window
    n_s0: int           # snapshots on [0, T0]
    gamma1: float
    gamma2: float
    gamma3: float
    m_cap: int
    m_l: int
    p: int
    tau: float = 1e-13
    lin_tol: float = 1e-14
    aug_tol: float = 1e-12
    method: str = "adaptive"      # or "parareal_I" / "parareal_II" (comparators of Sec. 4)
    fine: str = "implicit_euler"  # or "rk4": the explicit fine integrator (not the paper's)
    coarse_factor: int = 2        # Parareal-II: grid coarsening factor


def derive_params(w, T0: Optional[float] = None, dT: Optional[float] = None,
                  lin_tol: float = 1e-14, pod_tol3: Optional[float] = None,
                  method: str = "adaptive", fine: str = "implicit_euler",
                  coarse_factor: int = 2) -> Params:
    N = w.n_sub
    DeltaT = w.T / N
    S = steps_for(DeltaT, w.dt)
    dt = DeltaT / S
    T0 = DeltaT if T0 is None else T0
    S0 = steps_for(T0, dt)
    dT = DeltaT / 10.0 if dT is None else dT
    Lc = steps_for(DeltaT, dT)
    if w.n_snap > 0:
        dM = max(1, S // (w.n_snap - 1))
    else:
        dM = 5
    n_s = S // dM + 1
    n_s0 = S0 // dM + 1
    if w.n_snap > 0:
        n_s = min(n_s, w.n_snap)
        n_s0 = min(n_s0, w.n_snap)
    g12 = 1.0 - w.pod_tol
    g3 = 1.0 - (w.pod_tol * 4e-3 if pod_tol3 is None else pod_tol3)
    if method not in ("adaptive", "parareal_I", "parareal_II"):
        raise ValueError(f"unknown method {method!r}")
    if fine not in ("implicit_euler", "rk4"):
        raise ValueError(f"unknown fine integrator {fine!r}")
    return Params(N, DeltaT, S, dt, T0, S0, DeltaT / Lc, Lc, dM, n_s, n_s0, g12, g12, g3,
                  w.m_cap, w.m_l, w.p, lin_tol=lin_tol, method=method, fine=fine,
                  coarse_factor=coarse_factor)


# The fine propagator selected by the parameters (the module-level name stays patchable).
def fine_propagate(op, u0, t0, steps, dt, dM=0, n_snap=0, tol=1e-14, prm=None, **kw):
    if prm is not None and prm.fine == "rk4":
        return fine_propagate_rk4(op, u0, t0, steps, dt, dM, n_snap)
    return _fine_implicit_euler(op, u0, t0, steps, dt, dM, n_snap, tol=tol, **kw)


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    """||a - b|| / ||b||, eq. (error)."""
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a - b))


def sequential_fine(w, prm: Params, op=None) -> List[np.ndarray]:
    """U_n = F(0, t_n, u0), n = 0..N, marching one subinterval after another."""
    op = make_operator(w) if op is None else op
    u, _ = fine_propagate(op, w.u0(), 0.0, prm.S0, prm.dt, tol=prm.lin_tol, prm=prm)
    out = [u]
    for n in range(prm.N):
        u, _ = fine_propagate(op, u, prm.T0 + n * prm.DeltaT, prm.S, prm.dt, tol=prm.lin_tol,
                              prm=prm)
        out.append(u)
    return out


def coarse_operator(op, c: int):
    """The problem on the grid coarsened by c (Parareal-II): same flow and eps, the
    forcing and a stored velocity perturbation at the coarse points (injection, like the
    states)."""
    f = None if op.f is None else restrict(op.f, c)
    bp = op.stored_perturbation()
    pc = None if bp is None else np.stack([restrict(b, c) for b in bp])
    return Operator(Grid(op.grid.n // c, op.grid.L), op.flow, op.eps, f, pc)


def iteration0(w, prm: Params, op):
    """Case I: fine on [0, T0], V0 = POD_Mode(W, gamma1), U^0 by G_0 (eq. (formula4))."""
    if prm.method == "parareal_II":
        u_hat0, _ = fine_propagate(op, w.u0(), 0.0, prm.S0, prm.dt, tol=prm.lin_tol, prm=prm)
        op_c = coarse_operator(op, prm.coarse_factor)
        U = [u_hat0]
        for n in range(prm.N):
            U.append(coarse_grid_propagate(op_c, U[n], prm.T0 + n * prm.DeltaT, prm.Lc, prm.dT,
                                           prm.coarse_factor))
        return U, None, 0
    u_hat0, W = fine_propagate(op, w.u0(), 0.0, prm.S0, prm.dt, prm.dM, prm.n_s0,
                               tol=prm.lin_tol, prm=prm)
    V0, m0, _ = pod_mode(W, prm.gamma1, prm.m_cap, prm.tau)
    U = [u_hat0]
    for n in range(prm.N):
        x, _ = coarse_propagate(op, V0, U[n], prm.T0 + n * prm.DeltaT, prm.Lc, prm.dT)
        U.append(x.reshape(u_hat0.shape))
    return U, V0, m0


def parareal(w, prm: Params, k_max: int = 0, tol: float = 0.0, reference=None,
             op=None, record: bool = True):
    """Run Algorithm 2.  Returns a dict with the iterates U^k (list per k), increments,
    errors against `reference` (if given), POD dimensions and the fine end states F^k."""
    op = make_operator(w) if op is None else op
    N = prm.N
    k_max = N if k_max <= 0 else min(k_max, N)
    U_prev, V0, m0 = iteration0(w, prm, op)
    shape = U_prev[0].shape
    hist: Dict[str, list] = dict(U=[list(U_prev)], inc=[], err=[], m1=[], m2=[], aug=[],
                                 F=[])
    if reference is not None:
        hist["err"].append([rel_l2(U_prev[n], reference[n]) for n in range(N + 1)])
    # level-1 bases: latest[(n)] = list of (iteration, basis) in sweep order
    level1_store: Dict[int, Dict[int, np.ndarray]] = {}

    def level1(kk, nn):
        # The basis of subinterval nn at iteration kk: the one computed at the last
        # iteration <= kk that swept nn (its data is unchanged since then).
        store = level1_store.get(nn, {})
        cands = [it for it in store if it <= kk]
        return store[max(cands)] if cands else None

    k_done = 0
    plain = prm.method in ("parareal_I", "parareal_II")
    op_c = coarse_operator(op, prm.coarse_factor) if prm.method == "parareal_II" else None
    for k in range(1, k_max + 1):
        F: Dict[int, np.ndarray] = {}
        m1 = {}
        for n in range(k - 1, N):
            if plain:
                F[n], _ = fine_propagate(op, U_prev[n], prm.T0 + n * prm.DeltaT, prm.S, prm.dt,
                                         tol=prm.lin_tol, prm=prm)
                continue
            Fn, Wn = fine_propagate(op, U_prev[n], prm.T0 + n * prm.DeltaT, prm.S, prm.dt,
                                    prm.dM, prm.n_s, tol=prm.lin_tol, prm=prm)
            F[n] = Fn
            R1, m, _ = pod_mode(Wn, prm.gamma2, prm.m_cap, prm.tau)
            level1_store.setdefault(n, {})[k] = R1
            m1[n] = m
        U = [None] * (N + 1)
        for n in range(k):
            U[n] = U_prev[n]
        U[k] = F[k - 1]
        m2 = {}
        augs = {}
        for n in range(k, N):
            if plain:
                t_n = prm.T0 + n * prm.DeltaT
                if op_c is not None:
                    g_new = coarse_grid_propagate(op_c, U[n], t_n, prm.Lc, prm.dT, prm.coarse_factor)
                    g_old = coarse_grid_propagate(op_c, U_prev[n], t_n, prm.Lc, prm.dT,
                                                  prm.coarse_factor)
                    U[n + 1] = g_new + F[n] - g_old
                    continue
                g_new, _ = coarse_propagate(op, V0, U[n], t_n, prm.Lc, prm.dT)
                g_old, _ = coarse_propagate(op, V0, U_prev[n], t_n, prm.Lc, prm.dT)
                U[n + 1] = (g_new + F[n].reshape(-1) - g_old).reshape(shape)
                continue
            blocks = level2_blocks(level1, k, n, prm.m_l, prm.p, V0)
            R2, m, _ = pod_mode(np.concatenate(blocks, axis=1), prm.gamma3, prm.m_cap,
                                prm.tau)
            m2[n] = m
            V, augd = augment(R2, U[n], prm.aug_tol)
            augs[n] = augd
            t_n = prm.T0 + n * prm.DeltaT
            g_new, _ = coarse_propagate(op, V, U[n], t_n, prm.Lc, prm.dT)
            g_old, _ = coarse_propagate(op, V, U_prev[n], t_n, prm.Lc, prm.dT)
            U[n + 1] = (g_new + F[n].reshape(-1) - g_old).reshape(shape)
        # increment relative to the new iterate: ||U^k - U^{k-1}|| / ||U^k||
        inc =[float(np.linalg.norm(U[n] - U_prev[n]) / max(np.linalg.norm(U[n]), 1e-300))
               for n in range(N + 1)]
        hist["inc"].append(inc)
        hist["m1"].append(m1)
        hist["m2"].append(m2)
        hist["aug"].append(augs)
        if record:
            hist["U"].append(list(U))
            hist["F"].append(F)
        if reference is not None:
            hist["err"].append([rel_l2(U[n], reference[n]) for n in range(N + 1)])
        U_prev = U
        k_done = k
        if tol > 0:
            crit = hist["err"][-1] if reference is not None else inc
            if max(crit) <= tol:
                break
    hist["k"] = k_done
    hist["U_final"] = U_prev
    hist["V0"] = V0
    hist["m0"] = m0
    return hist
