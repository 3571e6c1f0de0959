"""Galerkin-reduced coarse propagator G and the augmentation of the POD space.

Reduced implicit Euler (Sec. 2.3, eqs. (eq8)/(eq00)): with a basis V (N_g x m) of the
POD space and M = I (reading R1), the coarse step l on [t_a, t_a + L*dT] solves

    (V^T V + dT V^T L_h(t_l) V) beta_l = V^T V beta_{l-1} + dT V^T f(t_l),
    t_l = t_a + l dT,

starting from the Galerkin projection of the initial value, V^T V beta_0 = V^T x, and
G returns V beta_L.  Each reduced system is solved by dense LU with partial pivoting.

Augmentation (Case II, eqs. (eqaug)/(eq12)): d~ = U - R R^T U, d = d~ / ||d~||, and the
basis becomes [R, d] so that U lies in the coarse space.  The bordered matrices of
eq. (eq13) are the blocks of [R, d]^T A [R, d]; the (2,1) block is read as d^T A R
(reading R13).  Following reading R11, d~ is orthogonalised against R once more and the
augmentation is skipped when ||d~|| <= aug_tol * ||U||.
"""
from __future__ import annotations

import numpy as np


def galerkin_project(op, V: np.ndarray, t: float):
    """(V^T V, V^T L_h(t) V) for a basis V stored as N_g x m columns."""
    shape = (op.grid.n,) * 3
    LV = np.stack([op.L(V[:, i].reshape(shape), t).reshape(-1) for i in range(V.shape[1])],
                  axis=1)
    return V.T @ V, V.T @ LV


def coarse_propagate(op, V: np.ndarray, x: np.ndarray, t_a: float, n_steps: int,
                     dT: float, with_forcing: bool = True):
    """G(t_a, t_a + n_steps*dT, P_V x): reduced implicit Euler in span V.

    Returns (V beta_L, beta_L).  The reduced matrices are re-assembled at every coarse
    time when the flow depends on time; otherwise once (Sec. 3.3: separable operators
    are assembled at the first step only)."""
    Mv = V.T @ V
    beta = np.linalg.solve(Mv, V.T @ x.reshape(-1))
    Lv = None
    for l in range(1, n_steps + 1):
        t = t_a + l * dT
        if Lv is None or op.time_dependent:
            _, Lv = galerkin_project(op, V, t)
        rhs = Mv @ beta
        if with_forcing and op.has_forcing:
            rhs = rhs + dT * (V.T @ op.forcing(t).reshape(-1))
        beta = np.linalg.solve(Mv + dT * Lv, rhs)
    return V @ beta, beta


def augment(R: np.ndarray, U: np.ndarray, aug_tol: float = 1e-12):
    """[R, d] with d~ = U - R R^T U (eq. (eqaug)), orthogonalised once more against R,
    d = d~ / ||d~|| (eq. (eq12)).  Returns (V, augmented?)."""
    u = U.reshape(-1)
    d = u - R @ (R.T @ u)
    d = d - R @ (R.T @ d)
    nd = np.linalg.norm(d)
    if nd <= aug_tol * np.linalg.norm(u):
        return R, False
    return np.concatenate([R, (d / nd)[:, None]], axis=1), True


# ------------------------------------------------------------------------------------
# Coarse-grid propagator of the comparator "Parareal-II" (Sec. 4): the same problem on a
# grid coarsened by a factor c in every direction (the paper coarsens the FEM mesh by
# three bisections, i.e. a factor 2), implicit Euler with the coarse step dT, restriction
# by injection and prolongation by trilinear interpolation on the periodic grid.

def restrict(u: np.ndarray, c: int) -> np.ndarray:
    """Injection: the values at the coarse points x_{c i}."""
    return np.ascontiguousarray(u[::c, ::c, ::c])


def prolong(uc: np.ndarray, c: int) -> np.ndarray:
    """Trilinear interpolation from the coarse points to every fine point (periodic)."""
    out = uc
    for axis in range(3):
        nc = out.shape[axis]
        w = np.arange(c) / c                        # offset of fine point j*c + a is a/c
        lo = np.repeat(out, c, axis=axis)           # u_c[j] at fine points j*c + a
        hi = np.repeat(np.roll(out, -1, axis=axis), c, axis=axis)
        shape = [1, 1, 1]
        shape[axis] = nc * c
        wt = np.tile(w, nc).reshape(shape)
        out = (1.0 - wt) * lo + wt * hi
    return out


def coarse_grid_propagate(op_c, x: np.ndarray, t_a: float, n_steps: int, dT: float, c: int):
    """P G_c(R x): n_steps implicit Euler steps of size dT on the coarse operator op_c
    (with its forcing), from the restriction of x, interpolated back."""
    from .fine import fine_propagate
    uc, _ = fine_propagate(op_c, restrict(x, c), t_a, n_steps, dT, tol=1e-14)
    return prolong(uc, c)
