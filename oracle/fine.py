"""Fine propagator F: implicit Euler in time, eq. (semi-dis-eq), on the FD grid.

One step from t_old to t_new = t_old + dt solves the algebraic system of eq. (algform)
with M = I (reading R1):

    (I + dt L_h(t_new)) u_new = u_old + dt f(t_new).

The paper does not name its linear solver (Sec. 3.3 only says "linear solvers of
approximately linear complexity"); following the build target this oracle uses
BiCGStab (van der Vorst, SIAM J. Sci. Stat. Comput. 13, 1992) started from u_old with
shadow residual r_hat = r_0, stopping when ||r||_2 <= tol * ||rhs||_2 (reading R14), or a
dense LU solve on tiny grids.

Snapshots (Case I, Sec. 2.3): the states at steps 0, dM, 2 dM, ..., (n_s - 1) dM, the
initial state included (reading R4).

An explicit alternative to the paper's implicit Euler (not used by the paper; the build
target names it): the classical fourth-order Runge-Kutta method (Kutta 1901) on the
semi-discrete system u' = -L_h(t) u + f(t), fine_propagate_rk4.
"""
from __future__ import annotations

import numpy as np


class SolverError(RuntimeError):
    pass


def bicgstab(apply_A, b: np.ndarray, x0: np.ndarray, tol: float, maxit: int = 200):
    """Textbook BiCGStab for A x = b.  Returns (x, iterations).

    Raises SolverError on breakdown (rho = 0, (r_hat, v) = 0, omega = 0) or when maxit
    iterations do not reach ||r|| <= tol ||b||.
    """
    x = x0.copy()
    r = b - apply_A(x)
    bnorm = np.linalg.norm(b)
    if np.linalg.norm(r) <= tol * bnorm:
        return x, 0
    r_hat = r.copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    for it in range(1, maxit + 1):
        rho = np.vdot(r_hat, r)
        if rho == 0.0:
            raise SolverError("BiCGStab breakdown: rho = 0")
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = apply_A(p)
        rv = np.vdot(r_hat, v)
        if rv == 0.0:
            raise SolverError("BiCGStab breakdown: (r_hat, v) = 0")
        alpha = rho / rv
        s = r - alpha * v
        if np.linalg.norm(s) <= tol * bnorm:
            x = x + alpha * p
            return x, it
        t = apply_A(s)
        tt = np.vdot(t, t)
        if tt == 0.0:
            raise SolverError("BiCGStab breakdown: (t, t) = 0")
        omega = np.vdot(t, s) / tt
        if omega == 0.0:
            raise SolverError("BiCGStab breakdown: omega = 0")
        x = x + alpha * p + omega * s
        r = s - omega * t
        if np.linalg.norm(r) <= tol * bnorm:
            return x, it
        rho_old = rho
    raise SolverError(f"BiCGStab did not reach tol {tol} in {maxit} iterations")


def implicit_euler_step(op, u_old: np.ndarray, t_new: float, dt: float,
                        tol: float = 1e-14, dense_A=None, maxit: int = 200):
    """One fine step (I + dt L(t_new)) u_new = u_old + dt f(t_new).

    dense_A: optional explicit matrix of L_h(t_new) (time-independent flows); when given,
    the step is a dense LU solve instead of BiCGStab.
    Returns (u_new, iterations) (iterations = 0 for the dense solve).
    """
    rhs = u_old + dt * op.forcing(t_new) if op.has_forcing else u_old.copy()
    if dense_A is not None:
        Ng = u_old.size
        A = np.eye(Ng) + dt * dense_A
        return np.linalg.solve(A, rhs.reshape(-1)).reshape(u_old.shape), 0

    def apply_A(x):
        return x + dt * op.L(x, t_new)

    return bicgstab(apply_A, rhs, u_old, tol, maxit)


def fine_propagate(op, u0: np.ndarray, t0: float, steps: int, dt: float, dM: int = 0,
                   n_snap: int = 0, tol: float = 1e-14, dense_A=None, stats=None):
    """F(t0, t0 + steps*dt, u0).  Returns (u_end, W) with W the N_g x n_snap snapshot
    matrix (states at steps 0, dM, ..., (n_snap-1) dM), or (u_end, None) if n_snap = 0."""
    u = u0.copy()
    W = None
    if n_snap > 0:
        W = np.zeros((u0.size, n_snap))
        W[:, 0] = u.reshape(-1)
    for j in range(1, steps + 1):
        u, its = implicit_euler_step(op, u, t0 + j * dt, dt, tol, dense_A)
        if stats is not None:
            stats.append(its)
        if n_snap > 0 and j % dM == 0 and j // dM < n_snap:
            W[:, j // dM] = u.reshape(-1)
    return u, W


def rk4_step(op, u: np.ndarray, t: float, dt: float) -> np.ndarray:
    """One classical Runge-Kutta step of u' = g(t, u) = -L_h(t) u + f(t) from t to t + dt:
    k1 = g(t, u), k2 = g(t + dt/2, u + dt/2 k1), k3 = g(t + dt/2, u + dt/2 k2),
    k4 = g(t + dt, u + dt k3), u_new = u + dt/6 (k1 + 2 k2 + 2 k3 + k4)."""
    def g(tt, v):
        out = -op.L(v, tt)
        if op.has_forcing:
            out = out + op.forcing(tt)
        return out
    k1 = g(t, u)
    k2 = g(t + dt / 2, u + dt / 2 * k1)
    k3 = g(t + dt / 2, u + dt / 2 * k2)
    k4 = g(t + dt, u + dt * k3)
    return u + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)


def fine_propagate_rk4(op, u0: np.ndarray, t0: float, steps: int, dt: float, dM: int = 0,
                       n_snap: int = 0):
    """F(t0, t0 + steps*dt, u0) with rk4_step; snapshots as in fine_propagate."""
    u = u0.copy()
    W = None
    if n_snap > 0:
        W = np.zeros((u0.size, n_snap))
        W[:, 0] = u.reshape(-1)
    for j in range(1, steps + 1):
        u = rk4_step(op, u, t0 + (j - 1) * dt, dt)
        if n_snap > 0 and j % dM == 0 and j // dM < n_snap:
            W[:, j // dM] = u.reshape(-1)
    return u, W
