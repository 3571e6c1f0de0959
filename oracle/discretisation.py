"""Spatial operator of the advection-diffusion problem, eq. (eq1) of Sec. 4.

    u_t - eps * Lap(u) + B(x, t) . grad(u) + c u = f   on the periodic cube [0, L]^3, c = 0.

The paper discretises in space with P1 finite elements (Sec. 2.2, eqs. (eq5)-(algform)).
This oracle uses the second-order finite-difference analogue on a uniform periodic grid
(reading R0): x_i = i h, h = L / n, and

    (L_h u)_i = sum_d b_d(x_i, t) (u_{i+e_d} - u_{i-e_d}) / (2h)
              - eps * sum_d (u_{i+e_d} - 2 u_i + u_{i-e_d}) / h^2 .

With this grid the mass matrix of eq. (algform) is the identity (reading R1), so the
fine algebraic system is (I + dt L_h(t_new)) u_new = u_old + dt f(t_new).

Arrays are indexed [z][y][x]; numpy axis 2 is x, axis 1 is y, axis 0 is z.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional, Tuple

import numpy as np

AXES = (2, 1, 0)  # x, y, z as numpy axes of a [z][y][x] array


@dataclasses.dataclass(frozen=True)
class Grid:
    n: int
    L: float = 2.0 * math.pi

    @property
    def h(self) -> float:
        return self.L / self.n

    @property
    def Ng(self) -> int:
        return self.n ** 3

    def coords(self) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
        """Broadcastable coordinate arrays X (x), Y (y), Z (z) of a [z][y][x] grid."""
        s = np.arange(self.n, dtype=np.float64) * self.h
        return s[None, None, :], s[None, :, None], s[:, None, None]


def velocity(flow, grid: Grid, t: float = 0.0, pert: Optional[np.ndarray] = None):
    """The three components (b_x, b_y, b_z) of the advection field at time t.

    abc:  (A sin z + C cos y, B sin x + A cos z, C sin y + B cos x); the paper's ABC flow
          (Sec. 4.2) with A = B = C = 1 at phase sin(w t) = 0.
    kolmogorov: (sin(k y), 0, 0), the classical Kolmogorov forcing profile.
    const: constant (b0, b1, b2), used by the Fourier-symbol check.
    paper_kolmogorov: (cos y, cos z, cos x) + (sin z, sin x, sin y) cos t, eq. (koleq).
    paper_abc: ABC with all arguments shifted by sin(w t), Sec. 4.2.
    A steady kind with flow.pert_seed > 0 carries the seeded divergence-free perturbation
    b' of the input recipe on top (a stored 3 x n^3 field); `pert` overrides it with a
    given stored field (the injected one on a coarser grid).
    """
    base = _analytic_velocity(flow, grid, t)
    if pert is None and getattr(flow, "pert_seed", 0) > 0:
        pert = flow.pert(grid.n)
    if pert is None:
        return base
    if time_dependent(flow):
        raise ValueError("the velocity perturbation applies to steady flows only")
    return tuple(b + p for b, p in zip(base, pert))


def _analytic_velocity(flow, grid: Grid, t: float):
    X, Y, Z = grid.coords()
    one = np.ones((grid.n,) * 3)
    kind = flow.kind
    if kind == "abc":
        A, B, C = flow.A, flow.B, flow.C
        return (A * np.sin(Z) + C * np.cos(Y)) * one, \
               (B * np.sin(X) + A * np.cos(Z)) * one, \
               (C * np.sin(Y) + B * np.cos(X)) * one
    if kind == "kolmogorov":
        return np.sin(flow.k * Y) * one, 0.0 * one, 0.0 * one
    if kind == "const":
        return flow.b0 * one, flow.b1 * one, flow.b2 * one
    if kind == "paper_kolmogorov":
        c = math.cos(t)
        return (np.cos(Y) + np.sin(Z) * c) * one, \
               (np.cos(Z) + np.sin(X) * c) * one, \
               (np.cos(X) + np.sin(Y) * c) * one
    if kind == "paper_abc":
        ph = math.sin(flow.w * t)
        return (np.sin(Z + ph) + np.cos(Y + ph)) * one, \
               (np.sin(X + ph) + np.cos(Z + ph)) * one, \
               (np.sin(Y + ph) + np.cos(X + ph)) * one
    raise ValueError(f"unknown flow kind {kind!r}")


def time_dependent(flow) -> bool:
    return flow.kind in ("paper_kolmogorov", "paper_abc")


def apply_L(u: np.ndarray, vel, eps: float, h: float) -> np.ndarray:
    """(L_h u) = b . grad_h u - eps Lap_h u with central differences (see module doc)."""
    out = np.zeros_like(u)
    for axis, b in zip(AXES, vel):
        up = np.roll(u, -1, axis=axis)   # u_{i+e_d}
        um = np.roll(u, +1, axis=axis)   # u_{i-e_d}
        out += b * (up - um) / (2.0 * h)
        out -= eps * (up - 2.0 * u + um) / (h * h)
    return out


def apply_LT(u: np.ndarray, vel, eps: float, h: float) -> np.ndarray:
    """Transpose of L_h: (L_h^T u)_i = sum_j (L_h)_{j i} u_j.

    Row j of L_h holds +b_d(j)/(2h) at column j+e_d and -b_d(j)/(2h) at column j-e_d, so
    column i collects +b_d(i-e_d)/(2h) u_{i-e_d} and -b_d(i+e_d)/(2h) u_{i+e_d}.
    The diffusion part is symmetric.
    """
    out = np.zeros_like(u)
    for axis, b in zip(AXES, vel):
        bu = b * u
        out += (np.roll(bu, +1, axis=axis) - np.roll(bu, -1, axis=axis)) / (2.0 * h)
        up = np.roll(u, -1, axis=axis)
        um = np.roll(u, +1, axis=axis)
        out -= eps * (up - 2.0 * u + um) / (h * h)
    return out


def assemble_L_dense(grid: Grid, vel, eps: float) -> np.ndarray:
    """The N_g x N_g matrix of L_h written entry by entry (for brute-force checks, n <= 10)."""
    n, h = grid.n, grid.h
    Ng = grid.Ng
    A = np.zeros((Ng, Ng))
    bx, by, bz = (np.asarray(b) for b in vel)

    def idx(x, y, z):
        return (x % n) + n * ((y % n) + n * (z % n))

    for z in range(n):
        for y in range(n):
            for x in range(n):
                i = idx(x, y, z)
                A[i, i] += 6.0 * eps / (h * h)
                for (dx, dy, dz), b in (((1, 0, 0), bx[z, y, x]), ((0, 1, 0), by[z, y, x]),
                                        ((0, 0, 1), bz[z, y, x])):
                    A[i, idx(x + dx, y + dy, z + dz)] += b / (2.0 * h) - eps / (h * h)
                    A[i, idx(x - dx, y - dy, z - dz)] += -b / (2.0 * h) - eps / (h * h)
    return A


@dataclasses.dataclass
class Operator:
    """The problem data the propagators need: grid, flow, eps, forcing f(x) (or None) and
    an explicit stored velocity perturbation (None: the flow's own, if any)."""
    grid: Grid
    flow: object
    eps: float
    f: Optional[np.ndarray] = None
    pert: Optional[np.ndarray] = None

    def __post_init__(self):
        # the stored field is built once, not at every operator application
        if self.pert is None and getattr(self.flow, "pert_seed", 0) > 0:
            self.pert = self.flow.pert(self.grid.n)

    def vel(self, t: float):
        return velocity(self.flow, self.grid, t, self.pert)

    def stored_perturbation(self) -> Optional[np.ndarray]:
        if self.pert is not None:
            return self.pert
        return self.flow.pert(self.grid.n) if getattr(self.flow, "pert_seed", 0) > 0 else None

    def L(self, u: np.ndarray, t: float) -> np.ndarray:
        return apply_L(u, self.vel(t), self.eps, self.grid.h)

    def LT(self, u: np.ndarray, t: float) -> np.ndarray:
        return apply_LT(u, self.vel(t), self.eps, self.grid.h)

    def forcing(self, t: float) -> np.ndarray:
        """f(x, t).  The seeded forcing is time independent; the paper's own flows carry
        the forcing of eq. (koleq) / Sec. 4.2 on top of it."""
        n = self.grid.n
        base = np.zeros((n, n, n)) if self.f is None else self.f
        kind = self.flow.kind
        if kind == "paper_kolmogorov":
            X, Y, Z = self.grid.coords()
            return base + (-np.cos(Y) - np.sin(Z) * math.cos(t)) * np.ones((n,) * 3)
        if kind == "paper_abc":
            X, Y, Z = self.grid.coords()
            ph = math.sin(self.flow.w * t)
            return base + (-np.sin(Z + ph) - np.cos(Y + ph)) * np.ones((n,) * 3)
        return base

    @property
    def time_dependent(self) -> bool:
        return time_dependent(self.flow)

    @property
    def has_forcing(self) -> bool:
        return self.f is not None or self.time_dependent


def make_operator(w) -> Operator:
    """Operator for a ``pr_inputs.Workload``."""
    return Operator(Grid(w.n), w.flow, w.eps, w.f())
