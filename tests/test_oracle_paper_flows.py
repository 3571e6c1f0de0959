"""Pins of the oracle's time-dependent flows of Sec. 4 (no GPU): eq. (koleq), the
Kolmogorov-type field B = (cos y, cos z, cos x) + (sin z, sin x, sin y) cos t with
f = -cos y - sin z cos t, and the ABC field of Sec. 4.2 with every argument shifted by
sin(w t) and f = -sin(z + sin w t) - cos(y + sin w t)."""
import math

import numpy as np
import pytest

import oracle as O
from oracle.coarse import coarse_propagate
from oracle.discretisation import Operator, velocity
from oracle.fine import fine_propagate
from pr_inputs import Flow, initial_state

KOL = Flow("paper_kolmogorov")
ABC = Flow("paper_abc", w=1.0)


def coords(n):
    g = O.Grid(n)
    X, Y, Z = g.coords()
    return g, X, Y, Z


@pytest.mark.parametrize("t", [0.0, 0.7, math.pi / 2, 2.5])
def test_paper_kolmogorov_velocity_and_forcing_closed_form(t):
    g, X, Y, Z = coords(8)
    bx, by, bz = velocity(KOL, g, t)
    one = np.ones((8, 8, 8))
    assert np.allclose(bx, (np.cos(Y) + np.sin(Z) * math.cos(t)) * one, atol=0, rtol=0)
    assert np.allclose(by, (np.cos(Z) + np.sin(X) * math.cos(t)) * one, atol=0, rtol=0)
    assert np.allclose(bz, (np.cos(X) + np.sin(Y) * math.cos(t)) * one, atol=0, rtol=0)
    f = Operator(g, KOL, 0.1, None).forcing(t)
    assert np.allclose(f, (-np.cos(Y) - np.sin(Z) * math.cos(t)) * one, atol=1e-15)


def test_paper_kolmogorov_at_cos_t_zero_is_the_steady_part():
    g, X, Y, Z = coords(6)
    bx, by, bz = velocity(KOL, g, math.pi / 2)
    assert np.max(np.abs(bx - np.cos(Y))) < 1e-15
    assert np.max(np.abs(bz - np.cos(X))) < 1e-15


def test_paper_abc_at_zero_phase_is_the_steady_abc_flow():
    # sin(w t) = 0 at t = 0 and t = pi: the field is the ABC flow with A = B = C = 1
    g = O.Grid(8)
    for t in (0.0, math.pi):
        b = velocity(ABC, g, t)
        ref = velocity(Flow("abc"), g, 0.0)
        for c, r in zip(b, ref):
            assert np.max(np.abs(c - r)) < 1e-15


def test_paper_abc_phase_is_a_shift_of_every_argument():
    # with phase p = sin(w t), B(x, t) = B_abc(x + p, y + p, z + p): shifting the grid
    # function of the steady field by a whole number of cells reproduces the phase
    n = 16
    g = O.Grid(n)
    t = math.asin(2 * math.pi / n)        # p = h: one cell
    b = velocity(ABC, g, t)
    ref = velocity(Flow("abc"), g, 0.0)
    for c, r in zip(b, ref):
        shifted = np.roll(np.roll(np.roll(r, -1, 0), -1, 1), -1, 2)
        assert np.max(np.abs(c - shifted)) < 1e-13
    f = Operator(g, ABC, 0.1, None).forcing(t)
    _, X, Y, Z = coords(n)
    ph = 2 * math.pi / n
    assert np.max(np.abs(f - (-np.sin(Z + ph) - np.cos(Y + ph)))) < 1e-14


@pytest.mark.parametrize("flow", [KOL, ABC], ids=["kolmogorov", "abc"])
def test_fine_propagator_conserves_the_mean(flow):
    # every component b_d is independent of x_d (divergence free, discretely too) and the
    # forcing has zero mean, so the grid mean of u is invariant
    g = O.Grid(8)
    op = Operator(g, flow, 0.05, None)
    u0 = initial_state(8, seed=4) + 0.3
    u, _ = fine_propagate(op, u0, 0.4, 12, 0.01)
    assert abs(u.mean() - u0.mean()) < 1e-13


@pytest.mark.parametrize("flow", [KOL, ABC], ids=["kolmogorov", "abc"])
def test_time_dependent_coarse_with_complete_basis_equals_dense_fine(flow):
    # V = I, dT = dt: the reduced implicit Euler re-assembled at every coarse time equals
    # implicit Euler with the dense matrix of L_h(t_new) and f(t_new) at every step
    g = O.Grid(5)
    op = Operator(g, flow, 0.05, None)
    u = initial_state(5, seed=2)
    t0, dt, steps = 0.3, 0.05, 6
    x = u.reshape(-1).copy()
    for j in range(1, steps + 1):
        t = t0 + j * dt
        A = np.eye(g.Ng) + dt * O.assemble_L_dense(g, op.vel(t), op.eps)
        x = np.linalg.solve(A, x + dt * op.forcing(t).reshape(-1))
    gx, _ = coarse_propagate(op, np.eye(g.Ng), u, t0, steps, dt)
    assert np.linalg.norm(gx - x) < 1e-12 * np.linalg.norm(x)
    fx, _ = fine_propagate(op, u, t0, steps, dt)
    assert np.linalg.norm(fx.reshape(-1) - x) < 1e-12 * np.linalg.norm(x)


def test_time_dependence_matters():
    # the same step taken with the flow frozen at t0 differs: the propagators do evaluate
    # the field at the new time
    g = O.Grid(6)
    op = Operator(g, KOL, 0.05, None)
    u = initial_state(6, seed=3)
    a, _ = fine_propagate(op, u, 0.0, 4, 0.2)
    frozen = Operator(g, Flow("const"), 0.05, op.forcing(0.0))   # f frozen at t = 0
    vel0 = op.vel(0.0)
    frozen.vel = lambda t: vel0                                   # b frozen at t = 0
    b, _ = fine_propagate(frozen, u, 0.0, 4, 0.2)
    assert np.linalg.norm(a - b) > 1e-3 * np.linalg.norm(a)
