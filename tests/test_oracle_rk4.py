"""Pins of the oracle's explicit fine integrator (classical Runge-Kutta, fourth order) on
u' = -L_h(t) u + f(t) (no GPU): the amplification polynomial on a Fourier mode, fourth-
order convergence to the exact solution of the semi-discrete mode equation, invariants,
and parareal finite termination with this fine propagator."""
import cmath
import math

import numpy as np
import pytest

import oracle as O
import pr_inputs as pi
from oracle.discretisation import Operator
from oracle.fine import fine_propagate_rk4, rk4_step
from pr_inputs import Flow, initial_state
from test_oracle_operator import symbol


def mode(n, k):
    g = O.Grid(n)
    X, Y, Z = g.coords()
    return g, (k[0] * X + k[1] * Y + k[2] * Z) * np.ones((n,) * 3)


@pytest.mark.parametrize("k", [(1, 2, 0), (3, -1, 2)])
def test_rk4_multiplies_a_mode_by_its_amplification_polynomial(k):
    # u = Re(exp(i k.x)), L_h u = Re(lambda exp(i k.x)): each step multiplies the complex
    # amplitude by R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24, z = -dt lambda
    b = (1.1, 0.5, -0.8)
    eps, dt, steps = 0.05, 0.02, 5
    g, ph = mode(12, k)
    op = Operator(g, Flow("const", b0=b[0], b1=b[1], b2=b[2]), eps, None)
    z = -dt * symbol(k, b, eps, g.h)
    R = 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    u, _ = fine_propagate_rk4(op, np.cos(ph), 0.0, steps, dt)
    assert np.max(np.abs(u - np.real(R ** steps * np.exp(1j * ph)))) < 1e-13


def test_rk4_is_fourth_order():
    # error against exp(-lambda t) shrinks 16-fold per halving of dt
    k, b, eps, T = (2, 1, 0), (0.9, -0.4, 0.3), 0.1, 0.4
    g, ph = mode(10, k)
    op = Operator(g, Flow("const", b0=b[0], b1=b[1], b2=b[2]), eps, None)
    lam = symbol(k, b, eps, g.h)
    exact = np.real(cmath.exp(-lam * T) * np.exp(1j * ph))
    errs = []
    for steps in (4, 8, 16):
        u, _ = fine_propagate_rk4(op, np.cos(ph), 0.0, steps, T / steps)
        errs.append(np.max(np.abs(u - exact)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 14 < r1 < 18 and 14 < r2 < 18, (r1, r2)


def test_rk4_stages_see_their_own_times():
    # u' = f(t) with L = 0 (b = 0, eps tiny) integrates f exactly for cubic time
    # dependence; with the paper's forcing -cos y - sin z cos t the quadrature error of
    # one step is O(dt^5): compare with the exact integral
    g = O.Grid(6)
    op = Operator(g, Flow("paper_kolmogorov"), 1e-300, None)
    op.vel = lambda t: (0.0, 0.0, 0.0)
    X, Y, Z = g.coords()
    u0 = np.zeros((6, 6, 6))
    t, dt = 0.3, 0.1
    u1 = rk4_step(op, u0, t, dt)
    exact = (-np.cos(Y) * dt - np.sin(Z) * (math.sin(t + dt) - math.sin(t))) * np.ones((6,) * 3)
    assert np.max(np.abs(u1 - exact)) < 1e-7


@pytest.mark.parametrize("flow", [Flow("abc"), Flow("paper_abc", w=1.0)], ids=["abc", "paper_abc"])
def test_rk4_conserves_the_mean(flow):
    g = O.Grid(8)
    op = Operator(g, flow, 0.05, None)
    u0 = initial_state(8, seed=5) + 0.2
    u, _ = fine_propagate_rk4(op, u0, 0.1, 10, 0.01)
    assert abs(u.mean() - u0.mean()) < 1e-14


def test_parareal_with_rk4_fine_propagator_terminates_on_its_sequential_solution():
    w = pi.tiny(n=6, n_sub=4, T=0.04, dt=2e-3, f_seed=3)
    prm = O.derive_params(w, fine="rk4")
    ref = O.sequential_fine(w, prm)
    hist = O.parareal(w, prm, reference=ref)
    assert max(hist["err"][-1]) < 1e-13
    # and the reference really is the explicit one: it differs from implicit Euler by O(dt)
    ref_ie = O.sequential_fine(w, O.derive_params(w))
    assert O.rel_l2(ref[-1], ref_ie[-1]) > 1e-6
