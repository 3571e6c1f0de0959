"""Pins of the oracle's operator and fine propagator against closed forms, brute force
and invariants (no GPU).

* Fourier symbol: for constant b and u = exp(i k.x) the FD operator of eq. (eq1) acts as
  multiplication by  lambda_h(k) = eps sum_j 4 sin^2(k_j h/2)/h^2 + i sum_j b_j sin(k_j h)/h,
  and one implicit Euler step, eq. (semi-dis-eq), divides the mode by 1 + dt lambda_h.
* Dense brute force: the operator assembled entry by entry on an 8^3 grid, and the dense
  LU solve of the implicit Euler system, against the matrix-free operator and BiCGStab.
* Invariants: mean conservation for a discretely divergence-free flow with zero-mean
  forcing, skew-symmetry of central advection, energy decay without forcing.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle.discretisation import Operator
from oracle.fine import SolverError, bicgstab, fine_propagate, implicit_euler_step
from pr_inputs import Flow, initial_state, forcing


def symbol(k, b, eps, h):
    lam = 0.0 + 0.0j
    for kj, bj in zip(k, b):
        lam += eps * 4.0 * math.sin(kj * h / 2.0) ** 2 / h ** 2 + 1j * bj * math.sin(kj * h) / h
    return lam


@pytest.mark.parametrize("k", [(1, 0, 0), (2, -3, 1), (0, 5, 7), (4, 4, 4)])
def test_fourier_symbol_of_L_and_LT(k):
    g = O.Grid(16)
    b = (0.7, -1.3, 0.4)
    flow = Flow("const", b0=b[0], b1=b[1], b2=b[2])
    eps = 0.03
    X, Y, Z = g.coords()
    u = np.exp(1j * (k[0] * X + k[1] * Y + k[2] * Z)) * np.ones((16,) * 3)
    vel = O.velocity(flow, g)
    lam = symbol(k, b, eps, g.h)
    Lu = O.apply_L(u, vel, eps, g.h)
    assert np.max(np.abs(Lu - lam * u)) < 1e-11 * max(1.0, abs(lam))
    # L^T has the conjugate symbol (advection flips sign)
    LTu = O.apply_LT(u, vel, eps, g.h)
    assert np.max(np.abs(LTu - np.conj(lam) * u)) < 1e-11 * max(1.0, abs(lam))


@pytest.mark.parametrize("k", [(1, 2, 0), (3, -1, 2)])
def test_implicit_euler_divides_mode_by_one_plus_dt_lambda(k):
    g = O.Grid(12)
    b = (1.1, 0.5, -0.8)
    eps, dt = 0.05, 0.01
    op = Operator(g, Flow("const", b0=b[0], b1=b[1], b2=b[2]), eps, None)
    X, Y, Z = g.coords()
    ph = (k[0] * X + k[1] * Y + k[2] * Z) * np.ones((12,) * 3)
    u0 = np.cos(ph)
    u1, its = implicit_euler_step(op, u0, dt, dt, tol=1e-15)
    amp = 1.0 / (1.0 + dt * symbol(k, b, eps, g.h))
    expect = np.real(amp * np.exp(1j * ph))
    assert its > 0
    assert np.max(np.abs(u1 - expect)) < 1e-13


def test_dense_assembly_matches_matrix_free_operator():
    g = O.Grid(8)
    vel = O.velocity(Flow("abc", A=1.0, B=0.7, C=1.3), g)
    eps = 0.02
    A = O.assemble_L_dense(g, vel, eps)
    u = initial_state(8, seed=11)
    assert np.allclose(O.apply_L(u, vel, eps, g.h).reshape(-1), A @ u.reshape(-1),
                       rtol=0, atol=1e-12)
    assert np.allclose(O.apply_LT(u, vel, eps, g.h).reshape(-1), A.T @ u.reshape(-1),
                       rtol=0, atol=1e-12)


def test_bicgstab_step_matches_dense_lu_on_8cubed():
    g = O.Grid(8)
    f = forcing(8, seed=5)
    op = Operator(g, Flow("abc"), 0.05, f)
    A = O.assemble_L_dense(g, op.vel(0.0), op.eps)
    u = initial_state(8, seed=3)
    for j in range(1, 6):
        ub, its = implicit_euler_step(op, u, j * 0.01, 0.01, tol=1e-15)
        ud, _ = implicit_euler_step(op, u, j * 0.01, 0.01, dense_A=A)
        assert its >= 1
        assert np.linalg.norm(ub - ud) <= 1e-13 * np.linalg.norm(ud)
        u = ud


def test_mean_conserved_for_divergence_free_flow_and_zero_mean_forcing():
    g = O.Grid(10)
    f = forcing(10, seed=9)
    assert abs(f.mean()) < 1e-15
    op = Operator(g, Flow("abc"), 0.01, f)
    u0 = initial_state(10, seed=4) + 0.3
    u, _ = fine_propagate(op, u0, 0.0, 20, 0.01, tol=1e-15)
    assert abs(u.mean() - u0.mean()) < 1e-13


@pytest.mark.parametrize("flow", [Flow("abc"), Flow("kolmogorov", k=2),
                                  Flow("paper_kolmogorov"), Flow("paper_abc")])
def test_central_advection_is_skew(flow):
    g = O.Grid(10)
    vel = O.velocity(flow, g, t=0.37)
    u = initial_state(10, seed=1)
    v = forcing(10, seed=2)
    a = np.vdot(v, O.apply_L(u, vel, 0.0, g.h))
    b = np.vdot(O.apply_L(v, vel, 0.0, g.h), u)
    assert abs(a + b) < 1e-12 * (abs(a) + 1e-300) + 1e-12


def test_energy_decays_without_forcing():
    g = O.Grid(10)
    op = Operator(g, Flow("kolmogorov", k=3), 0.02, None)
    u = initial_state(10, seed=6)
    e_prev = np.linalg.norm(u)
    for j in range(1, 11):
        u, _ = implicit_euler_step(op, u, j * 0.01, 0.01, tol=1e-15)
        e = np.linalg.norm(u)
        assert e <= e_prev * (1 + 1e-14)
        e_prev = e


def test_snapshots_are_states_at_multiples_of_dM():
    g = O.Grid(8)
    op = Operator(g, Flow("abc"), 0.05, None)
    u0 = initial_state(8)
    uS, W = fine_propagate(op, u0, 0.0, 10, 0.01, dM=5, n_snap=3, tol=1e-15)
    u5, _ = fine_propagate(op, u0, 0.0, 5, 0.01, tol=1e-15)
    assert np.array_equal(W[:, 0], u0.reshape(-1))
    assert np.array_equal(W[:, 1], u5.reshape(-1))
    assert np.array_equal(W[:, 2], uS.reshape(-1))


def test_bicgstab_reports_nonconvergence():
    g = O.Grid(8)
    op = Operator(g, Flow("abc"), 0.05, None)
    u0 = initial_state(8)
    with pytest.raises(SolverError):
        implicit_euler_step(op, u0, 0.5, 0.5, tol=1e-15, maxit=1)


def test_bicgstab_zero_rhs_converges_immediately():
    x, its = bicgstab(lambda v: 2.0 * v, np.zeros(5), np.zeros(5), 1e-14)
    assert its == 0 and not x.any()
