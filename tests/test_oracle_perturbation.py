"""Pins of the seeded velocity perturbation of the 256^3 Kolmogorov case and of the
oracle's operator and propagators on a perturbed flow (no GPU).  The perturbation
b' = curl_h Psi is stored per point; unlike the analytic fields, b'_d depends on x_d, so
the advection matrix is not skew-symmetric and L^T is not L with the sign of b flipped."""
import numpy as np
import pytest

import oracle as O
from oracle.coarse import coarse_propagate
from oracle.discretisation import Operator, apply_L, apply_LT, velocity
from oracle.fine import fine_propagate
from pr_inputs import Flow, initial_state, perturbation

KOL8P = Flow("kolmogorov", k=2, pert_seed=4)


def cdiv(b, h):
    return sum((np.roll(c, -1, ax) - np.roll(c, 1, ax)) / (2 * h) for c, ax in zip(b, (2, 1, 0)))


@pytest.mark.parametrize("n,seed,amp", [(8, 4, 0.05), (12, 1, 0.2), (16, 7, 0.05)])
def test_perturbation_amplitude_divergence_and_mean(n, seed, amp):
    b = perturbation(n, seed, amp)
    assert b.shape == (3, n, n, n)
    assert np.max(np.abs(b)) == pytest.approx(amp, rel=1e-15)
    h = 2 * np.pi / n
    # central differences along different axes commute: div_h curl_h = 0 to rounding
    assert np.max(np.abs(cdiv(b, h))) < 1e-14 * amp / h
    # a difference of periodic values sums to zero: every component has zero mean
    assert np.max(np.abs(b.mean(axis=(1, 2, 3)))) < 1e-15
    # the seed matters and the field is not the trivial one
    assert np.max(np.abs(b - perturbation(n, seed + 1, amp))) > 0.1 * amp


def test_perturbed_velocity_is_the_sum_and_steady_only():
    g = O.Grid(8)
    base = velocity(Flow("kolmogorov", k=2), g)
    pert = perturbation(8, 4)
    for v, b, p in zip(velocity(KOL8P, g, 0.3), base, pert):
        assert np.array_equal(v, b + p)
    with pytest.raises(ValueError):
        velocity(Flow("paper_abc", pert_seed=1), g, 0.0)


def test_perturbed_operator_matches_dense_matrix_and_its_transpose():
    g = O.Grid(6)
    vel = velocity(Flow("abc", pert_seed=2, pert_amp=0.3), g)
    A = O.assemble_L_dense(g, vel, 0.04)
    u = initial_state(6, seed=5)
    assert np.max(np.abs(apply_L(u, vel, 0.04, g.h).reshape(-1) - A @ u.reshape(-1))) < 1e-13
    assert np.max(np.abs(apply_LT(u, vel, 0.04, g.h).reshape(-1) - A.T @ u.reshape(-1))) < 1e-13
    # advection part only: not skew-symmetric any more (b'_d varies along x_d) ...
    Ad = O.assemble_L_dense(g, vel, 0.0)
    assert np.max(np.abs(Ad + Ad.T)) > 1e-3
    # ... but its columns still sum to zero (discrete divergence zero): sum_i (A u)_i = 0
    assert np.max(np.abs(Ad.sum(axis=0))) < 1e-13


def test_perturbed_fine_step_equals_dense_solve_and_conserves_the_mean():
    g = O.Grid(6)
    op = Operator(g, Flow("kolmogorov", k=1, pert_seed=3, pert_amp=0.3), 0.02, None)
    u = initial_state(6, seed=2) + 0.2
    dt, steps = 0.05, 5
    A = np.eye(g.Ng) + dt * O.assemble_L_dense(g, op.vel(0.0), op.eps)
    x = u.reshape(-1).copy()
    for _ in range(steps):
        x = np.linalg.solve(A, x)
    fx, _ = fine_propagate(op, u, 0.0, steps, dt)
    assert np.linalg.norm(fx.reshape(-1) - x) < 1e-12 * np.linalg.norm(x)
    assert abs(fx.mean() - u.mean()) < 1e-14


def test_perturbed_complete_basis_coarse_equals_fine():
    g = O.Grid(5)
    op = Operator(g, Flow("abc", pert_seed=5, pert_amp=0.2), 0.05, None)
    u = initial_state(5, seed=2)
    gx, _ = coarse_propagate(op, np.eye(g.Ng), u, 0.1, 4, 0.03)
    fx, _ = fine_propagate(op, u, 0.1, 4, 0.03)
    assert np.linalg.norm(gx - fx.reshape(-1)) < 1e-12 * np.linalg.norm(fx)


def test_perturbation_changes_the_solution():
    g = O.Grid(8)
    u = initial_state(8, seed=1)
    a, _ = fine_propagate(Operator(g, Flow("kolmogorov", k=2), 0.01, None), u, 0.0, 10, 0.02)
    b, _ = fine_propagate(Operator(g, KOL8P, 0.01, None), u, 0.0, 10, 0.02)
    assert np.linalg.norm(a - b) > 1e-4 * np.linalg.norm(a)


def test_parareal_II_coarse_operator_injects_the_stored_perturbation():
    from oracle.coarse import restrict
    from oracle.parareal import coarse_operator
    g = O.Grid(8)
    op = Operator(g, KOL8P, 0.02, None)
    opc = coarse_operator(op, 2)
    full = perturbation(8, KOL8P.pert_seed, KOL8P.pert_amp)
    base_c = velocity(Flow("kolmogorov", k=2), opc.grid)
    for d, v in enumerate(opc.vel(0.0)):
        assert np.array_equal(v, base_c[d] + restrict(full[d], 2))
    # not the field drawn afresh on the coarse grid
    assert np.max(np.abs(opc.pert - perturbation(4, KOL8P.pert_seed, KOL8P.pert_amp))) > 1e-3
