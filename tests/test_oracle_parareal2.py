"""Pins of the oracle's comparator "Parareal-II" (Sec. 4: plain parareal whose coarse
propagator works on a coarser grid), no GPU: restriction by injection and trilinear
prolongation against their definitions on polynomials and modes, the coarse-grid
propagator, finite termination, and the one-iteration limit G = F."""
import math

import numpy as np
import pytest

import oracle as O
import pr_inputs as pi
from oracle.coarse import coarse_grid_propagate, prolong, restrict
from oracle.discretisation import Grid, Operator
from oracle.fine import fine_propagate
from oracle.parareal import coarse_operator


def test_injection_of_the_interpolant_is_the_identity():
    uc = np.random.default_rng(0).standard_normal((5, 5, 5))
    for c in (2, 3):
        assert np.array_equal(restrict(prolong(uc, c), c), uc)


def test_prolongation_is_trilinear_on_the_periodic_grid():
    rng = np.random.default_rng(1)
    uc = rng.standard_normal((4, 4, 4))
    u = prolong(uc, 2)
    # a fine point between two coarse points along x is their mean, the cell centre the
    # mean of its eight corners
    assert abs(u[0, 0, 1] - 0.5 * (uc[0, 0, 0] + uc[0, 0, 1])) < 1e-15
    assert abs(u[0, 0, 7] - 0.5 * (uc[0, 0, 3] + uc[0, 0, 0])) < 1e-15      # wraps
    corners = [uc[z, y, x] for z in (1, 2) for y in (2, 3) for x in (0, 1)]
    assert abs(u[3, 5, 1] - np.mean(corners)) < 1e-15
    # a function linear in one direction within a period is reproduced between nodes
    lin = np.tile(np.arange(4.0)[None, None, :], (4, 4, 1))
    assert np.allclose(prolong(lin, 2)[:, :, 3], 1.5)
    assert np.allclose(prolong(np.full((3, 3, 3), 2.5), 3), 2.5)


def test_restriction_of_a_resolved_mode_is_its_coarse_sampling():
    n, c = 12, 2
    g = Grid(n)
    X, Y, Z = g.coords()
    u = np.sin(X + 2 * Y) * np.cos(Z) * np.ones((n,) * 3)
    gc = Grid(n // c)
    Xc, Yc, Zc = gc.coords()
    assert np.max(np.abs(restrict(u, c) - np.sin(Xc + 2 * Yc) * np.cos(Zc))) < 1e-15


def test_coarse_grid_propagator_is_implicit_euler_on_the_coarse_problem():
    w = pi.tiny(n=8, n_sub=2, f_seed=3)
    op = O.make_operator(w)
    op_c = coarse_operator(op, 2)
    assert op_c.grid.n == 4 and np.array_equal(op_c.f, op.f[::2, ::2, ::2])
    x = w.u0()
    got = coarse_grid_propagate(op_c, x, 0.3, 3, 0.01, 2)
    uc, _ = fine_propagate(op_c, x[::2, ::2, ::2].copy(), 0.3, 3, 0.01, tol=1e-14)
    assert np.array_equal(got, prolong(uc, 2))


def test_parareal_II_reaches_the_sequential_solution_at_k_equals_N():
    w = pi.tiny(n=8, n_sub=4, T=0.08, dt=2e-3, f_seed=2)
    prm = O.derive_params(w, method="parareal_II")
    ref = O.sequential_fine(w, prm)
    hist = O.parareal(w, prm, reference=ref)
    assert hist["k"] == w.n_sub
    assert max(hist["err"][0]) > 1e-4
    assert max(hist["err"][-1]) < 1e-13


def test_parareal_II_without_coarsening_and_dT_dt_converges_in_one_iteration():
    # coarse_factor 1 and dT = dt make G = F exactly
    w = pi.tiny(n=6, n_sub=3, T=0.03, dt=2e-3, f_seed=1)
    prm = O.derive_params(w, dT=2e-3, method="parareal_II", coarse_factor=1)
    ref = O.sequential_fine(w, prm)
    hist = O.parareal(w, prm, k_max=1, reference=ref)
    assert max(hist["err"][1]) < 1e-12
