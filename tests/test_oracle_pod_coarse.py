"""Pins of the oracle's POD (Algorithm 1, Case II) and coarse propagator (eqs. (eq8),
(eq13), (eqaug)) against the SVD, hand-computed criteria, exact reconstruction and
dense/complete-basis brute force (no GPU)."""
import numpy as np
import pytest

import oracle as O
from oracle.coarse import augment, coarse_propagate, galerkin_project
from oracle.discretisation import Operator
from oracle.fine import fine_propagate
from oracle.pod import cholqr, level2_blocks, pod_mode, pod_select
from pr_inputs import Flow, forcing, initial_state


def rng(seed=0):
    return np.random.default_rng(seed)


def test_pod_eigenvalues_are_squared_singular_values():
    W = rng(1).standard_normal((500, 12))
    _, _, lam = pod_mode(W, 1.0)
    s = np.linalg.svd(W, compute_uv=False)
    assert np.allclose(lam, s ** 2, rtol=1e-12, atol=0)


def test_pod_basis_orthonormal_and_reconstructs_full_rank_snapshots():
    W = rng(2).standard_normal((400, 9)) @ np.diag(np.logspace(0, -3, 9))
    R, m, _ = pod_mode(W, 1.0, cap=0, tau=1e-13)
    assert m == 9
    assert np.max(np.abs(R.T @ R - np.eye(m))) < 1e-13
    assert np.linalg.norm(W - R @ (R.T @ W)) < 1e-12 * np.linalg.norm(W)


def test_pod_recovers_span_of_rank_deficient_snapshots():
    A = rng(3).standard_normal((300, 4))
    B = rng(4).standard_normal((10, 4))
    W = A @ B.T                     # rank 4, 10 snapshots
    R, m, lam = pod_mode(W, 1.0, tau=1e-10)
    assert m == 4
    assert np.all(lam[4:] <= 1e-10 * lam[0])
    P = R @ R.T
    assert np.linalg.norm(P @ A - A) < 1e-10 * np.linalg.norm(A)


def test_pod_modes_are_scaled_snapshot_combinations():
    # r_i = W y_i / sqrt(lambda_i) before re-orthonormalisation has unit norm and
    # spans the leading eigenvectors of W W^T
    W = rng(5).standard_normal((200, 6))
    R, m, lam = pod_mode(W, 1.0, reorth=False)
    assert np.allclose(np.linalg.norm(R, axis=0), 1.0, atol=1e-12)
    U, s, _ = np.linalg.svd(W, full_matrices=False)
    for i in range(m):
        assert abs(abs(U[:, i] @ R[:, i]) - 1.0) < 1e-10


@pytest.mark.parametrize("gamma,cap,expect", [
    (0.9, 0, 1), (0.95, 0, 2), (0.999, 0, 3), (1.0, 0, 3), (1.0, 2, 2)])
def test_criterion_sums_square_roots(gamma, cap, expect):
    # sqrt(lambda) = 10, 1, 0.1, 1e-10 ; the last is numerically zero (tau = 1e-13)
    lam = np.array([100.0, 1.0, 0.01, 1e-20])
    assert pod_select(lam, gamma, 1e-13, cap) == expect


def test_criterion_distinguishes_sqrt_from_plain_eigenvalues():
    lam = np.array([100.0, 1.0, 0.01])
    # sum of sqrt: 11.1, 0.99*11.1 = 10.989 > 10 -> m = 2 (plain sums would give m = 1)
    assert pod_select(lam, 0.99, 1e-13) == 2


def test_criterion_zero_snapshots():
    assert pod_select(np.zeros(5), 0.9, 1e-13) == 0


def test_cholqr_keeps_span_and_orthonormalises():
    R0 = rng(6).standard_normal((300, 7)) @ np.triu(rng(7).standard_normal((7, 7)) + 3 * np.eye(7))
    Q = cholqr(R0, passes=2)
    assert np.max(np.abs(Q.T @ Q - np.eye(7))) < 1e-14
    assert np.linalg.norm(Q @ (Q.T @ R0) - R0) < 1e-12 * np.linalg.norm(R0)


def test_one_cholqr_pass_orthonormalises_pod_projections():
    # R = W Y Lambda^{-1/2} of snapshots with a 1e-11 eigenvalue ratio is orthonormal only
    # to ~1e-7; one Cholesky QR pass restores rounding-level orthonormality (reading R7)
    A = np.linalg.qr(rng(8).standard_normal((2000, 6)))[0] @ np.diag(np.logspace(0, -5.5, 6))
    W = A @ np.linalg.qr(rng(9).standard_normal((6, 6)))[0]
    lam, Y = np.linalg.eigh(W.T @ W)
    o = np.argsort(lam)[::-1]
    R = W @ Y[:, o] / np.sqrt(lam[o])
    assert np.max(np.abs(R.T @ R - np.eye(6))) > 1e-9
    Q = cholqr(R)
    assert np.max(np.abs(Q.T @ Q - np.eye(6))) < 1e-14


def test_level2_blocks_order_and_missing_blocks():
    store = {(2, 3): "R2_3", (2, 4): "R2_4", (1, 4): "R1_4", (2, 2): "R2_2"}
    get = lambda kk, nn: store.get((kk, nn))
    assert level2_blocks(get, 2, 4, 1, 1, "V0") == ["R2_3", "R2_4", "R1_4"]
    assert level2_blocks(get, 2, 4, 2, 0, "V0") == ["R2_2", "R2_3", "R2_4"]
    assert level2_blocks(get, 2, 4, 0, 0, "V0") == ["R2_4"]
    # iteration 1: previous-iteration block missing -> V0 once
    assert level2_blocks(get, 1, 4, 0, 2, "V0") == ["R1_4", "V0"]


def test_augmentation_makes_U_exactly_representable():
    R, _ = np.linalg.qr(rng(8).standard_normal((256, 5)))
    U = rng(9).standard_normal(256)
    V, augd = augment(R, U)
    assert augd and V.shape[1] == 6
    assert np.max(np.abs(V.T @ V - np.eye(6))) < 1e-14
    P_U = V @ np.linalg.solve(V.T @ V, V.T @ U)
    assert np.linalg.norm(P_U - U) < 1e-13 * np.linalg.norm(U)


def test_augmentation_skipped_when_U_in_span():
    R, _ = np.linalg.qr(rng(10).standard_normal((256, 5)))
    U = R @ np.array([1.0, -2.0, 0.5, 0.0, 3.0])
    V, augd = augment(R, U)
    assert not augd and V.shape[1] == 5


def test_galerkin_matrices_match_dense_projection():
    g = O.Grid(8)
    op = Operator(g, Flow("abc"), 0.03, None)
    V, _ = np.linalg.qr(rng(11).standard_normal((512, 6)))
    Mv, Lv = galerkin_project(op, V, 0.0)
    A = O.assemble_L_dense(g, op.vel(0.0), op.eps)
    assert np.max(np.abs(Mv - np.eye(6))) < 1e-14
    assert np.max(np.abs(Lv - V.T @ A @ V)) < 1e-11


@pytest.mark.parametrize("with_f", [False, True])
def test_complete_basis_coarse_equals_fine(with_f):
    # V = identity (every grid function representable) and dT = dt: the reduced
    # implicit Euler of eq. (eq8) is the fine implicit Euler of eq. (algform).
    g = O.Grid(6)
    op = Operator(g, Flow("abc"), 0.05, forcing(6, seed=3) if with_f else None)
    V = np.eye(g.Ng)
    u0 = initial_state(6, seed=2)
    gx, _ = coarse_propagate(op, V, u0, 0.2, 7, 0.01)
    A = O.assemble_L_dense(g, op.vel(0.0), op.eps)
    fx, _ = fine_propagate(op, u0, 0.2, 7, 0.01, dense_A=A)
    assert np.linalg.norm(gx - fx.reshape(-1)) < 1e-12 * np.linalg.norm(fx)


def test_coarse_propagator_invariant_to_basis_rotation():
    g = O.Grid(8)
    op = Operator(g, Flow("kolmogorov", k=2), 0.02, forcing(8, seed=1))
    V, _ = np.linalg.qr(rng(12).standard_normal((512, 5)))
    Q, _ = np.linalg.qr(rng(13).standard_normal((5, 5)))
    x = initial_state(8)
    a, _ = coarse_propagate(op, V, x, 0.0, 4, 0.02)
    b, _ = coarse_propagate(op, V @ Q, x, 0.0, 4, 0.02)
    assert np.linalg.norm(a - b) < 1e-13 * np.linalg.norm(a)


def test_augmented_coarse_propagator_independent_of_gram_schmidt_passes():
    # Reading R11: G in V = [R, d~ / ||d~||] depends only on span{R, U}, so one
    # Gram-Schmidt pass (the CUDA sweep) and two (the oracle's augment) give the same G to
    # rounding, the mass matrix V^T V absorbing what one pass leaves in span R.  Also for
    # a basis that is orthonormal only to ~1e-9 and for U close to span R.
    g = O.Grid(8)
    op = Operator(g, Flow("abc"), 0.03, forcing(8, seed=2))
    R, _ = np.linalg.qr(rng(14).standard_normal((512, 5)))
    for noise, near in ((0.0, 1.0), (1e-9, 1.0), (0.0, 1e-6)):
        Rn = R + noise * rng(15).standard_normal(R.shape)
        U = Rn @ rng(16).standard_normal(5) + near * rng(17).standard_normal(512)
        V2, augd = augment(Rn, U)
        assert augd
        d1 = U - Rn @ (Rn.T @ U)
        V1 = np.concatenate([Rn, (d1 / np.linalg.norm(d1))[:, None]], axis=1)
        a, _ = coarse_propagate(op, V2, U, 0.1, 6, 0.02)
        b, _ = coarse_propagate(op, V1, U, 0.1, 6, 0.02)
        assert np.linalg.norm(a - b) < 1e-11 * np.linalg.norm(a), (noise, near)
        # a different direction (d~ of another vector) does change G
        w = rng(18).standard_normal(512)
        dw = w - Rn @ (Rn.T @ w)
        e, _ = coarse_propagate(op, np.concatenate([Rn, (dw / np.linalg.norm(dw))[:, None]], axis=1), U, 0.1,
                                6, 0.02)
        assert np.linalg.norm(e - a) > 1e-6 * np.linalg.norm(a)
