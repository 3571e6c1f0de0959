"""POD of snapshot matrices: Algorithm 1 (POD_Mode) and the two-level POD of Case II.

POD_Mode(W, gamma) (Sec. 2.3, Case I, and Algorithm 1), with M = I (reading R1):
  1. eigen-decompose the Gram matrix W^T M W: lambda_1 >= ... >= lambda_r > 0 = ...;
  2. m = min{ k : sum_{i<=k} sqrt(lambda_i) >= gamma * sum_{i<=r} sqrt(lambda_i) }
     (the paper sums square roots of the eigenvalues; kept as printed, reading R6);
  3. R_tilde = first m columns of R, r_i = W y_i / sqrt(lambda_i).
Readings: "lambda = 0" means lambda_i <= tau * lambda_1 (R5); an optional cap bounds m
(R6); the returned basis is re-orthonormalised by one Cholesky QR pass, which keeps its
span (R7).  R = W Y Lambda^{-1/2} is orthonormal up to eps * lambda_1 / lambda_m; one
Cholesky QR pass brings that to rounding level, its error being eps * cond(R)^2 with
cond(R) ~ 1.

Case II level 2, eq. (W^k_n): the level-1 bases of the m_l left neighbours, of this
subinterval and of the p previous iterations are concatenated and compressed again
with gamma_3.
"""
from __future__ import annotations

import numpy as np


def pod_select(lam: np.ndarray, gamma: float, tau: float, cap: int = 0) -> int:
    """POD dimension m from eigenvalues sorted in descending order (Algorithm 1, step 2)."""
    if lam.size == 0 or lam[0] <= 0.0:
        return 0
    r = int(np.sum(lam > tau * lam[0]))
    sq = np.sqrt(lam[:r])
    total = np.sum(sq)
    csum = np.cumsum(sq)
    m = int(np.argmax(csum >= gamma * total)) + 1
    if cap > 0:
        m = min(m, cap)
    return min(m, r)


def cholqr(R: np.ndarray, passes: int = 1) -> np.ndarray:
    """Cholesky QR: R <- R L^{-T} with R^T R = L L^T (reading R7), `passes` times."""
    for _ in range(passes):
        G = R.T @ R
        Lc = np.linalg.cholesky(G)
        R = np.linalg.solve(Lc, R.T).T     # R L^{-T}
    return R


def pod_mode(W: np.ndarray, gamma: float, cap: int = 0, tau: float = 1e-13,
             reorth: bool = True):
    """Algorithm 1.  W is N_g x n_s.  Returns (R_tilde (N_g x m), m, lambda)."""
    G = W.T @ W
    lam, Y = np.linalg.eigh(G)
    order = np.argsort(lam)[::-1]
    lam, Y = lam[order], Y[:, order]
    m = pod_select(lam, gamma, tau, cap)
    if m == 0:
        return np.zeros((W.shape[0], 0)), 0, lam
    R = W @ Y[:, :m] / np.sqrt(lam[:m])
    if reorth:
        R = cholqr(R)
    return R, m, lam


def level2_blocks(level1, k: int, n: int, m_l: int, p: int, V0):
    """The blocks of W^k_n, eq. (W^k_n):
        [R^k_{n-m_l,0}, ..., R^k_{n,0}, R^{k-1}_{n,0}, ..., R^{k-p}_{n,0}].

    level1(kk, nn) returns the level-1 basis of subinterval nn at iteration kk, or None if
    it does not exist (nn < 0 or kk < 1).  A missing block is replaced by the Case-I
    basis V0, at most once (reading R8).
    """
    blocks = []
    used_v0 = False
    wanted = [(k, n - j) for j in range(m_l, -1, -1)] + [(k - j, n) for j in range(1, p + 1)]
    for kk, nn in wanted:
        B = level1(kk, nn) if (kk >= 1 and nn >= 0) else None
        if B is None:
            if used_v0:
                continue
            B = V0
            used_v0 = True
        blocks.append(B)
    return blocks
