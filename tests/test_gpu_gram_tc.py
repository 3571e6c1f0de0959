"""The tensor-core Gram (pr_op_gram, tensor = 1): G = W^T W of FP64 columns from error-free
BF16 digit products on tcgen05, against exactly rounded sums and the FP64 kernel.

Step 1 of POD_Mode (Algorithm 1) needs the Gram to ~1e-14 of its norm (larger errors
move eigenvalues at the rank threshold, see the parity notes).  The digit scheme loses
only the truncation of each value to 2^-53 of its column's largest magnitude (so at most
2^-53 (max|x| sum|y| + max|y| sum|x|) in an entry) and the FP64 additions of the partial
sums (like any FP64 Gram); each entry is checked against that bound with a factor 4 of
slack, and against the FP64 kernel at 1e-14 of the Gram's largest entry.
"""
import math

import numpy as np
import pytest

import pr_inputs as pi

pytestmark = pytest.mark.gpu


def _exact_dot(x, y):
    """The exactly rounded sum of x_p y_p: every product split into two doubles (Dekker,
    Veltkamp splitting), then math.fsum."""
    c = 134217729.0   # 2^27 + 1
    def split(a):
        t = c * a
        hi = t - (t - a)
        return hi, a - hi
    xh, xl = split(x)
    yh, yl = split(y)
    p = x * y
    e = ((xh * yh - p) + xh * yl + xl * yh) + xl * yl
    return math.fsum(np.concatenate([p, e]))


def _columns(n, K, B, seed):
    rng = np.random.default_rng(seed)
    Ng = n ** 3
    W = np.empty((B, K, Ng))
    for b in range(B):
        for i in range(K):
            f = pi.initial_state(n, seed=100 * b + i + 1).reshape(-1)
            scale = 10.0 ** rng.uniform(-3, 3)
            W[b, i] = scale * (f + 1e-3 * rng.standard_normal(Ng))
    if K > 2:
        W[0, 1] = 0.0                  # a zero column
        W[0, 2] = W[0, 0] * (1 + 1e-9)  # a nearly parallel one
    return W


@pytest.mark.parametrize("n,K,B", [(8, 5, 1), (12, 33, 2), (16, 64, 3)])
def test_tensor_gram_matches_exact_sums(gpu, n, K, B):
    bd, torch = gpu
    w = pi.Workload("gram", n, pi.Flow("abc"), 0.05, 1.0, 4, 1e-3, n_snap=64, m_cap=32)
    s = bd.Parareal.from_workload(w, precision=bd.PR_FP32)
    W = _columns(n, K, B, seed=K)
    Wt = torch.from_numpy(W).to("cuda")
    Gt = s.op_gram(Wt, tensor=True).cpu().numpy()
    G64 = s.op_gram(Wt, tensor=False).cpu().numpy()
    s.close()
    worst_tc = worst_64 = 0.0
    for b in range(B):
        for i in range(K):
            for j in range(i, K):
                if K > 16 and (i * 7 + j * 13) % 5:   # a sample of the entries at larger K
                    continue
                ex = _exact_dot(W[b, i], W[b, j])
                x, y = W[b, i], W[b, j]
                bound = 2.0 ** -50 * float(np.sum(np.abs(x * y)) + np.abs(x).max() * np.abs(y).sum()
                                          + np.abs(y).max() * np.abs(x).sum()) + 1e-300
                worst_tc = max(worst_tc, abs(Gt[b, i, j] - ex) / bound)
                worst_64 = max(worst_64, abs(G64[b, i, j] - ex) / bound)
                assert Gt[b, i, j] == Gt[b, j, i]
    print(f"n={n} K={K} B={B}: Gram error / bound: tensor cores {worst_tc:.3f}, FP64 kernel {worst_64:.3f}")
    assert worst_tc < 1.0, worst_tc
    rel = np.abs(Gt - G64).max() / np.abs(G64).max()
    assert rel < 1e-14, rel


@pytest.mark.parametrize("wl", ["tiny_forced", "abc16"])
def test_fp32_mode_with_tensor_grams_against_oracle(gpu, wl):
    """The FP32 mode with every symmetric POD Gram on the tensor cores (level 1 and the
    Cholesky-QR Grams, PR_GRAM_TENSOR) against the FP64 oracle, within the FP32-mode bar
    max(1e-5, 10 x the oracle's change under 1e-8 fine perturbations) at every (k, n)."""
    import oracle as O
    from test_gpu_parity import TOL32, oracle_envelope, rel
    bd, torch = gpu
    w = {"tiny_forced": pi.tiny(n=10, n_sub=5, T=0.1, dt=2e-3, f_seed=2, flow=pi.Flow("kolmogorov", k=2)),
         "abc16": pi.ABC_16}[wl]
    prm = O.derive_params(w)
    K = min(w.n_sub, 3)
    hist, env = oracle_envelope(w, prm, K, 1e-8, where="fine")
    s = bd.Parareal.from_workload(w, precision=bd.PR_FP32, gram_mode=bd.PR_GRAM_TENSOR)
    s.set_initial(w.u0(), w.f())
    s.iteration0()
    Us = [s.interfaces()]
    for k in range(1, K + 1):
        s.iterate(k)
        Us.append(s.interfaces())
    s.close()
    worst = 0.0
    for k in range(K + 1):
        for n in range(w.n_sub + 1):
            e = rel(Us[k][n], hist["U"][k][n])
            tol = max(TOL32, 10 * env[k][n])
            worst = max(worst, e / tol)
            assert e < tol, (k, n, e, env[k][n])
    print(f"{wl} FP32 mode, tensor-core Grams: worst error / tolerance {worst:.3f}")


# ---- the narrow form (K <= 32): bit-exact against a digit-level emulation ----------------
#
# For K <= 32 columns the kernel sums the digit products exactly (128-bit integers) and
# rounds once, so its result is a function of the inputs alone: each value truncated
# toward zero to y = trunc(x 2^(56 - e)) (e = exponent of the column's largest magnitude
# + 3), y cut into balanced base-128 digits D_0 (most significant) .. D_7, and
#   G[i, j] = round( sum_{s, t: min(s, t) <= 3} 2^(-7 (s + t + 2)) sum_p D_s(p, i) D_t(p, j)
#                    * 2^(e_i + e_j) ).
# The emulation below computes that with Python integers (no code shared with the kernel).

def _col_exp(x):
    m = float(np.abs(x).max())
    if m == 0.0:
        return 0
    return math.frexp(m)[1] - 1 + 3          # unbiased exponent of the maximum, + 3


def _digits(x, e):
    y = np.trunc(np.ldexp(x, 56 - e)).astype(np.int64)   # exact: |y| < 2^54
    z = y + sum(64 << (7 * k) for k in range(8))
    return np.stack([((z >> (7 * (7 - s))) & 127) - 64 for s in range(8)])   # D_s, s = 0 most significant


def _emulated_gram(W):
    from fractions import Fraction
    K = W.shape[0]
    es = [_col_exp(W[i]) for i in range(K)]
    D = np.stack([_digits(W[i], es[i]) for i in range(K)], axis=1)   # (8, K, P)
    G = np.zeros((K, K))
    dots = {}
    for s in range(8):
        for t in range(8):
            if min(s, t) <= 3:
                dots[s, t] = D[s] @ D[t].T      # int64, exact (|sum| < P 2^12)
    for i in range(K):
        for j in range(i, K):
            S = sum(int(dots[s, t][i, j]) << (7 * (14 - s - t)) for (s, t) in dots)
            G[i, j] = G[j, i] = float(Fraction(S) * Fraction(2) ** (es[i] + es[j] - 112))
    return G


def _hard_columns(n, K, B, seed):
    """Seeded smooth fields at scales 1e-30 .. 1e30 plus the awkward cases: a zero column,
    exact zeros and negative zeros inside a column, subnormal entries inside a normal
    column, a column spanning 25 orders of magnitude, a column with a single nonzero."""
    rng = np.random.default_rng(seed)
    Ng = n ** 3
    W = np.empty((B, K, Ng))
    for b in range(B):
        for i in range(K):
            f = pi.initial_state(n, seed=1000 * b + i + 7).reshape(-1)
            W[b, i] = 10.0 ** rng.uniform(-30, 30) * (f + 1e-3 * rng.standard_normal(Ng))
    W[0, 0, ::7] = 0.0
    W[0, 0, 1::7] = -0.0
    if K > 1:
        W[0, 1] = 0.0
    if K > 2:
        W[0, 2, ::5] = 5e-320                                   # subnormals
    if K > 3:
        W[0, 3] *= 10.0 ** rng.uniform(-25, 0, Ng)              # wide dynamic range
    if K > 4:
        W[0, 4] = 0.0
        W[0, 4, Ng // 2] = -3.0
    return W


@pytest.mark.parametrize("n,K,B", [
    (8, 5, 1),      # 512 points: one unit of 8 stages
    (9, 7, 2),      # 729 points (odd): odd columns only 8-byte aligned, a 25-point tail
    (10, 32, 2),    # 1,000 points: two units, the second ragged (488 = 7 x 64 + 40)
    (16, 17, 3),    # 4,096 points: eight units an item, 17 of 32 columns
    (72, 6, 1),     # 373,248 points: units of 5,832 points, two accumulation windows each
])
def test_narrow_tensor_gram_is_exactly_the_digit_sum(gpu, n, K, B):
    bd, torch = gpu
    w = pi.Workload("gram", n, pi.Flow("abc"), 0.05, 1.0, 4, 1e-3, n_snap=64, m_cap=32)
    s = bd.Parareal.from_workload(w, precision=bd.PR_FP32)
    W = _hard_columns(n, K, B, seed=n * K)
    Wt = torch.from_numpy(W).to("cuda")
    Gt = s.op_gram(Wt, tensor=True).cpu().numpy()
    s.close()
    for b in range(B):
        Ge = _emulated_gram(W[b])
        bad = np.argwhere(Gt[b].view(np.int64) != Ge.view(np.int64))
        assert bad.size == 0, (b, bad[:4].tolist(), [(Gt[b][tuple(ij)], Ge[tuple(ij)]) for ij in bad[:4]])


@pytest.mark.parametrize("n,K,B", [(12, 32, 2), (20, 24, 5)])
def test_narrow_tensor_gram_within_the_fp64_bound(gpu, n, K, B):
    """The narrow form against exactly rounded dot products, within the bound of the wide
    test (its dropped digit pairs are a subset of the wide form's)."""
    bd, torch = gpu
    w = pi.Workload("gram", n, pi.Flow("abc"), 0.05, 1.0, 4, 1e-3, n_snap=64, m_cap=32)
    s = bd.Parareal.from_workload(w, precision=bd.PR_FP32)
    W = _columns(n, K, B, seed=K + 1)
    Wt = torch.from_numpy(W).to("cuda")
    Gt = s.op_gram(Wt, tensor=True).cpu().numpy()
    s.close()
    worst = 0.0
    for b in range(B):
        for i in range(K):
            for j in range(i, K):
                if (i * 7 + j * 13) % 3:
                    continue
                x, y = W[b, i], W[b, j]
                ex = _exact_dot(x, y)
                bound = 2.0 ** -50 * float(np.sum(np.abs(x * y)) + np.abs(x).max() * np.abs(y).sum()
                                          + np.abs(y).max() * np.abs(x).sum()) + 1e-300
                worst = max(worst, abs(Gt[b, i, j] - ex) / bound)
    assert worst < 1.0, worst


@pytest.mark.parametrize("K", [4, 24, 32, 60, 96])
def test_double_float_gram_agrees(gpu, K):
    """pr_op_gram's double-float kernel (tensor = 2, the FP32 mode's default) against the
    tensor-core (up to 64 columns) and FP64 kernels on the same columns: all FP64-accurate.
    60 and 96 columns (465 and 1176 output tiles) exceed the kernel's 384 threads and take
    two and four passes over each chunk."""
    bd, torch = gpu
    n, B = 16, 3
    w = pi.Workload("gram", n, pi.Flow("abc"), 0.05, 1.0, 4, 1e-3, n_snap=64, m_cap=32)
    s = bd.Parareal.from_workload(w, precision=bd.PR_FP32)
    W = _columns(n, K, B, seed=K + 5)
    Wt = torch.from_numpy(W).to("cuda")
    Gd = s.op_gram(Wt, tensor=False, df=True).cpu().numpy()
    Gt = s.op_gram(Wt, tensor=True).cpu().numpy() if K <= 64 else None
    G64 = s.op_gram(Wt, tensor=False).cpu().numpy()
    s.close()
    for b in range(B):
        sc = np.abs(G64[b]).max()
        assert np.abs(Gd[b] - G64[b]).max() < 1e-14 * sc
        assert np.array_equal(Gd[b], Gd[b].T)
        if Gt is not None:
            assert np.abs(Gt[b] - G64[b]).max() < 1e-14 * sc


@pytest.mark.parametrize("K", [16, 40])
def test_tensor_gram_wait_timeout_is_reported_and_the_device_stays_usable(gpu, K):
    """Failure path of the tensor-core Grams (narrow form for 16 columns, wide for 40):
    with a spin limit of 0 every mbarrier wait that is not already complete gives up at
    once; the kernel records PR_ERR_TIMEOUT, waits (with its own bound) for the MMAs in
    flight, frees its tensor memory and returns.  The host reads the status, and a fresh
    context on the same device computes the Gram correctly afterwards."""
    bd, torch = gpu
    n, B = 16, 3
    w = pi.Workload("gram", n, pi.Flow("abc"), 0.05, 1.0, 4, 1e-3, n_snap=64, m_cap=32)
    W = _columns(n, K, B, seed=K + 9)
    Wt = torch.from_numpy(W).to("cuda")
    s = bd.Parareal.from_workload(w, precision=bd.PR_FP32, spin_limit=0)
    with pytest.raises(bd.PRError) as ei:
        s.op_gram(Wt, tensor=True)
    assert ei.value.status == 6
    s.close()
    s2 = bd.Parareal.from_workload(w, precision=bd.PR_FP32)
    Gt = s2.op_gram(Wt, tensor=True).cpu().numpy()
    G64 = s2.op_gram(Wt, tensor=False).cpu().numpy()
    s2.close()
    for b in range(B):
        assert np.abs(Gt[b] - G64[b]).max() < 1e-14 * np.abs(G64[b]).max()
