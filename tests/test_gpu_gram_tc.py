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
