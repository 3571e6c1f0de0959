"""Pins of the oracle's stopping rule (reading R12 of Algorithm 2's "while not converged")
and of how well the whole-iteration result is determined by its inputs (no GPU).

Stopping rule: parareal stops after the first iteration k >= 1 at which
max_n ||U^k_n - U^{k-1}_n|| / ||U^k_n|| <= tol (increments), or, with a reference, the
error of eq. (error) max_n ||U^k_n - U_n|| / ||U_n|| <= tol; else at k = N or k_max.
The pins recompute both criteria here from the recorded iterates with plain norms and
check the stop against them, and check that the iterate returned is the one of that k.

Conditioning: the POD of Algorithm 1 truncates the spectrum of a Gram matrix whose
eigenvalues fall over many decades, and the augmentation of eqs. (eqaug)/(eq12)
normalises a residual d~ that can be tiny.  So perturbations at the level of FP64
rounding in the inputs of the POD change the iterates far more than 1e-12: two correct
FP64 implementations that round differently cannot agree to 1e-12 at every (k, n) on
such a workload.  These pins measure it on the 16^3 ABC workload with the oracle alone.
"""
import sys

import numpy as np
import pytest

import oracle as O
import pr_inputs as pi


def _norm_rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.sqrt(np.sum((a - b) ** 2)) / np.sqrt(np.sum(b ** 2)))


@pytest.fixture(scope="module")
def history():
    w = pi.tiny(n=8, n_sub=5, T=0.1, dt=2e-3, f_seed=7, flow=pi.Flow("kolmogorov", k=2),
                eps=0.02)
    prm = O.derive_params(w)
    ref = O.sequential_fine(w, prm)
    full = O.parareal(w, prm, k_max=prm.N, reference=ref)
    return w, prm, ref, full


def _first_k(values, tol):
    for k, v in enumerate(values, start=1):
        if v <= tol:
            return k
    return None


def test_stop_on_error_against_reference(history):
    w, prm, ref, full = history
    N = prm.N
    # errors of eq. (error) recomputed from the recorded iterates
    errs = [max(_norm_rel(full["U"][k][n], ref[n]) for n in range(N + 1)) for k in range(1, N + 1)]
    assert errs[-1] < 1e-12                         # finite termination at k = N
    # a tolerance strictly between two consecutive errors stops at the later iteration
    k_star = next(k for k in range(2, N + 1) if errs[k - 1] < 0.5 * errs[k - 2])
    tol = float(np.sqrt(errs[k_star - 1] * errs[k_star - 2]))
    assert _first_k(errs, tol) == k_star
    h = O.parareal(w, prm, k_max=N, tol=tol, reference=ref)
    assert h["k"] == k_star
    for n in range(N + 1):
        assert np.array_equal(h["U_final"][n], full["U"][k_star][n])


def test_stop_on_increment(history):
    w, prm, ref, full = history
    N = prm.N
    incs = [max(np.linalg.norm((full["U"][k][n] - full["U"][k - 1][n]).ravel())
                / np.linalg.norm(full["U"][k][n].ravel()) for n in range(N + 1))
            for k in range(1, N + 1)]
    # increments shrink as the iterates converge; U^N = U^{N-1} except at n = N
    k_star = next(k for k in range(2, N + 1) if incs[k - 1] < 0.5 * incs[k - 2])
    tol = float(np.sqrt(incs[k_star - 1] * incs[k_star - 2]))
    k_expect = _first_k(incs, tol)
    h = O.parareal(w, prm, k_max=N, tol=tol)
    assert h["k"] == k_expect
    assert max(h["inc"][-1]) <= tol
    for n in range(N + 1):
        assert np.array_equal(h["U_final"][n], full["U"][k_expect][n])


def test_stop_bounds(history):
    w, prm, ref, full = history
    # a tolerance every iterate meets still performs one iteration
    assert O.parareal(w, prm, k_max=prm.N, tol=1e6, reference=ref)["k"] == 1
    # an unreachable tolerance stops at k_max, then at N (finite termination)
    assert O.parareal(w, prm, k_max=2, tol=1e-300, reference=ref)["k"] == 2
    assert O.parareal(w, prm, k_max=0, tol=1e-300, reference=ref)["k"] == prm.N


# ------------------------------------------------------------------------ conditioning
def _perturbed_gram_run(w, prm, k_max, rho, seed=3):
    """The oracle with every POD Gram matrix perturbed by symmetric noise of relative size
    rho (the size of FP64 summation rounding in a Gram of a few thousand points)."""
    pod = sys.modules["oracle.pod"]
    rng = np.random.default_rng(seed)
    orig = pod.np.linalg.eigh

    def eigh(G):
        E = rng.standard_normal(G.shape)
        return orig(G + rho * np.abs(G).max() * 0.5 * (E + E.T))

    shim = type(sys)("np_shim")
    shim.__dict__.update(np.__dict__)
    shim.linalg = type(sys)("linalg_shim")
    shim.linalg.__dict__.update(np.linalg.__dict__)
    shim.linalg.eigh = eigh
    pod.np = shim
    try:
        return O.parareal(w, prm, k_max=k_max)
    finally:
        pod.np = np


def test_pod_truncation_is_ill_conditioned_on_abc16():
    # The Case-I window of the 16^3 ABC workload: the sqrt-lambda criterion keeps m = 4
    # modes and lambda_4 / lambda_1 ~ 2e-8, so the kept subspace moves by ~ rho *
    # lambda_1 / (lambda_4 - lambda_5) under a Gram perturbation rho (Davis-Kahan).
    w = pi.ABC_16
    prm = O.derive_params(w)
    op = O.make_operator(w)
    _, W = O.fine_propagate(op, w.u0(), 0.0, prm.S0, prm.dt, prm.dM, prm.n_s0, tol=prm.lin_tol)
    lam = np.sort(np.linalg.eigvalsh(W.T @ W))[::-1]
    _, m, _ = O.pod_mode(W, prm.gamma1, prm.m_cap, prm.tau)
    assert m == 4
    assert lam[3] / lam[0] < 1e-7 and lam[0] / (lam[3] - lam[4]) > 1e7


def _recording_pod_dims():
    """Wrap the oracle's pod_mode so that the POD dimension of every call is recorded."""
    pod_mod = sys.modules["oracle.pod"]
    par_mod = sys.modules["oracle.parareal"]
    dims = []
    orig = pod_mod.pod_mode

    def rec(*args, **kw):
        out = orig(*args, **kw)
        dims.append(out[1])
        return out
    return dims, orig, rec, (pod_mod, par_mod)


def test_rounding_level_gram_noise_moves_abc16_iterates_beyond_1e_12():
    # 1e-15 relative noise in the Gram matrices (FP64 rounding of sums over 4096 points)
    # changes the oracle's own iterates by more than 1e-12 already at k = 0 and by orders
    # of magnitude more at k = 1, where the augmentation normalises residuals as small as
    # 5e-9 ||U||.  No pair of FP64 implementations that round differently can therefore
    # meet 1e-12 at every (k, n) of this workload.  Every discrete decision is the same in
    # both runs (each POD dimension, each augment / skip), so running the oracle with the
    # other side's decisions forced on it would not close the gap either: the kept
    # subspaces themselves move (Davis-Kahan, previous test).
    w = pi.ABC_16
    prm = O.derive_params(w)
    dims, orig, rec, mods = _recording_pod_dims()
    for m_ in mods:
        m_.pod_mode = rec
    try:
        h = O.parareal(w, prm, k_max=1)
        dims_ref = list(dims)
        dims.clear()
        hp = _perturbed_gram_run(w, prm, 1, 1e-15)
    finally:
        for m_ in mods:
            m_.pod_mode = orig
    assert dims == dims_ref and len(dims) > prm.N, (dims, dims_ref)
    assert hp["aug"] == h["aug"] and hp["m1"] == h["m1"] and hp["m2"] == h["m2"]
    d0 = max(_norm_rel(hp["U"][0][n], h["U"][0][n]) for n in range(prm.N + 1))
    d1 = max(_norm_rel(hp["U"][1][n], h["U"][1][n]) for n in range(prm.N + 1))
    assert d0 > 1e-12, d0
    assert d1 > 1e-9, d1


def test_skipping_small_augmentations_costs_accuracy():
    # Reading R11 skips the augmentation only when U is in span R to rounding
    # (||d~|| <= 1e-12 ||U||).  A threshold that also skips small but resolvable residuals
    # (1e-6) gives up the exactness P U = U that the augmentation exists for, and the
    # iteration converges to a worse error.
    w = pi.tiny(n=8, n_sub=4, T=0.08, dt=2e-3)
    prm = O.derive_params(w)
    ref = O.sequential_fine(w, prm)
    errs = {}
    for at in (1e-12, 1e-6):
        prm.aug_tol = at
        h = O.parareal(w, prm, k_max=3, reference=ref)
        errs[at] = [max(e) for e in h["err"]]
    assert sum(h_aug for h_aug in O.parareal(w, O.derive_params(w), k_max=2)["aug"][1].values()) > 0
    assert errs[1e-12][2] < 0.1 * errs[1e-6][2], errs
