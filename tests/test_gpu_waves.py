"""Wave mode (pr_opts.wave): each iteration streamed over waves of subintervals, the form
that runs the 128^3 x 256 and 256^3 x 128 workloads on one GPU.

* On the 64^3 Kolmogorov workload the wave form (per wave: fine sweep, level-1 POD,
  level-2 POD, Galerkin matrices and its share of the coarse sweep; one generation of
  level-1 bases) gives bit-identical iterates to the single-launch form in both precision
  modes, ragged last wave included.
* Against the oracle: flat 1e-12 in the FP64 mode up to k = N, the FP32-mode bar on the
  16^3 ABC workload.
* At full size (128^3 with 256 subintervals, 256^3 with 128) one iteration runs, and its
  results are checked on samples the oracle can compute (fine steps from the GPU's own
  interface states, the POD of the GPU's own snapshot windows) and on properties that
  hold at any size (U^1_1 = F_0 exactly, conservation of the mean, orthonormal bases).
"""
import dataclasses

import numpy as np
import pytest

import oracle as O
import pr_inputs as pi
from test_gpu_parity import TOL32, TOL64, davis_kahan_tol, oracle_envelope, rel, span_dist

pytestmark = pytest.mark.gpu


def _iterates(bd, w, K, precision, **kw):
    s = bd.Parareal.from_workload(w, precision=precision, **kw)
    s.set_initial(w.u0(), w.f())
    s.iteration0()
    out = [s.interfaces()]
    for k in range(1, K + 1):
        s.iterate(k)
        out.append(s.interfaces())
    return s, out


@pytest.mark.parametrize("precision", [0, 1])
def test_wave_form_bit_identical_on_kol64(gpu, precision):
    bd, torch = gpu
    w = pi.KOL_64
    K = 3
    G = 9   # CTAs per subinterval, fixed so that both forms reduce in the same order
    s1, U1 = _iterates(bd, w, K, precision, group_ctas=G)
    m1 = s1.diagnostics()
    s1.close()
    s2, U2 = _iterates(bd, w, K, precision, group_ctas=G, wave=12)   # waves 12 x 5 + 4 (ragged)
    m2 = s2.diagnostics()
    s2.close()
    for k in range(K + 1):
        assert np.array_equal(U1[k], U2[k]), (k, float(np.max(np.abs(U1[k] - U2[k]))))
    assert np.array_equal(m1["m1"], m2["m1"]) and np.array_equal(m1["m2"], m2["m2"])
    torch.cuda.empty_cache()


def test_wave_workspace_is_smaller(gpu):
    bd, torch = gpu
    w = pi.KOL_64
    full = bd.Parareal.from_workload(w, precision=bd.PR_FP32, workspace=False)
    wave = bd.Parareal.from_workload(w, precision=bd.PR_FP32, workspace=False, wave=8)
    nf, nw = full.workspace_bytes(), wave.workspace_bytes()
    # the snapshot store keeps 8 windows instead of 64; the level-2 bases, 8 of 64; the
    # level-1 bases lose a generation (and gain one wave's)
    snap_window = w.n_snap * w.Ng * 8
    basis = w.m_cap * w.Ng * 8
    assert nf - nw > 56 * snap_window + 56 * basis + 56 * basis, (nf, nw)
    full.close()
    wave.close()


def test_wave_form_against_oracle_fp64(gpu):
    """FP64 mode in waves of 3 (a ragged last wave) at a flat 1e-12 at every (k, n) up to
    k = N (a workload whose rounding response is below 1e-13)."""
    bd, torch = gpu
    w = pi.tiny(n=8, n_sub=4, T=0.08, dt=2e-3)
    prm = O.derive_params(w)
    hist = O.parareal(w, prm, k_max=w.n_sub)
    s, Us = _iterates(bd, w, w.n_sub, bd.PR_FP64, wave=3)
    assert s.fine_ms()[1] == 1            # k = N: one subinterval left, one wave
    s.close()
    worst = max(rel(Us[k][n], hist["U"][k][n]) for k in range(w.n_sub + 1) for n in range(w.n_sub + 1))
    assert worst < TOL64, worst


def test_wave_form_against_oracle_fp32(gpu):
    """FP32 mode in waves of 3 on the 16^3 ABC workload: within max(1e-5, 10 x the oracle's
    change under 1e-8 fine perturbations) at every (k, n)."""
    bd, torch = gpu
    w = pi.ABC_16
    prm = O.derive_params(w)
    K = 3
    hist, env = oracle_envelope(w, prm, K, 1e-8, where="fine")
    s, Us = _iterates(bd, w, K, bd.PR_FP32, wave=3)
    s.close()
    for k in range(K + 1):
        for n in range(w.n_sub + 1):
            e = rel(Us[k][n], hist["U"][k][n])
            assert e < max(TOL32, 10 * env[k][n]), (k, n, e, env[k][n])


def test_wave_mode_rewind_and_limits(gpu):
    bd, torch = gpu
    w = pi.tiny(n=8, n_sub=5, T=0.1, dt=2e-3)
    s = bd.Parareal.from_workload(w, precision=bd.PR_FP64, wave=2)
    s.set_initial(w.u0(), w.f())
    s.iteration0()
    s.iterate(1)
    a = s.interfaces()
    s.rewind()                      # iteration 1 used V0, not level-1 bases of k = 0
    s.iterate(1)
    assert np.array_equal(a, s.interfaces())
    s.iterate(2)
    with pytest.raises(bd.PRError) as ei:
        s.rewind()                  # the level-1 bases of iteration 1 were replaced
    assert ei.value.status == 8
    with pytest.raises(bd.PRError):
        s.snapshots(0)              # only the last wave's windows are resident
    assert s.snapshots(4).shape[0] == s.n_s
    s.close()
    with pytest.raises(bd.PRError):   # waves stream the adaptive method only
        bd.Parareal.from_workload(w, precision=bd.PR_FP64, wave=2, method=bd.PR_METHOD_PARAREAL_I)


def _full_size_checks(bd, torch, w, wave, sample_n, steps_check):
    """One iteration of the full workload in wave mode (FP32 mode); checks on samples the
    oracle can compute and on invariants."""
    torch.cuda.empty_cache()
    s = bd.Parareal.from_workload(w, precision=bd.PR_FP32, wave=wave)
    free, total = torch.cuda.mem_get_info()
    print(f"{w.name}: workspace {s.workspace_bytes() / 2**30:.1f} GiB (free after binding "
          f"{free / 2**30:.1f} of {total / 2**30:.1f} GiB)")
    try:
        s.set_initial(w.u0(), w.f())
        s.iteration0()
        U0 = s.interface(sample_n)
        s.iterate(1)
        ms, launches = s.fine_ms()
        assert launches == -(-w.n_sub // wave)
        print(f"{w.name}: fine kernel {ms:.0f} ms over {launches} waves")
        d = s.diagnostics()
        assert np.all(d["m1"] >= 1) and np.all(d["m1"] <= w.m_cap)
        assert np.all(d["m2"][1:] >= 1) and np.all(d["m2"][1:] <= w.m_cap)
        # reading R10: U^1_1 = F(U^0_0) exactly
        assert np.array_equal(s.interface(1), s.fine_end(0))
        # divergence-free flow, zero-mean forcing: every step conserves the mean, up to the
        # FP32 mode's evaluation of the residual (R20: ~1e-7 of delta_t L u per step; the
        # measured drift after 128 x 391 steps is 4e-8 of the initial rms)
        u0 = w.u0()
        mean0, rms0 = float(np.mean(u0)), float(np.sqrt(np.mean(u0 * u0)))
        for n in (1, w.n_sub // 2, w.n_sub):
            u = s.interface(n)
            assert np.all(np.isfinite(u))
            assert abs(float(np.mean(u)) - mean0) < 1e-6 * rms0, (n, float(np.mean(u)))
        # sampled fine parity: the oracle's first snapshot interval of subinterval sample_n
        # (which the last wave holds) from the GPU's own U^0, against the GPU's snapshot
        prm = O.derive_params(w)
        W = s.snapshots(sample_n)
        assert rel(W[0], U0) < 1e-14   # the FP32 mode's state is a float pair (~48 bits)
        if steps_check:
            op = O.make_operator(w)
            u_or, _ = O.fine_propagate(op, U0, prm.T0 + sample_n * prm.DeltaT, steps_check, prm.dt, tol=1e-14)
            assert prm.dM == steps_check
            assert rel(W[1], u_or) < TOL32, rel(W[1], u_or)
        # level-1 POD of the GPU's own window against the GPU's basis: same span within the
        # Davis-Kahan bound of its double-float Gram; orthonormal bases at both levels
        Wm = W.reshape(W.shape[0], -1).T
        del W
        Ro, mo, lam = O.pod_mode(Wm, prm.gamma2, prm.m_cap, prm.tau)
        del Wm
        Rg = s.basis(1, sample_n).T
        assert Rg.shape[1] == mo
        assert span_dist(Rg, Ro) < davis_kahan_tol(lam, mo, 1e-14), span_dist(Rg, Ro)
        assert np.abs(Rg.T @ Rg - np.eye(mo)).max() < 1e-12
        R2 = s.basis(2, sample_n).T
        assert np.abs(R2.T @ R2 - np.eye(R2.shape[1])).max() < 1e-12
    finally:
        s.close()
        del s
        torch.cuda.empty_cache()


def test_abc128_full_size_iteration(gpu):
    # 128^3 = 2,097,152 points (the paper's DOF count), 256 subintervals x 391 steps,
    # 64 snapshots per window, POD rank <= 32: waves of 32 subintervals
    bd, torch = gpu
    w = pi.ABC_128
    _full_size_checks(bd, torch, w, 32, w.n_sub - 1, 6)


def test_kol256_full_size_iteration(gpu):
    # 256^3 = 16.8M points with the stored divergence-free perturbation, 128 subintervals
    # x 625 steps, 16 snapshots per window, POD rank <= 8: waves of 8 subintervals (fine
    # steps at 256^3 against the oracle: test_gpu_fullsize)
    bd, torch = gpu
    w = pi.KOL_256
    _full_size_checks(bd, torch, w, 8, w.n_sub - 1, None)
