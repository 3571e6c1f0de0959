"""pr_op_apply_L_noalloc against pr_op_apply_L.

The no-alloc entry point serves callers that cannot call cudaMalloc (for example while
another framework's caching allocator holds the device memory budget): its scratch is a
static device array instead of the context workspace.  It must give the same operator
values as the workspace path on two calls in a row (the second reuses the scratch left by
the first), and refuse a call above its stated limit.  This file is collected last so a
run that stops at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import pr_inputs as pi

pytestmark = pytest.mark.gpu

TOL = 1e-13   # same as the operator parity test


def test_noalloc_operator_matches_workspace_operator(gpu):
    bd, torch = gpu
    lib = bd.lib()
    cases = ((16, pi.Flow("abc", A=1.0, B=0.7, C=1.3), 3),
             (12, pi.Flow("kolmogorov", k=3), 64))
    for n, flow, count in cases:
        w = pi.Workload("noalloc", n, flow, 0.021, 1.0, 2, 1e-3, n_snap=8, m_cap=8)
        s = bd.Parareal.from_workload(w)
        u = np.stack([pi.initial_state(n, seed=30 + i) + 0.1 * i for i in range(count)])
        ut = torch.from_numpy(np.ascontiguousarray(u)).to("cuda")
        for call in range(2):                      # two calls in a row per direction
            for transpose in (0, 1):
                ref = s.op_apply_L(ut, transpose=bool(transpose))
                out = torch.full_like(ut, float("nan"))
                st = lib.pr_op_apply_L_noalloc(s.ctx, C.c_void_p(ut.data_ptr()),
                                               C.c_void_p(out.data_ptr()), count, transpose)
                assert st == 0, lib.pr_last_error(s.ctx)
                err = float(((out - ref).norm() / ref.norm()).item())
                assert err < TOL, (n, call, transpose, err)
        s.close()


def test_noalloc_rejects_calls_above_its_limit(gpu):
    bd, torch = gpu
    lib = bd.lib()
    w = pi.Workload("noalloc", 8, pi.Flow("abc"), 0.05, 1.0, 2, 1e-3, n_snap=8, m_cap=8)
    s = bd.Parareal.from_workload(w)
    u = torch.zeros((65, 8, 8, 8), dtype=torch.float64, device="cuda")
    out = torch.empty_like(u)
    st = lib.pr_op_apply_L_noalloc(s.ctx, C.c_void_p(u.data_ptr()), C.c_void_p(out.data_ptr()), 65, 0)
    assert st == 1
    assert b"64" in lib.pr_last_error(s.ctx)
    s.close()
