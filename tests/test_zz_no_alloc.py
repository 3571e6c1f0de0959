"""pr_op_apply_L_noalloc against pr_op_apply_L and the oracle's operator.

The no-alloc entry point serves callers that cannot call cudaMalloc (for example while
another framework's caching allocator holds the device memory budget): its scratch is a
static device array instead of the context workspace.  It must give the same operator
values as the workspace path on two calls in a row (the second reuses the scratch left by
the first), match the FP64 oracle's operator (with and without a stored velocity
perturbation), allocate no device memory on a context that never bound a workspace, and
refuse a call above its stated limit.  This file is collected last so a run that stops at
the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
import pr_inputs as pi
from oracle.discretisation import Operator

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


def _noalloc(lib, s, ut, out, count, transpose):
    st = lib.pr_op_apply_L_noalloc(s.ctx, C.c_void_p(ut.data_ptr()), C.c_void_p(out.data_ptr()), count, transpose)
    assert st == 0, lib.pr_last_error(s.ctx)


def test_noalloc_first_call_on_a_fresh_context_allocates_nothing(gpu):
    """A context that never bound a workspace calls the no-alloc operator before anything
    else: device free memory is unchanged across two calls, and the values match the
    oracle's operator (and pr_op_apply_L, run afterwards)."""
    bd, torch = gpu
    lib = bd.lib()
    n, count = 12, 3
    flow = pi.Flow("abc", A=0.9, B=1.2, C=0.8)
    w = pi.Workload("noalloc_fresh", n, flow, 0.033, 1.0, 2, 1e-3, n_snap=8, m_cap=8)
    u = np.stack([pi.initial_state(n, seed=50 + i) for i in range(count)])
    ut = torch.from_numpy(u).to("cuda")
    outs = [torch.full_like(ut, float("nan")) for _ in range(2)]
    # load the library's module on this device first (lazy module loading places the
    # static scratch array then), on a throwaway context
    warm = bd.Parareal.from_workload(w, workspace=False)
    _noalloc(lib, warm, ut, outs[0], count, 0)
    warm.close()
    torch.cuda.synchronize()
    s = bd.Parareal.from_workload(w, workspace=False)
    free0, _ = torch.cuda.mem_get_info()
    for call, transpose in ((0, 0), (1, 1)):
        _noalloc(lib, s, ut, outs[call], count, transpose)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    op = Operator(O.Grid(n), flow, 0.033)
    for i in range(count):
        for call, fn in ((0, op.L), (1, op.LT)):
            ref = fn(u[i], 0.0).reshape(-1)
            got = outs[call][i].cpu().numpy().reshape(-1)
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < TOL
    # the workspace path afterwards gives the same values
    ref_ws = s.op_apply_L(ut, transpose=False)
    _noalloc(lib, s, ut, outs[0], count, 0)
    assert float(((outs[0] - ref_ws).norm() / ref_ws.norm()).item()) < TOL
    s.close()


def test_noalloc_with_stored_perturbation(gpu):
    """A stored velocity perturbation lives in the workspace: once it is bound and
    pr_set_initial has uploaded the field, the no-alloc operator reads it and matches the
    oracle's perturbed operator and pr_op_apply_L, on two calls in a row."""
    bd, torch = gpu
    lib = bd.lib()
    n, count = 12, 2
    flow = pi.Flow("kolmogorov", k=2, pert_seed=3, pert_amp=0.05)
    w = pi.Workload("noalloc_pert", n, flow, 0.02, 1.0, 2, 1e-3, n_snap=8, m_cap=8)
    s = bd.Parareal.from_workload(w)
    s.set_initial(w.u0(), None)
    u = np.stack([pi.initial_state(n, seed=60 + i) for i in range(count)])
    ut = torch.from_numpy(u).to("cuda")
    op = O.make_operator(w)
    for call in range(2):
        for transpose in (0, 1):
            out = torch.full_like(ut, float("nan"))
            _noalloc(lib, s, ut, out, count, transpose)
            ref_ws = s.op_apply_L(ut, transpose=bool(transpose))
            assert float(((out - ref_ws).norm() / ref_ws.norm()).item()) < TOL
            for i in range(count):
                ref = (op.LT if transpose else op.L)(u[i], 0.0).reshape(-1)
                got = out[i].cpu().numpy().reshape(-1)
                assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < TOL, (call, transpose, i)
    s.close()
