"""ctypes binding of the C ABI in include/parareal.h (same function names).

Argument marshalling only: every step of the method runs in the CUDA library.  PyTorch
supplies device memory (the workspace and caller tensors) and the stream.  Importing
this module fails loudly if the library has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Optional, Sequence

import numpy as np

from .build import lib_path

PR_OK = 0
STATUS = {0: "PR_OK", 1: "PR_ERR_INVALID_ARG", 2: "PR_ERR_OOM", 3: "PR_ERR_CUDA",
          4: "PR_ERR_NOT_CONVERGED", 5: "PR_ERR_BREAKDOWN", 6: "PR_ERR_TIMEOUT",
          7: "PR_ERR_NONFINITE", 8: "PR_ERR_STATE", 9: "PR_ERR_UNSUPPORTED"}
PR_FLOW_ABC, PR_FLOW_KOLMOGOROV, PR_FLOW_CONST = 0, 1, 2
PR_FLOW_PAPER_KOLMOGOROV, PR_FLOW_PAPER_ABC = 3, 4
PR_FP64, PR_FP32 = 0, 1
PR_METHOD_ADAPTIVE, PR_METHOD_PARAREAL_I, PR_METHOD_PARAREAL_II = 0, 1, 2
PR_GRAM_AUTO, PR_GRAM_DF, PR_GRAM_TENSOR = 0, 1, 2
PR_FINE_IMPLICIT_EULER, PR_FINE_RK4 = 0, 1


class pr_grid(C.Structure):
    _fields_ = [("n", C.c_int), ("L", C.c_double)]


class pr_flow(C.Structure):
    _fields_ = [("kind", C.c_int), ("A", C.c_double), ("B", C.c_double), ("C", C.c_double),
                ("k", C.c_int), ("b", C.c_double * 3), ("w", C.c_double),
                ("pert", C.POINTER(C.c_double))]


class pr_opts(C.Structure):
    _fields_ = [("T0", C.c_double), ("dT", C.c_double), ("n_snap", C.c_int), ("m_cap", C.c_int),
                ("m_l", C.c_int), ("p", C.c_int), ("pod_tol3", C.c_double),
                ("rank_tau", C.c_double), ("precision", C.c_int), ("lin_tol", C.c_double),
                ("lin_maxit", C.c_int), ("aug_tol", C.c_double), ("group_ctas", C.c_int),
                ("ctas_per_sm", C.c_int), ("spin_limit", C.c_longlong), ("method", C.c_int),
                ("fine", C.c_int), ("wave", C.c_int), ("gram_mode", C.c_int)]


class pr_report(C.Structure):
    _fields_ = [("k", C.c_int), ("converged", C.c_int), ("max_inc", C.c_double),
                ("max_err", C.c_double), ("t_iter0", C.c_double), ("t_fine", C.c_double),
                ("t_pod", C.c_double), ("t_coarse", C.c_double), ("t_check", C.c_double),
                ("t_total", C.c_double), ("fine_dof_steps", C.c_double),
                ("lin_iters_mean", C.c_double), ("lin_iters_max", C.c_int), ("m0", C.c_int),
                ("m1_max", C.c_int), ("m2_max", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class pr_server_opts(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("max_active", C.c_int), ("batch_fine", C.c_int)]


class pr_request(C.Structure):
    _fields_ = [("grid", pr_grid), ("flow", pr_flow), ("eps", C.c_double), ("T", C.c_double),
                ("n_sub", C.c_int), ("dt_fine", C.c_double), ("pod_tol", C.c_double),
                ("opts", pr_opts), ("u0", C.POINTER(C.c_double)), ("f", C.POINTER(C.c_double)),
                ("tol", C.c_double), ("k_max", C.c_int)]


PR_REQ_PENDING, PR_REQ_ACTIVE, PR_REQ_DONE, PR_REQ_FAILED = 0, 1, 2, 3

_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)
_SIGS = {
    "pr_opts_init": (None, [C.POINTER(pr_opts)]),
    "pr_create": (C.c_int, [C.POINTER(pr_grid), C.POINTER(pr_flow), C.c_double, C.c_double,
                            C.c_int, C.c_double, C.c_double, C.POINTER(pr_opts), C.POINTER(_P)]),
    "pr_destroy": (None, [_P]),
    "pr_get_sizes": (C.c_int, [_P, _I, _I, _I, _I, _I, _I, _D, _D]),
    "pr_workspace_bytes": (C.c_size_t, [_P]),
    "pr_bind_workspace": (C.c_int, [_P, _P, C.c_size_t]),
    "pr_set_stream": (C.c_int, [_P, _P]),
    "pr_set_initial": (C.c_int, [_P, _D, _D]),
    "pr_iteration0": (C.c_int, [_P]),
    "pr_fine_sweep": (C.c_int, [_P, C.c_int]),
    "pr_pod_update": (C.c_int, [_P, C.c_int]),
    "pr_coarse_sweep": (C.c_int, [_P, C.c_int]),
    "pr_check": (C.c_int, [_P, C.c_int, _D, _D]),
    "pr_solve": (C.c_int, [_P, C.c_double, C.c_int, _D, C.POINTER(pr_report)]),
    "pr_compute_reference": (C.c_int, [_P, C.c_int]),
    "pr_set_reference": (C.c_int, [_P, _P, C.c_int]),
    "pr_get_interface": (C.c_int, [_P, C.c_int, _D]),
    "pr_get_interfaces": (C.c_int, [_P, _D]),
    "pr_set_interfaces": (C.c_int, [_P, _D, C.c_int]),
    "pr_get_diagnostics": (C.c_int, [_P, _D, _D, _I, _I, _I]),
    "pr_get_lin_stats": (C.c_int, [_P, _I, _I]),
    "pr_sync": (C.c_int, [_P]),
    "pr_last_error": (C.c_char_p, [_P]),
    "pr_status_string": (C.c_char_p, [C.c_int]),
    "pr_launch_count": (C.c_longlong, []),
    "pr_rewind": (C.c_int, [_P]),
    "pr_get_fine_end": (C.c_int, [_P, C.c_int, _D]),
    "pr_get_snapshots": (C.c_int, [_P, C.c_int, _P]),
    "pr_get_basis": (C.c_int, [_P, C.c_int, C.c_int, _P, _I]),
    "pr_op_apply_L": (C.c_int, [_P, _P, _P, C.c_int, C.c_int]),
    "pr_op_apply_L_df": (C.c_int, [_P, _P, _P, C.c_int]),
    "pr_op_fine": (C.c_int, [_P, _P, _P, _P, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int]),
    "pr_op_pod": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, _P, _I]),
    "pr_op_coarse_update": (C.c_int, [_P, _P, C.c_int, _P, _P, _P, _P]),
    "pr_op_apply_L_noalloc": (C.c_int, [_P, _P, _P, C.c_int, C.c_int]),
    "pr_fine_sweep_batch": (C.c_int, [C.POINTER(_P), _I, C.c_int]),
    "pr_tune_fine": (C.c_int, [_P, C.c_int, _I, _D]),
    "pr_server_opts_init": (None, [C.POINTER(pr_server_opts)]),
    "pr_server_create": (C.c_int, [C.POINTER(pr_server_opts), C.POINTER(_P)]),
    "pr_server_destroy": (None, [_P]),
    "pr_server_submit": (C.c_int, [_P, C.POINTER(pr_request), _I]),
    "pr_server_step": (C.c_int, [_P, _I, _I]),
    "pr_server_query": (C.c_int, [_P, C.c_int, _I, _I, _D]),
    "pr_get_fine_ms": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "pr_op_gram": (C.c_int, [_P, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int]),
    "pr_server_result": (C.c_int, [_P, C.c_int, _D]),
    "pr_server_request_error": (C.c_char_p, [_P, C.c_int]),
    "pr_server_last_error": (C.c_char_p, [_P]),
}

_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is not built; run "
                               "`python -m paper_2601_10981_gb300.build` (needs nvcc)")
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class PRError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _tptr(t) -> Optional[int]:
    return None if t is None else C.c_void_p(t.data_ptr())


def opts(**kw) -> pr_opts:
    o = pr_opts()
    lib().pr_opts_init(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def flow_struct(kind: str, A=1.0, B=1.0, Cc=1.0, k=1, b=(0.0, 0.0, 0.0), w=1.0, pert=None) -> pr_flow:
    """pr_flow; pert: optional stored velocity perturbation, array (3, n, n, n) float64
    (kept alive by the returned struct; pr_create copies it)."""
    f = pr_flow()
    f.kind = {"abc": PR_FLOW_ABC, "kolmogorov": PR_FLOW_KOLMOGOROV, "const": PR_FLOW_CONST,
              "paper_kolmogorov": PR_FLOW_PAPER_KOLMOGOROV, "paper_abc": PR_FLOW_PAPER_ABC}[kind]
    f.A, f.B, f.C, f.k = A, B, Cc, k
    f.b[0], f.b[1], f.b[2] = b
    f.w = w
    if pert is not None:
        arr = np.ascontiguousarray(pert, dtype=np.float64)
        f._pert_keep = arr
        f.pert = arr.ctypes.data_as(C.POINTER(C.c_double))
    return f


def flow_of(fl, n: int) -> pr_flow:
    """pr_flow of a pr_inputs.Flow on an n^3 grid (with its stored perturbation, if any)."""
    pert = fl.pert(n) if getattr(fl, "pert_seed", 0) > 0 else None
    return flow_struct(fl.kind, fl.A, fl.B, fl.C, fl.k, (fl.b0, fl.b1, fl.b2), fl.w, pert)


class Parareal:
    """One adaptive-parareal problem on the GPU (an owned pr_ctx).

    The workspace is a torch uint8 tensor on the current device; work runs on the torch
    current stream of the device at construction time."""

    def __init__(self, n: int, flow: pr_flow, eps: float, T: float, n_sub: int, dt: float,
                 pod_tol: float = 5e-6, options: Optional[pr_opts] = None, L: float = 0.0,
                 stream=None, workspace: bool = True):
        import torch
        self._lib = lib()
        g = pr_grid(n, L)
        ctx = C.c_void_p()
        st = self._lib.pr_create(C.byref(g), C.byref(flow), eps, T, n_sub, dt, pod_tol,
                                 C.byref(options) if options is not None else None, C.byref(ctx))
        if st != PR_OK:
            raise PRError(st, "pr_create failed")
        self.ctx = ctx
        self.n, self.N, self.Ng = n, n_sub, n ** 3
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._check(self._lib.pr_set_stream(self.ctx, C.c_void_p(self.stream.cuda_stream)))
        self.ws = None
        if workspace:
            nbytes = int(self._lib.pr_workspace_bytes(self.ctx))
            self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            base = self.ws.data_ptr()
            aligned = (base + 255) // 256 * 256
            self._check(self._lib.pr_bind_workspace(self.ctx, C.c_void_p(aligned), nbytes))
        sizes = [C.c_int() for _ in range(6)]
        dte, dT = C.c_double(), C.c_double()
        self._lib.pr_get_sizes(self.ctx, *[C.byref(s) for s in sizes], C.byref(dte), C.byref(dT))
        self.S, self.S0, self.dM, self.n_s, self.n_s0, self.Lc = (s.value for s in sizes)
        self.dt_eff, self.DeltaT = dte.value, dT.value
        self.fp32 = bool(options is not None and options.precision == PR_FP32)

    @classmethod
    def from_workload(cls, w, precision: int = PR_FP64, workspace: bool = True, **opt_kw):
        fl = w.flow
        flow = flow_of(fl, w.n)
        o = opts(n_snap=w.n_snap, m_cap=w.m_cap, m_l=w.m_l, p=w.p, precision=precision, **opt_kw)
        obj = cls(w.n, flow, w.eps, w.T, w.n_sub, w.dt, w.pod_tol, o, workspace=workspace)
        return obj

    def workspace_bytes(self) -> int:
        """pr_workspace_bytes: device bytes the context needs."""
        return int(self._lib.pr_workspace_bytes(self.ctx))

    # ------------------------------------------------------------------ errors
    def _check(self, st: int):
        if st != PR_OK:
            msg = self._lib.pr_last_error(self.ctx).decode() if getattr(self, "ctx", None) else ""
            raise PRError(st, msg)

    def status(self, st: int) -> int:
        return st

    def close(self):
        if getattr(self, "ctx", None):
            self._lib.pr_destroy(self.ctx)
            self.ctx = None
        self.ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ phases
    def set_initial(self, u0: np.ndarray, f: Optional[np.ndarray] = None):
        u0 = np.ascontiguousarray(u0, dtype=np.float64).reshape(-1)
        f = None if f is None else np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        self._check(self._lib.pr_set_initial(self.ctx, _dptr(u0), _dptr(f)))

    def iteration0(self):
        self._check(self._lib.pr_iteration0(self.ctx))

    def fine_sweep(self, k: int):
        self._check(self._lib.pr_fine_sweep(self.ctx, k))

    def pod_update(self, k: int):
        self._check(self._lib.pr_pod_update(self.ctx, k))

    def coarse_sweep(self, k: int):
        self._check(self._lib.pr_coarse_sweep(self.ctx, k))

    def check(self, k: int):
        mi, me = C.c_double(), C.c_double()
        self._check(self._lib.pr_check(self.ctx, k, C.byref(mi), C.byref(me)))
        return mi.value, me.value

    def iterate(self, k: int):
        self.fine_sweep(k)
        self.pod_update(k)
        self.coarse_sweep(k)
        return self.check(k)

    def solve(self, tol: float, k_max: int = 0, ref: Optional[np.ndarray] = None) -> dict:
        rep = pr_report()
        r = None if ref is None else np.ascontiguousarray(ref, dtype=np.float64).reshape(-1)
        self._check(self._lib.pr_solve(self.ctx, tol, k_max, _dptr(r), C.byref(rep)))
        return rep.as_dict()

    def compute_reference(self, fp64: bool = True):
        self._check(self._lib.pr_compute_reference(self.ctx, 1 if fp64 else 0))

    def set_reference(self, U):
        if hasattr(U, "data_ptr"):
            self._check(self._lib.pr_set_reference(self.ctx, C.c_void_p(U.data_ptr()), 1))
        else:
            a = np.ascontiguousarray(U, dtype=np.float64).reshape(-1)
            self._check(self._lib.pr_set_reference(self.ctx, a.ctypes.data_as(C.c_void_p), 0))

    def interfaces(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        """U^k_0..U^k_N; out: an optional C-contiguous float64 host array of N+1 grid
        functions to fill (e.g. pinned memory, for a direct device-to-host copy)."""
        if out is None:
            out = np.empty((self.N + 1, self.n, self.n, self.n))
        elif not (out.dtype == np.float64 and out.flags.c_contiguous and out.size == (self.N + 1) * self.Ng):
            raise ValueError("out must be a C-contiguous float64 array of (N+1) n^3 values")
        self._check(self._lib.pr_get_interfaces(self.ctx, _dptr(out)))
        return out

    def interface(self, n: int) -> np.ndarray:
        out = np.empty((self.n, self.n, self.n))
        self._check(self._lib.pr_get_interface(self.ctx, n, _dptr(out)))
        return out

    def set_interfaces(self, U: np.ndarray, k_done: int):
        U = np.ascontiguousarray(U, dtype=np.float64).reshape(-1)
        self._check(self._lib.pr_set_interfaces(self.ctx, _dptr(U), k_done))

    def diagnostics(self):
        N = self.N
        inc, err = np.zeros(N + 1), np.zeros(N + 1)
        m0 = C.c_int()
        m1, m2 = np.zeros(N, dtype=np.int32), np.zeros(N, dtype=np.int32)
        self._check(self._lib.pr_get_diagnostics(self.ctx, _dptr(inc), _dptr(err), C.byref(m0),
                                                  m1.ctypes.data_as(_I), m2.ctypes.data_as(_I)))
        return dict(inc=inc, err=err, m0=m0.value, m1=m1, m2=m2)

    def fine_ms(self):
        """(ms, launches): device time of the fine-kernel launches of the last fine sweep."""
        ms, nl = C.c_double(), C.c_int()
        self._check(self._lib.pr_get_fine_ms(self.ctx, C.byref(ms), C.byref(nl)))
        return ms.value, nl.value

    def lin_stats(self):
        tot, mx = np.zeros(self.N, dtype=np.int32), np.zeros(self.N, dtype=np.int32)
        self._check(self._lib.pr_get_lin_stats(self.ctx, tot.ctypes.data_as(_I), mx.ctypes.data_as(_I)))
        return tot, mx

    def rewind(self):
        self._check(self._lib.pr_rewind(self.ctx))

    def fine_end(self, n: int) -> np.ndarray:
        out = np.empty((self.n, self.n, self.n))
        self._check(self._lib.pr_get_fine_end(self.ctx, n, _dptr(out)))
        return out

    def snapshots(self, n: int) -> np.ndarray:
        out = np.empty((self.n_s, self.Ng), dtype=np.float64)
        self._check(self._lib.pr_get_snapshots(self.ctx, n, out.ctypes.data_as(C.c_void_p)))
        return out

    def basis(self, level: int, n: int = 0) -> np.ndarray:
        m = C.c_int()
        self._check(self._lib.pr_get_basis(self.ctx, level, n, None, C.byref(m)))
        out = np.empty((m.value, self.Ng), dtype=np.float64)
        if m.value:
            self._check(self._lib.pr_get_basis(self.ctx, level, n, out.ctypes.data_as(C.c_void_p),
                                               C.byref(m)))
        return out

    def sync(self):
        self._check(self._lib.pr_sync(self.ctx))

    def tune_fine(self, steps: int = 8):
        """pr_tune_fine: the fastest CTA-group size of the fine launch (kept in the context)
        and its time in ms."""
        G, ms = C.c_int(), C.c_double()
        self._check(self._lib.pr_tune_fine(self.ctx, steps, C.byref(G), C.byref(ms)))
        return G.value, ms.value

    # ------------------------------------------------------------------ single ops
    def op_apply_L(self, u, transpose: bool = False, df: bool = False):
        """u: torch float64 tensor (count, n, n, n) on the GPU.  df: the double-float form
        of the FP32 mode's Galerkin projection (pr_op_apply_L_df; L only, not L^T)."""
        out = self.torch.empty_like(u)
        count = u.shape[0] if u.dim() == 4 else 1
        if df:
            if transpose:
                raise ValueError("the double-float operator form has no transpose")
            self._check(self._lib.pr_op_apply_L_df(self.ctx, _tptr(u), _tptr(out), count))
        else:
            self._check(self._lib.pr_op_apply_L(self.ctx, _tptr(u), _tptr(out), count, int(transpose)))
        return out

    def op_fine(self, u, steps: int, dM: int = 1, n_snap: int = 0, t0: float = 0.0):
        B = u.shape[0]
        out = self.torch.empty_like(u)
        snap = None
        if n_snap > 0:
            snap = self.torch.zeros((B, n_snap) + tuple(u.shape[1:]), dtype=self.torch.float64,
                                    device=u.device)
        self._check(self._lib.pr_op_fine(self.ctx, _tptr(u), _tptr(out), _tptr(snap), B, t0,
                                         steps, dM, n_snap))
        return out, snap

    def op_pod(self, W, gamma: float, cap: int = 0):
        """W: (B, n_cols, n, n, n) float64 or float32 tensor; returns the (float64) bases and
        the POD dimensions."""
        B, ncol = W.shape[0], W.shape[1]
        mmax = min(cap, ncol) if cap > 0 else ncol
        R = self.torch.zeros((B, mmax) + tuple(W.shape[2:]), dtype=self.torch.float64,
                             device=W.device)
        m = np.zeros(B, dtype=np.int32)
        w32 = 1 if W.dtype == self.torch.float32 else 0
        self._check(self._lib.pr_op_pod(self.ctx, _tptr(W), w32, ncol, B, gamma, cap, _tptr(R),
                                        m.ctypes.data_as(_I)))
        return R, m

    def op_gram(self, W, tensor: bool = True, df: bool = False):
        """G_b = W_b^T W_b of a (B, n_cols, n^3) float64 CUDA tensor; returns (B, n_cols, n_cols).
        tensor: tensor cores; else df: double-float on the FP32 pipe; else FP64."""
        torch = self.torch
        B, K = W.shape[0], W.shape[1]
        G = torch.empty((B, K, K), dtype=torch.float64, device=W.device)
        mode = 1 if tensor else (2 if df else 0)
        self._check(self._lib.pr_op_gram(self.ctx, C.c_void_p(W.data_ptr()), K, B, C.c_void_p(G.data_ptr()),
                                         mode))
        return G

    def op_coarse_update(self, R, m: int, U, Uprev, F):
        out = self.torch.empty_like(U)
        self._check(self._lib.pr_op_coarse_update(self.ctx, _tptr(R), m, _tptr(U), _tptr(Uprev),
                                                  _tptr(F), _tptr(out)))
        return out


def launch_count() -> int:
    return int(lib().pr_launch_count())


def fine_sweep_batch(problems: Sequence[Parareal], ks: Sequence[int]):
    """pr_fine_sweep_batch: the fine sweeps of several problems in one persistent launch."""
    arr = (C.c_void_p * len(problems))(*[p.ctx.value for p in problems])
    kk = (C.c_int * len(ks))(*ks)
    st = lib().pr_fine_sweep_batch(arr, kk, len(problems))
    if st != PR_OK:
        raise PRError(st, lib().pr_last_error(problems[0].ctx).decode())


class Server:
    """pr_server: continuous batching of parareal requests on one GPU."""

    def __init__(self, hbm_budget: int = 0, max_active: int = 0, batch_fine: bool = True):
        self._lib = lib()
        o = pr_server_opts()
        self._lib.pr_server_opts_init(C.byref(o))
        o.hbm_budget, o.max_active, o.batch_fine = hbm_budget, max_active, int(batch_fine)
        srv = C.c_void_p()
        st = self._lib.pr_server_create(C.byref(o), C.byref(srv))
        if st != PR_OK:
            raise PRError(st, "pr_server_create failed")
        self.srv = srv
        self._n = {}

    def _check(self, st: int):
        if st != PR_OK:
            raise PRError(st, self._lib.pr_server_last_error(self.srv).decode())

    def submit(self, w, u0: np.ndarray, f: Optional[np.ndarray] = None, tol: float = 1e-6,
               k_max: int = 0, precision: int = PR_FP32, **opt_kw) -> int:
        """Queue the problem of workload w (pr_inputs.Workload fields) with initial state u0."""
        fl = w.flow
        r = pr_request()
        r.grid = pr_grid(w.n, 0.0)
        flow = flow_of(fl, w.n)   # alive through pr_server_submit, which copies the perturbation
        r.flow = flow
        r.eps, r.T, r.n_sub, r.dt_fine, r.pod_tol = w.eps, w.T, w.n_sub, w.dt, w.pod_tol
        r.opts = opts(n_snap=w.n_snap, m_cap=w.m_cap, m_l=w.m_l, p=w.p, precision=precision, **opt_kw)
        u0 = np.ascontiguousarray(u0, dtype=np.float64).reshape(-1)
        fa = None if f is None else np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        r.u0 = _dptr(u0)
        r.f = _dptr(fa)
        r.tol, r.k_max = tol, k_max
        rid = C.c_int()
        self._check(self._lib.pr_server_submit(self.srv, C.byref(r), C.byref(rid)))
        self._n[rid.value] = w.n
        return rid.value

    def step(self):
        a, p = C.c_int(), C.c_int()
        self._check(self._lib.pr_server_step(self.srv, C.byref(a), C.byref(p)))
        return a.value, p.value

    def query(self, rid: int):
        st, k, inc = C.c_int(), C.c_int(), C.c_double()
        self._check(self._lib.pr_server_query(self.srv, rid, C.byref(st), C.byref(k), C.byref(inc)))
        return st.value, k.value, inc.value

    def result(self, rid: int) -> np.ndarray:
        n = self._n[rid]
        out = np.empty((n, n, n))
        self._check(self._lib.pr_server_result(self.srv, rid, _dptr(out)))
        return out

    def request_error(self, rid: int) -> str:
        return self._lib.pr_server_request_error(self.srv, rid).decode()

    def close(self):
        if getattr(self, "srv", None):
            self._lib.pr_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
