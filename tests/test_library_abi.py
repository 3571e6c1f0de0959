"""The C-ABI library builds, loads and exports every function include/parareal.h declares,
and the binding covers exactly those names.  Host-only calls (no device work) check the
option defaults and argument validation."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "parareal.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*\*?\s*\**\s*(pr_[A-Za-z0-9_]+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2601_10981_gb300 import build
    if not os.path.exists(build.lib_path()):
        build.build()
    from paper_2601_10981_gb300 import binding
    return binding.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for core in ("pr_create", "pr_fine_sweep", "pr_pod_update", "pr_coarse_sweep", "pr_solve",
                 "pr_destroy", "pr_set_initial", "pr_iteration0", "pr_check"):
        assert core in names
    assert len(names) >= 30


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_binding_covers_exactly_the_header():
    from paper_2601_10981_gb300 import binding
    assert sorted(binding._SIGS) == declared_functions()


def test_opts_defaults(lib):
    from paper_2601_10981_gb300 import binding
    o = binding.opts()
    assert (o.m_l, o.p, o.precision, o.lin_maxit) == (1, 1, 0, 200)
    assert o.aug_tol == 1e-12 and o.spin_limit == 1 << 22 and o.m_cap == 0


def test_status_strings(lib):
    assert lib.pr_status_string(0) == b"ok"
    assert lib.pr_status_string(6) == b"in-kernel barrier timed out"


def test_create_validates_arguments_before_touching_the_device(lib):
    from paper_2601_10981_gb300 import binding as b
    flow = b.flow_struct("abc")
    out = C.c_void_p()

    def create(n=16, eps=0.05, T=1.0, N=4, dt=1e-3, tol=5e-6, **kw):
        g = b.pr_grid(n, 0.0)
        o = b.opts(**kw)
        return lib.pr_create(C.byref(g), C.byref(flow), eps, T, N, dt, tol, C.byref(o), C.byref(out))

    assert create(n=2) == 9             # grid below the stencil's minimum
    assert create(n=300) == 9           # above the fine kernel's row tiling
    assert create(eps=0.0) == 1
    assert create(T=-1.0) == 1
    assert create(N=0) == 1
    assert create(dt=0.0) == 1
    assert create(tol=1.5) == 1
    assert create(m_l=2) == 9
    assert create(p=-1) == 9
    assert create(precision=5) == 1
    bad = b.flow_struct("abc")
    bad.kind = 7
    g = b.pr_grid(16, 0.0)
    assert lib.pr_create(C.byref(g), C.byref(bad), 0.1, 1.0, 4, 1e-3, 5e-6, None, C.byref(out)) == 1
    assert lib.pr_create(C.byref(g), C.byref(flow), 0.1, 1.0, 4, 1e-3, 5e-6, None, None) == 1
