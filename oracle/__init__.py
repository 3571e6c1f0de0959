"""Plain FP64 CPU oracle of the MOR-based adaptive parareal method (arXiv 2601.10981).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this package.
The CUDA library never calls it and shares no code with it; both sides receive the same
seeded inputs from ``pr_inputs``.

The oracle is written for a reader checking it against the paper: numpy arrays, library
primitives (matmul, ``eigh``, ``solve``, ``cholesky``) as single steps, no blocking or
fusion.  Modules:

* ``discretisation`` - periodic finite-difference form of the operator in eq. (eq1)
  (the FD analogue of the P1 FEM of Sec. 2.2), velocity fields of Sec. 4.
* ``fine``           - implicit Euler fine propagator, eq. (semi-dis-eq)/(algform), with a
  textbook BiCGStab or a dense LU solve per step.
* ``pod``            - POD_Mode (Algorithm 1) with one Cholesky QR re-orthonormalisation,
  and the two-level POD of Case II, eq. (W^k_n).
* ``coarse``         - the Galerkin-reduced coarse propagator, eqs. (eq8)/(eq00)/(eq13), and
  the augmentation of eqs. (eqaug)/(eq12).
* ``parareal``       - Algorithm 2 with the update of eq. (formula4), the sequential fine
  reference and the error of eq. (error).

Every function is pinned by a ``-m "not gpu"`` test (Fourier symbol, dense brute force,
invariants, SVD identity, finite termination, complete-basis and dense-Galerkin checks);
see ``tests/test_oracle_*.py``.
"""
from .discretisation import (Grid, velocity, apply_L, apply_LT, assemble_L_dense,
                             make_operator)
from .fine import bicgstab, implicit_euler_step, fine_propagate
from .pod import pod_mode, cholqr, level2_blocks
from .coarse import coarse_propagate, augment, galerkin_project
from .parareal import Params, derive_params, iteration0, parareal, sequential_fine, rel_l2

__all__ = [
    "Grid", "velocity", "apply_L", "apply_LT", "assemble_L_dense", "make_operator",
    "bicgstab", "implicit_euler_step", "fine_propagate",
    "pod_mode", "cholqr", "level2_blocks",
    "coarse_propagate", "augment", "galerkin_project",
    "Params", "derive_params", "iteration0", "parareal", "sequential_fine", "rel_l2",
]
