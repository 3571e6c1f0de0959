"""Seeded synthetic inputs for the adaptive-parareal hot path.

This module builds the inputs that both the CUDA library and the CPU oracle receive:

* the workload recipes (grid size, velocity field, viscosity, horizon, number of time
  subintervals, fine step, snapshot count, POD rank cap), and
* the seeded fields: the initial state ``u0``, the forcing ``f`` and the optional
  divergence-free velocity perturbation ``b'``.

It holds none of the method's arithmetic (no operator, no time stepping, no POD); it
only draws random numbers and evaluates finite Fourier sums on the periodic grid.
Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), written out here from its published definition.

Field recipe (the paper's test problems are smooth periodic fields on [0, 2*pi]^3,
Sec. 4, eq. (eq1)):

    u0(x) = sin x sin y sin z + sum_{k in K(3)} a_k cos(k.x) + b_k sin(k.x)
    f(x)  =                     sum_{k in K(4)} a_k cos(k.x) + b_k sin(k.x)

where K(r) is the half-space of non-zero integer wave vectors with |k|_2 <= r (first
non-zero component positive, so every real mode appears once) and a_k, b_k are drawn
in the half-space order (kz, ky, kx ascending) from U[-0.1, 0.1].  Grid points are
x_i = i*h, h = L/n, and arrays are laid out [z][y][x] (x fastest, C order).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

TWO_PI = 2.0 * math.pi
_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 counter-based generator (Steele et al. 2014)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_pm(self, amp: float) -> float:
        """Uniform double in [-amp, amp)."""
        return amp * (2.0 * self.uniform() - 1.0)


def half_space_modes(kmax: int):
    """Non-zero integer wave vectors (kx, ky, kz) with |k|^2 <= kmax^2, one per +-k pair."""
    modes = []
    for kz in range(-kmax, kmax + 1):
        for ky in range(-kmax, kmax + 1):
            for kx in range(-kmax, kmax + 1):
                k2 = kx * kx + ky * ky + kz * kz
                if k2 == 0 or k2 > kmax * kmax:
                    continue
                if kz > 0 or (kz == 0 and (ky > 0 or (ky == 0 and kx > 0))):
                    modes.append((kx, ky, kz))
    return modes


def grid_1d(n: int, L: float = TWO_PI) -> np.ndarray:
    return np.arange(n, dtype=np.float64) * (L / n)


def fourier_field(n: int, kmax: int, seed: int, amp: float = 0.1,
                  L: float = TWO_PI) -> np.ndarray:
    """sum_k a_k cos(k.x) + b_k sin(k.x) over K(kmax), coefficients from SplitMix64(seed)."""
    rng = SplitMix64(seed)
    x = grid_1d(n, L) * (TWO_PI / L)  # phase per unit wave number
    # a cos(k.x) + b sin(k.x) = Re((a - i b) e^{i k.x}); the coefficients are drawn mode by
    # mode in half-space order and the sum is taken per kz over (ky, kx) planes, so that
    # the n^3 work is one product per distinct kz
    coef = {}
    for (kx, ky, kz) in half_space_modes(kmax):
        a = rng.uniform_pm(amp)
        b = rng.uniform_pm(amp)
        coef.setdefault(kz, {}).setdefault(ky, []).append((kx, a - 1j * b))
    e = lambda k: np.exp(1j * k * x)
    out = np.zeros((n, n, n), dtype=np.float64)
    for kz, rows in coef.items():
        plane = np.zeros((n, n), dtype=np.complex128)   # [y][x]
        for ky, terms in rows.items():
            cx = sum(c * e(kx) for kx, c in terms)
            plane += e(ky)[:, None] * cx[None, :]
        out += (e(kz)[:, None, None] * plane[None, :, :]).real
    return out


def initial_state(n: int, seed: int = 1, L: float = TWO_PI) -> np.ndarray:
    """u0 = sin x sin y sin z + seeded modes with |k| <= 3, amplitude 0.1."""
    x = grid_1d(n, L)
    s = np.sin(x)
    base = s[:, None, None] * s[None, :, None] * s[None, None, :]
    return base + fourier_field(n, 3, seed, 0.1, L)


def forcing(n: int, seed: int, L: float = TWO_PI) -> np.ndarray:
    """Zero-mean smooth forcing: seeded modes with |k| <= 4, amplitude 0.1."""
    return fourier_field(n, 4, seed, 0.1, L)


def perturbation(n: int, seed: int, amp: float = 0.05, L: float = TWO_PI) -> np.ndarray:
    """Seeded velocity perturbation b' = curl_h Psi, shape (3, n, n, n) = (b'_x, b'_y, b'_z).

    Psi = (Psi_x, Psi_y, Psi_z) are three seeded fields with |k| <= 4 (seeds 3*seed,
    3*seed + 1, 3*seed + 2), and curl_h takes central differences (f_{i+1} - f_{i-1})/(2h).
    Central differences along different axes commute, so the central-difference
    divergence of b' vanishes (up to rounding): the field is discretely divergence-free
    for the advection stencil.  b' is scaled so that max_{d, i} |b'_d(x_i)| = amp.
    This is part of the field's definition, not of the method.
    """
    h = L / n
    psi = [fourier_field(n, 4, 3 * seed + c, 1.0, L) for c in range(3)]

    def d(f, axis):   # axis: 2 = x, 1 = y, 0 = z of a [z][y][x] array
        return (np.roll(f, -1, axis=axis) - np.roll(f, 1, axis=axis)) / (2.0 * h)

    bx = d(psi[2], 1) - d(psi[1], 0)
    by = d(psi[0], 0) - d(psi[2], 2)
    bz = d(psi[1], 2) - d(psi[0], 1)
    b = np.stack([bx, by, bz])
    return b * (amp / np.max(np.abs(b)))


@dataclasses.dataclass(frozen=True)
class Flow:
    """Velocity field b(x, t) of the advection term.

    kind: 'abc'   b = (A sin z + C cos y, B sin x + A cos z, C sin y + B cos x)
          'kolmogorov'  b = (sin(k y), 0, 0)
          'const' b = (b0, b1, b2)
          'paper_kolmogorov'  b = (cos y, cos z, cos x) + (sin z, sin x, sin y) cos t
          'paper_abc'  ABC with every argument shifted by sin(w t)
    pert_seed > 0 adds the steady divergence-free perturbation
    perturbation(n, pert_seed, pert_amp) to a steady kind.
    """
    kind: str = "abc"
    A: float = 1.0
    B: float = 1.0
    C: float = 1.0
    k: int = 1
    w: float = 1.0
    b0: float = 0.0
    b1: float = 0.0
    b2: float = 0.0
    pert_seed: int = 0
    pert_amp: float = 0.05

    def pert(self, n: int) -> Optional[np.ndarray]:
        """The perturbation on an n^3 grid, or None."""
        return perturbation(n, self.pert_seed, self.pert_amp) if self.pert_seed > 0 else None


@dataclasses.dataclass(frozen=True)
class Workload:
    """One parareal problem: grid, flow, viscosity, horizon and discretisation sizes.

    n_snap = 0 means "snapshot every 5 fine steps" (the paper's delta_M); a positive
    n_snap fixes the number of snapshots per subinterval window instead.
    m_cap = 0 means no cap on the POD rank.
    """
    name: str
    n: int
    flow: Flow
    eps: float
    T: float
    n_sub: int
    dt: float
    n_snap: int = 0
    m_cap: int = 0
    k_max: int = 0
    u0_seed: int = 1
    f_seed: Optional[int] = None
    pod_tol: float = 5e-6
    m_l: int = 1
    p: int = 1

    @property
    def Ng(self) -> int:
        return self.n ** 3

    def u0(self) -> np.ndarray:
        return initial_state(self.n, self.u0_seed)

    def f(self) -> Optional[np.ndarray]:
        return None if self.f_seed is None else forcing(self.n, self.f_seed)


# The workloads this library is measured and checked on.
ABC_16 = Workload("abc16_eps0.05_N8", 16, Flow("abc"), 0.05, 1.0, 8, 1e-3,
                  n_snap=0, m_cap=8, k_max=8, u0_seed=1)
KOL_64 = Workload("kolmogorov4_64_eps0.01_N64", 64, Flow("kolmogorov", k=4), 0.01, 10.0, 64,
                  1e-3, n_snap=32, m_cap=16, k_max=0, u0_seed=1, f_seed=2)
ABC_128 = Workload("abc128_eps0.005_N256", 128, Flow("abc"), 0.005, 50.0, 256, 5e-4,
                   n_snap=64, m_cap=32, k_max=0, u0_seed=1)

KOL_256 = Workload("kolmogorov8_256_pert_eps0.002_N128", 256,
                   Flow("kolmogorov", k=8, pert_seed=4, pert_amp=0.05), 0.002, 20.0, 128, 2.5e-4,
                   n_snap=16, m_cap=8, k_max=0, u0_seed=1)

WORKLOADS = {w.name: w for w in (ABC_16, KOL_64, ABC_128, KOL_256)}


def tiny(n: int = 8, n_sub: int = 4, flow: Flow = Flow("abc"), eps: float = 0.05,
         T: float = 0.08, dt: float = 2e-3, f_seed: Optional[int] = None,
         m_cap: int = 6, n_snap: int = 0, m_l: int = 1, p: int = 1,
         pod_tol: float = 5e-6, name: str = "tiny") -> Workload:
    """A small workload the oracle finishes in well under a second."""
    return Workload(name, n, flow, eps, T, n_sub, dt, n_snap=n_snap, m_cap=m_cap,
                    u0_seed=1, f_seed=f_seed, m_l=m_l, p=p, pod_tol=pod_tol)


def serving_stream(n_requests: int = 200, rate: float = 5.0, seed: int = 5):
    """Mixed request stream: Poisson arrivals, random grid/flow/eps/horizon/subintervals."""
    rng = SplitMix64(seed)
    t = 0.0
    reqs = []
    for i in range(n_requests):
        t += -math.log(1.0 - rng.uniform()) / rate
        n = (32, 64, 96, 128)[int(rng.uniform() * 4)]
        if rng.uniform() < 0.5:
            flow = Flow("abc")
        else:
            flow = Flow("kolmogorov", k=(2, 4, 8)[int(rng.uniform() * 3)])
        eps = math.exp(math.log(0.002) + rng.uniform() * (math.log(0.05) - math.log(0.002)))
        T = 1.0 + 19.0 * rng.uniform()
        n_sub = (16, 32, 64)[int(rng.uniform() * 3)]
        reqs.append(dict(arrival=t, workload=Workload(
            f"req{i}", n, flow, eps, T, n_sub, 1e-3, n_snap=32, m_cap=16, u0_seed=1 + i)))
    return reqs
