"""Cost model and speedup estimate of the adaptive parareal method (Sec. 3.3 and the
per-iteration accounting of Sec. 4), applied to measured phase times.

Per parareal iteration k >= 1 (Sec. 4.1): T_total = T_F + T_U + T_C + N (T_G + T_A), where
T_F is the fine propagation of one subinterval, T_U the reduced-system build, T_C the POD
build, T_G the coarse propagation and T_A the augmentation of one subinterval.  On a
machine that runs all subintervals concurrently the estimated speedup over the
sequential fine solve is  T_F N / (T_total (k + 1))  (the cheaper iteration 0 counted as
one more iteration).  The asymptotic form of eq. (speedup) is
N / ((1 + C_p3 m_max dt N / (C_f DeltaT)) k).
"""
from __future__ import annotations


def iteration_total(T_F: float, T_G: float, T_U: float, T_C: float, T_A: float, N: int) -> float:
    """Wall time of one parareal iteration, T_F + T_U + T_C + N (T_G + T_A)."""
    return T_F + T_U + T_C + N * (T_G + T_A)


def speedup_estimate(T_F: float, N: int, T_total: float, k: int) -> float:
    """T_F N / (T_total (k + 1)): sequential fine cost over the parareal cost of k
    iterations plus iteration 0."""
    return T_F * N / (T_total * (k + 1))


def speedup_model(N: int, k_max: int, m_max: int, dt: float, DeltaT: float,
                  Cp3_over_Cf: float) -> float:
    """eq. (speedup): N / ((1 + (C_p3 m_max / C_f)(dt / DeltaT) N) k_max)."""
    return N / ((1.0 + Cp3_over_Cf * m_max * (dt / DeltaT) * N) * k_max)


def cost_seq(N: int, DeltaT: float, T0: float, dt: float, tau_F: float) -> float:
    """(N DeltaT/dt + T0/dt) tau_F: the fine propagator over [0, T] one step at a time."""
    return (N * DeltaT / dt + T0 / dt) * tau_F


def cost_par(N: int, k_max: int, DeltaT: float, T0: float, dt: float, dT: float, tau_F: float,
             tau_G: float, T_C: float, T_U: float, T_A: float) -> float:
    """Sec. 3.3: T0/dt tau_F + T_C + T_U + N DeltaT/dT tau_G
       + sum_{k=1}^{k_max} (DeltaT/dt tau_F + T_C + T_U + (N - k)(T_A + DeltaT/dT tau_G))."""
    c = T0 / dt * tau_F + T_C + T_U + N * DeltaT / dT * tau_G
    for k in range(1, k_max + 1):
        c += DeltaT / dt * tau_F + T_C + T_U + (N - k) * (T_A + DeltaT / dT * tau_G)
    return c
