"""KPM density of states, Eq. 4.  TEST INFRASTRUCTURE ONLY.

Eq. 4 defines rho(E) = (2 / Omega) Tr[delta(E - H)].  The library returns the
density per orbital and per eV, (1/N) Tr[delta(E - H)], which integrates to 1;
multiplying by 2 (spin) and by N / Omega gives Eq. 4.

With rescaled energy x = (E - b) / a and KPM moments mu_n (``kpm``):

    rho(E) = [ g_0 mu_0 + 2 sum_{n=1}^{M-1} g_n mu_n T_n(x) ] / (pi a sqrt(1 - x^2))

for |x| < 1 and 0 otherwise.  Damping kernels (Weisse et al., RMP 78, 275):

    Jackson  g_n = [ (M - n + 1) cos(pi n / (M + 1))
                     + sin(pi n / (M + 1)) cot(pi / (M + 1)) ] / (M + 1)
    Lorentz  g_n = sinh(lam (1 - n / M)) / sinh(lam)
    none     g_n = 1
"""
from __future__ import annotations

import numpy as np

from .descriptors import chebyshev_T

JACKSON, LORENTZ, NONE = 0, 1, 2


def kernel_coefficients(M, kind=JACKSON, lam=4.0):
    n = np.arange(M, dtype=np.float64)
    if kind == JACKSON:
        q = np.pi / (M + 1)
        return ((M - n + 1) * np.cos(q * n) + np.sin(q * n) / np.tan(q)) / (M + 1)
    if kind == LORENTZ:
        return np.sinh(lam * (1.0 - n / M)) / np.sinh(lam)
    return np.ones(M)


def density_of_states(mu, a, b, energies, kind=JACKSON, lam=4.0):
    mu = np.asarray(mu, np.float64)
    M = mu.size
    g = kernel_coefficients(M, kind, lam)
    x = (np.asarray(energies, np.float64) - b) / a
    inside = np.abs(x) < 1.0
    xs = np.where(inside, x, 0.0)
    T = chebyshev_T(M, xs)                          # [M, K]
    coef = g * mu
    coef[1:] *= 2.0
    series = coef @ T
    rho = series / (np.pi * a * np.sqrt(1.0 - xs * xs))
    return np.where(inside, rho, 0.0)
