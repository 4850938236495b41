"""Spectral bounds for the Chebyshev rescaling (Sec. 2.4).  TEST INFRASTRUCTURE ONLY.

The Chebyshev expansion of the LSQT method needs the spectrum of H inside
[-1, 1] after H~ = (H - b) / a.  Two FP64 estimates are combined:

* Gershgorin: every eigenvalue lies in [min_i(H_ii - R_i), max_i(H_ii + R_i)]
  with R_i = sum_{j != i} |H_ij| -- a guaranteed enclosure.
* Lanczos: k steps of the symmetric Lanczos three-term recurrence (no
  reorthogonalisation) from a seeded real start vector q, giving a
  tridiagonal T_k whose extreme eigenvalues (Ritz values theta_min,
  theta_max) are found by Sturm-sequence bisection.

Combination used here:
  delta = 0.01 (theta_max - theta_min)
  E_max = min(G_max, theta_max + delta),  E_min = max(G_min, theta_min - delta)
  a = (E_max - E_min) / (2 - eps),  b = (E_max + E_min) / 2,  eps = 0.01.

The Lanczos start vector is q_i = u(seed, 0, i) - 1/2 (u as in ``kpm``),
normalised.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .kpm import uniform


def gershgorin(H):
    H = sp.csr_matrix(H)
    diag = H.diagonal()
    absrow = np.asarray(abs(H).sum(axis=1)).reshape(-1) - np.abs(diag)
    return float(np.min(diag - absrow)), float(np.max(diag + absrow))


def lanczos_tridiagonal(H, k, seed):
    """alpha [m], beta [m-1] of the Lanczos tridiagonal, m <= k."""
    n = H.shape[0]
    q = uniform(seed, np.zeros(n, np.uint64), np.arange(n, dtype=np.uint64)) - 0.5
    q = q / np.sqrt(np.dot(q, q))
    q_prev = np.zeros(n)
    beta_prev = 0.0
    alpha, beta = [], []
    for j in range(k):
        w = H @ q - beta_prev * q_prev
        a = float(np.dot(q, w))
        w = w - a * q
        alpha.append(a)
        bnorm = float(np.sqrt(np.dot(w, w)))
        if j == k - 1 or bnorm <= 1e-300:
            break
        beta.append(bnorm)
        q_prev, q = q, w / bnorm
        beta_prev = bnorm
    return np.array(alpha), np.array(beta)


def sturm_count(alpha, beta, x):
    """Number of eigenvalues of tridiag(alpha, beta) strictly below x."""
    count = 0
    d = 1.0
    for i in range(alpha.size):
        off = beta[i - 1] ** 2 if i > 0 else 0.0
        d = (alpha[i] - x) - (off / d if i > 0 else 0.0)
        if d == 0.0:
            d = -1e-300
        if d < 0.0:
            count += 1
    return count


def tridiagonal_extremes(alpha, beta, iters=200):
    """(theta_min, theta_max) of tridiag(alpha, beta) by bisection."""
    m = alpha.size
    ext = np.zeros(m)
    ext[:-1] += np.abs(beta)
    ext[1:] += np.abs(beta)
    lo0, hi0 = float(np.min(alpha - ext)), float(np.max(alpha + ext))

    def bisect(target_count_at_least):
        lo, hi = lo0, hi0
        for _ in range(iters):
            mid = 0.5 * (lo + hi)
            if mid <= lo or mid >= hi:
                break
            if sturm_count(alpha, beta, mid) >= target_count_at_least:
                hi = mid
            else:
                lo = mid
        return 0.5 * (lo + hi)

    return bisect(1), bisect(m)


def spectral_bounds(H, lanczos_steps=64, seed=7, eps=0.01, margin=0.01):
    """(E_min, E_max, a, b) as described in the module docstring."""
    gmin, gmax = gershgorin(H)
    alpha, beta = lanczos_tridiagonal(H, lanczos_steps, seed)
    tmin, tmax = tridiagonal_extremes(alpha, beta)
    delta = margin * (tmax - tmin)
    emax = min(gmax, tmax + delta)
    emin = max(gmin, tmin - delta)
    a = (emax - emin) / (2.0 - eps)
    b = 0.5 * (emax + emin)
    return emin, emax, a, b
