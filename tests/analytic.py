"""Closed-form references used to pin the oracle (no oracle code here).

* Nearest-neighbour graphene band structure E(k) = +-|t| |1 + e^{i k.a1} + e^{i k.a2}|
  (Wallace, Phys. Rev. 71, 622 (1947); Castro Neto et al., RMP 81, 109 (2009), Eq. 6).
* Its density of states in closed form with the complete elliptic integral
  (Hobson & Nierenberg, Phys. Rev. 89, 662 (1953); Castro Neto et al., Eq. 14),
  per 2-atom unit cell, so it integrates to 2.
"""
import numpy as np
from scipy.special import ellipk


def nn_graphene_bands_torus(n1, n2, t):
    """All 2 n1 n2 eigenvalues of NN graphene on an n1 x n2 primitive torus."""
    m1, m2 = np.meshgrid(np.arange(n1), np.arange(n2), indexing="ij")
    f = 1.0 + np.exp(2j * np.pi * m1 / n1) + np.exp(2j * np.pi * m2 / n2)
    e = abs(t) * np.abs(f).reshape(-1)
    return np.sort(np.concatenate([-e, e]))


def nn_graphene_band_samples(nk, t):
    """+-|t||f(k)| on an nk x nk uniform grid of the Brillouin zone."""
    return nn_graphene_bands_torus(nk, nk, t)


def nn_graphene_dos_closed_form(E, t):
    """DOS per atom per eV (integrates to 1) of infinite NN graphene."""
    t = abs(t)
    E = np.atleast_1d(np.asarray(E, np.float64))
    out = np.zeros_like(E)
    for k, en in enumerate(E):
        e = abs(en / t)
        if e == 0.0 or e >= 3.0:
            continue
        q = (1.0 + e) ** 2 - ((e * e - 1.0) ** 2) / 4.0
        if e < 1.0:
            z0, z1 = q, 4.0 * e
        else:
            z0, z1 = 4.0 * e, q
        out[k] = 2.0 * e / (t * np.pi ** 2) / np.sqrt(z0) * ellipk(z1 / z0) / 2.0
    return out


def chebyshev_moments_of_levels(levels, a, b, M):
    """mu_n = mean over levels of T_n((E - b)/a) = cos(n arccos x)."""
    x = np.clip((np.asarray(levels) - b) / a, -1.0, 1.0)
    th = np.arccos(x)
    n = np.arange(M)[:, None]
    return np.cos(n * th[None, :]).mean(axis=1)
