"""Analytic environment-dependent teacher TB model.  TEST INFRASTRUCTURE ONLY.

The paper trains on DFT band structures (Sec. 2.3, Eq. 3) that are not
available here; the teacher below generates the labels instead.  It is an
orthogonal pz Hamiltonian of the form of Eq. 1 with one orbital per atom:

    t_ij  = P[Z_i, Z_j] * exp(-beta (r_ij / a_cc - 1))
            * (1 + gamma (n_i + n_j - 6) / 6) * f_c(r_ij)
    eps_i = onsite[Z_i]

with n_i the number of neighbours of atom i closer than r_count and f_c the
smooth cosine cutoff f_c(r) = (1 + cos(pi r / r_cut)) / 2 for r < r_cut, else
0 (the "smooth cutoff function" named below Eq. 2; the cosine form is this
build's reading).  Hoppings are symmetric (t_ij = t_ji), as the pz-pz case of
the symmetry stated after Eq. 2 requires.
"""
from __future__ import annotations

import numpy as np


def cutoff(r, rcut):
    """Smooth cosine cutoff f_c(r) = (1 + cos(pi r / rcut)) / 2 on r < rcut."""
    r = np.asarray(r, np.float64)
    return np.where(r < rcut, 0.5 * (1.0 + np.cos(np.pi * r / rcut)), 0.0)


def distances(dvec):
    return np.sqrt(np.sum(np.asarray(dvec, np.float64) ** 2, axis=-1))


def coordination(indptr, dist, r_count):
    """n_i = #{j in N(i): r_ij < r_count} (integer per atom)."""
    n = len(indptr) - 1
    close = (np.asarray(dist) < r_count).astype(np.int64)
    counts = np.zeros(n, np.int64)
    rows = np.repeat(np.arange(n), np.diff(indptr))
    np.add.at(counts, rows, close)
    return counts


def hopping(r, zi, zj, ni, nj, params):
    """Teacher hopping t(r; Z_i, Z_j, n_i, n_j) in eV (vectorised)."""
    r = np.asarray(r, np.float64)
    pref = np.asarray(params.hop_prefactor, np.float64)[zi, zj]
    radial = np.exp(-params.beta * (r / params.a_cc - 1.0))
    env = 1.0 + params.gamma * ((np.asarray(ni) + np.asarray(nj)) - 6.0) / 6.0
    return pref * radial * env * cutoff(r, params.rcut)


def teacher_elements(species, indptr, indices, dvec, params):
    """Per-CSR-entry hoppings t_ij and per-atom onsite energies eps_i."""
    species = np.asarray(species)
    dist = distances(dvec)
    n_count = coordination(indptr, dist, params.r_count)
    rows = np.repeat(np.arange(len(indptr) - 1), np.diff(indptr))
    t = hopping(dist, species[rows], species[indices], n_count[rows], n_count[indices], params)
    eps = np.asarray(params.onsite, np.float64)[species]
    return t, eps, n_count
