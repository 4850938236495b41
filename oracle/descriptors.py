"""Radial Chebyshev descriptors of Eq. 2.  TEST INFRASTRUCTURE ONLY.

    f_k(r)  = (1/2) [T_k(2 (r / r_cut - 1)^2 - 1) + 1] f_c(r),   k = 0..7
    C_n(r)  = sum_k c^{Z_i Z_j}_{nk} f_k(r)
    v_i     = sum_{j in N(i)} C_n(r_ij)                     (node feature)

The per-edge input of the per-pair MLP (the reduced form of e_ij in Eq. 2,
with the environment network taken as the identity) is the 32-vector

    x_ij = [ C(r_ij), v_i, v_j, C(r_ij) * (v_i + v_j) ]

T_k is evaluated by the three-term recurrence T_0 = 1, T_1 = x,
T_{k+1} = 2 x T_k - T_{k-1}.
"""
from __future__ import annotations

import numpy as np

from .teacher import cutoff


def chebyshev_T(n_terms, x):
    """[n_terms, ...] array of T_0(x) .. T_{n_terms-1}(x) by recurrence."""
    x = np.asarray(x, np.float64)
    out = np.empty((n_terms,) + x.shape)
    out[0] = 1.0
    if n_terms > 1:
        out[1] = x
    for k in range(1, n_terms - 1):
        out[k + 1] = 2.0 * x * out[k] - out[k - 1]
    return out


def radial_basis(r, rcut, n_basis=8):
    """f_k(r) for k = 0..n_basis-1, shape [..., n_basis]."""
    r = np.asarray(r, np.float64)
    x = 2.0 * (r / rcut - 1.0) ** 2 - 1.0
    t = chebyshev_T(n_basis, x)                       # [K, ...]
    f = 0.5 * (t + 1.0) * cutoff(r, rcut)[None]
    return np.moveaxis(f, 0, -1)


def mixed_descriptor(r, zi, zj, cmix, rcut):
    """C_n(r_ij) = sum_k c^{Z_i Z_j}_{nk} f_k(r_ij), shape [E, n_basis]."""
    f = radial_basis(r, rcut, cmix.shape[-1])             # [E, K]
    c = np.asarray(cmix, np.float64)[zi, zj]             # [E, N, K]
    return np.einsum("enk,ek->en", c, f)


def node_features(n_atoms, indptr, C):
    """v_i = sum over the CSR row of C_n(r_ij)."""
    rows = np.repeat(np.arange(n_atoms), np.diff(indptr))
    v = np.zeros((n_atoms, C.shape[1]))
    np.add.at(v, rows, C)
    return v


def edge_features(indptr, indices, C, v):
    """x_ij = [C, v_i, v_j, C * (v_i + v_j)] for every CSR entry, [E, 32]."""
    rows = np.repeat(np.arange(len(indptr) - 1), np.diff(indptr))
    vi, vj = v[rows], v[indices]
    return np.concatenate([C, vi, vj, C * (vi + vj)], axis=1)


def descriptors(species, indptr, indices, dvec, cmix, rcut):
    """Convenience: (C per edge, v per atom, x per edge)."""
    species = np.asarray(species)
    r = np.sqrt(np.sum(np.asarray(dvec, np.float64) ** 2, axis=-1))
    rows = np.repeat(np.arange(len(indptr) - 1), np.diff(indptr))
    C = mixed_descriptor(r, species[rows], species[indices], cmix, rcut)
    v = node_features(len(indptr) - 1, indptr, C)
    x = edge_features(indptr, indices, C, v)
    return C, v, x
