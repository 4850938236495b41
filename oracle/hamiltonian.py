"""Sparse orthogonal TB Hamiltonian of Eq. 1.  TEST INFRASTRUCTURE ONLY.

    H = sum_i eps_i c_i^+ c_i + sum_{j in N(i)} t_ij c_i^+ c_j

stored as a SciPy CSR matrix in FP64 (diagonal included).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def csr_hamiltonian(n, indptr, indices, hop, onsite):
    off = sp.csr_matrix((np.asarray(hop, np.float64), np.asarray(indices), np.asarray(indptr)),
                        shape=(n, n))
    return (off + sp.diags(np.asarray(onsite, np.float64))).tocsr()


def symmetrize_directed(indptr, indices, y_dir):
    """H_ij = (y(i->j) + y(j->i)) / 2 for every stored entry (i, j).

    Implements the pz-pz case H_ij = H_ji of the symmetry stated after Eq. 2
    for a network whose raw output depends on the edge direction.
    """
    n = len(indptr) - 1
    m = sp.csr_matrix((np.asarray(y_dir, np.float64), indices, indptr), shape=(n, n))
    s = 0.5 * (m + m.T)
    s = s.tocsr()
    rows = np.repeat(np.arange(n), np.diff(indptr))
    return np.asarray(s[rows, indices]).reshape(-1)
