"""Multi-orbital (s, p, d) Slater-Koster Hamiltonian (the SK form of Eq. 1 with
the angular factors P_lambda(r_ij) of Sec. 3; the paper's 100-million-atom
graphene DOS uses an s, p and d model, Sec. 3).  TEST INFRASTRUCTURE ONLY.

Orbitals per atom, in this order (9):
    s, p_x, p_y, p_z, d_xy, d_yz, d_zx, d_{x^2-y^2}, d_{3z^2-r^2}

A hopping block H_ij (9 x 9) follows from the ten two-centre integrals
V = (ss_sigma, sp_sigma, pp_sigma, pp_pi, sd_sigma, pd_sigma, pd_pi,
dd_sigma, dd_pi, dd_delta) of the bond by rotation, not by the closed-form
table: in the bond frame (j at +z from i) the block B is diagonal in the
magnetic quantum number,
    B[s,s] = ss_sigma, B[s,p_z] = sp_sigma, B[p_z,p_z] = pp_sigma,
    B[p_x,p_x] = B[p_y,p_y] = pp_pi, B[s,d_z2] = sd_sigma,
    B[p_z,d_z2] = pd_sigma, B[p_x,d_zx] = B[p_y,d_yz] = pd_pi,
    B[d_z2,d_z2] = dd_sigma, B[d_zx,d_zx] = B[d_yz,d_yz] = dd_pi,
    B[d_xy,d_xy] = B[d_x2-y2,d_x2-y2] = dd_delta,
with B[b,a] = (-1)^(l_a + l_b) B[a,b] (parity); then H_ij = D(Q) B D(Q)^T
for any rotation Q taking e_z to the bond direction, with D = diag(1, D1, D2)
the real-orbital rotation matrices: D1 = Q on (x, y, z), and D2 acting on
the d orbitals as symmetric traceless tensors (T -> Q T Q^T) projected on an
orthonormal tensor basis of the five d orbitals.  B is invariant under
rotations about z, so the choice of Q about the bond does not matter.

The synthetic teacher (no trained network here) gives every integral the
distance form of the pz teacher:
    V_k(r) = V0_k exp(-beta (r / a_cc - 1)) f_c(r),
onsite energies E_s, E_p, E_d per orbital type, one species.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .teacher import cutoff

N_ORB = 9
L_OF = np.array([0, 1, 1, 1, 2, 2, 2, 2, 2])
S, PX, PY, PZ, DXY, DYZ, DZX, DX2, DZ2 = range(9)
INTEGRALS = ("ss_sigma", "sp_sigma", "pp_sigma", "pp_pi", "sd_sigma", "pd_sigma", "pd_pi", "dd_sigma", "dd_pi",
             "dd_delta")


@dataclass
class SKParams:
    v0: np.ndarray          # [10] prefactors (eV), order of INTEGRALS
    onsite: np.ndarray      # [3] E_s, E_p, E_d (eV)
    a_cc: float = 1.42
    beta: float = 3.0
    rcut: float = 3.0


def bond_frame_block(v):
    """B (9 x 9) in the bond frame from the ten integrals v."""
    ss, sps, pps, ppp, sds, pds, pdp, dds, ddp, ddd = [float(x) for x in v]
    B = np.zeros((9, 9))
    B[S, S] = ss
    B[S, PZ] = sps
    B[PZ, PZ] = pps
    B[PX, PX] = B[PY, PY] = ppp
    B[S, DZ2] = sds
    B[PZ, DZ2] = pds
    B[PX, DZX] = B[PY, DYZ] = pdp
    B[DZ2, DZ2] = dds
    B[DZX, DZX] = B[DYZ, DYZ] = ddp
    B[DXY, DXY] = B[DX2, DX2] = ddd
    for a in range(9):
        for b in range(a + 1, 9):
            if B[a, b] != 0.0:
                B[b, a] = (-1) ** (L_OF[a] + L_OF[b]) * B[a, b]
    return B


def _d_tensors():
    """Orthonormal (Frobenius) symmetric traceless tensors of the five real d
    orbitals, in the order d_xy, d_yz, d_zx, d_x2-y2, d_3z2-r2 (a d orbital
    is x^T T x / r^2 up to normalisation)."""
    T = np.zeros((5, 3, 3))
    T[0][0, 1] = T[0][1, 0] = 1.0
    T[1][1, 2] = T[1][2, 1] = 1.0
    T[2][2, 0] = T[2][0, 2] = 1.0
    T[3][0, 0], T[3][1, 1] = 1.0, -1.0
    T[4][0, 0], T[4][1, 1], T[4][2, 2] = -1.0, -1.0, 2.0
    for k in range(5):
        T[k] /= np.linalg.norm(T[k])
    return T


_DT = _d_tensors()


def rotation_to(d):
    """A rotation matrix Q with Q e_z = d / |d|."""
    z = np.asarray(d, np.float64) / np.linalg.norm(d)
    helper = np.array([1.0, 0.0, 0.0]) if abs(z[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    x = helper - z * np.dot(helper, z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return np.stack([x, y, z], axis=1)    # columns: images of e_x, e_y, e_z


def orbital_rotation(Q):
    """D = diag(1, D1, D2) for the 9 real orbitals."""
    D = np.zeros((9, 9))
    D[0, 0] = 1.0
    D[1:4, 1:4] = Q
    for a in range(5):
        for b in range(5):
            D[4 + a, 4 + b] = np.sum(_DT[a] * (Q @ _DT[b] @ Q.T))
    return D


def hopping_block(d, v):
    """H_ij (9 x 9) for bond vector d = r_j - r_i and integrals v."""
    D = orbital_rotation(rotation_to(d))
    return D @ bond_frame_block(v) @ D.T


def integrals(r, p: SKParams):
    """V_k(r) for the ten integrals (0 beyond r_cut)."""
    r = np.asarray(r, np.float64)
    radial = np.exp(-p.beta * (r / p.a_cc - 1.0)) * cutoff(r, p.rcut)
    return np.asarray(p.v0, np.float64)[None, :] * radial[..., None]


def onsite_vector(p: SKParams):
    e = np.asarray(p.onsite, np.float64)
    return np.array([e[0], e[1], e[1], e[1], e[2], e[2], e[2], e[2], e[2]])


def sk_hamiltonian(n_atoms, indptr, indices, disp, p: SKParams):
    """Sparse 9N x 9N H: orbital index 9 i + a."""
    rows, cols, vals = [], [], []
    V = integrals(np.linalg.norm(disp, axis=1), p)
    for i in range(n_atoms):
        for e in range(indptr[i], indptr[i + 1]):
            j = int(indices[e])
            blk = hopping_block(disp[e], V[e])
            r = 9 * i + np.repeat(np.arange(9), 9)
            c = 9 * j + np.tile(np.arange(9), 9)
            rows.append(r)
            cols.append(c)
            vals.append(blk.reshape(-1))
    on = onsite_vector(p)
    rows.append(np.arange(9 * n_atoms))
    cols.append(np.arange(9 * n_atoms))
    vals.append(np.tile(on, n_atoms))
    H = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(9 * n_atoms, 9 * n_atoms))
    H.sum_duplicates()
    return H


def gershgorin(H):
    """Row-sum enclosure of the spectrum of a sparse symmetric H."""
    H = sp.csr_matrix(H)
    diag = H.diagonal()
    radius = np.asarray(abs(H).sum(axis=1)).reshape(-1) - np.abs(diag)
    return float(np.min(diag - radius)), float(np.max(diag + radius))
