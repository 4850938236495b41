"""Environment network of Eq. 2, the SK-form pz hopping and band-energy
training with the loss of Eq. 3 (the band form, Sec. 3).  TEST
INFRASTRUCTURE ONLY.

Model (the hopping H_ij = sum_lambda MLP_lambda(e_ij) P_lambda(r_ij_hat) and
the onsite H_ii = MLP_alpha(v_i) of Sec. 3, for one pz orbital per atom):

    v_i   = sum_{j in N(i)} C(r_ij)                       node feature (Eq. 2)
    u_ij  = v_i + v_j      (= sum_{k in N(i)} C(r_ik) + sum_{l in N(j)} C(r_jl))
    m_ij  = MLP_e(u_ij):   8 -> 32 (SiLU) -> 8             environment network
    e_ij  = C(r_ij) * m_ij                               edge feature (Eq. 2)
    y_ij  = MLP_lambda(e_ij): 8 -> 32 (SiLU) -> 32 (SiLU) -> 2   (sigma, pi)
    t_ij  = y_sigma n_z^2 + y_pi (1 - n_z^2),   n_z = d_z / r
            (the pz-pz Slater-Koster angular factors)
    eps_i = eps0[Z_i] + MLP_alpha(v_i)[Z_i]:  8 -> 32 (SiLU) -> 3

u, C(r) and n_z^2 are the same for i -> j and j -> i, so H is symmetric
without a symmetrisation step (the pz-pz case of the symmetry after Eq. 2).

Bloch sum (periodic cells; every stored neighbour (i, j) carries its bond
vector d = r_j + T - r_i of one image):

    H(k)_ij = sum over stored (i, j, d) of t e^{i k.d}  +  eps_i delta_ij

Bands E_b(k) are the eigenvalues of H(k) in ascending order.  Loss (Eq. 3),
summed over the cells c, k-points and bands b of a batch:

    D = E_pred - E_ref,   S = sum w_b |D|,   L = S^2 + sum w_b D^2,
    dL/dE = 2 S w_b sign(D) + 2 w_b D        (sign(0) = 0)

Gradients with respect to the Hamiltonian follow the Hellmann-Feynman
theorem for non-degenerate bands: dE_b/dt_e = Re(conj(psi_b[i]) psi_b[j]
e^{i k.d_e}) for a stored element e = (i, j, d_e), dE_b/deps_i = |psi_b[i]|^2.

Parameters are one flat vector in the order of ENV_LAYOUT (weights row-major
[out][in]).
"""
from __future__ import annotations

import numpy as np

from . import descriptors as ode

ENV_LAYOUT = (("We1", (32, 8)), ("be1", (32,)), ("We2", (8, 32)), ("be2", (8,)),
              ("Wh1", (32, 8)), ("bh1", (32,)), ("Wh2", (32, 32)), ("bh2", (32,)),
              ("Wh3", (2, 32)), ("bh3", (2,)),
              ("Wo1", (32, 8)), ("bo1", (32,)), ("Wo2", (3, 32)), ("bo2", (3,)))
ENV_NPARAM = int(sum(np.prod(s) for _, s in ENV_LAYOUT))


def unpack(flat):
    flat = np.asarray(flat, np.float64)
    assert flat.size == ENV_NPARAM
    out, k = {}, 0
    for name, shape in ENV_LAYOUT:
        m = int(np.prod(shape))
        out[name] = flat[k:k + m].reshape(shape)
        k += m
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], np.float64).reshape(-1) for name, _ in ENV_LAYOUT])


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def silu(z):
    return z * sigmoid(z)


def silu_grad(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


# ------------------------------------------------------------------ inputs

def edge_inputs(species, indptr, indices, dvec, cmix, rcut):
    """(C [E, 8], u [E, 8], n_z^2 [E], v [N, 8]) for the CSR neighbour list."""
    species = np.asarray(species)
    dvec = np.asarray(dvec, np.float64)
    r = np.sqrt(np.sum(dvec * dvec, axis=1))
    rows = np.repeat(np.arange(len(indptr) - 1), np.diff(indptr))
    C = ode.mixed_descriptor(r, species[rows], species[indices], cmix, rcut)
    v = ode.node_features(len(indptr) - 1, indptr, C)
    u = v[rows] + v[indices]
    nz2 = (dvec[:, 2] / r) ** 2
    return C, u, nz2, v


# ------------------------------------------------------------------ network

def hopping_forward(flat, C, u, nz2):
    p = unpack(flat)
    z1 = u @ p["We1"].T + p["be1"]
    h1 = silu(z1)
    m = h1 @ p["We2"].T + p["be2"]
    e = C * m
    z2 = e @ p["Wh1"].T + p["bh1"]
    h2 = silu(z2)
    z3 = h2 @ p["Wh2"].T + p["bh2"]
    h3 = silu(z3)
    y = h3 @ p["Wh3"].T + p["bh3"]
    t = y[:, 0] * nz2 + y[:, 1] * (1.0 - nz2)
    return t, dict(C=C, u=u, nz2=nz2, z1=z1, h1=h1, m=m, e=e, z2=z2, h2=h2, z3=z3, h3=h3)


def hopping_backward(flat, cache, gt):
    """dL/dparams (flat) from dL/dt per edge."""
    p = unpack(flat)
    c = cache
    gt = np.asarray(gt, np.float64)
    dy = np.stack([gt * c["nz2"], gt * (1.0 - c["nz2"])], axis=1)
    g = {name: np.zeros(shape) for name, shape in ENV_LAYOUT}
    g["Wh3"] = dy.T @ c["h3"]
    g["bh3"] = dy.sum(0)
    dz3 = (dy @ p["Wh3"]) * silu_grad(c["z3"])
    g["Wh2"] = dz3.T @ c["h2"]
    g["bh2"] = dz3.sum(0)
    dz2 = (dz3 @ p["Wh2"]) * silu_grad(c["z2"])
    g["Wh1"] = dz2.T @ c["e"]
    g["bh1"] = dz2.sum(0)
    dm = (dz2 @ p["Wh1"]) * c["C"]
    g["We2"] = dm.T @ c["h1"]
    g["be2"] = dm.sum(0)
    dz1 = (dm @ p["We2"]) * silu_grad(c["z1"])
    g["We1"] = dz1.T @ c["u"]
    g["be1"] = dz1.sum(0)
    return pack(g)


def onsite_forward(flat, v, species, eps0):
    p = unpack(flat)
    species = np.asarray(species)
    z = v @ p["Wo1"].T + p["bo1"]
    h = silu(z)
    out = h @ p["Wo2"].T + p["bo2"]
    eps = np.asarray(eps0, np.float64)[species] + out[np.arange(len(species)), species]
    return eps, dict(v=v, z=z, h=h, species=species)


def onsite_backward(flat, cache, geps):
    p = unpack(flat)
    c = cache
    n = len(c["species"])
    dout = np.zeros((n, 3))
    dout[np.arange(n), c["species"]] = geps
    g = {name: np.zeros(shape) for name, shape in ENV_LAYOUT}
    g["Wo2"] = dout.T @ c["h"]
    g["bo2"] = dout.sum(0)
    dz = (dout @ p["Wo2"]) * silu_grad(c["z"])
    g["Wo1"] = dz.T @ c["v"]
    g["bo1"] = dz.sum(0)
    return pack(g)


# ------------------------------------------------------------------ bands

def bloch_hamiltonian(n, indptr, indices, dvec, t, eps, k):
    """Dense complex H(k) [n, n] of one periodic cell."""
    Hk = np.zeros((n, n), complex)
    k = np.asarray(k, np.float64)
    for i in range(n):
        for e in range(indptr[i], indptr[i + 1]):
            Hk[i, indices[e]] += t[e] * np.exp(1j * np.dot(k, dvec[e]))
        Hk[i, i] += eps[i]
    return Hk


def bands(n, indptr, indices, dvec, t, eps, kpts):
    """(E [nk, n] ascending, psi [nk, n, n] with psi[q][:, b] the b-th
    eigenvector) by the library's dense Hermitian eigensolver."""
    E = np.empty((len(kpts), n))
    psi = np.empty((len(kpts), n, n), complex)
    for q, k in enumerate(kpts):
        E[q], psi[q] = np.linalg.eigh(bloch_hamiltonian(n, indptr, indices, dvec, t, eps, k))
    return E, psi


def band_loss(E, E_ref, w):
    """(L, dL/dE) of Eq. 3 over arrays [..., n_bands] with band weights w."""
    D = np.asarray(E, np.float64) - np.asarray(E_ref, np.float64)
    w = np.broadcast_to(np.asarray(w, np.float64), D.shape)
    S = float(np.sum(w * np.abs(D)))
    L = S * S + float(np.sum(w * D * D))
    return L, 2.0 * S * w * np.sign(D) + 2.0 * w * D


def band_gradient(indptr, indices, dvec, kpts, psi, dLdE):
    """(dL/dt per stored element, dL/deps per atom) of one cell."""
    n = len(indptr) - 1
    rows = np.repeat(np.arange(n), np.diff(indptr))
    gt = np.zeros(len(indices))
    geps = np.zeros(n)
    for q, k in enumerate(kpts):
        P = psi[q]                       # [atom, band]
        g = np.asarray(dLdE[q], np.float64)
        phase = np.exp(1j * (np.asarray(dvec, np.float64) @ np.asarray(k, np.float64)))
        # sum_b g_b conj(psi_b[i]) psi_b[j] e^{i k.d}
        gt += np.real(np.einsum("eb,eb,b->e", np.conj(P[rows]), P[indices], g) * phase)
        geps += np.einsum("ib,b->i", np.abs(P) ** 2, g)
    return gt, geps


# ------------------------------------------------------------------ training step

def cell_loss_and_grad(flat, cells, kpts, E_ref, w, eps0):
    """Eq. 3 over a batch of cells and its gradient with respect to the flat
    parameters.  cells: list of dicts with n, species, indptr, indices, dvec,
    C, u, nz2, v.  E_ref [cells, nk, n]."""
    Es, caches = [], []
    for c in cells:
        t, hc = hopping_forward(flat, c["C"], c["u"], c["nz2"])
        eps, oc = onsite_forward(flat, c["v"], c["species"], eps0)
        E, psi = bands(c["n"], c["indptr"], c["indices"], c["dvec"], t, eps, kpts)
        Es.append(E)
        caches.append((hc, oc, psi))
    L, dLdE = band_loss(np.stack(Es), E_ref, w)
    grad = np.zeros(ENV_NPARAM)
    for c, (hc, oc, psi), g in zip(cells, caches, dLdE):
        gt, geps = band_gradient(c["indptr"], c["indices"], c["dvec"], kpts, psi, g)
        grad += hopping_backward(flat, hc, gt) + onsite_backward(flat, oc, geps)
    return L, grad, np.stack(Es)
