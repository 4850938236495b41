"""The per-pair SiLU MLP, its loss and the AdamW update.  TEST INFRASTRUCTURE ONLY.

Network (Sec. 3: "an MLP with a SiLU nonlinear activation function"), one
evaluation per directed edge i->j with input x_ij from ``descriptors``:

    xn = (x - mean) * inv_std                 frozen input normalisation
    z1 = xn W1^T + b1,  h1 = silu(z1)          32 -> 64
    z2 = h1 W2^T + b2,  h2 = silu(z2)          64 -> 64
    y  = h2 W3^T + b3                          64 -> 2   (y0 hopping, y1 onsite share)

Hamiltonian from the outputs:  H_ij = (y0(i->j) + y0(j->i)) / 2 and
eps_i = eps0[Z_i] + sum_j y1(i->j).

Loss of the form of Eq. 3, applied to Hamiltonian-element residuals instead
of band energies (no DFT bands here), all weights w = 1 and normalised by the
number of residuals n:

    L = ( sum_k |D_k| / n )^2 + sum_k D_k^2 / n

over D = { y0(i->j) - t_ij for every directed edge } U { eps_i - eps_i^teacher }.
The subgradient of |D| at 0 is taken as 0.

AdamW (Sec. 2.1) with decoupled weight decay, as in Loshchilov & Hutter
(ICLR 2019): p <- p (1 - lr wd); m <- b1 m + (1 - b1) g;
v <- b2 v + (1 - b2) g^2; p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
"""
from __future__ import annotations

import numpy as np

PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))


def silu(z):
    return z * sigmoid(z)


def silu_grad(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def forward(params, x, mean, inv_std):
    p = {k: np.asarray(v, np.float64) for k, v in params.items()}
    xn = (np.asarray(x, np.float64) - mean) * inv_std
    z1 = xn @ p["W1"].T + p["b1"]
    h1 = silu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = silu(z2)
    y = h2 @ p["W3"].T + p["b3"]
    return y, dict(xn=xn, z1=z1, h1=h1, z2=z2, h2=h2)


def backward(params, cache, dy):
    p = {k: np.asarray(v, np.float64) for k, v in params.items()}
    dy = np.asarray(dy, np.float64)
    g = {}
    g["W3"] = dy.T @ cache["h2"]
    g["b3"] = dy.sum(axis=0)
    dz2 = (dy @ p["W3"]) * silu_grad(cache["z2"])
    g["W2"] = dz2.T @ cache["h1"]
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * silu_grad(cache["z1"])
    g["W1"] = dz1.T @ cache["xn"]
    g["b1"] = dz1.sum(axis=0)
    return g


def hamiltonian_residuals(y, edge_row, edge_valid, t_target, n_atoms, species, eps0, eps_target):
    """Residuals of the learned H against the teacher.

    y [E, 2] per directed edge; edge_row [E] the row i of each edge;
    edge_valid [E] bool (padding edges excluded).  Returns (D_hop [E] with
    zeros on padding, D_onsite [N], eps_pred [N]).
    """
    y = np.asarray(y, np.float64)
    valid = np.asarray(edge_valid, bool)
    d_hop = np.where(valid, y[:, 0] - np.asarray(t_target, np.float64), 0.0)
    eps_pred = np.asarray(eps0, np.float64)[np.asarray(species)].copy()
    np.add.at(eps_pred, np.asarray(edge_row)[valid], y[valid, 1])
    d_on = eps_pred - np.asarray(eps_target, np.float64)
    return d_hop, d_on, eps_pred


def loss_eq3(d_hop, d_on, edge_valid):
    """L and dL/dD for both residual sets (padding edges get zero gradient)."""
    valid = np.asarray(edge_valid, bool)
    n = int(valid.sum()) + d_on.size
    s_abs = (np.abs(d_hop[valid]).sum() + np.abs(d_on).sum()) / n
    s_sq = (np.square(d_hop[valid]).sum() + np.square(d_on).sum()) / n
    loss = s_abs * s_abs + s_sq
    g_hop = np.where(valid, 2.0 * s_abs * np.sign(d_hop) / n + 2.0 * d_hop / n, 0.0)
    g_on = 2.0 * s_abs * np.sign(d_on) / n + 2.0 * d_on / n
    return loss, g_hop, g_on


def output_gradient(g_hop, g_on, edge_row, edge_valid):
    """dL/dy per edge: y0 gets its hopping residual gradient, y1 the onsite
    residual gradient of its row (eps_i sums y1 over the row)."""
    valid = np.asarray(edge_valid, bool)
    dy = np.zeros((g_hop.size, 2))
    dy[:, 0] = g_hop
    dy[:, 1] = np.where(valid, np.asarray(g_on)[np.asarray(edge_row)], 0.0)
    return dy


def learned_hamiltonian(indptr, indices, y, species, eps0):
    """(H_ij per CSR entry, eps_i) from per-directed-edge outputs y [E, 2]."""
    from .hamiltonian import symmetrize_directed
    n = len(indptr) - 1
    hop = symmetrize_directed(indptr, indices, y[:, 0])
    rows = np.repeat(np.arange(n), np.diff(indptr))
    eps = np.asarray(eps0, np.float64)[np.asarray(species)].copy()
    np.add.at(eps, rows, y[:, 1])
    return hop, eps


def adamw_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=0.0):
    """One AdamW step (t counts from 1).  Returns new (params, m, v)."""
    new_p, new_m, new_v = {}, {}, {}
    for k in params:
        p = np.asarray(params[k], np.float64) * (1.0 - lr * wd)
        g = np.asarray(grads[k], np.float64)
        mk = beta1 * np.asarray(m[k], np.float64) + (1.0 - beta1) * g
        vk = beta2 * np.asarray(v[k], np.float64) + (1.0 - beta2) * g * g
        mhat = mk / (1.0 - beta1 ** t)
        vhat = vk / (1.0 - beta2 ** t)
        new_p[k] = p - lr * mhat / (np.sqrt(vhat) + eps)
        new_m[k], new_v[k] = mk, vk
    return new_p, new_m, new_v


def cosine_lr(step, total, lr0, lr_min=0.0):
    return lr_min + 0.5 * (lr0 - lr_min) * (1.0 + np.cos(np.pi * min(step, total) / total))
