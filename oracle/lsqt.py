"""Velocity-autocorrelation (VAC) conductivity of the LSQT method, Eq. 3 (sigma),
Sec. 2.4.  TEST INFRASTRUCTURE ONLY.

Eq. 3 (sigma) gives the conductivity at energy E and correlation time t as

    sigma(E, t) = (2 e^2 / Omega) int_0^t Tr[ delta(E - H) Re(V V(tau)) ] dtau,
    V(tau) = exp(i H tau / hbar) V exp(-i H tau / hbar),

with the states propagated in steps of 0.1 fs (Sec. 2.4).  The library
returns the per-orbital quantities

    C(E, tau)   = (1/N) Re Tr[ delta(E - H) V V(tau) ]        (A^2 / fs^2 / eV)
    S(E, t)     = int_0^t C(E, tau) dtau  (trapezoid rule)    (A^2 / fs / eV)

so that sigma(E, t) = (2 e^2 N / Omega) S(E, t).  Steps, in order:

* velocity    V = (i / hbar) [H, X]: V_ij = (i / hbar) (x_j - x_i) H_ij with
              x_j - x_i the minimum-image displacement along the transport
              direction (the displacement the neighbour list returns);
* trace       Tr[delta V U(tau)^+ V U(tau)] = Tr[V U^+ V U delta] is
              estimated with random-phase vectors phi (E[phi phi^+] = 1) as
              <phi_L(tau)| V delta(E - H) |phi_R(tau)>, where
              phi_L(0) = V phi, phi_R(0) = phi and both are propagated by
              U(tau) = exp(-i H tau / hbar) (U commutes with delta(E - H));
* propagation U(dt) applied as the matrix exponential (SciPy expm_multiply);
* energy      delta(E - H) by the Jackson-damped Chebyshev series of
              H~ = (H - b)/a: moments mu_n(tau) = Re <V phi_L(tau)| T_n(H~)
              |phi_R(tau)> / N (V is Hermitian), and C(E, tau) is the series
              of dos.density_of_states applied to mu_n(tau).

The random phases are those of ``kpm`` (vectors first .. first + R - 1).
With the N basis vectors instead of random ones the trace is exact.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.linalg import expm_multiply

from . import dos as odos
from .kpm import random_phase_vectors, rescale

HBAR = 0.6582119569   # eV fs (CODATA 2018: hbar = 6.582119569e-16 eV s)


def velocity_matrix(n, indptr, indices, hop, disp, direction=(1.0, 0.0, 0.0)):
    """V = (i / hbar) [H, X] as a complex CSR matrix from the hopping values
    of the neighbour list (indptr, indices, hop) and its displacements
    disp[e] = r_j - r_i (minimum image)."""
    e = np.asarray(direction, np.float64)
    dx = np.asarray(disp, np.float64) @ e
    data = (1j / HBAR) * dx * np.asarray(hop, np.float64)
    return sp.csr_matrix((data, np.asarray(indices), np.asarray(indptr)), shape=(n, n))


def propagate(H, psi, dt):
    """U(dt) psi = exp(-i H dt / hbar) psi."""
    return expm_multiply((-1j * dt / HBAR) * sp.csr_matrix(H, dtype=np.complex128), psi)


def vac_moments_of_vectors(H, V, phi, a, b, M, n_steps, dt):
    """mu[j, r, n] = Re <V phi_L(t_j)| T_n(H~) |phi_R(t_j)> / N for the
    columns phi[:, r], t_j = j dt, j = 0 .. n_steps."""
    n = H.shape[0]
    Ht = rescale(H, a, b)
    phi = np.asarray(phi, np.complex128)
    phi_l = V @ phi
    phi_r = phi.copy()
    out = np.zeros((n_steps + 1, phi.shape[1], M))
    for j in range(n_steps + 1):
        w = V @ phi_l                       # <V phi_L| = (V phi_L)^+
        v_prev = phi_r
        out[j, :, 0] = np.sum(np.conj(w) * v_prev, axis=0).real / n
        if M > 1:
            v_cur = Ht @ v_prev
            out[j, :, 1] = np.sum(np.conj(w) * v_cur, axis=0).real / n
            for k in range(2, M):
                v_next = 2.0 * (Ht @ v_cur) - v_prev
                out[j, :, k] = np.sum(np.conj(w) * v_next, axis=0).real / n
                v_prev, v_cur = v_cur, v_next
        if j < n_steps:
            phi_l = propagate(H, phi_l, dt)
            phi_r = propagate(H, phi_r, dt)
    return out


def vac_moments(H, V, a, b, M, R, seed, n_steps, dt, first=0):
    """Stochastic VAC moments [n_steps + 1, R, M] with random vectors
    first .. first + R - 1."""
    phi = random_phase_vectors(seed, H.shape[0], R, first)
    return vac_moments_of_vectors(H, V, phi, a, b, M, n_steps, dt)


def vac_moments_exact_trace(H, V, a, b, M, n_steps, dt):
    """The trace over all N basis vectors: [n_steps + 1, M]."""
    n = H.shape[0]
    return vac_moments_of_vectors(H, V, np.eye(n), a, b, M, n_steps, dt).sum(axis=1)


def correlation(mu_t, a, b, energies, kind=odos.JACKSON):
    """C(E, t_j) [n_steps + 1, K] from moments mu_t [n_steps + 1, M] (already
    averaged over vectors) by the Chebyshev series of the DOS."""
    return np.stack([odos.density_of_states(m, a, b, energies, kind) for m in np.asarray(mu_t)])


def running_integral(C, dt):
    """S(E, t_j) = int_0^{t_j} C dtau by the trapezoid rule, S(E, 0) = 0."""
    C = np.asarray(C, np.float64)
    S = np.zeros_like(C)
    for j in range(1, C.shape[0]):
        S[j] = S[j - 1] + 0.5 * dt * (C[j - 1] + C[j])
    return S
