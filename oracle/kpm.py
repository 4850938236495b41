"""Kernel polynomial method moments (LSQT core, Sec. 2.4).  TEST INFRASTRUCTURE ONLY.

Sec. 2.4 names the ingredients -- Chebyshev expansion, KPM, sparse
matrix-vector products and the random phase approximation -- and cites the
standard formulation (Weisse, Wellein, Alvermann & Fehske, Rev. Mod. Phys. 78,
275 (2006)), whose conventions are used here:

* rescaling      H~ = (H - b) / a maps the spectrum into [-1, 1];
* random phases  v0[i, r] = exp(i phi), phi = 2 pi u(seed, r, i);
* recursion      v1 = H~ v0,  v_{n+1} = 2 H~ v_n - v_{n-1};
* moments        mu_n^(r) = Re( sum_i conj(v0[i, r]) v_n[i, r] ) / N,
                 mu_n = mean_r mu_n^(r)  (so mu_0 = 1).

The uniform deviate u is counter based so that any implementation can
reproduce it from its definition:

    u(seed, r, i) = (splitmix64(seed XOR splitmix64(r * 2^32 + i)) >> 11) * 2^-53

where splitmix64(x) is one output of the SplitMix64 generator whose state is x
(Steele, Lea & Flood, OOPSLA 2014): z = x + 0x9E3779B97F4A7C15;
z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9; z = (z ^ (z >> 27)) * 0x94D049BB133111EB;
return z ^ (z >> 31)  (all arithmetic modulo 2^64).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x):
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniform(seed, r, i):
    """u(seed, r, i) in [0, 1), vectorised over arrays r and i."""
    r = np.asarray(r, np.uint64)
    i = np.asarray(i, np.uint64)
    inner = splitmix64((r << np.uint64(32)) + i)
    z = splitmix64(np.uint64(seed) ^ inner)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def random_phase_vectors(seed, n, R, first=0):
    """v0 [N, R] complex128 with unit-modulus entries: random vectors
    first .. first + R - 1 of the ensemble."""
    i = np.arange(n, dtype=np.uint64)[:, None]
    r = np.arange(first, first + R, dtype=np.uint64)[None, :]
    phi = 2.0 * np.pi * uniform(seed, r, i)
    return np.cos(phi) + 1j * np.sin(phi)


def rescale(H, a, b):
    """H~ = (H - b I) / a as a CSR matrix in FP64."""
    n = H.shape[0]
    return ((H - b * sp.identity(n, format="csr")) / a).tocsr()


def chebyshev_moments(Ht, v0, M):
    """Per-vector moments mu^(r)_n, n = 0..M-1, and max |Im <v0|v_n>| / N.

    Ht: rescaled Hamiltonian (sparse or dense, real); v0: [N, R] complex.
    Returns (mu [R, M] float64, max_imag float).
    """
    n = v0.shape[0]
    R = v0.shape[1]
    mu = np.zeros((R, M))
    max_imag = 0.0

    def record(k, v):
        nonlocal max_imag
        dots = np.sum(np.conj(v0) * v, axis=0) / n
        mu[:, k] = dots.real
        max_imag = max(max_imag, float(np.max(np.abs(dots.imag))))

    v_prev = v0.copy()
    record(0, v_prev)
    if M == 1:
        return mu, max_imag
    v_cur = Ht @ v_prev
    record(1, v_cur)
    for k in range(2, M):
        v_next = 2.0 * (Ht @ v_cur) - v_prev
        record(k, v_next)
        v_prev, v_cur = v_cur, v_next
    return mu, max_imag


def exact_trace_moments(Ht, M):
    """mu_n = Tr T_n(H~) / N, by running the same recursion on every basis
    vector e_i (the deterministic limit of the stochastic trace)."""
    n = Ht.shape[0]
    eye = np.eye(n)
    mu, _ = chebyshev_moments(Ht, eye.astype(np.complex128), M)
    return mu.sum(axis=0)


def kpm_moments(H, a, b, M, R, seed, first=0):
    """Full oracle step: rescale, draw v0 (vectors first .. first + R - 1),
    recurse.  Returns (mu [M], mu_r [R, M])."""
    Ht = rescale(H, a, b)
    v0 = random_phase_vectors(seed, H.shape[0], R, first)
    mu_r, _ = chebyshev_moments(Ht, v0, M)
    return mu_r.mean(axis=0), mu_r
