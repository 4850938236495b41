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


def chebyshev_moments_of_levels(levels, a, b, M, chunk=1 << 15):
    """mu_n = mean over levels of T_n((E - b)/a).

    Small level sets use T_n(x) = cos(n arccos x); large ones the three-term
    recurrence T_{n+1} = 2 x T_n - T_{n-1} on cache-sized chunks."""
    x = np.clip((np.asarray(levels, np.float64) - b) / a, -1.0, 1.0)
    if x.size <= 100000:
        n = np.arange(M)[:, None]
        return np.cos(n * np.arccos(x)[None, :]).mean(axis=1)
    acc = np.zeros(M)
    for s in range(0, x.size, chunk):
        xc = x[s:s + chunk]
        t0 = np.ones_like(xc)
        t1 = xc.copy()
        acc[0] += t0.sum()
        if M > 1:
            acc[1] += t1.sum()
        two_x = 2.0 * xc
        for k in range(2, M):
            t2 = two_x * t1
            t2 -= t0
            acc[k] += t2.sum()
            t0, t1 = t1, t2
    return acc / x.size


def rect_cell_bloch_levels(nx, ny, shell_hoppings, a_cc=1.42, onsite=0.0, chunk=200000):
    """All 4 nx ny eigenvalues of pristine graphene on an nx x ny torus of
    4-atom rectangular cells (3 a_cc by sqrt(3) a_cc, basis (0,0), (a,0),
    (1.5a, h), (2.5a, h)), with hoppings given per neighbour shell as
    {distance: t}.  Bloch's theorem: H(k)_{bb'} = sum_T t(|d|) e^{i k.d},
    d = r_b' + T - r_b, for k on the torus grid."""
    h = 0.5 * np.sqrt(3.0) * a_cc
    lx, ly = 3.0 * a_cc, np.sqrt(3.0) * a_cc
    basis = np.array([[0.0, 0.0], [a_cc, 0.0], [1.5 * a_cc, h], [2.5 * a_cc, h]])
    terms = []                                   # (b, b', d, t)
    for b in range(4):
        for bp in range(4):
            for tx in (-1, 0, 1):
                for ty in (-1, 0, 1):
                    d = basis[bp] + np.array([tx * lx, ty * ly]) - basis[b]
                    r = float(np.hypot(*d))
                    for dist, t in shell_hoppings.items():
                        if abs(r - dist) < 1e-6:
                            terms.append((b, bp, d, t))
    m1, m2 = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    kx = (2 * np.pi * m1 / (nx * lx)).reshape(-1)
    ky = (2 * np.pi * m2 / (ny * ly)).reshape(-1)
    out = []
    for s in range(0, kx.size, chunk):
        k = np.stack([kx[s:s + chunk], ky[s:s + chunk]], axis=1)
        Hk = np.zeros((k.shape[0], 4, 4), np.complex128)
        for b in range(4):
            Hk[:, b, b] += onsite
        for b, bp, d, t in terms:
            Hk[:, b, bp] += t * np.exp(1j * (k @ d))
        out.append(np.linalg.eigvalsh(Hk).reshape(-1))
    return np.concatenate(out)


HBAR_EV_FS = 0.6582119569   # CODATA 2018


def _rect_cell_terms(shell_hoppings, a_cc=1.42):
    h = 0.5 * np.sqrt(3.0) * a_cc
    lx, ly = 3.0 * a_cc, np.sqrt(3.0) * a_cc
    basis = np.array([[0.0, 0.0], [a_cc, 0.0], [1.5 * a_cc, h], [2.5 * a_cc, h]])
    terms = []
    for b in range(4):
        for bp in range(4):
            for tx in (-1, 0, 1):
                for ty in (-1, 0, 1):
                    d = basis[bp] + np.array([tx * lx, ty * ly]) - basis[b]
                    r = float(np.hypot(*d))
                    for dist, t in shell_hoppings.items():
                        if abs(r - dist) < 1e-6:
                            terms.append((b, bp, d, t))
    return terms, lx, ly


def rect_cell_bloch_vac_moments(nx, ny, shell_hoppings, a, b, M, times, direction=(1.0, 0.0), a_cc=1.42):
    """Exact per-orbital VAC moments of pristine graphene on an nx x ny torus
    of rectangular cells, by Bloch's theorem:
        mu_n(t) = (1/N) Re Tr[T_n(H~) V U(t)^+ V U(t)],  U(t) = exp(-i H t / hbar),
    with H(k)_{bb'} = sum t e^{i k.d} and the velocity V(k) = (1/hbar) dH(k)/dk
    along `direction` (d = r_b' + T - r_b, the atomic positions in the phase).
    In the eigenbasis of H(k): sum_{a,b} T_n(e~_a) |V_ab|^2 cos((e_b - e_a) t / hbar)."""
    terms, lx, ly = _rect_cell_terms(shell_hoppings, a_cc)
    e = np.asarray(direction, np.float64)
    m1, m2 = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    k = np.stack([(2 * np.pi * m1 / (nx * lx)).reshape(-1), (2 * np.pi * m2 / (ny * ly)).reshape(-1)], axis=1)
    Hk = np.zeros((k.shape[0], 4, 4), np.complex128)
    Vk = np.zeros((k.shape[0], 4, 4), np.complex128)
    for bb, bp, d, t in terms:
        ph = np.exp(1j * (k @ d))
        Hk[:, bb, bp] += t * ph
        Vk[:, bb, bp] += (1j / HBAR_EV_FS) * float(d @ e) * t * ph
    w, W = np.linalg.eigh(Hk)
    Ve = np.conj(np.transpose(W, (0, 2, 1))) @ Vk @ W           # V in the eigenbasis
    P = np.abs(Ve) ** 2                                           # |V_ab|^2
    x = np.clip((w - b) / a, -1.0, 1.0)                           # [nk, 4]
    Tn = np.cos(np.arange(M)[:, None, None] * np.arccos(x)[None])  # [M, nk, 4]
    N = 4 * nx * ny
    out = np.zeros((len(times), M))
    for j, t in enumerate(times):
        c = np.cos((w[:, None, :] - w[:, :, None]) * t / HBAR_EV_FS)   # [nk, a, b]: cos((e_b - e_a) t)
        A = np.sum(P * c, axis=2)                                        # [nk, a]
        out[j] = np.einsum("mka,ka->m", Tn, A) / N
    return out


def ring_vac_moments(n, t, eps0, a, b, M):
    """Exact per-orbital VAC moments of a ring of n sites (spacing 1 A,
    hopping t, onsite eps0): V = (i t / hbar)(S - S^+) commutes with H, so
    mu_n(t) = (1/n) sum_k T_n(e~_k) v_k^2 for all t, with
    e_k = eps0 + 2 t cos k, v_k = -2 t sin k / hbar, k = 2 pi m / n."""
    kk = 2 * np.pi * np.arange(n) / n
    ek = eps0 + 2 * t * np.cos(kk)
    vk = -2 * t * np.sin(kk) / HBAR_EV_FS
    x = np.clip((ek - b) / a, -1.0, 1.0)
    Tn = np.cos(np.arange(M)[:, None] * np.arccos(x)[None, :])
    return (Tn * vk[None, :] ** 2).sum(axis=1) / n
