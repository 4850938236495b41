"""Pins for oracle.hamiltonian, oracle.bounds, oracle.kpm and oracle.dos:
dense diagonalisation, the textbook graphene band structure and DOS, KPM
invariants, the published SplitMix64 outputs and the KPM sum rule."""
import math
import os

import numpy as np
import pytest

from oracle import bounds as bo
from oracle import dos as ds
from oracle import hamiltonian as ha
from oracle import kpm
from oracle import neighbors as nb
from oracle import teacher as te
from paper_2509_06525_gb300 import synth
from tests import analytic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_splitmix64_published_outputs():
    # successive outputs of SplitMix64 started from state 0; the generator's
    # state after k steps is k * gamma, so output k is splitmix64(k * gamma)
    gamma = 0x9E3779B97F4A7C15
    for k, (hexval,) in enumerate(_read_golden("splitmix64_seed0.txt")):
        state = np.uint64((k * gamma) % (1 << 64))
        assert int(kpm.splitmix64(state)) == int(hexval, 16)


def test_uniform_range_and_independence():
    u = kpm.uniform(42, np.zeros(100000, np.uint64), np.arange(100000, dtype=np.uint64))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3
    u2 = kpm.uniform(42, np.ones(100000, np.uint64), np.arange(100000, dtype=np.uint64))
    assert abs(np.corrcoef(u, u2)[0, 1]) < 0.02
    v0 = kpm.random_phase_vectors(42, 1000, 3)
    np.testing.assert_allclose(np.abs(v0), 1.0, atol=1e-15)


def _nn_graphene_H(n1, n2, t=-2.7):
    s = synth.graphene_primitive(n1, n2)
    indptr, idx, _ = nb.neighbors(s.positions, s.box, s.pbc, 1.8)
    H = ha.csr_hamiltonian(s.n, indptr, idx, np.full(idx.size, t), np.zeros(s.n))
    return s, H


def test_nn_graphene_spectrum_closed_form():
    s, H = _nn_graphene_H(20, 20)
    ev = np.linalg.eigvalsh(H.toarray())
    np.testing.assert_allclose(ev, analytic.nn_graphene_bands_torus(20, 20, -2.7), atol=1e-11)


def _teacher_H(n1=20, n2=20, sigma=0.05, seed=1001):
    s = synth.graphene_primitive(n1, n2, sigma, seed)
    p = synth.teacher_graphene()
    indptr, idx, d = nb.neighbors(s.positions, s.box, s.pbc, p.rcut)
    t, eps, _ = te.teacher_elements(s.species, indptr, idx, d, p)
    return s, ha.csr_hamiltonian(s.n, indptr, idx, t, eps)


@pytest.fixture(scope="module")
def teacher800():
    s, H = _teacher_H()
    ev = np.linalg.eigvalsh(H.toarray())
    return s, H, ev


def test_teacher_H_symmetric(teacher800):
    _, H, _ = teacher800
    assert abs(H - H.T).max() == 0.0


def test_gershgorin_and_lanczos_bracket_spectrum(teacher800):
    _, H, ev = teacher800
    gmin, gmax = bo.gershgorin(H)
    assert gmin <= ev[0] and ev[-1] <= gmax
    alpha, beta = bo.lanczos_tridiagonal(H, 64, 7)
    tmin, tmax = bo.tridiagonal_extremes(alpha, beta)
    # Ritz values lie inside the spectrum and converge to its extremes
    assert ev[0] - 1e-9 <= tmin and tmax <= ev[-1] + 1e-9
    assert abs(tmin - ev[0]) < 5e-3 and abs(tmax - ev[-1]) < 5e-3
    emin, emax, a, b = bo.spectral_bounds(H, 64, 7)
    assert emin <= ev[0] and ev[-1] <= emax
    assert np.all(np.abs((ev - b) / a) <= 1.0 - 0.004)


def test_tridiagonal_extremes_match_dense():
    rng = np.random.default_rng(0)
    alpha = rng.normal(size=40)
    beta = rng.uniform(0.1, 1.0, size=39)
    T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
    ev = np.linalg.eigvalsh(T)
    lo, hi = bo.tridiagonal_extremes(alpha, beta)
    assert abs(lo - ev[0]) < 1e-12 and abs(hi - ev[-1]) < 1e-12
    for x in np.linspace(ev[0] - 1, ev[-1] + 1, 37):
        assert bo.sturm_count(alpha, beta, x) == int(np.sum(ev < x))


def test_exact_trace_moments_match_diagonalisation(teacher800):
    _, H, ev = teacher800
    emin, emax, a, b = bo.spectral_bounds(H, 64, 7)
    Ht = kpm.rescale(H, a, b)
    mu = kpm.exact_trace_moments(Ht.toarray(), 512)
    ref = analytic.chebyshev_moments_of_levels(ev, a, b, 512)
    np.testing.assert_allclose(mu, ref, atol=1e-10)


def test_moment_invariants(teacher800):
    _, H, _ = teacher800
    emin, emax, a, b = bo.spectral_bounds(H, 64, 7)
    mu, mu_r = kpm.kpm_moments(H, a, b, 512, 8, 42)
    assert np.all(np.abs(mu_r[:, 0] - 1.0) <= 1e-14)
    assert np.all(np.abs(mu_r) <= 1.0 + 1e-12)


def test_odd_moments_vanish_on_bipartite_lattice():
    s, H = _nn_graphene_H(10, 10)
    a = 1.01 * 3 * 2.7
    Ht = kpm.rescale(H, a, 0.0)
    mu = kpm.exact_trace_moments(Ht.toarray(), 64)
    assert np.max(np.abs(mu[1::2])) < 1e-13
    # random phases: pair every vector r with its sublattice-flipped copy S r;
    # S H S = -H makes the odd moments of the pair cancel exactly
    v0 = kpm.random_phase_vectors(42, s.n, 4)
    sign = np.where(np.arange(s.n) % 2 == 0, 1.0, -1.0)[:, None]
    mu_r, _ = kpm.chebyshev_moments(Ht, np.concatenate([v0, sign * v0], axis=1), 64)
    pair = mu_r[:4] + mu_r[4:]
    assert np.max(np.abs(pair[:, 1::2])) < 1e-13
    assert np.max(np.abs(mu_r[:, 1::2])) > 1e-4     # each alone is not zero


def test_stochastic_moments_within_statistical_bound(teacher800):
    _, H, ev = teacher800
    emin, emax, a, b = bo.spectral_bounds(H, 64, 7)
    R = 64
    mu, mu_r = kpm.kpm_moments(H, a, b, 128, R, 42)
    ref = analytic.chebyshev_moments_of_levels(ev, a, b, 128)
    sigma = mu_r.std(axis=0, ddof=1)
    assert np.all(np.abs(mu - ref)[1:] <= 6.0 * sigma[1:] / math.sqrt(R) + 1e-12)


def test_jackson_kernel_properties():
    for M in (16, 512, 1024):
        g = ds.kernel_coefficients(M, ds.JACKSON)
        assert abs(g[0] - 1.0) < 1e-13
        assert np.all(np.diff(g) < 0) and g[-1] > 0


def test_dos_sum_rule_gauss_chebyshev():
    # integral of rho dE = g0 mu0 = 1 exactly; Gauss-Chebyshev quadrature of
    # order K > M is exact for the polynomial part
    rng = np.random.default_rng(3)
    mu = np.concatenate([[1.0], rng.uniform(-0.3, 0.3, 127)])
    a, b = 2.5, 0.3
    K = 400
    x = np.cos(np.pi * (np.arange(K) + 0.5) / K)
    rho = ds.density_of_states(mu, a, b, a * x + b)
    integral = np.pi / K * np.sum(rho * np.sqrt(1 - x * x)) * a
    assert abs(integral - 1.0) < 1e-12


def test_single_level_peak():
    # moments of one level at x0: mu_n = T_n(x0); the Jackson DOS peaks there
    # with a width close to pi / M (Weisse et al. 2006, Sec. II.C)
    M, x0 = 256, 0.3
    mu = np.cos(np.arange(M) * np.arccos(x0))
    x = np.linspace(-0.999, 0.999, 20001)
    rho = ds.density_of_states(mu, 1.0, 0.0, x)
    assert abs(x[np.argmax(rho)] - x0) < 2e-3
    mean = np.trapezoid(rho * x, x)
    sd = math.sqrt(np.trapezoid(rho * (x - mean) ** 2, x))
    assert abs(mean - x0) < 1e-3
    assert 0.5 * math.pi / M < sd < 2.0 * math.pi / M


@pytest.mark.slow
def test_nn_graphene_dos_against_closed_form():
    """KPM on a 200k-atom NN graphene sheet vs the textbook DOS, and the
    exact k-grid moments vs the elliptic-integral closed form."""
    t = -2.7
    s = synth.graphene_rect(250, 200)
    indptr, idx, _ = nb.neighbors(s.positions, s.box, s.pbc, 1.8)
    H = ha.csr_hamiltonian(s.n, indptr, idx, np.full(idx.size, t), np.zeros(s.n))
    a, b, M = 3 * 2.7 / 0.99, 0.0, 192
    mu, _ = kpm.kpm_moments(H, a, b, M, 4, 42)
    E = np.linspace(-7.5, 7.5, 601)
    rho_kpm = ds.density_of_states(mu, a, b, E)
    levels = analytic.nn_graphene_band_samples(600, t)
    mu_k = analytic.chebyshev_moments_of_levels(levels, a, b, M)
    rho_k = ds.density_of_states(mu_k, a, b, E)
    l1 = np.sum(np.abs(rho_kpm - rho_k)) / np.sum(np.abs(rho_k))
    assert l1 < 1e-2
    # smooth regions away from the van Hove points (|E| = |t|), the Dirac
    # point and the band edges: the damped expansion follows the closed form
    exact = analytic.nn_graphene_dos_closed_form(E, t)
    e = np.abs(E) / 2.7
    sel = ((e > 0.25) & (e < 0.75)) | ((e > 1.35) & (e < 2.6))
    rel = np.abs(rho_k[sel] - exact[sel]) / exact[sel]
    assert np.max(rel) < 0.05
