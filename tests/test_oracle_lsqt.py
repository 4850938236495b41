"""Pins of the VAC conductivity oracle (Eq. 3 (sigma), Sec. 2.4) against
results fixed by the mathematics: time evolution against the eigen-
decomposition, a ring where [H, V] = 0 (closed-form k sums, time
independent), graphene's exact Bloch VAC on the 4-atom rectangular cell
(with interband terms, both directions), the trapezoid rule, the spectral
sum rule and the stochastic error bound."""
import math

import numpy as np
import scipy.sparse as sp

from oracle import hamiltonian as oha
from oracle import lsqt
from oracle import neighbors as onb
from oracle import teacher as ote
from paper_2509_06525_gb300 import synth
from tests import analytic


def _ring(n, t=-1.3, eps0=0.2):
    pos = np.zeros((n, 3))
    pos[:, 0] = np.arange(n, dtype=np.float64)
    box = np.diag([float(n), 30.0, 30.0])
    pbc = np.array([1, 0, 0], np.int32)
    ip, idx, d = onb.neighbors(pos, box, pbc, 1.5)
    hop = np.full(idx.size, t)
    H = oha.csr_hamiltonian(n, ip, idx, hop, np.full(n, eps0))
    V = lsqt.velocity_matrix(n, ip, idx, hop, d)
    return H, V


def test_hbar_value():
    # hbar = h / (2 pi), h = 4.135667696e-15 eV s (CODATA 2018, exact SI value)
    assert abs(lsqt.HBAR - 4.135667696e-15 / (2 * math.pi) * 1e15) < 1e-10


def test_velocity_is_hermitian_and_commutator_form():
    H, V = _ring(12)
    Vd = V.toarray()
    np.testing.assert_allclose(Vd, Vd.conj().T, atol=1e-15)
    # V = (i/hbar)[H, X] with X the unwrapped positions, away from the seam
    X = np.diag(np.arange(12, dtype=np.float64))
    comm = (1j / lsqt.HBAR) * (H.toarray() @ X - X @ H.toarray())
    np.testing.assert_allclose(Vd[2:10, 2:10], comm[2:10, 2:10], atol=1e-13)


def test_propagation_equals_eigendecomposition_and_is_unitary():
    rng = np.random.default_rng(4)
    A = rng.normal(size=(30, 30))
    H = sp.csr_matrix(0.5 * (A + A.T))
    psi = rng.normal(size=(30, 3)) + 1j * rng.normal(size=(30, 3))
    w, W = np.linalg.eigh(H.toarray())
    for dt in (0.1, 0.7):
        U = W @ np.diag(np.exp(-1j * w * dt / lsqt.HBAR)) @ W.conj().T
        out = lsqt.propagate(H, psi, dt)
        np.testing.assert_allclose(out, U @ psi, atol=1e-12)
        np.testing.assert_allclose(np.linalg.norm(out, axis=0), np.linalg.norm(psi, axis=0), rtol=1e-13)


def test_ring_moments_are_time_independent_closed_form():
    n, t, eps0 = 40, -1.3, 0.2
    H, V = _ring(n, t, eps0)
    a, b, M = 2.8, 0.2, 48
    mu = lsqt.vac_moments_exact_trace(H, V, a, b, M, 4, 0.3)
    ref = analytic.ring_vac_moments(n, t, eps0, a, b, M)
    for j in range(mu.shape[0]):
        np.testing.assert_allclose(mu[j], ref, rtol=0, atol=1e-11)


def test_graphene_moments_equal_bloch_vac_with_interband_terms():
    nx, ny = 4, 6
    s = synth.graphene_rect(nx, ny)
    p = synth.teacher_graphene()
    ip, idx, d = onb.neighbors(s.positions, s.box, s.pbc, p.rcut)
    t, eps, _ = ote.teacher_elements(s.species, ip, idx, d, p)
    H = oha.csr_hamiltonian(s.n, ip, idx, t, eps)
    a_cc = p.a_cc
    shells = {a_cc: float(ote.hopping(a_cc, 0, 0, 3, 3, p)),
              math.sqrt(3) * a_cc: float(ote.hopping(math.sqrt(3) * a_cc, 0, 0, 3, 3, p)),
              2 * a_cc: float(ote.hopping(2 * a_cc, 0, 0, 3, 3, p))}
    a, b, M, dt, steps = 4.8, -0.1, 32, 0.25, 4
    for direction in ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0)):
        V = lsqt.velocity_matrix(s.n, ip, idx, t, d, direction)
        mu = lsqt.vac_moments_exact_trace(H, V, a, b, M, steps, dt)
        ref = analytic.rect_cell_bloch_vac_moments(nx, ny, shells, a, b, M, dt * np.arange(steps + 1),
                                                   direction[:2])
        np.testing.assert_allclose(mu, ref, rtol=0, atol=1e-10)
        # interband terms make the correlation decay: mu_0(t) changes with t
        assert abs(mu[-1, 0] - mu[0, 0]) > 1e-3 * abs(mu[0, 0])


def test_running_integral_trapezoid_is_exact_for_linear():
    tgrid = 0.1 * np.arange(11)
    C = np.stack([2.0 + 3.0 * tgrid, -1.0 + 0.5 * tgrid], axis=1)
    S = lsqt.running_integral(C, 0.1)
    np.testing.assert_allclose(S[:, 0], 2.0 * tgrid + 1.5 * tgrid ** 2, atol=1e-13)
    np.testing.assert_allclose(S[:, 1], -tgrid + 0.25 * tgrid ** 2, atol=1e-13)


def test_correlation_sum_rule():
    """int C(E, t) dE = mu_0(t): Gauss-Chebyshev quadrature integrates the
    damped series exactly (the same rule pins the DOS)."""
    H, V = _ring(30)
    a, b, M = 2.8, 0.2, 40
    mu = lsqt.vac_moments_exact_trace(H, V, a, b, M, 2, 0.2) / 1.0
    K = 4 * M
    x = np.cos(np.pi * (np.arange(K) + 0.5) / K)
    E = b + a * x
    C = lsqt.correlation(mu, a, b, E)
    w = np.pi / K * np.sqrt(1.0 - x * x) * a
    np.testing.assert_allclose(C @ w, mu[:, 0], rtol=1e-12)


def test_stochastic_estimate_within_statistical_bound():
    s = synth.graphene_rect(6, 6, 0.1, 7)
    p = synth.teacher_graphene()
    ip, idx, d = onb.neighbors(s.positions, s.box, s.pbc, p.rcut)
    t, eps, _ = ote.teacher_elements(s.species, ip, idx, d, p)
    H = oha.csr_hamiltonian(s.n, ip, idx, t, eps)
    V = lsqt.velocity_matrix(s.n, ip, idx, t, d)
    a, b, M, R = 4.8, -0.1, 16, 48
    exact = lsqt.vac_moments_exact_trace(H, V, a, b, M, 2, 0.3)
    st = lsqt.vac_moments(H, V, a, b, M, R, 99, 2, 0.3)
    mean, spread = st.mean(axis=1), st.std(axis=1, ddof=1)
    assert np.all(np.abs(mean - exact) <= 6.0 * spread / np.sqrt(R) + 1e-12)
