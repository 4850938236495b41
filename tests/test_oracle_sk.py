"""Pins of the s, p, d Slater-Koster oracle (rotation construction) against
results fixed independently: the bond-frame block along z, entries of the
closed-form Slater-Koster table (Slater & Koster, Phys. Rev. 94, 1498
(1954), Table I) covering all ten integrals at random directions, the
invariance of a flake's spectrum under a rotation, Hermiticity, and the
reduction of planar graphene with only pp_pi to the pz model."""
import math

import numpy as np
import pytest

from oracle import hamiltonian as oha
from oracle import neighbors as onb
from oracle import slater_koster as osk
from paper_2509_06525_gb300 import synth

V = np.array([-5.0, 5.4, 6.2, -2.9, -2.0, -2.4, 1.2, -1.8, 1.0, -0.3])
SS, SPS, PPS, PPP, SDS, PDS, PDP, DDS, DDP, DDD = V
S, PX, PY, PZ, DXY, DYZ, DZX, DX2, DZ2 = range(9)
R3 = math.sqrt(3.0)


def test_block_along_z_is_the_bond_frame_block():
    np.testing.assert_allclose(osk.hopping_block([0.0, 0.0, 1.7], V), osk.bond_frame_block(V), atol=1e-15)


@pytest.mark.parametrize("seed", range(6))
def test_entries_match_the_closed_form_table(seed):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=3)
    l, m, n = d / np.linalg.norm(d)
    H = osk.hopping_block(d, V)
    table = {
        (S, S): SS,
        (S, PX): l * SPS,
        (PX, S): -l * SPS,
        (PX, PX): l * l * PPS + (1 - l * l) * PPP,
        (PX, PY): l * m * (PPS - PPP),
        (PX, PZ): l * n * (PPS - PPP),
        (S, DXY): R3 * l * m * SDS,
        (S, DZ2): (n * n - 0.5 * (l * l + m * m)) * SDS,
        (S, DX2): 0.5 * R3 * (l * l - m * m) * SDS,
        (PX, DXY): R3 * l * l * m * PDS + m * (1 - 2 * l * l) * PDP,
        (PZ, DZ2): n * (n * n - 0.5 * (l * l + m * m)) * PDS + R3 * n * (l * l + m * m) * PDP,
        (PX, DX2): 0.5 * R3 * l * (l * l - m * m) * PDS + l * (1 - l * l + m * m) * PDP,
        (DXY, DXY): 3 * l * l * m * m * DDS + (l * l + m * m - 4 * l * l * m * m) * DDP
        + (n * n + l * l * m * m) * DDD,
        (DXY, DYZ): 3 * l * m * m * n * DDS + l * n * (1 - 4 * m * m) * DDP + l * n * (m * m - 1) * DDD,
        (DZ2, DZ2): (n * n - 0.5 * (l * l + m * m)) ** 2 * DDS + 3 * n * n * (l * l + m * m) * DDP
        + 0.75 * (l * l + m * m) ** 2 * DDD,
        (DX2, DX2): 0.75 * (l * l - m * m) ** 2 * DDS + (l * l + m * m - (l * l - m * m) ** 2) * DDP
        + (n * n + 0.25 * (l * l - m * m) ** 2) * DDD,
    }
    for (a, b), ref in table.items():
        assert abs(H[a, b] - ref) < 1e-12, (a, b, H[a, b], ref)


def _flake():
    s = synth.graphene_rect(3, 3, 0.15, 4)
    keep = s.positions[:, 0] < 6.0
    return s.positions[keep]


def _cluster_h(pos, p):
    box = np.diag([200.0, 200.0, 200.0])
    pbc = np.array([0, 0, 0], np.int32)
    ip, idx, d = onb.neighbors(pos, box, pbc, p.rcut)
    return osk.sk_hamiltonian(pos.shape[0], ip, idx, d, p)


def test_spectrum_invariant_under_rotation():
    p = osk.SKParams(V, np.array([-7.5, 0.0, 14.0]))
    pos = _flake() + 50.0
    H = _cluster_h(pos, p)
    rng = np.random.default_rng(1)
    Qr, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    c = pos.mean(axis=0)
    H2 = _cluster_h((pos - c) @ Qr.T + c, p)
    e1 = np.linalg.eigvalsh(H.toarray())
    e2 = np.linalg.eigvalsh(H2.toarray())
    np.testing.assert_allclose(e1, e2, atol=1e-10)


def test_periodic_sheet_hamiltonian_is_symmetric():
    s = synth.graphene_rect(4, 4, 0.1, 2)
    p = osk.SKParams(V, np.array([-7.5, 0.0, 14.0]))
    ip, idx, d = onb.neighbors(s.positions, s.box, s.pbc, p.rcut)
    H = osk.sk_hamiltonian(s.n, ip, idx, d, p).toarray()
    np.testing.assert_allclose(H, H.T, atol=1e-13)


def test_planar_graphene_with_only_pp_pi_reduces_to_the_pz_model():
    s = synth.graphene_rect(5, 4)                     # pristine, planar
    v = np.zeros(10)
    v[3] = -2.7                                       # pp_pi only
    p = osk.SKParams(v, np.array([0.0, 0.4, 0.0]))
    ip, idx, d = onb.neighbors(s.positions, s.box, s.pbc, p.rcut)
    H = osk.sk_hamiltonian(s.n, ip, idx, d, p).toarray()
    pz = 9 * np.arange(s.n) + PZ
    others = np.setdiff1d(np.arange(9 * s.n), pz)
    assert np.max(np.abs(H[np.ix_(pz, others)])) < 1e-14        # pz decouples
    t = osk.integrals(np.linalg.norm(d, axis=1), p)[:, 3]         # pp_pi(r), n = 0 in plane
    Hpz = oha.csr_hamiltonian(s.n, ip, idx, t, np.full(s.n, 0.4)).toarray()
    np.testing.assert_allclose(H[np.ix_(pz, pz)], Hpz, atol=1e-13)
