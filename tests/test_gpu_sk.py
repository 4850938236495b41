"""GPU parity of the matrix-free s, p, d Slater-Koster path against the
oracle's rotation construction: the compressed SK form of every bond, the
Gershgorin bounds, and the KPM moments of the 9N-orbital Hamiltonian (FP32
vectors, tolerance 2e-4 as for the pz KPM), on thermal (non-planar) sheets,
a triclinic cell, a ragged size and a multi-CTA size; plus mu_0 = 1 and
|mu_n| <= 1 at 1e6 atoms (9e6 orbitals)."""
import numpy as np
import pytest
import torch

from oracle import kpm as okpm
from oracle import neighbors as onb
from oracle import slater_koster as osk
from paper_2509_06525_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_2509_06525_gb300 import build, gputb
    build.build()
    assert torch.cuda.is_available()
    return gputb


STRUCTS = {
    "rect_thermal": lambda: synth.graphene_rect(6, 5, 0.1, 3),
    "prim_triclinic": lambda: synth.graphene_primitive(8, 8, 0.1, 5),
    "ragged": lambda: synth.graphene_rect(7, 9, 0.1, 8),
    "rect_4800": lambda: synth.graphene_rect(40, 30, 0.1, 13),
}


def _params(sk):
    return osk.SKParams(sk.v0, sk.onsite, sk.a_cc, sk.beta, sk.rcut)


@pytest.fixture(scope="module", params=list(STRUCTS))
def case(request, g):
    s = STRUCTS[request.param]()
    sk = synth.teacher_sk_graphene()
    pos = torch.tensor(s.positions, device="cuda")
    nb = g.build_neighbors(pos, s.box, s.pbc, sk.rcut, r_count=0.0)
    geom = g.sk_geometry(pos, s.box, s.pbc, nb, sk)
    ip, idx, d = onb.neighbors(s.positions, s.box, s.pbc, sk.rcut)
    H = osk.sk_hamiltonian(s.n, ip, idx, d, _params(sk))
    return s, sk, nb, geom, ip, idx, d, H


def test_compressed_sk_form_matches_oracle(g, case):
    s, sk, nb, geom, ip, idx, d, H = case
    gm = geom.cpu().numpy()
    sp_, col, cnt = nb.slice_ptr.cpu().numpy(), nb.col.cpu().numpy(), nb.cnt.cpu().numpy()
    V = osk.integrals(np.linalg.norm(d, axis=1), _params(sk))
    for i in range(s.n):
        k, lane = divmod(i, 32)
        for q in range(cnt[i]):
            e = sp_[k] + lane + 32 * q
            j = col[e]
            eo = ip[i] + q                           # both sides sort neighbours by j
            assert idx[eo] == j
            u = d[eo] / np.linalg.norm(d[eo])
            np.testing.assert_allclose(gm[0:3, e], u, rtol=0, atol=2e-7)
            np.testing.assert_allclose(gm[3:, e], V[eo], rtol=2e-6, atol=1e-9)


def test_gershgorin_bounds_match_oracle(g, case):
    s, sk, nb, geom, ip, idx, d, H = case
    emin, emax, a, b = g.sk_bounds(nb, geom, sk)
    gmin, gmax = osk.gershgorin(H)
    assert emin <= gmin and emax >= gmax                  # still an enclosure
    np.testing.assert_allclose([emin, emax], [gmin, gmax], rtol=2e-5)
    np.testing.assert_allclose([a, b], [(emax - emin) / 1.99, 0.5 * (emax + emin)], rtol=1e-12)


@pytest.mark.parametrize("first", [0, 3])
def test_kpm_moments_match_oracle(g, case, first):
    s, sk, nb, geom, ip, idx, d, H = case
    gmin, gmax = osk.gershgorin(H)
    a, b = 1.001 * (gmax - gmin) / 1.99, 0.5 * (gmax + gmin)
    M = 96
    mu = g.sk_kpm_moments(nb, geom, sk, a, b, M, 21, first_vector=first).cpu().numpy()
    _, mu_ref = okpm.kpm_moments(H, a, b, M, 1, 21, first=first)
    assert abs(mu[0] - 1.0) < 1e-6
    assert np.max(np.abs(mu - mu_ref[0])) <= 2e-4


def test_moment_invariants_at_one_million_atoms(g):
    s = synth.graphene_rect(500, 500, 0.1, 1002)
    sk = synth.teacher_sk_graphene()
    pos = torch.tensor(s.positions, device="cuda")
    nb = g.build_neighbors(pos, s.box, s.pbc, sk.rcut, r_count=0.0)
    geom = g.sk_geometry(pos, s.box, s.pbc, nb, sk)
    emin, emax, a, b = g.sk_bounds(nb, geom, sk)
    mu = g.sk_kpm_moments(nb, geom, sk, a, b, 256, 42).cpu().numpy()
    assert abs(mu[0] - 1.0) < 1e-6
    assert np.all(np.abs(mu) <= 1.0 + 1e-6) and np.all(np.isfinite(mu))
    # the first moment is the mean onsite energy of the rescaled H: (E_s + 3 E_p + 5 E_d)/9 - b, over a
    mean_on = (sk.onsite[0] + 3 * sk.onsite[1] + 5 * sk.onsite[2]) / 9.0
    assert abs(mu[1] - (mean_on - b) / a) < 3.0 / np.sqrt(9 * s.n)
