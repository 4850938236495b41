"""GPU parity of the VAC conductivity path (Eq. 3 (sigma), Sec. 2.4) against
the FP64 oracle: velocity values, VAC moments (FP64 rel 1e-10 and FP32 rel
1e-4 of the largest moment), vector blocks, the correlation / running
integral, and the time independence of a ring's moments ([H, V] = 0) at
100k sites."""
import numpy as np
import pytest
import torch

from oracle import bounds as obo
from oracle import hamiltonian as oha
from oracle import lsqt as olsqt
from oracle import neighbors as onb
from oracle import teacher as ote
from paper_2509_06525_gb300 import synth
from tests.sell_helpers import sell_matrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_2509_06525_gb300 import build, gputb
    build.build()
    assert torch.cuda.is_available()
    return gputb


def _case(name):
    if name == "prim800":
        s, p = synth.graphene_primitive(20, 20, 0.05, 1001), synth.teacher_graphene()
    elif name == "junction_ragged":
        s, p = synth.hbn_graphene_junction(6, 7, 0.1, 9), synth.teacher_hbn_graphene()
        s.positions, s.species = s.positions[:-5].copy(), s.species[:-5].copy()
    else:
        s, p = synth.graphene_rect(60, 40, 0.1, 21), synth.teacher_graphene()   # 9600 atoms, many CTAs
    ip, idx, d = onb.neighbors(s.positions, s.box, s.pbc, p.rcut)
    t, eps, _ = ote.teacher_elements(s.species, ip, idx, d, p)
    H = oha.csr_hamiltonian(s.n, ip, idx, t, eps)
    _, _, a, b = obo.spectral_bounds(H, 64, 7)
    return s, p, ip, idx, d, t, eps, H, a, b


@pytest.fixture(scope="module", params=["prim800", "junction_ragged", "rect9600"])
def case(request):
    return _case(request.param)


def _dense_from_sell(n, slice_ptr, col, val):
    sp_, c, v = slice_ptr.cpu().numpy(), col.cpu().numpy(), val.cpu().numpy()
    D = np.zeros((n, n))
    for i in range(n):
        k, lane = divmod(i, 32)
        w = (sp_[k + 1] - sp_[k]) // 32
        for s in range(w):
            e = sp_[k] + lane + 32 * s
            D[i, c[e]] += v[e]
    return D


def test_velocity_values_match_oracle(g, case):
    s, p, ip, idx, d, t, eps, H, a, b = case
    if s.n > 2000:
        pytest.skip("dense comparison on the small cases")
    Hd = sell_matrix(ip, idx, t, eps, s.n, torch.float64)
    pos = torch.tensor(s.positions, device="cuda")
    for e in ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.6, 0.8, 0.0)):
        vv = g.velocity_values(pos, s.box, s.pbc, p.rcut, Hd, e)
        got = _dense_from_sell(s.n, Hd.slice_ptr, Hd.col, vv)
        ref = (olsqt.velocity_matrix(s.n, ip, idx, t, d, e).toarray() / (1j / olsqt.HBAR)).real
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(got, -got.T, atol=1e-12)   # V Hermitian: vval antisymmetric


@pytest.mark.parametrize("dtype,R,tol", [(torch.float64, 4, 1e-10), (torch.float64, 8, 1e-10),
                                         (torch.float32, 1, 1e-4), (torch.float32, 8, 1e-4),
                                         (torch.float32, 16, 1e-4)])
def test_vac_moments_match_oracle(g, case, dtype, R, tol):
    s, p, ip, idx, d, t, eps, H, a, b = case
    M, steps, dt, seed = 48, 3, 0.3, 5
    Hd = sell_matrix(ip, idx, t, eps, s.n, dtype)
    pos = torch.tensor(s.positions, device="cuda")
    vv = g.velocity_values(pos, s.box, s.pbc, p.rcut, Hd)
    mu = g.lsqt_vac(Hd, vv, a, b, M, R, seed, steps, dt).cpu().numpy()
    V = olsqt.velocity_matrix(s.n, ip, idx, t, d)
    ref = olsqt.vac_moments(H, V, a, b, M, R, seed, steps, dt)
    assert mu.shape == ref.shape
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(mu - ref)) <= tol * scale


def test_vector_blocks_compose_the_ensemble(g):
    s, p, ip, idx, d, t, eps, H, a, b = _case("prim800")
    Hd = sell_matrix(ip, idx, t, eps, s.n, torch.float64)
    vv = g.velocity_values(torch.tensor(s.positions, device="cuda"), s.box, s.pbc, p.rcut, Hd)
    full = g.lsqt_vac(Hd, vv, a, b, 32, 8, 7, 2, 0.2).cpu().numpy()
    lo = g.lsqt_vac(Hd, vv, a, b, 32, 4, 7, 2, 0.2, first_vector=0).cpu().numpy()
    hi = g.lsqt_vac(Hd, vv, a, b, 32, 4, 7, 2, 0.2, first_vector=4).cpu().numpy()
    scale = np.max(np.abs(full))
    np.testing.assert_allclose(np.concatenate([lo, hi], axis=1), full, rtol=0, atol=1e-12 * scale)


def test_correlation_and_running_integral_match_oracle(g):
    s, p, ip, idx, d, t, eps, H, a, b = _case("junction_ragged")
    V = olsqt.velocity_matrix(s.n, ip, idx, t, d)
    dt = 0.25
    mu = olsqt.vac_moments(H, V, a, b, 64, 4, 3, 6, dt)          # oracle moments as the input
    E = np.linspace(b - 0.98 * a, b + 0.98 * a, 301)
    C_ref = olsqt.correlation(mu.mean(axis=1), a, b, E)
    S_ref = olsqt.running_integral(C_ref, dt)
    C, S = g.lsqt_correlation(torch.tensor(mu, device="cuda"), a, b, torch.tensor(E, device="cuda"), dt)
    np.testing.assert_allclose(C.cpu().numpy(), C_ref, rtol=1e-10, atol=1e-12 * np.max(np.abs(C_ref)))
    np.testing.assert_allclose(S.cpu().numpy(), S_ref, rtol=1e-10, atol=1e-12 * np.max(np.abs(S_ref)))


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-11), (torch.float32, 2e-4)])
def test_ring_moments_time_independent_at_100k_sites(g, dtype, tol):
    """[H, V] = 0 on a ring makes <V phi_L(t)| T_n |phi_R(t)> independent of t
    for every vector, so all time points must repeat t = 0."""
    n = 100_000
    pos = np.zeros((n, 3))
    pos[:, 0] = np.arange(n, dtype=np.float64)
    box = np.diag([float(n), 30.0, 30.0])
    pbc = np.array([1, 0, 0], np.int32)
    rows = np.arange(n)
    indptr = np.arange(0, 2 * n + 1, 2)
    idx = np.stack([(rows - 1) % n, (rows + 1) % n], axis=1).reshape(-1)
    idx = np.sort(idx.reshape(n, 2), axis=1).reshape(-1)
    hop = np.full(2 * n, -1.3)
    Hd = sell_matrix(indptr, idx, hop, np.full(n, 0.2), n, dtype)
    vv = g.velocity_values(torch.tensor(pos, device="cuda"), box, pbc, 1.5, Hd)
    mu = g.lsqt_vac(Hd, vv, 2.8, 0.2, 32, 4, 11, 5, 0.4).cpu().numpy()
    scale = np.max(np.abs(mu[0]))
    assert np.max(np.abs(mu - mu[0][None])) <= tol * scale
    # and t = 0 equals the oracle's closed form in expectation: mean v^2 = 2 t^2 / hbar^2
    assert abs(mu[0, :, 0].mean() - 2 * 1.3 ** 2 / olsqt.HBAR ** 2) < 0.02 * 2 * 1.3 ** 2 / olsqt.HBAR ** 2


def test_lsqt_errors(g):
    s, p, ip, idx, d, t, eps, H, a, b = _case("prim800")
    Hd = sell_matrix(ip, idx, t, eps, s.n, torch.float64)
    vv = g.velocity_values(torch.tensor(s.positions, device="cuda"), s.box, s.pbc, p.rcut, Hd)
    with pytest.raises(g.GputbError):
        g.lsqt_vac(Hd, vv, a, b, 16, 32, 1, 1, 0.1)          # R = 32 not supported
    with pytest.raises(g.GputbError):
        g.lsqt_vac(Hd, vv, a, b, 16, 4, 1, 1, -0.1)          # dt <= 0
    with pytest.raises(g.GputbError):
        g.lsqt_vac(Hd, vv, a, b, 16, 4, 1, 1, 100.0)         # a dt / hbar > 200
