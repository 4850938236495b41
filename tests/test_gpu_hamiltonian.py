"""GPU parity of tb_build_neighbors, tb_build_hamiltonian_teacher and
tb_spectral_bounds against the FP64 oracle, and the whole plain path
(positions -> neighbours -> teacher H -> bounds -> KPM -> DOS).

Neighbour and ELL indices must match bit for bit; teacher values to FP64
rounding (rel 1e-13) or to one FP32 rounding; bounds to rel 1e-9."""
import numpy as np
import pytest
import torch

from oracle import bounds as obo
from oracle import dos as ods
from oracle import hamiltonian as oha
from oracle import kpm as okpm
from oracle import neighbors as onb
from oracle import teacher as ote
from paper_2509_06525_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_2509_06525_gb300 import build, gputb
    build.build()
    return gputb


def _dev(s):
    return (torch.tensor(s.positions, device="cuda"), torch.tensor(s.species, device="cuda"))


def _sell_rows(nb):
    """Decode the device SELL structure into per-row neighbour arrays."""
    sp = nb.slice_ptr.cpu().numpy()
    col = nb.col.cpu().numpy()
    cnt = nb.cnt.cpu().numpy()
    rows = []
    for i in range(nb.n):
        k, lane = divmod(i, 32)
        w = (sp[k + 1] - sp[k]) // 32
        pos = sp[k] + lane + 32 * np.arange(w)
        c = col[pos]
        assert np.all(c[cnt[i]:] == i), "padding must hold col = i"
        rows.append(c[:cnt[i]])
    # slice widths are the row maxima
    for k in range(len(sp) - 1):
        assert (sp[k + 1] - sp[k]) // 32 == cnt[32 * k:32 * k + 32].max()
    return rows


def _margin_ok(dvec, rcut):
    r = np.sqrt((dvec ** 2).sum(1))
    return np.min(np.abs(r - rcut)) > 1e-9


STRUCTS = {
    "prim800": lambda: synth.graphene_primitive(20, 20, 0.05, 1001),
    "rect_thermal": lambda: synth.graphene_rect(40, 30, 0.1, 77),
    "junction": lambda: synth.hbn_graphene_junction(24, 20, 0.1, 5),
    "ragged": lambda: synth.graphene_rect(7, 9, 0.1, 3),
}


@pytest.mark.parametrize("name", list(STRUCTS))
def test_neighbors_bit_exact(g, name):
    s = STRUCTS[name]()
    pos, _ = _dev(s)
    nb = g.build_neighbors(pos, s.box, s.pbc, 3.0, r_count=1.8, max_width=16)
    indptr, idx, d = onb.neighbors(s.positions, s.box, s.pbc, 3.0)
    assert _margin_ok(d, 3.0)
    rows = _sell_rows(nb)
    for i in range(s.n):
        np.testing.assert_array_equal(rows[i], idx[indptr[i]:indptr[i + 1]])
    ncount = ote.coordination(indptr, ote.distances(d), 1.8)
    np.testing.assert_array_equal(nb.ncount.cpu().numpy(), ncount)


def test_neighbors_random_triclinic_3d(g):
    rng = np.random.default_rng(4)
    box = np.array([[9.0, 0.0, 0.0], [3.7, 8.1, 0.0], [1.1, -0.9, 7.5]])
    pos = rng.uniform(0.0, 1.0, size=(100, 3)) @ box   # ~30 neighbours per atom
    pbc = np.array([1, 1, 1], np.int32)
    nb = g.build_neighbors(torch.tensor(pos, device="cuda"), box, pbc, 3.4, r_count=0.0, max_width=64)
    indptr, idx, d = onb.neighbors_bruteforce(pos, box, pbc, 3.4)
    assert _margin_ok(d, 3.4)
    rows = _sell_rows(nb)
    for i in range(pos.shape[0]):
        np.testing.assert_array_equal(rows[i], idx[indptr[i]:indptr[i + 1]])


def test_neighbor_errors(g):
    s = synth.graphene_rect(6, 6, 0.1, 1)
    pos, _ = _dev(s)
    with pytest.raises(g.GputbError) as e:
        g.build_neighbors(pos, s.box, s.pbc, 3.0, max_width=8)
    assert e.value.status == g.TB_ERR_ELL_OVERFLOW
    small = synth.graphene_rect(1, 6)
    with pytest.raises(g.GputbError) as e:
        g.build_neighbors(torch.tensor(small.positions, device="cuda"), small.box, small.pbc, 3.0)
    assert e.value.status == g.TB_ERR_BOX
    bad = s.positions.copy()
    bad[5, 1] = np.nan
    with pytest.raises(g.GputbError) as e:
        g.build_neighbors(torch.tensor(bad, device="cuda"), s.box, s.pbc, 3.0)
    assert e.value.status == g.TB_ERR_NOT_FINITE


def _oracle_teacher(s, params):
    indptr, idx, d = onb.neighbors(s.positions, s.box, s.pbc, params.rcut)
    t, eps, _ = ote.teacher_elements(s.species, indptr, idx, d, params)
    return indptr, idx, t, eps


def _sell_values(H, nb):
    sp = nb.slice_ptr.cpu().numpy()
    val = H.val.cpu().numpy()
    cnt = nb.cnt.cpu().numpy()
    out = []
    for i in range(nb.n):
        k, lane = divmod(i, 32)
        w = (sp[k + 1] - sp[k]) // 32
        pos = sp[k] + lane + 32 * np.arange(w)
        assert np.all(val[pos[cnt[i]:]] == 0.0)
        out.append(val[pos[:cnt[i]]])
    return np.concatenate(out)


@pytest.mark.parametrize("name,params", [("prim800", synth.teacher_graphene()),
                                         ("junction", synth.teacher_hbn_graphene())])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_teacher_values(g, name, params, dtype):
    s = STRUCTS[name]()
    pos, spc = _dev(s)
    nb = g.build_neighbors(pos, s.box, s.pbc, params.rcut, r_count=params.r_count)
    H = g.build_hamiltonian_teacher(pos, spc, s.box, s.pbc, nb, params, dtype=dtype)
    indptr, idx, t, eps = _oracle_teacher(s, params)
    v = _sell_values(H, nb)
    if dtype == torch.float64:
        np.testing.assert_allclose(v, t, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(H.diag.cpu().numpy(), eps, rtol=0, atol=0)
    else:
        # FP32 exp/cos: within a few FP32 ulp of the FP64 teacher
        np.testing.assert_allclose(v, t.astype(np.float32), rtol=2.0 ** -20, atol=1e-12)


def test_spectral_bounds_match_oracle(g):
    s = STRUCTS["prim800"]()
    params = synth.teacher_graphene()
    pos, spc = _dev(s)
    nb = g.build_neighbors(pos, s.box, s.pbc, params.rcut, r_count=params.r_count)
    H = g.build_hamiltonian_teacher(pos, spc, s.box, s.pbc, nb, params, dtype=torch.float64)
    bd = g.spectral_bounds(H, 64, synth.LANCZOS_SEED)
    indptr, idx, t, eps = _oracle_teacher(s, params)
    Hc = oha.csr_hamiltonian(s.n, indptr, idx, t, eps)
    emin, emax, a, b = obo.spectral_bounds(Hc, 64, synth.LANCZOS_SEED)
    np.testing.assert_allclose([bd.emin, bd.emax, bd.a, bd.b], [emin, emax, a, b], rtol=1e-9, atol=1e-12)
    ev = np.linalg.eigvalsh(Hc.toarray())
    assert bd.emin <= ev[0] and ev[-1] <= bd.emax
    gmin, gmax = obo.gershgorin(Hc)
    np.testing.assert_allclose([bd.g_min, bd.g_max], [gmin, gmax], rtol=1e-13)


@pytest.mark.parametrize("name", ["prim800", "junction_ragged", "rect100k_ragged"])
def test_spectral_bounds_fp32_values_match_oracle(g, name):
    """FP32 Hamiltonian: the GPU Lanczos runs in double-float arithmetic
    (about 48 significant bits); against the FP64 oracle on the same
    FP32-rounded values the bounds agree to rel 1e-9, and both enclose the
    spectrum.  The 100k-atom case spans many CTAs with a ragged last slice."""
    from tests.sell_helpers import sell_matrix
    if name == "prim800":
        s, params = synth.graphene_primitive(20, 20, 0.05, 1001), synth.teacher_graphene()
    elif name == "junction_ragged":
        s, params = synth.hbn_graphene_junction(6, 7, 0.1, 9), synth.teacher_hbn_graphene()
        s.positions, s.species = s.positions[:-5].copy(), s.species[:-5].copy()
    else:
        s, params = synth.graphene_rect(101, 251, 0.1, 31), synth.teacher_graphene()
    indptr, idx, t, eps = _oracle_teacher(s, params)
    t32 = t.astype(np.float32).astype(np.float64)
    e32 = eps.astype(np.float32).astype(np.float64)
    Hd = sell_matrix(indptr, idx, t32, e32, s.n, torch.float32)
    bd = g.spectral_bounds(Hd, 64, synth.LANCZOS_SEED)
    Hc = oha.csr_hamiltonian(s.n, indptr, idx, t32, e32)
    emin, emax, a, b = obo.spectral_bounds(Hc, 64, synth.LANCZOS_SEED)
    np.testing.assert_allclose([bd.emin, bd.emax, bd.a, bd.b], [emin, emax, a, b], rtol=1e-9, atol=1e-12)
    gmin, gmax = obo.gershgorin(Hc)
    np.testing.assert_allclose([bd.g_min, bd.g_max], [gmin, gmax], rtol=1e-13)
    if s.n <= 1000:
        ev = np.linalg.eigvalsh(Hc.toarray())
        assert bd.emin <= ev[0] and ev[-1] <= bd.emax


def test_plain_path_end_to_end(g):
    """positions -> GPU path -> DOS, against the oracle path on the same input."""
    w = synth.WORKLOADS["graphene-800-fp64"]
    s = synth.graphene_primitive(w["n1"], w["n2"], w["sigma"], w["seed"])
    params = synth.teacher_graphene()
    pos, spc = _dev(s)
    nb = g.build_neighbors(pos, s.box, s.pbc, params.rcut, r_count=params.r_count)
    H = g.build_hamiltonian_teacher(pos, spc, s.box, s.pbc, nb, params, dtype=torch.float64)
    bd = g.spectral_bounds(H, 64, synth.LANCZOS_SEED)
    indptr, idx, t, eps = _oracle_teacher(s, params)
    Hc = oha.csr_hamiltonian(s.n, indptr, idx, t, eps)
    emin, emax, a, b = obo.spectral_bounds(Hc, 64, synth.LANCZOS_SEED)
    # moments with the bounds passed explicitly to both sides
    mu = g.kpm_moments(H, a, b, w["M"], w["R"], synth.KPM_SEED)
    mu_ref_mean, mu_ref = okpm.kpm_moments(Hc, a, b, w["M"], w["R"], synth.KPM_SEED)
    assert np.max(np.abs(mu.cpu().numpy() - mu_ref)) <= 1e-12
    E = np.linspace(emin, emax, w["K"])
    rho = g.kpm_dos(mu, a, b, torch.tensor(E, device="cuda")).cpu().numpy()
    rho_ref = ods.density_of_states(mu_ref_mean, a, b, E)
    assert np.sum(np.abs(rho - rho_ref)) / np.sum(np.abs(rho_ref)) <= 1e-3
    # and with the GPU's own bounds the DOS still agrees
    mu2 = g.kpm_moments(H, bd.a, bd.b, w["M"], w["R"], synth.KPM_SEED)
    rho2 = g.kpm_dos(mu2, bd.a, bd.b, torch.tensor(E, device="cuda")).cpu().numpy()
    assert np.sum(np.abs(rho2 - rho_ref)) / np.sum(np.abs(rho_ref)) <= 1e-3


@pytest.mark.slow
def test_neighbors_full_size_sampled_rows(g):
    """10-million-atom 300 K sheet (the learned-path workload): sampled rows
    against the oracle's brute force of the definition."""
    w = synth.WORKLOADS["graphene-10M-learned"]
    s = synth.graphene_rect(w["nx"], w["ny"], w["sigma"], w["seed"])
    pos = torch.tensor(s.positions, device="cuda")
    nb = g.build_neighbors(pos, s.box, s.pbc, 3.0, r_count=1.8, max_width=16)
    rng = np.random.default_rng(0)
    rows = np.concatenate([[0, 1, s.n - 1], rng.choice(s.n, 13, replace=False)])
    sp = nb.slice_ptr.cpu().numpy()
    cnt = nb.cnt.cpu().numpy()
    for i, (ref, dv) in zip(rows, onb.neighbors_of_rows(s.positions, s.box, s.pbc, 3.0, rows)):
        k, lane = divmod(int(i), 32)
        pos_e = sp[k] + lane + 32 * np.arange(cnt[i])
        got = nb.col[torch.tensor(pos_e, device="cuda")].cpu().numpy()
        np.testing.assert_array_equal(got, ref)
    assert int(nb.cnt.max()) <= 16


@pytest.mark.parametrize("name,params", [("prim800", synth.teacher_graphene()),
                                         ("junction", synth.teacher_hbn_graphene())])
def test_teacher_fp32_symmetric_bit_for_bit(g, name, params):
    """The FP32 teacher forms bond lengths from FP32-pair positions; every
    step is sign-symmetric, so H_ij and H_ji agree bit for bit, across the
    periodic seams of the triclinic primitive sheet too."""
    s = STRUCTS[name]()
    pos, spc = _dev(s)
    nb = g.build_neighbors(pos, s.box, s.pbc, params.rcut, r_count=params.r_count)
    H = g.build_hamiltonian_teacher(pos, spc, s.box, s.pbc, nb, params, dtype=torch.float32)
    indptr, idx, t, eps = _oracle_teacher(s, params)
    v = _sell_values(H, nb)
    rows = np.repeat(np.arange(s.n), np.diff(indptr))
    for e in range(len(idx)):
        i, j = rows[e], idx[e]
        back = indptr[j] + int(np.searchsorted(idx[indptr[j]:indptr[j + 1]], i))
        assert idx[back] == i and v[e] == v[back], (i, j)
