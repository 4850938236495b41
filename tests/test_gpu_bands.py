"""GPU parity of the environment-network model and the band-energy training
path (Eq. 2 edge feature, Sec. 3 SK form and H(R) -> H(k) -> E_pre, Eq. 3
band loss) against the FP64 oracle, through the C ABI.

Bars (FP32 arithmetic on the device, FP64 in the oracle):
* bond inputs: C and u rel 2e-5, n_z^2 and d abs 2e-6 (1e-6 of r_cut);
* hoppings and onsite terms: rel 1e-5 of the largest (FP32 network sums
  of 8..32 terms, accurate SiLU);
* bands: on the device's own H(k), |dE| <= 1e-5 ||H(k)||_2 and
  ||H psi - E psi|| <= 2e-5 ||H(k)||_2, orthonormal to 8 n 2^-24 (FP32
  Jacobi, each column rotated about 8 n times);
  against the oracle's model, within Weyl's bound max_i sum_j |dH_ij| of
  the element differences (itself <= 1e-4 of the band width) plus 1e-5;
* loss statistics rel 1e-6, dL/dE rel 1e-5 (same eigenvalues fed to both);
* Hellmann-Feynman gradients and the network gradient: rel L2 1e-4 when fed
  the same upstream gradient; the whole training gradient: rel L2 1e-3.
"""
import numpy as np
import pytest
import torch

from oracle import env_bands as oe
from oracle import neighbors as onb
from oracle import teacher as ote
from paper_2509_06525_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_2509_06525_gb300 import build, gputb
    build.build()
    return gputb


@pytest.fixture(scope="module")
def bands():
    from paper_2509_06525_gb300 import bands as b
    return b


CMIX = synth.descriptor_mixing("identity")


def _slots(sp, cnt, row):
    return sp[row >> 5] + (row & 31) + 32 * np.arange(cnt[row])


def _oracle_cell(s, rcut=3.0):
    indptr, idx, d = onb.neighbors(s.positions, s.box, s.pbc, rcut)
    C, u, nz2, v = oe.edge_inputs(s.species, indptr, idx, d, CMIX.astype(float), rcut)
    return dict(n=s.n, species=s.species, indptr=indptr, indices=idx, dvec=d, C=C, u=u, nz2=nz2, v=v)


def _sell_to_csr(batch, c):
    """SELL positions of cell c's elements in the oracle's CSR order."""
    sp = batch.slice_ptr.cpu().numpy()
    cnt = batch.cnt.cpu().numpy()
    P = batch.rows_per_cell
    return np.concatenate([_slots(sp, cnt, c * P + i) for i in range(batch.n_atoms)]).astype(np.int64)


def _structure_with_vacancy(seed):
    s = synth.graphene_rect(2, 3, 0.1, seed)
    keep = np.arange(s.n) != 5
    return synth.Structure(s.positions[keep], s.species[keep], s.box, s.pbc, name="graphene-2x3-vacancy")


def test_env_hamiltonian_vs_oracle(g):
    """A 400-atom h-BN/graphene junction (three species: every onsite
    network output is used) with a random model: H from positions, from
    stored bond inputs, and against the oracle."""
    s = synth.hbn_graphene_junction(10, 10, 0.1, 17)
    p = synth.teacher_hbn_graphene()
    flat = synth.init_env_mlp(8, -1.0)
    eps0 = np.array([0.2, -0.1, 0.05])
    model = g.EnvModel(flat, CMIX, eps0)
    pos = torch.tensor(s.positions, device="cuda")
    spc = torch.tensor(s.species, device="cuda")
    nb = g.build_neighbors(pos, s.box, s.pbc, p.rcut, r_count=p.r_count, max_width=16)
    v = g.compute_descriptors(pos, spc, s.box, s.pbc, p.rcut, nb, model.cmix)
    feat = g.env_edge_inputs(pos, spc, s.box, s.pbc, p.rcut, nb, model.cmix, v)
    g.env_set_variant(1)   # FP32 pipes: the arithmetic of env_forward
    try:
        H = g.build_hamiltonian_env(pos, spc, s.box, s.pbc, p.rcut, nb, model, v=v)
    finally:
        g.env_set_variant(0)
    val, diag = g.env_forward(s.n, nb.slice_ptr, nb.cnt, feat, v, spc, model, nb.total)
    torch.cuda.synchronize()
    assert torch.equal(H.val, val) and torch.equal(H.diag, diag)

    o = _oracle_cell(s, p.rcut)
    sp, cnt = nb.slice_ptr.cpu().numpy(), nb.cnt.cpu().numpy()
    pos_e = np.concatenate([_slots(sp, cnt, i) for i in range(s.n)])
    f = feat.cpu().numpy()[pos_e].astype(np.float64)
    np.testing.assert_array_equal(nb.col.cpu().numpy()[pos_e], o["indices"])
    np.testing.assert_allclose(f[:, :8], o["C"], rtol=2e-5, atol=2e-5)
    np.testing.assert_allclose(f[:, 8:16], o["u"], rtol=2e-5, atol=2e-5)
    np.testing.assert_allclose(f[:, 16], o["nz2"], atol=2e-6)
    np.testing.assert_allclose(f[:, 17:20], o["dvec"], atol=2e-6)

    t_ref, _ = oe.hopping_forward(flat.astype(np.float64), o["C"], o["u"], o["nz2"])
    e_ref, _ = oe.onsite_forward(flat.astype(np.float64), o["v"], s.species, eps0.astype(np.float32))
    t = val.cpu().numpy()[pos_e].astype(np.float64)
    assert np.max(np.abs(t - t_ref)) <= 1e-5 * np.max(np.abs(t_ref))
    assert np.max(np.abs(diag.cpu().numpy() - e_ref)) <= 1e-5 * np.max(np.abs(e_ref))
    # symmetric bit for bit: the (j, i) element equals the (i, j) one
    rows = np.repeat(np.arange(s.n), np.diff(o["indptr"]))
    tv = val.cpu().numpy()
    for e in range(0, len(pos_e), 7):
        i, j = rows[e], o["indices"][e]
        back = _slots(sp, cnt, j)[int(np.searchsorted(o["indices"][o["indptr"][j]:o["indptr"][j + 1]], i))]
        assert tv[pos_e[e]] == tv[back]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_env_hamiltonian_tensor_cores_vs_oracle(g, dtype):
    """The default kernel of H from positions: the hopping network on the
    tensor cores (BF16 layer inputs and weights, FP32 accumulation, hardware
    tanh in SiLU).  A 48,000-atom h-BN/graphene junction: every CTA takes
    several 128-slot tiles, the last tile is ragged.  Bars: each layer input
    and weight carries a BF16 rounding (2^-9 relative); over four layers
    with sums of 8..32 terms this gives rel L2 <= 1e-2 and max <= 3e-2 of
    max|t| against the FP64 oracle.  Identical bond inputs give identical
    rows, so H stays symmetric bit for bit; the onsite terms (FP32 network)
    keep the FP32 bar; padding slots stay untouched."""
    s = synth.hbn_graphene_junction(120, 100, 0.1, 23)
    p = synth.teacher_hbn_graphene()
    flat = synth.init_env_mlp(8, -1.0)
    eps0 = np.array([0.2, -0.1, 0.05])
    model = g.EnvModel(flat, CMIX, eps0)
    pos = torch.tensor(s.positions, device="cuda")
    spc = torch.tensor(s.species, device="cuda")
    nb = g.build_neighbors(pos, s.box, s.pbc, p.rcut, r_count=p.r_count, max_width=16)
    v = g.compute_descriptors(pos, spc, s.box, s.pbc, p.rcut, nb, model.cmix)
    H = g.build_hamiltonian_env(pos, spc, s.box, s.pbc, p.rcut, nb, model, v=v, dtype=dtype)
    torch.cuda.synchronize()
    sp, cnt = nb.slice_ptr.cpu().numpy(), nb.cnt.cpu().numpy()
    assert -(-int(sp[-1]) // 128) >= 3 * 152 * 8          # tiles >= 3 x the largest grid

    o = _oracle_cell(s, p.rcut)
    pos_e = np.concatenate([_slots(sp, cnt, i) for i in range(s.n)])
    t_ref, _ = oe.hopping_forward(flat.astype(np.float64), o["C"], o["u"], o["nz2"])
    e_ref, _ = oe.onsite_forward(flat.astype(np.float64), o["v"], s.species, eps0.astype(np.float32))
    tv = H.val.cpu().numpy().astype(np.float64)
    t = tv[pos_e]
    scale = np.max(np.abs(t_ref))
    assert np.linalg.norm(t - t_ref) <= 1e-2 * np.linalg.norm(t_ref)
    assert np.max(np.abs(t - t_ref)) <= 3e-2 * scale
    assert np.max(np.abs(H.diag.cpu().numpy() - e_ref)) <= 1e-5 * np.max(np.abs(e_ref))
    pad = np.ones(len(tv), dtype=bool)
    pad[pos_e] = False
    assert np.all(tv[pad] == 0.0)
    rows = np.repeat(np.arange(s.n), np.diff(o["indptr"]))
    for e in range(0, len(pos_e), 11):
        i, j = rows[e], o["indices"][e]
        back = _slots(sp, cnt, j)[int(np.searchsorted(o["indices"][o["indptr"][j]:o["indptr"][j + 1]], i))]
        assert tv[pos_e[e]] == tv[back]


@pytest.mark.parametrize("shape", ["24", "23-odd", "64-max", "pristine-gamma"])
def test_bloch_bands_vs_oracle(g, bands, shape):
    """The eigensolver on the device's own H (tight), then the bands of the
    device's model against the oracle's within Weyl's bound: |dE| <=
    ||dH||_2 <= max row sum of |dH| over the differences of the Hamiltonian
    elements (FP32 descriptors and network), plus the eigensolver's share."""
    p = synth.teacher_graphene()
    if shape == "24":
        cells = synth.band_training_cells(3, 100)
    elif shape == "23-odd":
        cells = [_structure_with_vacancy(sd) for sd in (1, 2)]
    elif shape == "64-max":
        cells = synth.band_training_cells(2, 200, nx=4, ny=4)
    else:
        cells = [synth.graphene_rect(2, 3, 0.0, 0)]
    kpts = synth.band_kgrid(cells[0].box, 2, 2)
    if shape == "pristine-gamma":
        kpts = np.concatenate([np.zeros((1, 3)), kpts])
    flat = synth.init_env_mlp(9, -1.5)
    model = g.EnvModel(flat, CMIX, np.zeros(3))
    batch = bands.build_cell_batch(cells, p, CMIX, kpts)
    val, diag = g.env_forward(batch.n_rows, batch.slice_ptr, batch.cnt, batch.feat, batch.v, batch.species, model,
                              batch.total)
    evals, evecs = bands.bands_of(batch, val, diag)
    E, Psi = evals.cpu().numpy(), evecs.cpu().numpy()
    vd, dd = val.cpu().numpy().astype(np.float64), diag.cpu().numpy().astype(np.float64)
    td, edt = batch.t_teacher.cpu().numpy().astype(np.float64), batch.eps_teacher.cpu().numpy().astype(np.float64)
    P = batch.rows_per_cell
    for c, s in enumerate(cells):
        o = _oracle_cell(s)
        pos_e = _sell_to_csr(batch, c)
        rows = np.repeat(np.arange(s.n), np.diff(o["indptr"]))
        t_dev, e_dev = vd[pos_e], dd[c * P:c * P + s.n]
        # 1. eigensolver: the oracle's dense solver on the device's H
        E_same, _ = oe.bands(s.n, o["indptr"], o["indices"], o["dvec"], t_dev, e_dev, kpts)
        for q, k in enumerate(kpts):
            Hk = oe.bloch_hamiltonian(s.n, o["indptr"], o["indices"], o["dvec"], t_dev, e_dev, k)
            nrm = np.linalg.norm(Hk, 2)
            assert np.max(np.abs(E[c, q] - E_same[q])) <= 1e-5 * nrm, (shape, q)
            V = Psi[c, q].astype(np.complex128)
            res = np.linalg.norm(Hk @ V - V * E[c, q][None, :], axis=0)
            assert res.max() <= 2e-5 * nrm
            assert np.max(np.abs(V.conj().T @ V - np.eye(s.n))) <= 8 * s.n * 2.0 ** -24
        # 2. the device model's bands against the oracle model's
        t_ref, _ = oe.hopping_forward(flat.astype(np.float64), o["C"], o["u"], o["nz2"])
        e_ref, _ = oe.onsite_forward(flat.astype(np.float64), o["v"], s.species, np.zeros(3))
        E_ref, _ = oe.bands(s.n, o["indptr"], o["indices"], o["dvec"], t_ref, e_ref, kpts)
        weyl = np.max(np.abs(e_dev - e_ref) + np.bincount(rows, np.abs(t_dev - t_ref), s.n))
        assert weyl <= 1e-4 * np.max(np.abs(E_ref)), weyl
        nrm = np.max(np.abs(E_ref))
        assert np.max(np.abs(E[c] - E_ref)) <= weyl + 1e-5 * nrm, (shape, float(np.max(np.abs(E[c] - E_ref))), weyl)
        # 3. the teacher's reference bands
        tt, et, _ = ote.teacher_elements(s.species, o["indptr"], o["indices"], o["dvec"], p)
        Et, _ = oe.bands(s.n, o["indptr"], o["indices"], o["dvec"], tt, et, kpts)
        weyl_t = np.max(np.abs(edt[c * P:c * P + s.n] - et) + np.bincount(rows, np.abs(td[pos_e] - tt), s.n))
        assert np.max(np.abs(batch.e_ref.cpu().numpy()[c] - Et)) <= weyl_t + 1e-5 * np.max(np.abs(Et))


def test_single_atom_cell(g, bands):
    """One atom in a 7 A periodic cell: no neighbour, H(k) = eps."""
    s = synth.Structure(np.array([[1.0, 2.0, 0.0]]), np.array([1], np.int32),
                        np.diag([7.0, 7.0, 20.0]), name="single-atom")
    p = synth.teacher_hbn_graphene()
    batch = bands.build_cell_batch([s], p, CMIX, synth.band_kgrid(s.box, 2, 1))
    np.testing.assert_array_equal(batch.e_ref.cpu().numpy(), np.full((1, 2, 1), np.float32(p.onsite[1])))


def test_band_loss_and_gradient_vs_oracle(g, bands):
    p = synth.teacher_graphene()
    cells = synth.band_training_cells(3, 300)
    kpts = synth.band_kgrid(cells[0].box, 2, 2)
    flat = synth.init_env_mlp(10, -1.0)
    model = g.EnvModel(flat, CMIX, np.zeros(3))
    batch = bands.build_cell_batch(cells, p, CMIX, kpts)
    n_spec = len(cells) * len(kpts)
    w = bands.band_weights(batch.n_atoms, (4, 20), n_spec)
    tr = bands.BandTrainer(model, batch)
    stats, grad, evals = tr.loss_and_grad(w)
    torch.cuda.synchronize()
    E = evals.cpu().numpy().astype(np.float64)
    E_ref = batch.e_ref.cpu().numpy().astype(np.float64)
    wn = w.cpu().numpy().astype(np.float64)

    # the loss on the same eigenvalues
    L, dLdE = oe.band_loss(E, E_ref, wn)
    st = stats.cpu().numpy()
    assert abs(st[2] - L) <= 1e-6 * L
    dLdE_dev, _ = g.band_loss(evals, batch.e_ref, w)
    np.testing.assert_allclose(dLdE_dev.cpu().numpy(), dLdE, rtol=1e-5, atol=1e-5 * np.max(np.abs(dLdE)))

    # Hellmann-Feynman gradient per element and the network gradient, each fed
    # the device's upstream gradient
    g_val, g_diag = tr.g_val.cpu().numpy(), tr.g_diag.cpu().numpy()
    grad_net = np.zeros(oe.ENV_NPARAM)
    cells_o = []
    for c, s in enumerate(cells):
        o = _oracle_cell(s)
        cells_o.append(o)
        pos_e = _sell_to_csr(batch, c)
        t_ref, hc = oe.hopping_forward(flat.astype(np.float64), o["C"], o["u"], o["nz2"])
        e_ref, oc = oe.onsite_forward(flat.astype(np.float64), o["v"], s.species, np.zeros(3))
        _, psi = oe.bands(s.n, o["indptr"], o["indices"], o["dvec"], t_ref, e_ref, kpts)
        gt, ge = oe.band_gradient(o["indptr"], o["indices"], o["dvec"], kpts, psi, dLdE[c])
        gt_dev = g_val[pos_e].astype(np.float64)
        ge_dev = g_diag[c * batch.rows_per_cell:c * batch.rows_per_cell + s.n].astype(np.float64)
        assert np.linalg.norm(gt_dev - gt) <= 1e-4 * np.linalg.norm(gt)
        assert np.linalg.norm(ge_dev - ge) <= 1e-4 * np.linalg.norm(ge)
        grad_net += oe.hopping_backward(flat.astype(np.float64), hc, gt_dev)
        grad_net += oe.onsite_backward(flat.astype(np.float64), oc, ge_dev)
    gd = grad.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gd - grad_net) <= 1e-4 * np.linalg.norm(grad_net)

    # the whole chain against the oracle's own
    Lo, go, _ = oe.cell_loss_and_grad(flat.astype(np.float64), cells_o, kpts, E_ref, wn, np.zeros(3))
    assert abs(st[2] - Lo) <= 1e-4 * Lo
    assert np.linalg.norm(gd - go) <= 1e-3 * np.linalg.norm(go)

    # reproducible: the same step gives the same gradient bit for bit
    _, grad2, _ = tr.loss_and_grad(w)
    assert torch.equal(grad, grad2)


def test_bad_cell_layout_is_an_error(g, bands):
    """Declaring 12 atoms per cell when the neighbours reach row 23 is
    rejected (every access stays inside the declared rows)."""
    p = synth.teacher_graphene()
    cells = synth.band_training_cells(2, 400)
    batch = bands.build_cell_batch(cells, p, CMIX, synth.band_kgrid(cells[0].box, 1, 1))
    with pytest.raises(g.GputbError) as err:
        g.bloch_bands(batch.n_cells, 12, batch.rows_per_cell, batch.slice_ptr, batch.col, batch.cnt, batch.feat,
                      batch.t_teacher, batch.eps_teacher, batch.kpts)
    assert err.value.status == g.TB_ERR_INVALID_ARG
    with pytest.raises(g.GputbError):
        g.bloch_bands(batch.n_cells, 65, 96, batch.slice_ptr, batch.col, batch.cnt, batch.feat, batch.t_teacher,
                      batch.eps_teacher, batch.kpts)


def test_band_training_reduces_the_loss(g, bands):
    """Band-expansion training on 16 disordered 24-atom cells: the loss of
    Eq. 3 and the band error fall well below their initial values."""
    p = synth.teacher_graphene()
    cells = synth.band_training_cells(16, 500)
    kpts = synth.band_kgrid(cells[0].box, 2, 2)
    batch = bands.build_cell_batch(cells, p, CMIX, kpts)
    model = g.EnvModel(synth.init_env_mlp(11, -1.0), CMIX, np.zeros(3))
    w_all = bands.band_weights(batch.n_atoms, (0, batch.n_atoms), batch.n_cells * len(kpts))
    tr = bands.BandTrainer(model, batch)
    L0 = float(tr.loss_and_grad(w_all)[0][2].item())
    mae0 = bands.band_mae(model, batch)
    hist = bands.train_bands(model, batch, [(150, (8, 16)), (150, (4, 20)), (300, (0, 24))], lr=3e-3)
    L1 = float(tr.loss_and_grad(w_all)[0][2].item())
    mae1 = bands.band_mae(model, batch)
    print(f"band MAE {mae0:.4f} -> {mae1:.4f} eV; full-window loss {L0:.4g} -> {L1:.4g}; "
          f"last logged {hist[-1]}")
    assert L1 < 0.1 * L0
    assert mae1 < 0.25 * mae0
