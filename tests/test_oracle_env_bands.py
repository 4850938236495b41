"""Pins of the environment-network model and band-energy loss oracle
(Eq. 2 edge feature, Sec. 3 SK form, Eq. 3 band loss) against closed forms,
the Bloch theorem and finite differences."""
import math

import numpy as np
import pytest

from oracle import env_bands as oe
from oracle import neighbors as onb
from oracle import teacher as ote
from paper_2509_06525_gb300 import synth


def _cell(nx=2, ny=3, sigma=0.1, seed=5):
    s = synth.graphene_rect(nx, ny, sigma, seed)
    indptr, idx, d = onb.neighbors(s.positions, s.box, s.pbc, 3.0)
    return s, indptr, idx, d


def _inputs(s, indptr, idx, d):
    C, u, nz2, v = oe.edge_inputs(s.species, indptr, idx, d, synth.descriptor_mixing("identity").astype(float), 3.0)
    return dict(n=s.n, species=s.species, indptr=indptr, indices=idx, dvec=d, C=C, u=u, nz2=nz2, v=v)


def test_layout():
    assert oe.ENV_NPARAM == 2349 == synth.ENV_NPARAM
    flat = np.arange(oe.ENV_NPARAM, dtype=float)
    np.testing.assert_array_equal(oe.pack(oe.unpack(flat)), flat)


def test_bloch_bands_fold_honeycomb_closed_form():
    """Pristine 2 x 3 rectangular supercell (24 atoms): at any k its bands
    are the honeycomb bands E(k + G) = t2 g2 +- |t1 f1 + t3 f3| of the
    primitive cell at the 12 cosets G of the supercell's reciprocal lattice
    modulo the primitive one (Bloch theorem).  Pins the phase e^{ik.d} and
    the image handling of bloch_hamiltonian."""
    p = synth.teacher_graphene()
    s, indptr, idx, d = _cell(sigma=0.0)
    t, eps, _ = ote.teacher_elements(s.species, indptr, idx, d, p)
    a = p.a_cc
    t1, t2, t3 = (float(ote.hopping(r, 0, 0, 3, 3, p)) for r in (a, math.sqrt(3) * a, 2 * a))
    delta = np.array([[a, 0.0], [-0.5 * a, 0.5 * math.sqrt(3) * a], [-0.5 * a, -0.5 * math.sqrt(3) * a]])
    second = [delta[0] - delta[1], delta[0] - delta[2], delta[2] - delta[1]]

    def honeycomb(k):
        f1 = np.sum(np.exp(1j * delta @ k))
        f3 = np.sum(np.exp(-2j * delta @ k))
        g2 = 2.0 * sum(math.cos(float(np.dot(k, v))) for v in second)
        return [t2 * g2 - abs(t1 * f1 + t3 * f3), t2 * g2 + abs(t1 * f1 + t3 * f3)]

    B1 = 2 * math.pi / s.box[0, 0]
    B2 = 2 * math.pi / s.box[1, 1]
    rng = np.random.default_rng(0)
    kpts = np.concatenate([rng.uniform(-1, 1, (3, 2)), np.zeros((3, 1))], axis=1)
    E, _ = oe.bands(s.n, indptr, idx, d, t, eps, kpts)
    for q, k in enumerate(kpts):
        ref = []
        for m1 in range(4):
            for m2 in range(3):
                ref += honeycomb(k[:2] + np.array([m1 * B1, m2 * B2]))
        np.testing.assert_allclose(E[q], np.sort(ref), atol=1e-12)


def test_bloch_hamiltonian_hermitian_and_periodic():
    s, indptr, idx, d = _cell()
    c = _inputs(s, indptr, idx, d)
    flat = synth.init_env_mlp(3, 0.5)
    t, _ = oe.hopping_forward(flat, c["C"], c["u"], c["nz2"])
    eps, _ = oe.onsite_forward(flat, c["v"], s.species, np.zeros(3))
    k = np.array([0.3, -0.7, 0.0])
    Hk = oe.bloch_hamiltonian(s.n, indptr, idx, d, t, eps, k)
    np.testing.assert_allclose(Hk, Hk.conj().T, atol=1e-13)
    G = np.array([2 * math.pi / s.box[0, 0], 2 * 2 * math.pi / s.box[1, 1], 0.0])
    E0 = np.linalg.eigvalsh(Hk)
    E1 = np.linalg.eigvalsh(oe.bloch_hamiltonian(s.n, indptr, idx, d, t, eps, k + G))
    np.testing.assert_allclose(E0, E1, atol=1e-12)


def test_env_hopping_symmetric():
    """t_ij = t_ji: the stored (j, i) element has the same inputs."""
    s, indptr, idx, d = _cell()
    c = _inputs(s, indptr, idx, d)
    t, _ = oe.hopping_forward(synth.init_env_mlp(4, 0.3), c["C"], c["u"], c["nz2"])
    rows = np.repeat(np.arange(s.n), np.diff(indptr))
    for e in range(len(idx)):
        i, j = rows[e], idx[e]
        back = indptr[j] + int(np.searchsorted(idx[indptr[j]:indptr[j + 1]], i))
        assert idx[back] == i
        assert abs(t[e] - t[back]) <= 1e-14 * max(1.0, abs(t[e]))


def test_edge_inputs_are_eq2_sums():
    """u_ij equals sum_{k in N(i)} C(r_ik) + sum_{l in N(j)} C(r_jl) taken
    edge by edge, and n_z^2 of a flat sheet is 0 (of a buckled one in [0, 1])."""
    s, indptr, idx, d = _cell()
    c = _inputs(s, indptr, idx, d)
    rows = np.repeat(np.arange(s.n), np.diff(indptr))
    for e in (0, 7, len(idx) - 1):
        i, j = rows[e], idx[e]
        ref = c["C"][indptr[i]:indptr[i + 1]].sum(0) + c["C"][indptr[j]:indptr[j + 1]].sum(0)
        np.testing.assert_allclose(c["u"][e], ref, rtol=1e-14)
    s.positions[:, 2] = 0.0
    flat_idx = onb.neighbors(s.positions, s.box, s.pbc, 3.0)
    assert np.all(_inputs(s, *flat_idx)["nz2"] == 0.0)
    assert np.all((c["nz2"] >= 0) & (c["nz2"] <= 1))


def test_band_loss_closed_form():
    E = np.array([[1.0, 2.0]])
    Er = np.array([[0.5, 2.5]])
    w = np.array([1.0, 2.0])
    L, g = oe.band_loss(E, Er, w)
    # S = 0.5 + 2 * 0.5 = 1.5; L = 1.5^2 + (0.25 + 2 * 0.25) = 3.0
    assert L == pytest.approx(3.0, abs=1e-15)
    np.testing.assert_allclose(g, [[2 * 1.5 * 1 + 2 * 0.5, -2 * 1.5 * 2 - 2 * 2 * 0.5]], atol=1e-15)
    # a zero residual contributes no subgradient
    _, g0 = oe.band_loss(np.array([[1.0]]), np.array([[1.0]]), np.array([3.0]))
    assert g0[0, 0] == 0.0


def test_network_backward_finite_difference():
    s, indptr, idx, d = _cell()
    c = _inputs(s, indptr, idx, d)
    rng = np.random.default_rng(1)
    flat = synth.init_env_mlp(6, 0.4).astype(float)
    a = rng.normal(size=len(idx))
    b = rng.normal(size=s.n)
    eps0 = np.array([0.1, -0.2, 0.3])

    def scalar(f):
        t, _ = oe.hopping_forward(f, c["C"], c["u"], c["nz2"])
        e, _ = oe.onsite_forward(f, c["v"], s.species, eps0)
        return float(a @ t + b @ e)

    t, hc = oe.hopping_forward(flat, c["C"], c["u"], c["nz2"])
    e, oc = oe.onsite_forward(flat, c["v"], s.species, eps0)
    g = oe.hopping_backward(flat, hc, a) + oe.onsite_backward(flat, oc, b)
    for trial in range(3):
        direction = rng.normal(size=flat.size)
        h = 1e-6
        fd = (scalar(flat + h * direction) - scalar(flat - h * direction)) / (2 * h)
        assert abs(fd - g @ direction) <= 1e-6 * max(1.0, abs(fd))
    # every parameter block receives gradient (no dropped layer)
    for name, block in oe.unpack(g).items():
        if name == "bo2":
            assert block[0] != 0.0 and block[1] == 0.0 and block[2] == 0.0   # only carbon rows
        else:
            assert np.any(block != 0.0), name


def test_hellmann_feynman_band_gradient():
    """dL/ds along a symmetric perturbation of the hoppings and onsite terms
    equals sum_e dL/dt_e dt_e/ds + sum_i dL/deps_i deps_i/ds."""
    s, indptr, idx, d = _cell(seed=9)
    rng = np.random.default_rng(2)
    rows = np.repeat(np.arange(s.n), np.diff(indptr))
    p = synth.teacher_graphene()
    t0, _, _ = ote.teacher_elements(s.species, indptr, idx, d, p)
    eps0 = rng.normal(0, 0.1, s.n)
    key = np.minimum(rows, idx) * s.n + np.maximum(rows, idx)
    _, inv = np.unique(key, return_inverse=True)
    dt = rng.normal(size=inv.max() + 1)[inv]          # symmetric direction
    de = rng.normal(size=s.n)
    kpts = synth.band_kgrid(s.box, 2, 2)
    E_ref = rng.normal(0, 0.5, (len(kpts), s.n)) + oe.bands(s.n, indptr, idx, d, t0, eps0, kpts)[0]
    w = rng.uniform(0.5, 1.5, s.n)

    def loss(x):
        E, _ = oe.bands(s.n, indptr, idx, d, t0 + x * dt, eps0 + x * de, kpts)
        return oe.band_loss(E, E_ref, w)[0]

    E, psi = oe.bands(s.n, indptr, idx, d, t0, eps0, kpts)
    gaps = np.diff(E, axis=1)
    assert gaps.min() > 1e-3                         # non-degenerate: HF applies
    _, dLdE = oe.band_loss(E, E_ref, w)
    gt, geps = oe.band_gradient(indptr, idx, d, kpts, psi, dLdE)
    h = 1e-6
    fd = (loss(h) - loss(-h)) / (2 * h)
    assert abs(fd - (gt @ dt + geps @ de)) <= 1e-6 * max(1.0, abs(fd))


def test_training_gradient_finite_difference():
    """The whole chain: parameters -> t, eps -> H(k) -> bands -> Eq. 3."""
    cells = [_inputs(*_cell(seed=sd)) for sd in (11, 12)]
    kpts = synth.band_kgrid(synth.graphene_rect(2, 3).box, 2, 1)
    rng = np.random.default_rng(3)
    flat = synth.init_env_mlp(7, -1.0).astype(float)
    E_ref = np.stack([rng.normal(0, 1, (len(kpts), c["n"])) for c in cells])
    w = np.linspace(1.0, 0.5, cells[0]["n"])
    eps0 = np.zeros(3)
    L, g, _ = oe.cell_loss_and_grad(flat, cells, kpts, E_ref, w, eps0)
    direction = rng.normal(size=flat.size)
    h = 1e-6
    Lp = oe.cell_loss_and_grad(flat + h * direction, cells, kpts, E_ref, w, eps0)[0]
    Lm = oe.cell_loss_and_grad(flat - h * direction, cells, kpts, E_ref, w, eps0)[0]
    fd = (Lp - Lm) / (2 * h)
    assert abs(fd - g @ direction) <= 1e-5 * max(1.0, abs(fd))


def test_hand_wired_network():
    """A network with single nonzero paths, evaluated by hand with the
    exponential: pins which index is output and input in every layer, the
    product C * m of Eq. 2, the sigma/pi assignment of the SK factors and the
    species pick of the onsite network."""
    import math

    def silu(x):
        return x / (1.0 + math.exp(-x))

    p = {name: np.zeros(shape) for name, shape in oe.ENV_LAYOUT}
    p["We1"][0, 1] = 1.0          # z1[0] = u[1]
    p["We2"][2, 0] = 1.0          # m[2] = h1[0]
    p["be2"][2] = 0.25
    p["Wh1"][3, 2] = 1.0          # z2[3] = e[2] = C[2] m[2]
    p["Wh2"][4, 3] = 1.0          # z3[4] = h2[3]
    p["Wh3"][0, 4] = 2.0          # y_sigma = 2 h3[4] + 0.5
    p["Wh3"][1, 4] = 3.0          # y_pi = 3 h3[4] - 1
    p["bh3"][:] = (0.5, -1.0)
    p["Wo1"][5, 6] = 1.0          # z[5] = v[6]
    p["Wo2"][1, 5] = 2.0          # out[1] = 2 h[5] + 0.1
    p["bo2"][1] = 0.1
    flat = oe.pack(p)
    C = np.zeros((1, 8))
    C[0, 2] = 1.5
    u = np.zeros((1, 8))
    u[0, 1] = 2.0
    nz2 = np.array([0.25])
    t, _ = oe.hopping_forward(flat, C, u, nz2)
    # every other unit has a zero pre-activation and silu(0) = 0
    h1_0 = silu(2.0)
    m_2 = h1_0 + 0.25
    e_2 = 1.5 * m_2
    h2_3 = silu(e_2)
    h3_4 = silu(h2_3)
    y_sigma = 2.0 * h3_4 + 0.5
    y_pi = 3.0 * h3_4 - 1.0
    assert t[0] == pytest.approx(0.25 * y_sigma + 0.75 * y_pi, rel=1e-14)
    v = np.zeros((2, 8))
    v[:, 6] = 1.5
    eps, _ = oe.onsite_forward(flat, v, np.array([1, 0]), np.array([0.0, -0.3, 0.0]))
    assert eps[0] == pytest.approx(-0.3 + 0.1 + 2.0 * silu(1.5), rel=1e-14)
    assert eps[1] == 0.0          # species 0 reads out[0] = 0
