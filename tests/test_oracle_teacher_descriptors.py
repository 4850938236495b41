"""Pins for oracle.teacher and oracle.descriptors: closed-form special
cases of f_c, of the teacher hopping and of the Chebyshev radial basis of
Eq. 2, and the node-feature sum on pristine graphene."""
import math

import numpy as np
from numpy.polynomial import chebyshev as npcheb

from oracle import descriptors as de
from oracle import neighbors as nb
from oracle import teacher as te
from paper_2509_06525_gb300 import synth


def test_cutoff_special_values():
    rc = 3.0
    np.testing.assert_allclose(te.cutoff([0.0, rc / 2, rc, rc + 1e-9, 10.0], rc),
                               [1.0, 0.5, 0.0, 0.0, 0.0], atol=1e-15)
    # f_c(rc/3) = (1 + cos(pi/3)) / 2 = 3/4
    np.testing.assert_allclose(te.cutoff(rc / 3, rc), 0.75, atol=1e-15)


def test_teacher_special_cases():
    p = synth.teacher_hbn_graphene()
    a = p.a_cc
    # at r = a_cc and n_i + n_j = 6 both the radial and environment factors are 1
    for zi, zj in [(0, 0), (1, 2), (2, 1), (1, 0), (2, 0), (1, 1)]:
        t = te.hopping(a, zi, zj, 3, 3, p)
        assert abs(t - p.hop_prefactor[zi, zj] * te.cutoff(a, p.rcut)) < 1e-14
    # environment factor: n_i + n_j = 12 scales by 1 + gamma = 1.05
    assert abs(te.hopping(2.0, 0, 0, 6, 6, p) / te.hopping(2.0, 0, 0, 3, 3, p) - 1.05) < 1e-14
    assert abs(te.hopping(2.0, 0, 0, 0, 0, p) / te.hopping(2.0, 0, 0, 3, 3, p) - 0.95) < 1e-14
    # radial factor halves at r = a (1 + ln 2 / beta) once f_c is divided out
    r_half = a * (1.0 + math.log(2.0) / p.beta)
    ratio = (te.hopping(r_half, 0, 0, 3, 3, p) / te.cutoff(r_half, p.rcut)) / \
            (te.hopping(a, 0, 0, 3, 3, p) / te.cutoff(a, p.rcut))
    assert abs(ratio - 0.5) < 1e-14
    # symmetric in the species pair and zero beyond the cutoff
    assert te.hopping(1.5, 1, 2, 3, 2, p) == te.hopping(1.5, 2, 1, 2, 3, p)
    assert te.hopping(3.0, 0, 0, 3, 3, p) == 0.0


def test_teacher_pristine_graphene_values():
    # pristine graphene: n_i = 3 for every atom, so t(r) = -2.7 e^{-3(r/a-1)} f_c(r)
    s = synth.graphene_rect(3, 4)
    p = synth.teacher_graphene()
    indptr, idx, d = nb.neighbors(s.positions, s.box, s.pbc, p.rcut)
    t, eps, ncount = te.teacher_elements(s.species, indptr, idx, d, p)
    assert np.all(ncount == 3)
    assert np.all(eps == 0.0)
    r = te.distances(d)
    for shell in (p.a_cc, math.sqrt(3) * p.a_cc, 2 * p.a_cc):
        sel = np.abs(r - shell) < 1e-9
        expect = -2.7 * math.exp(-3.0 * (shell / p.a_cc - 1.0)) * 0.5 * (1 + math.cos(math.pi * shell / 3.0))
        np.testing.assert_allclose(t[sel], expect, rtol=1e-13)


def test_chebyshev_recurrence_matches_library_and_trig():
    x = np.linspace(-1, 1, 101)
    T = de.chebyshev_T(12, x)
    for k in range(12):
        coef = np.zeros(k + 1)
        coef[k] = 1.0
        np.testing.assert_allclose(T[k], npcheb.chebval(x, coef), atol=1e-13)
        np.testing.assert_allclose(T[k], np.cos(k * np.arccos(x)), atol=1e-12)


def test_radial_basis_special_points():
    rc = 3.0
    f0 = de.radial_basis(np.array([0.0]), rc)[0]
    np.testing.assert_allclose(f0, np.ones(8), atol=1e-15)         # T_k(1) = 1, f_c(0) = 1
    np.testing.assert_allclose(de.radial_basis(np.array([rc]), rc)[0], 0.0, atol=1e-15)
    r_mid = rc * (1.0 - 1.0 / math.sqrt(2.0))                      # argument x = 0
    k = np.arange(8)
    expect = 0.5 * (np.cos(k * np.pi / 2) + 1.0) * te.cutoff(r_mid, rc)
    np.testing.assert_allclose(de.radial_basis(np.array([r_mid]), rc)[0], expect, atol=1e-14)


def test_node_feature_of_pristine_graphene():
    s = synth.graphene_primitive(5, 5)
    indptr, idx, d = nb.neighbors(s.positions, s.box, s.pbc, 3.0)
    cmix = synth.descriptor_mixing("identity")
    C, v, x = de.descriptors(s.species, indptr, idx, d, cmix, 3.0)
    a = synth.A_CC
    shells = de.radial_basis(np.array([a, math.sqrt(3) * a, 2 * a]), 3.0)
    expect = 3 * shells[0] + 6 * shells[1] + 3 * shells[2]
    np.testing.assert_allclose(v, np.broadcast_to(expect, v.shape), atol=1e-12)
    # edge input layout: [C, v_i, v_j, C * (v_i + v_j)]
    e = 0
    np.testing.assert_allclose(x[e, :8], C[e])
    np.testing.assert_allclose(x[e, 24:], C[e] * 2 * expect, atol=1e-12)


def test_species_mixing_is_applied_per_ordered_pair():
    cmix = synth.descriptor_mixing("species").astype(np.float64)
    r = np.array([1.3, 2.0, 2.9])
    zi = np.array([1, 2, 0])
    zj = np.array([2, 1, 0])
    C = de.mixed_descriptor(r, zi, zj, cmix, 3.0)
    f = de.radial_basis(r, 3.0)
    for e in range(3):
        np.testing.assert_allclose(C[e], cmix[zi[e], zj[e]] @ f[e], atol=1e-14)
    # the ordered pair matters: (B, N) and (N, B) mix differently
    c_rev = de.mixed_descriptor(r[:1], zj[:1], zi[:1], cmix, 3.0)
    assert not np.allclose(C[0], c_rev[0])


def _chain3():
    """Three atoms on an open line, 1.42 A apart (no periodic direction):
    neighbours within 3 A by hand: 0 -> {1, 2}, 1 -> {0, 2}, 2 -> {0, 1};
    bond lengths 1.42 (0-1, 1-2) and 2.84 (0-2)."""
    pos = np.array([[0.0, 0.0, 0.0], [1.42, 0.0, 0.0], [2.84, 0.0, 0.0]]) + 10.0
    box = np.diag([40.0, 40.0, 40.0])
    pbc = np.array([0, 0, 0], np.int32)
    return pos, box, pbc


def _f_library(r, rc=3.0, k=8):
    """f_k(r) = (T_k(2(r/rc - 1)^2 - 1) + 1)/2 * (1 + cos(pi r/rc))/2 with T_k
    from numpy's Chebyshev series routine (a library evaluation, not the
    oracle's recurrence)."""
    xx = 2.0 * (r / rc - 1.0) ** 2 - 1.0
    t = np.array([npcheb.chebval(xx, np.eye(k)[m]) for m in range(k)])
    return 0.5 * (t + 1.0) * 0.5 * (1.0 + math.cos(math.pi * r / rc))


def test_edge_input_blocks_and_onsite_receiver_on_an_open_chain():
    """Eq. 2 / the per-pair network's input and outputs on a chain where the
    two endpoints of a bond have different environments (v_0 != v_1): the
    edge input of 0 -> 1 is [C(r_01), v_0, v_1, C(r_01) (v_0 + v_1)] -- the
    source atom's block first -- and the onsite share y1(i -> j) goes to the
    source atom i, the hopping H_ij to (y0(i->j) + y0(j->i))/2.  Swapping the
    v blocks, or crediting y1 to j, fails here."""
    pos, box, pbc = _chain3()
    indptr, idx, d = nb.neighbors(pos, box, pbc, 3.0)
    assert list(idx[indptr[0]:indptr[1]]) == [1, 2]
    assert list(idx[indptr[1]:indptr[2]]) == [0, 2]
    assert list(idx[indptr[2]:indptr[3]]) == [0, 1]
    cmix = synth.descriptor_mixing("identity")
    species = np.zeros(3, np.int32)
    C, v, x = de.descriptors(species, indptr, idx, d, cmix, 3.0)
    f1, f2 = _f_library(1.42), _f_library(2.84)
    v0, v1 = f1 + f2, 2.0 * f1
    np.testing.assert_allclose(v[0], v0, atol=1e-13)
    np.testing.assert_allclose(v[1], v1, atol=1e-13)
    np.testing.assert_allclose(v[2], v0, atol=1e-13)
    assert np.max(np.abs(v0 - v1)) > 1e-2
    e01 = indptr[0] + 0          # edge 0 -> 1
    expect = np.concatenate([f1, v0, v1, f1 * (v0 + v1)])
    np.testing.assert_allclose(x[e01], expect, atol=1e-13)
    e10 = indptr[1] + 0          # edge 1 -> 0: the blocks swap with the direction
    np.testing.assert_allclose(x[e10], np.concatenate([f1, v1, v0, f1 * (v1 + v0)]), atol=1e-13)

    from oracle import mlp as om
    # distinctive outputs per directed edge: y0 = 100 i + j, y1 = 10 i + j
    rows = np.repeat(np.arange(3), np.diff(indptr))
    y = np.stack([100.0 * rows + idx, 10.0 * rows + idx], axis=1)
    hop, eps = om.learned_hamiltonian(indptr, idx, y, species, np.array([0.5, 0.0, 0.0]))
    np.testing.assert_allclose(eps, [0.5 + 1 + 2, 0.5 + 10 + 12, 0.5 + 20 + 21])
    # H_01 = (y0(0->1) + y0(1->0)) / 2 = (1 + 100) / 2, H_02 = (2 + 200) / 2, H_12 = (102 + 201) / 2
    np.testing.assert_allclose(hop[indptr[0]:indptr[1]], [50.5, 101.0])
    np.testing.assert_allclose(hop[indptr[1]:indptr[2]], [50.5, 151.5])
    np.testing.assert_allclose(hop[indptr[2]:indptr[3]], [101.0, 151.5])
