"""Pins for oracle.neighbors (N(i) of Eq. 1): closed-form graphene shells,
an independent explicit-supercell brute force, k-d tree == brute force."""
import os

import numpy as np
import pytest

from oracle import neighbors as nb
from paper_2509_06525_gb300 import synth


def _golden_shells():
    path = os.path.join(os.path.dirname(__file__), "golden", "graphene_shells.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    return [(int(c), float(d)) for c, d in rows]


SHELLS = _golden_shells()   # 1NN, 2NN, 3NN of pristine graphene


def _shell_check(s, rcut):
    indptr, idx, d = nb.neighbors(s.positions, s.box, s.pbc, rcut)
    r = np.sqrt((d ** 2).sum(1))
    for i in range(s.n):
        ri = np.sort(r[indptr[i]:indptr[i + 1]])
        expect = np.concatenate([np.full(c, dist) for c, dist in SHELLS if dist < rcut])
        assert ri.size == expect.size
        np.testing.assert_allclose(ri, expect, rtol=0, atol=1e-12)


def test_shells_primitive_torus():
    _shell_check(synth.graphene_primitive(6, 5), 3.0)
    _shell_check(synth.graphene_primitive(6, 5), 1.8)


def test_shells_rect_cells():
    _shell_check(synth.graphene_rect(4, 5), 3.0)


def _supercell_reference(pos, box, pbc, rcut, reach=3):
    """Independent route: copy the atoms into an explicit (2 reach + 1)^d
    supercell and search without any periodicity."""
    n = pos.shape[0]
    ranges = [range(-reach, reach + 1) if pbc[k] else [0] for k in range(3)]
    imgs, owner = [], []
    for n1 in ranges[0]:
        for n2 in ranges[1]:
            for n3 in ranges[2]:
                imgs.append(pos + n1 * box[0] + n2 * box[1] + n3 * box[2])
                owner.append(np.arange(n))
    imgs = np.concatenate(imgs)
    owner = np.concatenate(owner)
    rows = []
    for i in range(n):
        dist = np.sqrt(((imgs - pos[i]) ** 2).sum(1))
        hit = (dist < rcut) & (owner != i)
        rows.append(np.sort(owner[hit]))
    return rows


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bruteforce_vs_supercell_triclinic(seed):
    rng = np.random.default_rng(seed)
    box = np.array([[9.0, 0.0, 0.0], [3.7, 8.1, 0.0], [1.1, -0.9, 7.5]])
    frac = rng.uniform(-0.2, 1.2, size=(70, 3))
    pos = frac @ box
    pbc = np.array([1, 1, 1])
    indptr, idx, d = nb.neighbors_bruteforce(pos, box, pbc, 3.4)
    ref = _supercell_reference(pos, box, pbc, 3.4)
    for i in range(pos.shape[0]):
        np.testing.assert_array_equal(idx[indptr[i]:indptr[i + 1]], ref[i])
    # displacement is the image vector: r_j + T - r_i with |d| < rcut
    rows = np.repeat(np.arange(pos.shape[0]), np.diff(indptr))
    frac_t = np.linalg.solve(box.T, (d - (pos[idx] - pos[rows])).T).T
    np.testing.assert_allclose(frac_t, np.rint(frac_t), atol=1e-9)


def test_bruteforce_vs_supercell_slab():
    s = synth.graphene_primitive(4, 4, sigma=0.3, seed=5)
    indptr, idx, _ = nb.neighbors_bruteforce(s.positions, s.box, s.pbc, 3.0)
    ref = _supercell_reference(s.positions, s.box, s.pbc, 3.0)
    for i in range(s.n):
        np.testing.assert_array_equal(idx[indptr[i]:indptr[i + 1]], ref[i])


def test_relation_is_symmetric_and_antisymmetric_displacement():
    s = synth.graphene_rect(3, 4, sigma=0.15, seed=3)
    indptr, idx, d = nb.neighbors_bruteforce(s.positions, s.box, s.pbc, 3.0)
    pairs = {}
    for i in range(s.n):
        for k in range(indptr[i], indptr[i + 1]):
            pairs[(i, int(idx[k]))] = d[k]
    for (i, j), dij in pairs.items():
        assert (j, i) in pairs
        np.testing.assert_array_equal(pairs[(j, i)], -dij)


def test_kdtree_equals_bruteforce():
    s = synth.graphene_rect(9, 8, sigma=0.12, seed=11)
    a = nb.neighbors_bruteforce(s.positions, s.box, s.pbc, 3.0)
    b = nb.neighbors_kdtree(s.positions, s.box, s.pbc, 3.0)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_allclose(a[2], b[2], atol=1e-12)


def test_rows_sampler_equals_bruteforce():
    s = synth.graphene_rect(6, 7, sigma=0.1, seed=2)
    indptr, idx, d = nb.neighbors_bruteforce(s.positions, s.box, s.pbc, 3.0)
    rows = [0, 5, 77, s.n - 1]
    for i, (ri, di) in zip(rows, nb.neighbors_of_rows(s.positions, s.box, s.pbc, 3.0, rows, chunk=50)):
        np.testing.assert_array_equal(ri, idx[indptr[i]:indptr[i + 1]])
        np.testing.assert_allclose(di, d[indptr[i]:indptr[i + 1]], atol=1e-12)


def test_small_box_rejected():
    s = synth.graphene_rect(1, 2)
    with pytest.raises(nb.BoxError):
        nb.neighbors_bruteforce(s.positions, s.box, s.pbc, 3.0)
