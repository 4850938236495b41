"""Neighbour lists N(i) of Eq. 1 (Sec. 3): every atom j != i that has a
periodic image within r_cut of atom i.  TEST INFRASTRUCTURE ONLY.

The plain definition is written out directly: for each pair and each lattice
translation T = n1 a1 + n2 a2 + n3 a3 (periodic directions only) the
displacement d = (r_j - r_i) + T is tested with |d|^2 < r_cut^2 in FP64.
Because every periodic perpendicular width must be at least 2 r_cut, at most
one image of j can satisfy the test, so the neighbour set and the
displacement d_ij are unique.

Outputs use CSR form: indptr [N+1], indices (sorted ascending within a row),
dvec [nnz, 3] (the displacement r_j + T - r_i of the unique image).
"""
from __future__ import annotations

import itertools

import numpy as np


class BoxError(ValueError):
    """A periodic perpendicular width is below 2 r_cut."""


def perpendicular_widths(box: np.ndarray) -> np.ndarray:
    """Distance between opposite faces of the cell, per lattice direction."""
    a1, a2, a3 = (np.asarray(box[k], np.float64) for k in range(3))
    vol = abs(np.dot(a1, np.cross(a2, a3)))
    return np.array([vol / np.linalg.norm(np.cross(a2, a3)),
                     vol / np.linalg.norm(np.cross(a3, a1)),
                     vol / np.linalg.norm(np.cross(a1, a2))])


def check_box(box, pbc, rcut):
    w = perpendicular_widths(box)
    for k in range(3):
        if pbc[k] and w[k] < 2.0 * rcut:
            raise BoxError(f"periodic width {w[k]:.4f} along a{k+1} < 2*rcut")


def _translations(box, pbc, reach=2):
    ranges = [range(-reach, reach + 1) if pbc[k] else range(0, 1) for k in range(3)]
    return np.array([n1 * box[0] + n2 * box[1] + n3 * box[2]
                     for n1, n2, n3 in itertools.product(*ranges)], np.float64)


def _check_in_reach(pos, box, pbc):
    # fractional coordinates must stay within [-0.5, 1.5) so that
    # translations with |n| <= 2 cover every image that can be within r_cut
    frac = np.linalg.solve(np.asarray(box, np.float64).T, pos.T).T
    for k in range(3):
        if pbc[k] and (frac[:, k].min() < -0.5 or frac[:, k].max() >= 1.5):
            raise ValueError("positions too far outside the cell for the brute-force oracle")


def _sq_norm(d):
    # ((dx*dx) + (dy*dy)) + (dz*dz), each step rounded separately
    return (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]


def neighbors_bruteforce(pos, box, pbc, rcut):
    """O(N^2 * images) brute force of the definition.  Small N only."""
    pos = np.asarray(pos, np.float64)
    box = np.asarray(box, np.float64)
    check_box(box, pbc, rcut)
    _check_in_reach(pos, box, pbc)
    n = pos.shape[0]
    shifts = _translations(box, pbc)
    r2 = rcut * rcut
    indptr = np.zeros(n + 1, np.int64)
    all_idx, all_d = [], []
    for i in range(n):
        d = (pos[None, :, :] - pos[i][None, None, :]) + shifts[:, None, :]  # [T, N, 3]
        hit = _sq_norm(d) < r2
        hit[:, i] = False
        t_idx, j_idx = np.nonzero(hit)
        order = np.argsort(j_idx, kind="stable")
        j_idx, t_idx = j_idx[order], t_idx[order]
        if np.any(np.diff(j_idx) == 0):
            raise BoxError("two images of one atom within r_cut")
        all_idx.append(j_idx)
        all_d.append(d[t_idx, j_idx])
        indptr[i + 1] = indptr[i] + j_idx.size
    indices = np.concatenate(all_idx).astype(np.int64) if n else np.zeros(0, np.int64)
    dvec = np.concatenate(all_d) if n else np.zeros((0, 3))
    return indptr, indices, dvec


def is_orthorhombic(box) -> bool:
    box = np.asarray(box)
    return bool(np.all(box[~np.eye(3, dtype=bool)] == 0.0))


def neighbors_kdtree(pos, box, pbc, rcut):
    """Same definition for orthorhombic boxes, using SciPy's cKDTree as the
    candidate-pair primitive; the strict '<' test and the minimum-image
    displacement are then applied per pair in FP64."""
    from scipy.spatial import cKDTree

    pos = np.asarray(pos, np.float64)
    box = np.asarray(box, np.float64)
    if not is_orthorhombic(box):
        raise ValueError("neighbors_kdtree needs an orthorhombic box")
    check_box(box, pbc, rcut)
    n = pos.shape[0]
    lengths = np.diag(box).copy()
    wrapped = pos.copy()
    boxsize = np.empty(3)
    for k in range(3):
        if pbc[k]:
            wrapped[:, k] = np.mod(wrapped[:, k], lengths[k])
            wrapped[:, k][wrapped[:, k] >= lengths[k]] = 0.0
            boxsize[k] = lengths[k]
        else:
            lo = wrapped[:, k].min()
            wrapped[:, k] -= lo
            boxsize[k] = wrapped[:, k].max() + 4.0 * rcut + 1.0
    tree = cKDTree(wrapped, boxsize=boxsize)
    pairs = tree.query_pairs(rcut * (1.0 + 1e-12) + 1e-12, output_type="ndarray")
    i = np.concatenate([pairs[:, 0], pairs[:, 1]]).astype(np.int64)
    j = np.concatenate([pairs[:, 1], pairs[:, 0]]).astype(np.int64)
    d = pos[j] - pos[i]
    for k in range(3):
        if pbc[k]:
            d[:, k] = d[:, k] - lengths[k] * np.rint(d[:, k] / lengths[k])
    keep = _sq_norm(d) < rcut * rcut
    i, j, d = i[keep], j[keep], d[keep]
    order = np.lexsort((j, i))
    i, j, d = i[order], j[order], d[order]
    indptr = np.zeros(n + 1, np.int64)
    np.add.at(indptr, i + 1, 1)
    indptr = np.cumsum(indptr)
    return indptr, j, d


def neighbors(pos, box, pbc, rcut):
    """Dispatch: brute force for small N, k-d tree for large orthorhombic cells."""
    n = np.asarray(pos).shape[0]
    if n <= 4000 or not is_orthorhombic(box):
        return neighbors_bruteforce(pos, box, pbc, rcut)
    return neighbors_kdtree(pos, box, pbc, rcut)


def neighbors_of_rows(pos, box, pbc, rcut, rows, chunk=1 << 22):
    """Brute force of the definition for a few sampled rows of a large system.

    Orthorhombic boxes use the per-component nearest image (exact for them);
    other boxes enumerate the lattice translations.  Returns a list of
    (indices sorted ascending, dvec) per requested row.
    """
    pos = np.asarray(pos, np.float64)
    box = np.asarray(box, np.float64)
    check_box(box, pbc, rcut)
    ortho = is_orthorhombic(box)
    lengths = np.diag(box)
    shifts = np.zeros((1, 3)) if ortho else _translations(box, pbc)
    r2 = rcut * rcut
    out = []
    n = pos.shape[0]
    for i in rows:
        idx_list, d_list = [], []
        for s in range(0, n, chunk):
            block = pos[s:s + chunk] - pos[i]
            if ortho:
                for k in range(3):
                    if pbc[k]:
                        block[:, k] -= lengths[k] * np.rint(block[:, k] / lengths[k])
            for t in shifts:
                d = block + t
                # cheap exact prefilter: every component within r_cut
                m = (np.abs(d[:, 0]) < rcut) & (np.abs(d[:, 1]) < rcut) & (np.abs(d[:, 2]) < rcut)
                if not m.any():
                    continue
                cand = np.nonzero(m)[0]
                dd = d[cand]
                ok = _sq_norm(dd) < r2
                jj = cand[ok] + s
                keep = jj != i
                idx_list.append(jj[keep])
                d_list.append(dd[ok][keep])
        idx = np.concatenate(idx_list) if idx_list else np.zeros(0, np.int64)
        dv = np.concatenate(d_list) if d_list else np.zeros((0, 3))
        order = np.argsort(idx, kind="stable")
        idx, dv = idx[order], dv[order]
        if np.any(np.diff(idx) == 0):
            raise BoxError("two images of one atom within r_cut")
        out.append((idx.astype(np.int64), dv))
    return out


def row_of(indptr, i):
    return slice(int(indptr[i]), int(indptr[i + 1]))
