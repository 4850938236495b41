"""Pin the Bloch-theorem helper used by the full-size GPU test: on a small
torus its eigenvalues must equal the dense diagonalisation of the oracle's
teacher Hamiltonian of the same pristine sheet."""
import math

import numpy as np

from oracle import hamiltonian as oha
from oracle import neighbors as onb
from oracle import teacher as ote
from paper_2509_06525_gb300 import synth
from tests import analytic


def test_rect_bloch_levels_equal_dense_teacher_spectrum():
    nx, ny = 6, 8
    s = synth.graphene_rect(nx, ny)
    p = synth.teacher_graphene()
    ip, idx, d = onb.neighbors(s.positions, s.box, s.pbc, p.rcut)
    t, eps, ncount = ote.teacher_elements(s.species, ip, idx, d, p)
    assert np.all(ncount == 3)
    ev = np.linalg.eigvalsh(oha.csr_hamiltonian(s.n, ip, idx, t, eps).toarray())
    a = p.a_cc
    shells = {a: float(ote.hopping(a, 0, 0, 3, 3, p)),
              math.sqrt(3) * a: float(ote.hopping(math.sqrt(3) * a, 0, 0, 3, 3, p)),
              2 * a: float(ote.hopping(2 * a, 0, 0, 3, 3, p))}
    levels = np.sort(analytic.rect_cell_bloch_levels(nx, ny, shells))
    np.testing.assert_allclose(levels, ev, atol=1e-11)


def test_sell_packing_matches_plain_definition():
    """The test-side SELL-32 packing (vectorised) places element s of row i at
    slice_ptr[i // 32] + s * 32 + i % 32, pads with col = i / value 0, and
    leaves phantom rows of the last slice at col = 0 / value 0: checked
    against a loop written from that definition on a ragged random matrix."""
    import numpy as np
    import scipy.sparse as sp
    from tests.sell_helpers import csr_to_sell
    rng = np.random.default_rng(5)
    n = 203
    A = sp.random(n, n, density=0.04, random_state=rng, format="csr")
    A.sort_indices()
    slice_ptr, col, val = csr_to_sell(A.indptr, A.indices, A.data, n)
    n_sl = (n + 31) // 32
    assert slice_ptr.shape == (n_sl + 1,)
    for k in range(n_sl):
        rows = range(32 * k, min(32 * k + 32, n))
        w = max(A.indptr[i + 1] - A.indptr[i] for i in rows)
        assert slice_ptr[k + 1] - slice_ptr[k] == 32 * w
        for lane in range(32):
            i = 32 * k + lane
            for s in range(w):
                e = slice_ptr[k] + s * 32 + lane
                if i >= n:
                    assert col[e] == 0 and val[e] == 0.0
                elif s < A.indptr[i + 1] - A.indptr[i]:
                    assert col[e] == A.indices[A.indptr[i] + s]
                    assert val[e] == A.data[A.indptr[i] + s]
                else:
                    assert col[e] == i and val[e] == 0.0
