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
