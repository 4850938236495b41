"""The double-float Lanczos of tb_spectral_bounds (FP32 Hamiltonians) runs
its SpMV on the band plan (tiles of 256 rows whose operands, the bands of
the Lanczos vector included, are bulk-copied into shared memory) wherever
the values and the diagonal are 16-byte aligned, and on global gathers
otherwise.  The two kernels perform the same operations in the same order,
so their bounds agree bit for bit; both agree with the FP64 oracle on the
same FP32-rounded values (rel 1e-9, as test_gpu_hamiltonian.py).  Sizes:
a 600k-atom sheet (every CTA of the banded SpMV takes several tiles, so the
two-stage ring wraps) and a random pattern mixed with a chain (tiles whose
columns need more than six bands take the gather path inside the banded
kernel)."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import bounds as obo
from oracle import hamiltonian as oha
from paper_2509_06525_gb300 import synth
from tests import oracle_pool
from tests.sell_helpers import sell_matrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_2509_06525_gb300 import build, gputb
    build.build()
    assert torch.cuda.is_available()
    return gputb


def _misaligned(g, H):
    """The same matrix with its values 4 bytes off a 16-byte boundary (the
    gather kernel)."""
    store = torch.empty(H.val.numel() + 1, dtype=H.val.dtype, device=H.val.device)
    val = store[1:]
    val.copy_(H.val)
    assert val.data_ptr() % 16 != 0
    return g.SellMatrix(H.n, H.slice_ptr, H.col, val, H.diag)


def _check(g, n, indptr, idx, t, eps):
    t32 = np.asarray(t, np.float32).astype(np.float64)
    e32 = np.asarray(eps, np.float32).astype(np.float64)
    Hd = sell_matrix(indptr, idx, t32, e32, n, torch.float32)
    assert Hd.val.data_ptr() % 16 == 0 and (Hd.diag is None or Hd.diag.data_ptr() % 16 == 0)
    banded = g.spectral_bounds(Hd, 64, synth.LANCZOS_SEED)
    gather = g.spectral_bounds(_misaligned(g, Hd), 64, synth.LANCZOS_SEED)
    assert [banded.emin, banded.emax, banded.a, banded.b] == [gather.emin, gather.emax, gather.a, gather.b]
    Hc = oha.csr_hamiltonian(n, indptr, idx, t32, e32)
    emin, emax, a, b = obo.spectral_bounds(Hc, 64, synth.LANCZOS_SEED)
    np.testing.assert_allclose([banded.emin, banded.emax, banded.a, banded.b], [emin, emax, a, b], rtol=1e-9,
                               atol=1e-12)


def test_banded_lanczos_multitile_sheet(g):
    s, p, H, ip, idx, t, eps = oracle_pool.oracle_hamiltonian(("junction", 300, 500, 0.1, 5152))
    tiles = -(-s.n // 256)
    assert tiles >= 3 * 3 * 152          # several tiles per CTA at up to 3 CTAs per SM
    _check(g, s.n, ip, idx, t, eps)


def test_banded_lanczos_scattered_tiles_gather(g):
    rng = np.random.default_rng(23)
    n = 6000
    A = sp.random(n, n, density=5 / n, random_state=rng, format="csr")
    A = (A + A.T).tocsr()
    A.setdiag(0)
    A.eliminate_zeros()
    A = A.tolil()
    for i in range(4000, n):
        A.rows[i], A.data[i] = [], []
    A = A.tocsr()
    chain = sp.diags([np.full(1999, -1.0), np.full(1999, -1.0)], [-1, 1], shape=(2000, 2000), format="csr")
    A = sp.bmat([[A[:4000, :4000], None], [None, chain]], format="csr")
    A.sort_indices()
    onsite = rng.uniform(-0.3, 0.3, n)
    _check(g, n, A.indptr, A.indices, A.data, onsite)
