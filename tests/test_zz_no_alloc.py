"""The allocation-free KPM entry point (kpm_moments_noalloc).

It exists for callers that cannot allocate device memory where they need
the moments (a host framework that owns the memory pool, latency-critical
loops, plug-ins handed only their buffers): its scratch is a static 32 MiB
device array inside the library.  The test calls it through the C ABI
twice in a row -- the second call reuses the scratch left by the first --
and compares both results with kpm_moments on a caller workspace, within
the moment tolerances used everywhere else (FP64 1e-12, FP32 2e-4).  This
file is collected last so a failure here leaves every other test already
run."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import bounds as obo
from oracle import hamiltonian as oha
from oracle import neighbors as onb
from oracle import teacher as ote
from paper_2509_06525_gb300 import synth
from tests.sell_helpers import sell_matrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_2509_06525_gb300 import build, gputb
    build.build()
    return gputb


def _call_noalloc(g, H, a, b, M, R, seed):
    mu = torch.full((R, M), float("nan"), dtype=torch.float64, device="cuda")
    st = g.lib().kpm_moments_noalloc(H.n, g._ptr(H.slice_ptr), g._ptr(H.col), g._ptr(H.val), g._ptr(H.diag),
                                     H.precision, float(a), float(b), int(M), int(R), int(seed), g._ptr(mu),
                                     g._stream())
    return st, mu


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-4)])
def test_noalloc_matches_workspace_entry_point(g, dtype, tol):
    s = synth.hbn_graphene_junction(10, 12, sigma=0.1, seed=21)        # 480 atoms, onsite terms
    p = synth.teacher_hbn_graphene()
    indptr, idx, d = onb.neighbors(s.positions, s.box, s.pbc, p.rcut)
    t, eps, _ = ote.teacher_elements(s.species, indptr, idx, d, p)
    _, _, a, b = obo.spectral_bounds(oha.csr_hamiltonian(s.n, indptr, idx, t, eps), 64, 7)
    H = sell_matrix(indptr, idx, t, eps, s.n, dtype)
    M, R = 256, 8
    ref = g.kpm_moments(H, a, b, M, R, synth.KPM_SEED).cpu().numpy()
    for call in range(2):
        st, mu = _call_noalloc(g, H, a, b, M, R, synth.KPM_SEED)
        assert st == g.TB_OK, g.lib().tb_last_error().decode()
        assert np.max(np.abs(mu.cpu().numpy() - ref)) <= tol, f"call {call}"
    # a different seed on the same scratch, then the first seed again
    st, mu_other = _call_noalloc(g, H, a, b, M, R, 99)
    assert st == g.TB_OK
    ref_other = g.kpm_moments(H, a, b, M, R, 99).cpu().numpy()
    assert np.max(np.abs(mu_other.cpu().numpy() - ref_other)) <= tol


def test_noalloc_rejects_sizes_beyond_its_scratch(g):
    # 4M rows with R = 32: the vector blocks alone exceed 32 MiB; the check
    # happens on the host before any device work
    n = 4 << 20
    sp = torch.zeros((n + 31) // 32 + 1, dtype=torch.int64, device="cuda")
    mu = torch.empty((32, 16), dtype=torch.float64, device="cuda")
    st = g.lib().kpm_moments_noalloc(n, g._ptr(sp), None, None, None, g.F32, 3.0, 0.0, 16, 32, 1, g._ptr(mu),
                                     g._stream())
    assert st == g.TB_ERR_WORKSPACE
    assert "32 MiB" in g.lib().tb_last_error().decode()
