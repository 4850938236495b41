"""Batched KPM over uneven snapshots (multi-frame averaging, Sec. 2.4).

Snapshot s of a batch must give exactly the moments of a standalone
kpm_moments run with seed + s (FP64: <= 1e-12 absolute; FP32: <= 2e-4),
and those must match the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import bounds as obo
from oracle import hamiltonian as oha
from oracle import kpm as okpm
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


@pytest.fixture(scope="module")
def snaps():
    """Five uneven h-BN/graphene junction snapshots (96 to ~1900 atoms; sizes
    that are not multiples of 32 or 256), with oracle H and bounds."""
    out = []
    p = synth.teacher_hbn_graphene()
    for k, (nx, ny) in enumerate([(4, 6), (10, 11), (14, 34), (6, 5), (20, 9)]):
        s = synth.hbn_graphene_junction(nx, ny, 0.1, 700 + k)
        if k == 3:
            s.positions, s.species = s.positions[:-7].copy(), s.species[:-7].copy()
        ip, idx, d = onb.neighbors(s.positions, s.box, s.pbc, p.rcut)
        t, eps, _ = ote.teacher_elements(s.species, ip, idx, d, p)
        H = oha.csr_hamiltonian(s.n, ip, idx, t, eps)
        _, _, a, b = obo.spectral_bounds(H, 64, 7)
        out.append((s, ip, idx, t, eps, H, a, b))
    return out


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 2e-4)])
@pytest.mark.parametrize("R", [1, 2, 8])
@pytest.mark.parametrize("doubling", [False, True])
def test_batched_equals_per_snapshot_and_oracle(g, snaps, dtype, tol, R, doubling):
    mats = [sell_matrix(ip, idx, t, eps, s.n, dtype) for (s, ip, idx, t, eps, H, a, b) in snaps]
    a = [x[6] for x in snaps]
    b = [x[7] for x in snaps]
    M, seed = 96, 31
    mu = g.kpm_moments_batched(mats, a, b, M, R, seed, doubling=doubling).cpu().numpy()
    for k, (s, ip, idx, t, eps, H, ak, bk) in enumerate(snaps):
        single = g.kpm_moments(mats[k], ak, bk, M, R, seed + k, doubling=doubling).cpu().numpy()
        assert np.max(np.abs(mu[k] - single)) <= tol
        _, ref = okpm.kpm_moments(H, ak, bk, M, R, seed + k)
        assert np.max(np.abs(mu[k] - ref)) <= tol


def test_batched_is_reproducible_and_reports_bounds(g, snaps):
    mats = [sell_matrix(ip, idx, t, eps, s.n, torch.float64) for (s, ip, idx, t, eps, H, a, b) in snaps]
    a = [x[6] for x in snaps]
    b = [x[7] for x in snaps]
    m1 = g.kpm_moments_batched(mats, a, b, 64, 4, 5).cpu().numpy()
    m2 = g.kpm_moments_batched(mats, a, b, 64, 4, 5).cpu().numpy()
    assert np.array_equal(m1, m2)
    bad = list(a)
    bad[2] = 0.3 * bad[2]
    with pytest.raises(g.GputbError) as e:
        g.kpm_moments_batched(mats, bad, b, 256, 1, 5)
    assert e.value.status in (g.TB_ERR_BOUNDS, g.TB_ERR_NOT_FINITE)


def test_phantom_rows_are_ignored_whatever_they_hold(g, snaps):
    """Rows i >= N of a snapshot's last slice may hold anything in the
    caller's value array; the batch must not pick it up."""
    from tests.sell_helpers import csr_to_sell
    mats, a, b = [], [], []
    for (s, ip, idx, t, eps, H, ak, bk) in snaps:
        sp, col, val = csr_to_sell(ip, idx, t, s.n)
        k_last = (s.n - 1) // 32
        for lane in range(s.n % 32 or 32, 32):          # phantom lanes of the last slice
            val[sp[k_last] + lane: sp[k_last + 1]: 32] = np.nan
        mats.append(g.SellMatrix(s.n, torch.tensor(sp, device="cuda"), torch.tensor(col, device="cuda"),
                                 torch.tensor(val, device="cuda"), torch.tensor(eps, device="cuda")))
        a.append(ak)
        b.append(bk)
    mu = g.kpm_moments_batched(mats, a, b, 64, 2, 3).cpu().numpy()
    assert np.all(np.isfinite(mu))
    for k, (s, ip, idx, t, eps, H, ak, bk) in enumerate(snaps):
        _, ref = okpm.kpm_moments(H, ak, bk, 64, 2, 3 + k)
        assert np.max(np.abs(mu[k] - ref)) <= 1e-12


def test_teacher_writes_zero_values_in_phantom_rows(g):
    s = synth.hbn_graphene_junction(5, 7, 0.1, 3)            # 140 atoms: 12 phantom rows
    p = synth.teacher_hbn_graphene()
    pos = torch.tensor(s.positions, device="cuda")
    nb = g.build_neighbors(pos, s.box, s.pbc, 3.0, 1.8)
    H = g.build_hamiltonian_teacher(pos, torch.tensor(s.species, device="cuda"), s.box, s.pbc, nb, p)
    sp = nb.slice_ptr.cpu().numpy()
    val = H.val.cpu().numpy()
    k = (s.n - 1) // 32
    for lane in range(s.n % 32, 32):
        assert np.all(val[sp[k] + lane: sp[k + 1]: 32] == 0.0)


def test_large_batch_spans_many_blocks_per_cta(g):
    """Many uneven snapshots (tens of thousands of rows in total) so that each
    CTA handles runs of blocks crossing snapshot boundaries, in both moment
    modes; every snapshot must equal its standalone run."""
    p = synth.teacher_hbn_graphene()
    mats, a, b = [], [], []
    rng = np.random.default_rng(0)
    for k in range(24):
        nx, ny = int(rng.integers(4, 30)), int(rng.integers(4, 40))   # >= 64 atoms (64 Lanczos steps)
        s = synth.hbn_graphene_junction(nx, ny, 0.1, 900 + k)
        pos = torch.tensor(s.positions, device="cuda")
        nb = g.build_neighbors(pos, s.box, s.pbc, 3.0, 1.8)
        H = g.build_hamiltonian_teacher(pos, torch.tensor(s.species, device="cuda"), s.box, s.pbc, nb, p,
                                        dtype=torch.float64)
        bd = g.spectral_bounds(H, 64, 7)
        mats.append(H)
        a.append(bd.a)
        b.append(bd.b)
    for doubling in (False, True):
        for R in (1, 8):
            mu = g.kpm_moments_batched(mats, a, b, 40, R, 9, doubling=doubling).cpu().numpy()
            for k in range(len(mats)):
                single = g.kpm_moments(mats[k], a[k], b[k], 40, R, 9 + k, doubling=doubling).cpu().numpy()
                assert np.max(np.abs(mu[k] - single)) <= 1e-12, (doubling, R, k)


def test_cached_graph_relaunch_and_recapture(g, snaps):
    """A second identical call launches the cached graph (same moments bit
    for bit); changing one snapshot's rescaling recaptures and matches the
    oracle for the new values; the batched autotuner's choice is correct."""
    mats = [sell_matrix(ip, idx, t, eps, s.n, torch.float32) for (s, ip, idx, t, eps, H, a, b) in snaps]
    a = [x[6] for x in snaps]
    b = [x[7] for x in snaps]
    m1 = g.kpm_moments_batched(mats, a, b, 64, 8, 3, doubling=True)
    m2 = g.kpm_moments_batched(mats, a, b, 64, 8, 3, doubling=True, mu=m1.clone())
    assert torch.equal(m1, m2)
    a2 = list(a)
    a2[1] = 1.25 * a2[1]
    m3 = g.kpm_moments_batched(mats, a2, b, 64, 8, 3, doubling=True).cpu().numpy()
    s, ip, idx, t, eps, H, _, bk = snaps[1]
    _, ref = okpm.kpm_moments(H, a2[1], bk, 64, 8, 3 + 1)
    assert np.max(np.abs(m3[1] - ref)) <= 2e-4
    best, times = g.kpm_moments_batched_autotune(mats, a, b, 8, doubling=True, reps=3)
    assert 0 <= best < g.kpm_shape_count(8, torch.float32) and len(times) == g.kpm_shape_count(8, torch.float32)
    try:
        m4 = g.kpm_moments_batched(mats, a, b, 64, 8, 3, doubling=True).cpu().numpy()
        for k, (s, ip, idx, t, eps, H, ak, bk) in enumerate(snaps):
            _, ref = okpm.kpm_moments(H, ak, bk, 64, 8, 3 + k)
            assert np.max(np.abs(m4[k] - ref)) <= 2e-4
    finally:
        g.kpm_clear_shapes()
