"""Oracle parity at sizes where every code path of the Chebyshev-step
kernels runs (Sec. 2.4: the KPM recursion, multi-frame averaging, the VAC
conductivity).

At the small sizes of test_gpu_kpm.py each CTA processes one tile at most.
Here the structures are large enough that, for every launch shape,
* a CTA of the bulk-copy ring processes more tiles than the ring has
  stages, so stages are reused and the mbarrier phase parity flips;
* a CTA of the direct-load kernel iterates its grid-stride loop;
* in the batched (segmented) form each CTA visits a contiguous span of
  blocks that crosses snapshot boundaries, so its runs end inside the span
  (one reduction per snapshot met) and at its end.
The launch geometry is asserted from the library's own grid query, and the
moments are compared element by element with the FP64 oracle on the same
seeded inputs.  Tolerances: FP64 moments <= 1e-12 absolute, FP32 <= 2e-4
absolute; VAC moments as test_gpu_lsqt.py (FP64 1e-10, FP32 1e-4 of the
largest moment).
"""
import numpy as np
import pytest
import torch

from oracle import bounds as obo
from oracle import kpm as okpm
from oracle import lsqt as olsqt
from oracle import neighbors as onb
from paper_2509_06525_gb300 import synth
from tests import oracle_pool
from tests.sell_helpers import sell_matrix

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 2e-4}
SHEET = ("junction", 300, 250, 0.1, 5150)      # 300,000 atoms, B/N onsite +2.3/-2.1 eV
M_SHEET = 64
SEED = 4242


@pytest.fixture(scope="module")
def g():
    from paper_2509_06525_gb300 import build, gputb
    build.build()
    assert torch.cuda.is_available()
    return gputb


@pytest.fixture(scope="module")
def sheet():
    s, p, H, ip, idx, t, eps = oracle_pool.oracle_hamiltonian(SHEET)
    _, _, a, b = obo.spectral_bounds(H, 64, synth.LANCZOS_SEED)
    return dict(s=s, p=p, H=H, ip=ip, idx=idx, t=t, eps=eps, a=a, b=b, mats={}, mu={})


def _mat(sheet, dtype):
    if dtype not in sheet["mats"]:
        sheet["mats"][dtype] = sell_matrix(sheet["ip"], sheet["idx"], sheet["t"], sheet["eps"], sheet["s"].n, dtype)
    return sheet["mats"][dtype]


def _shapes(g, R, dtype):
    return list(range(g.kpm_shape_count(R, dtype)))


@pytest.fixture(autouse=True)
def _clear_shapes(g):
    yield
    g.kpm_clear_shapes()


def _assert_multitile(g, n, R, dtype, doubling, shape):
    """Each CTA loops: more tiles than ring stages (pipelined shapes) or at
    least two grid-stride iterations (direct shapes)."""
    info = g.kpm_shape_info(R, dtype, shape)
    grid = g.kpm_shape_grid(n, R, dtype, doubling, shape)
    tiles = -(-n // info["rows_per_tile"])
    per_cta = tiles // grid
    need = info["stages"] + 1 if info["pipelined"] else 2
    assert per_cta >= need, (info, grid, tiles)


WIDE = ("junction", 400, 500, 0.1, 5151)        # 800,000 atoms


@pytest.fixture(scope="module")
def wide():
    s, p, H, ip, idx, t, eps = oracle_pool.oracle_hamiltonian(WIDE)
    _, _, a, b = obo.spectral_bounds(H, 64, synth.LANCZOS_SEED)
    _, mu = okpm.kpm_moments(H, a, b, M_SHEET, 1, SEED)
    return dict(s=s, ip=ip, idx=idx, t=t, eps=eps, a=a, b=b, mu={1: mu}, mats={})


@pytest.mark.parametrize("doubling", [False, True], ids=["direct", "doubling"])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
@pytest.mark.parametrize("R", [8, 16])
def test_multitile_ring_and_grid_stride_match_oracle(g, wide, R, dtype, doubling):
    """R = 8 and 16 vectors on the 800k-atom junction (oracle moments from a
    pool of processes over blocks of vectors)."""
    n = wide["s"].n
    if dtype not in wide["mats"]:
        wide["mats"][dtype] = sell_matrix(wide["ip"], wide["idx"], wide["t"], wide["eps"], n, dtype)
    Hd = wide["mats"][dtype]
    if R not in wide["mu"]:
        wide["mu"][R] = oracle_pool.kpm_moments_parallel(WIDE, wide["a"], wide["b"], M_SHEET, R, SEED)
    ref = wide["mu"][R]
    for shape in _shapes(g, R, dtype):
        _assert_multitile(g, n, R, dtype, doubling, shape)
        g.kpm_force_shape(R, dtype, shape)
        mu = g.kpm_moments(Hd, wide["a"], wide["b"], M_SHEET, R, SEED, doubling=doubling).cpu().numpy()
        err = np.max(np.abs(mu - ref))
        assert err <= TOL[dtype], (shape, err)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_one_vector_grid_stride_loop_matches_oracle(g, wide, dtype):
    """R = 1 (the 1e8-atom headline's block width): one thread per row on an
    800k-atom junction, so the direct kernel's grid-stride loop runs at least
    twice per CTA."""
    n = wide["s"].n
    Hd = sell_matrix(wide["ip"], wide["idx"], wide["t"], wide["eps"], n, dtype)
    for shape in _shapes(g, 1, dtype):
        for doubling in (False, True):
            _assert_multitile(g, n, 1, dtype, doubling, shape)
            g.kpm_force_shape(1, dtype, shape)
            mu = g.kpm_moments(Hd, wide["a"], wide["b"], M_SHEET, 1, SEED, doubling=doubling).cpu().numpy()
            assert np.max(np.abs(mu - wide["mu"][1])) <= TOL[dtype], (shape, doubling)


# eleven uneven junction snapshots, 4,800 .. 96,000 atoms (none a multiple of
# the 256-row tile), 425,040 atoms in all
BATCH = [(30, 42), (50, 60), (80, 70), (100, 95), (120, 110), (150, 120), (160, 150), (90, 80), (40, 30),
         (60, 55), (200, 100)]


@pytest.fixture(scope="module")
def batch():
    out = []
    for k, (nx, ny) in enumerate(BATCH):
        s, p, H, ip, idx, t, eps = oracle_pool.oracle_hamiltonian(("junction", nx, ny, 0.1, 6100 + k))
        _, _, a, b = obo.spectral_bounds(H, 64, synth.LANCZOS_SEED)
        out.append(dict(s=s, H=H, ip=ip, idx=idx, t=t, eps=eps, a=a, b=b))
    return out


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64], ids=["f32", "f64"])
def test_batched_runs_cross_snapshots_and_match_oracle(g, batch, dtype):
    R, M, seed = 8, 48, 91
    mats = [sell_matrix(x["ip"], x["idx"], x["t"], x["eps"], x["s"].n, dtype) for x in batch]
    a = [x["a"] for x in batch]
    b = [x["b"] for x in batch]
    refs = [okpm.kpm_moments(x["H"], x["a"], x["b"], M, R, seed + k)[1] for k, x in enumerate(batch)]
    n_pad = sum(-(-x["s"].n // 256) * 256 for x in batch)
    assert n_pad >= 400_000
    smallest = min(x["s"].n for x in batch)
    largest = max(x["s"].n for x in batch)
    for shape in _shapes(g, R, dtype):
        for doubling in (False, True):
            info = g.kpm_shape_info(R, dtype, shape)
            grid = g.kpm_shape_grid(n_pad, R, dtype, doubling, shape)
            blocks = n_pad // info["rows_per_tile"]
            # every CTA's span holds several blocks, and the spans are
            # shorter than the smallest snapshot, so that spans start and end
            # inside snapshots and some cross a snapshot boundary
            span = -(-blocks // grid)
            assert span >= 3
            assert span < smallest // info["rows_per_tile"]
            assert largest // info["rows_per_tile"] >= 2 * span
            g.kpm_force_shape(R, dtype, shape)
            mu = g.kpm_moments_batched(mats, a, b, M, R, seed, doubling=doubling).cpu().numpy()
            for k, ref in enumerate(refs):
                assert np.max(np.abs(mu[k] - ref)) <= TOL[dtype], (shape, doubling, k)


@pytest.mark.parametrize("dtype,R,tol", [(torch.float64, 4, 1e-10), (torch.float64, 8, 1e-10),
                                         (torch.float32, 8, 1e-4), (torch.float32, 16, 1e-4)])
def test_vac_moments_multitile_match_oracle(g, sheet, dtype, R, tol):
    """VAC moments (Eq. 3 (sigma)) on the 300k-atom junction: the moment
    recursion and the Chebyshev-Bessel propagation at 0.1 fs with every
    CTA looping over several tiles."""
    s, p = sheet["s"], sheet["p"]
    M, steps, dt, seed = 32, 2, 0.1, 17
    Hd = _mat(sheet, dtype)
    pos = torch.tensor(s.positions, device="cuda")
    vv = g.velocity_values(pos, s.box, s.pbc, p.rcut, Hd)
    ip, idx, d = onb.neighbors(s.positions, s.box, s.pbc, p.rcut)
    V = olsqt.velocity_matrix(s.n, ip, idx, sheet["t"], d)
    ref = olsqt.vac_moments(sheet["H"], V, sheet["a"], sheet["b"], M, R, seed, steps, dt)
    scale = np.max(np.abs(ref))
    for shape in _shapes(g, R, dtype):
        g.kpm_force_shape(R, dtype, shape)
        mu = g.lsqt_vac(Hd, vv, sheet["a"], sheet["b"], M, R, seed, steps, dt).cpu().numpy()
        assert np.max(np.abs(mu - ref)) <= tol * scale, shape


CFG2 = ("rect", 500, 500, 0.1, 1002)   # the 1,000,000-atom 300 K graphene sheet


def test_million_atom_fp32_error_growth_against_oracle(g):
    """1M-atom thermal graphene, R = 16 vectors in one blocked SpMM, M = 256:
    FP32 vectors (the bench's doubling mode and the direct mode) and FP64
    vectors against the FP64 oracle, element by element.  Also checks that
    the FP32 error does not grow faster than linearly in n (rounding of
    order n 2^-24 per element, averaged over N R entries)."""
    M, R = 256, 16
    s, p, H, ip, idx, t, eps = oracle_pool.oracle_hamiltonian(CFG2)
    _, _, a, b = obo.spectral_bounds(H, 64, synth.LANCZOS_SEED)
    ref = oracle_pool.kpm_moments_parallel(CFG2, a, b, M, R, synth.KPM_SEED)
    rows = []
    for dtype, doubling in ((torch.float32, True), (torch.float32, False), (torch.float64, True)):
        Hd = sell_matrix(ip, idx, t, eps, s.n, dtype)
        mu = g.kpm_moments(Hd, a, b, M, R, synth.KPM_SEED, doubling=doubling).cpu().numpy()
        dev = np.max(np.abs(mu - ref), axis=0)          # max over vectors, per moment n
        rows.append((dtype, doubling, dev))
        assert dev.max() <= TOL[dtype], (dtype, doubling, dev.max())
        del Hd
    dev32 = rows[0][2]
    bins = [float(dev32[k:k + 32].max()) for k in range(0, M, 32)]
    print("FP32 doubling max|dmu_n| per 32 moments:", ", ".join(f"{v:.2e}" for v in bins))
    # no faster than linear growth: the last bin within (M / 32) x the first two bins' level + slack
    assert bins[-1] <= (M / 32) * max(bins[0], bins[1], 1e-7) * 4
