"""GPU parity of kpm_moments / kpm_dos against the FP64 oracle.

Tolerances: FP64 moments <= 1e-12 absolute, FP32 moments <= 2e-4 absolute,
Jackson DOS <= 1e-3 relative L1 (sum|rho_gpu - rho_oracle| / sum|rho_oracle|).
The Hamiltonians here come from the oracle (packed into SELL-32 by the test)
so that this file isolates the KPM kernels."""
import numpy as np
import pytest
import torch

from oracle import bounds as obo
from oracle import dos as ods
from oracle import hamiltonian as oha
from oracle import kpm as okpm
from oracle import neighbors as onb
from oracle import teacher as ote
from paper_2509_06525_gb300 import synth
from tests.sell_helpers import sell_matrix

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-12
TOL_F32 = 2e-4
TOL_DOS = 1e-3


def _teacher_csr(s, params):
    indptr, idx, d = onb.neighbors(s.positions, s.box, s.pbc, params.rcut)
    t, eps, _ = ote.teacher_elements(s.species, indptr, idx, d, params)
    return indptr, idx, t, eps


@pytest.fixture(scope="module")
def gputb():
    from paper_2509_06525_gb300 import build, gputb as g
    build.build()
    assert torch.cuda.is_available()
    return g


def _shape_count(R, dtype):
    """Step shapes compiled for (R, precision), from the library's host-side
    shape table (no GPU needed); 5, the longest table, when the library
    cannot be loaded at collection time (then absent indices skip)."""
    try:
        from paper_2509_06525_gb300 import gputb as g
        return g.kpm_shape_count(R, dtype)
    except Exception:
        return 5


def _dname(dtype):
    return "f64" if dtype == torch.float64 else "f32"


def shape_cases(Rs, dtypes):
    """(R, dtype, shape) for every compiled launch shape of the Chebyshev
    step (direct loads, bulk-copy rings, banded steps; several complex
    numbers per thread, stage counts and register budgets)."""
    return [pytest.param(R, dt, k, id=f"R{R}-{_dname(dt)}-shape{k}")
            for R in Rs for dt in dtypes for k in range(_shape_count(R, dt))]


@pytest.fixture(autouse=True)
def _clear_shapes():
    yield
    from paper_2509_06525_gb300 import gputb as g
    if torch.cuda.is_available():
        g.kpm_clear_shapes()


def use_shape(g, shape, R, dtype):
    count = g.kpm_shape_count(R, dtype)
    if shape >= count:
        pytest.skip(f"R={R} {dtype} has {count} step shapes")
    g.kpm_force_shape(R, dtype, shape)


@pytest.fixture(params=[False, True], ids=["plain", "doubling"])
def doubling(request):
    """Moment doubling (mu_2k, mu_2k+1 from <v_k|v_k>, <v_k|v_k+1>) must give
    the oracle's directly defined moments within the same tolerances."""
    return request.param


@pytest.fixture(scope="module")
def cfg800():
    w = synth.WORKLOADS["graphene-800-fp64"]
    s = synth.graphene_primitive(w["n1"], w["n2"], w["sigma"], w["seed"])
    indptr, idx, t, eps = _teacher_csr(s, synth.teacher_graphene())
    H = oha.csr_hamiltonian(s.n, indptr, idx, t, eps)
    emin, emax, a, b = obo.spectral_bounds(H, 64, synth.LANCZOS_SEED)
    return s, indptr, idx, t, eps, H, a, b, w


@pytest.mark.parametrize("shape", range(_shape_count(8, torch.float64)), ids=lambda k: f"shape{k}")
def test_fp64_moments_match_oracle(gputb, cfg800, shape, doubling):
    s, indptr, idx, t, eps, H, a, b, w = cfg800
    M, R = w["M"], w["R"]
    use_shape(gputb, shape, R, torch.float64)
    Hd = sell_matrix(indptr, idx, t, eps, s.n, torch.float64)
    mu = gputb.kpm_moments(Hd, a, b, M, R, synth.KPM_SEED, doubling=doubling).cpu().numpy()
    _, mu_ref = okpm.kpm_moments(H, a, b, M, R, synth.KPM_SEED)
    assert np.max(np.abs(mu - mu_ref)) <= TOL_F64
    # bitwise reproducible
    mu2 = gputb.kpm_moments(Hd, a, b, M, R, synth.KPM_SEED, doubling=doubling).cpu().numpy()
    assert np.array_equal(mu, mu2)


@pytest.mark.parametrize("M", [2, 3, 4, 511])
def test_doubling_odd_and_tiny_moment_counts(gputb, cfg800, M):
    s, indptr, idx, t, eps, H, a, b, w = cfg800
    Hd = sell_matrix(indptr, idx, t, eps, s.n, torch.float64)
    mu = gputb.kpm_moments(Hd, a, b, M, 2, 11, doubling=True).cpu().numpy()
    _, mu_ref = okpm.kpm_moments(H, a, b, M, 2, 11)
    assert mu.shape == (2, M)
    assert np.max(np.abs(mu - mu_ref)) <= TOL_F64


@pytest.mark.parametrize("shape", range(_shape_count(8, torch.float32)), ids=lambda k: f"shape{k}")
def test_fp32_moments_match_oracle(gputb, cfg800, shape, doubling):
    s, indptr, idx, t, eps, H, a, b, w = cfg800
    M, R = w["M"], w["R"]
    use_shape(gputb, shape, R, torch.float32)
    Hd = sell_matrix(indptr, idx, t, eps, s.n, torch.float32)
    mu = gputb.kpm_moments(Hd, a, b, M, R, synth.KPM_SEED, doubling=doubling).cpu().numpy()
    _, mu_ref = okpm.kpm_moments(H, a, b, M, R, synth.KPM_SEED)
    assert np.max(np.abs(mu - mu_ref)) <= TOL_F32


def test_dos_matches_oracle(gputb, cfg800):
    s, indptr, idx, t, eps, H, a, b, w = cfg800
    M, R = w["M"], w["R"]
    Hd = sell_matrix(indptr, idx, t, eps, s.n, torch.float64)
    mu = gputb.kpm_moments(Hd, a, b, M, R, synth.KPM_SEED)
    emin, emax = b - a, b + a
    E = np.linspace(emin, emax, w["K"])
    rho = gputb.kpm_dos(mu, a, b, torch.tensor(E, device="cuda")).cpu().numpy()
    mu_ref, _ = okpm.kpm_moments(H, a, b, M, R, synth.KPM_SEED)
    rho_ref = ods.density_of_states(mu_ref, a, b, E)
    assert np.sum(np.abs(rho - rho_ref)) / np.sum(np.abs(rho_ref)) <= TOL_DOS
    # same moments into both DOS routines: agreement to rounding
    rho_same = ods.density_of_states(mu.mean(0).cpu().numpy(), a, b, E)
    np.testing.assert_allclose(rho, rho_same, rtol=1e-10, atol=1e-12)
    for kernel, kind in (("lorentz", ods.LORENTZ), ("none", ods.NONE)):
        r = gputb.kpm_dos(mu, a, b, torch.tensor(E, device="cuda"), kernel=kernel, lam=4.0).cpu().numpy()
        np.testing.assert_allclose(r, ods.density_of_states(mu.mean(0).cpu().numpy(), a, b, E, kind, 4.0),
                                   rtol=1e-9, atol=1e-11)




@pytest.mark.parametrize("R,dtype,shape", shape_cases([1, 2, 4, 8, 16, 32], [torch.float64, torch.float32]))
def test_all_block_widths_ragged_rows(gputb, R, dtype, shape, doubling):
    """Ragged N (not a multiple of 32), an h-BN junction with onsite terms
    (diag present), every supported R, every Chebyshev-step shape."""
    use_shape(gputb, shape, R, dtype)
    s = synth.hbn_graphene_junction(6, 7, sigma=0.1, seed=9)   # 168 atoms
    s.positions = s.positions[:-5].copy()                          # ragged, still periodic-valid
    s.species = s.species[:-5].copy()
    p = synth.teacher_hbn_graphene()
    indptr, idx, t, eps = _teacher_csr(s, p)
    H = oha.csr_hamiltonian(s.n, indptr, idx, t, eps)
    _, _, a, b = obo.spectral_bounds(H, 64, 7)
    M = 96
    Hd = sell_matrix(indptr, idx, t, eps, s.n, dtype)
    mu = gputb.kpm_moments(Hd, a, b, M, R, 1234, doubling=doubling).cpu().numpy()
    _, mu_ref = okpm.kpm_moments(H, a, b, M, R, 1234)
    tol = TOL_F64 if dtype == torch.float64 else TOL_F32
    assert np.max(np.abs(mu - mu_ref)) <= tol


@pytest.mark.parametrize("n", [1, 2, 31, 33, 300])
@pytest.mark.parametrize("R,dtype,shape", shape_cases([2, 8], [torch.float64]))
def test_tiny_systems(gputb, n, R, dtype, shape):
    use_shape(gputb, shape, R, torch.float64)
    rng = np.random.default_rng(n)
    dense = np.zeros((n, n))
    if n > 1:
        for i in range(n):
            j = (i + 1) % n
            if j != i:
                dense[i, j] = dense[j, i] = rng.uniform(-1, 1)
    onsite = rng.uniform(-0.5, 0.5, n)
    import scipy.sparse as sp
    off = sp.csr_matrix(dense)
    H = oha.csr_hamiltonian(n, off.indptr, off.indices, off.data, onsite)
    a, b = 3.0, 0.1
    Hd = sell_matrix(off.indptr, off.indices, off.data, onsite, n, torch.float64)
    mu = gputb.kpm_moments(Hd, a, b, 40, R, 5).cpu().numpy()
    _, mu_ref = okpm.kpm_moments(H, a, b, 40, R, 5)
    assert np.max(np.abs(mu - mu_ref)) <= TOL_F64


def test_bounds_violation_reported(gputb, cfg800):
    s, indptr, idx, t, eps, H, a, b, w = cfg800
    Hd = sell_matrix(indptr, idx, t, eps, s.n, torch.float64)
    with pytest.raises(gputb.GputbError) as ei:
        gputb.kpm_moments(Hd, 0.3 * a, b, 256, 1, 1)
    assert ei.value.status in (gputb.TB_ERR_BOUNDS, gputb.TB_ERR_NOT_FINITE)


@pytest.mark.parametrize("R,dtype,shape", shape_cases([8], [torch.float64, torch.float32]))
def test_wide_rows_fall_back_inside_the_pipeline(gputb, R, dtype, shape):
    """Rows wider than the pipeline's 16-slot tile budget (dense random
    pattern, 40 neighbours per row) take the direct-load path per tile."""
    import scipy.sparse as sp
    use_shape(gputb, shape, R, dtype)
    rng = np.random.default_rng(3)
    n = 700
    A = sp.random(n, n, density=40 / n, random_state=rng, format="csr")
    A = A + A.T
    A.setdiag(0)
    A.eliminate_zeros()
    A = A.tocsr()
    A.sort_indices()
    onsite = rng.uniform(-0.3, 0.3, n)
    H = oha.csr_hamiltonian(n, A.indptr, A.indices, A.data, onsite)
    _, _, a, b = obo.spectral_bounds(H, 64, 7)
    Hd = sell_matrix(A.indptr, A.indices, A.data, onsite, n, dtype)
    mu = gputb.kpm_moments(Hd, a, b, 64, R, 77).cpu().numpy()
    _, mu_ref = okpm.kpm_moments(H, a, b, 64, R, 77)
    assert np.max(np.abs(mu - mu_ref)) <= (TOL_F64 if dtype == torch.float64 else TOL_F32)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 2e-6)])
def test_first_vector_blocks_compose_the_ensemble(gputb, cfg800, dtype, tol):
    """Two calls over vectors 0-3 and 4-7 give the moments of one call over
    0-7 (up to the grouping of the partial sums), and the second block
    matches the oracle's vectors 4-7: how ranks split one ensemble."""
    s, indptr, idx, t, eps, H, a, b, w = cfg800
    Hd = sell_matrix(indptr, idx, t, eps, s.n, dtype)
    full = gputb.kpm_moments(Hd, a, b, 128, 8, 5, doubling=True).cpu().numpy()
    lo = gputb.kpm_moments(Hd, a, b, 128, 4, 5, doubling=True, first_vector=0).cpu().numpy()
    hi = gputb.kpm_moments(Hd, a, b, 128, 4, 5, doubling=True, first_vector=4).cpu().numpy()
    np.testing.assert_allclose(np.concatenate([lo, hi]), full, rtol=0, atol=tol)
    _, ref = okpm.kpm_moments(H, a, b, 128, 4, 5, first=4)
    assert np.max(np.abs(hi - ref)) <= (TOL_F64 if dtype == torch.float64 else TOL_F32)


def test_bounded_wait_gives_up_and_leaves_the_context_usable(gputb, cfg800):
    """The wait of the pipelined step (an mbarrier phase) runs on a phase
    that nothing completes: it must give up after its poll limit with
    TB_ERR_TIMEOUT, and the next call must work."""
    with pytest.raises(gputb.GputbError) as ei:
        gputb.debug_wait_timeout(2000)
    assert ei.value.status == gputb.TB_ERR_TIMEOUT
    s, indptr, idx, t, eps, H, a, b, w = cfg800
    Hd = sell_matrix(indptr, idx, t, eps, s.n, torch.float64)
    mu = gputb.kpm_moments(Hd, a, b, 64, 2, 3).cpu().numpy()
    _, mu_ref = okpm.kpm_moments(H, a, b, 64, 2, 3)
    assert np.max(np.abs(mu - mu_ref)) <= TOL_F64


@pytest.mark.parametrize("R,dtype,shape", shape_cases([1, 8, 16], [torch.float32]) + shape_cases([8], [torch.float64]))
def test_scattered_columns_take_the_gather_path(gputb, R, dtype, shape):
    """A random symmetric pattern (about 10 neighbours per row, anywhere in
    the matrix): slices fit the banded step's 16 slots, but a tile's columns
    fall in far more than 6 bands, so the banded shapes take their
    global-gather path for every tile; mixed with a cell-ordered block where
    tiles are banded."""
    import scipy.sparse as sp
    use_shape(gputb, shape, R, dtype)
    rng = np.random.default_rng(17)
    n = 3000
    A = sp.random(n, n, density=5 / n, random_state=rng, format="csr")
    A = (A + A.T).tocsr()
    A.setdiag(0)
    A.eliminate_zeros()
    # rows 2000.. get a banded nearest-neighbour chain instead
    A = A.tolil()
    for i in range(2000, n):
        A.rows[i], A.data[i] = [], []
    A = A.tocsr()
    chain = sp.diags([np.full(999, -1.0), np.full(999, -1.0)], [-1, 1], shape=(1000, 1000), format="csr")
    A = sp.bmat([[A[:2000, :2000], None], [None, chain]], format="csr")
    A.sort_indices()
    onsite = rng.uniform(-0.3, 0.3, n)
    H = oha.csr_hamiltonian(n, A.indptr, A.indices, A.data, onsite)
    _, _, a, b = obo.spectral_bounds(H, 64, 7)
    Hd = sell_matrix(A.indptr, A.indices, A.data, onsite, n, dtype)
    for doubling in (False, True):
        mu = gputb.kpm_moments(Hd, a, b, 64, R, 77, doubling=doubling).cpu().numpy()
        _, mu_ref = okpm.kpm_moments(H, a, b, 64, R, 77)
        assert np.max(np.abs(mu - mu_ref)) <= (TOL_F64 if dtype == torch.float64 else TOL_F32)


@pytest.mark.parametrize("R,dtype", [(1, torch.float32), (8, torch.float32), (8, torch.float64)])
def test_autotuned_shape_matches_oracle(gputb, R, dtype, tmp_path, monkeypatch):
    """tb_kpm_autotune times every shape on the caller's matrix and stores
    the fastest for its size class; the next kpm_moments call uses it and
    matches the oracle; the choice is written to the tuning cache file."""
    monkeypatch.setenv("GPUTB_TUNE_CACHE", str(tmp_path / "tuned.json"))
    s = synth.hbn_graphene_junction(40, 30, 0.1, 19)
    p = synth.teacher_hbn_graphene()
    indptr, idx, t, eps = _teacher_csr(s, p)
    H = oha.csr_hamiltonian(s.n, indptr, idx, t, eps)
    _, _, a, b = obo.spectral_bounds(H, 64, 7)
    Hd = sell_matrix(indptr, idx, t, eps, s.n, dtype)
    try:
        best, times = gputb.kpm_autotune(Hd, a, b, R, doubling=True, reps=3)
        assert len(times) == gputb.kpm_shape_count(R, dtype) and all(x > 0 for x in times)
        assert times[best] == min(times)
        assert gputb.kpm_get_shape(s.n, R, dtype, True) == best
        mu = gputb.kpm_moments(Hd, a, b, 96, R, 5, doubling=True).cpu().numpy()
        _, ref = okpm.kpm_moments(H, a, b, 96, R, 5)
        assert np.max(np.abs(mu - ref)) <= (TOL_F64 if dtype == torch.float64 else TOL_F32)
        import json
        data = json.load(open(tmp_path / "tuned.json"))
        entries = list(data.values())[0]
        assert any(e["shape"] == best and e["R"] == R for e in entries.values())
        gputb.kpm_clear_shapes()
        assert gputb.load_tuned_shapes() >= 1
        assert gputb.kpm_get_shape(s.n, R, dtype, True) == best
    finally:
        gputb.kpm_clear_shapes()
