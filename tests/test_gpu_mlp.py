"""GPU parity of the learned-Hamiltonian kernels against the FP64 oracle.

Tolerances (BF16 tensor-core arithmetic vs FP64, with the oracle evaluated
at the BF16-rounded weights and inputs): forward outputs rel L2 <= 1e-2;
gradients per tensor rel L2 <= 2e-2 and cosine >= 0.999; descriptors and
edge features (FP32 vs FP64) rel 2e-5; loss and dL/dy rel 1e-5; AdamW (FP32
vs FP64) rel 1e-5."""
import numpy as np
import pytest
import torch

from oracle import descriptors as ode
from oracle import mlp as omlp
from oracle import neighbors as onb
from oracle import teacher as ote
from paper_2509_06525_gb300 import synth
from tests.sell_helpers import csr_to_sell

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    from paper_2509_06525_gb300 import build, gputb
    build.build()
    return gputb


def bf16_round(a):
    return torch.tensor(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def sell_positions(slice_ptr, cnt):
    """SELL element index of every CSR entry (rows ascending, slots ascending)."""
    out = []
    for i, m in enumerate(cnt):
        k, lane = divmod(i, 32)
        out.append(slice_ptr[k] + lane + 32 * np.arange(m))
    return np.concatenate(out).astype(np.int64)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("kind", ["graphene", "junction"])
def test_descriptors_and_edge_features(g, kind):
    if kind == "graphene":
        s, cm = synth.graphene_primitive(20, 20, 0.1, 5), synth.descriptor_mixing("identity")
    else:
        s, cm = synth.hbn_graphene_junction(12, 10, 0.1, 6), synth.descriptor_mixing("species")
    pos = torch.tensor(s.positions, device="cuda")
    spc = torch.tensor(s.species, device="cuda")
    nb = g.build_neighbors(pos, s.box, s.pbc, 3.0, r_count=1.8)
    cmix = torch.tensor(cm.reshape(-1), device="cuda")
    v = g.compute_descriptors(pos, spc, s.box, s.pbc, 3.0, nb, cmix).cpu().numpy()
    xr, xb = g.edge_features(pos, spc, s.box, s.pbc, 3.0, nb, cmix, torch.tensor(v, device="cuda"))
    indptr, idx, d = onb.neighbors(s.positions, s.box, s.pbc, 3.0)
    C, v_ref, x_ref = ode.descriptors(s.species, indptr, idx, d, cm.astype(np.float64), 3.0)
    np.testing.assert_allclose(v, v_ref, rtol=2e-5, atol=2e-5)
    pos_e = sell_positions(nb.slice_ptr.cpu().numpy(), nb.cnt.cpu().numpy())
    xr = xr.cpu().numpy()
    np.testing.assert_allclose(xr[pos_e], x_ref, rtol=2e-5, atol=5e-5)
    mask = np.ones(xr.shape[0], bool)
    mask[pos_e] = False
    assert np.all(xr[mask] == 0.0)
    np.testing.assert_array_equal(xb.to(torch.float32).cpu().numpy(),
                                  torch.tensor(xr).to(torch.bfloat16).to(torch.float32).numpy())
    fmask = np.ones(32, np.float32)
    fmask[8:16] = 0.0
    mean, std, inv = g.feature_stats(torch.tensor(xr, device="cuda"), s.n, nb.slice_ptr, nb.cnt, mask=fmask)
    np.testing.assert_allclose(mean.cpu().numpy(), x_ref.mean(0), rtol=1e-4, atol=1e-5)
    np.testing.assert_allclose(std.cpu().numpy(), x_ref.std(0), rtol=1e-4, atol=1e-5)
    # the normalisation: mask / max(std, 1e-6), from the library
    sd = std.cpu().numpy()
    np.testing.assert_allclose(inv.cpu().numpy(), fmask / np.maximum(sd, np.float32(1e-6)), rtol=1e-6)
    np.testing.assert_array_equal(g.inverse_std(std).cpu().numpy(), np.float32(1.0) / np.maximum(sd, np.float32(1e-6)))


def _model(g, seed, bias=True):
    p = synth.init_mlp(seed)
    if bias:
        rng = np.random.default_rng(seed + 1)
        for k in ("b1", "b2", "b3"):
            p[k] = rng.normal(0, 0.2, p[k].shape).astype(np.float32)
    return p, g.MLPModel(p, synth.descriptor_mixing("identity"), np.zeros(3))


def _oracle_params_bf16(p):
    return {k: (bf16_round(v) if k.startswith("W") else np.asarray(v, np.float64)) for k, v in p.items()}


@pytest.mark.parametrize("E", [1000, 5003])
def test_forward_and_backward_match_oracle(g, E):
    p, model = _model(g, 3)
    rng = np.random.default_rng(E)
    x = bf16_round(rng.normal(size=(E, 32)))
    dy = rng.normal(size=(E, 2)).astype(np.float32)
    xb = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).cuda()
    y = g.mlp_forward(xb, model).cpu().numpy()
    po = _oracle_params_bf16(p)
    y_ref, cache = omlp.forward(po, x, np.zeros(32), np.ones(32))
    for c in range(2):
        assert rel_l2(y[:, c], y_ref[:, c]) <= 1e-2, c
    grad = g.mlp_backward(xb, model, torch.tensor(dy, device="cuda")).cpu().numpy()
    gref = omlp.backward(po, cache, dy.astype(np.float64))
    gg = g.unpack_params(grad)
    for k in omlp.PARAM_NAMES:
        a, b = gg[k].reshape(-1).astype(np.float64), gref[k].reshape(-1)
        cos = float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))
        assert rel_l2(a, b) <= 2e-2 and cos >= 0.999, (k, rel_l2(a, b), cos)
    # reproducible: fixed-order reduction
    grad2 = g.mlp_backward(xb, model, torch.tensor(dy, device="cuda")).cpu().numpy()
    assert np.array_equal(grad, grad2)


def test_loss_and_output_gradient(g):
    s = synth.hbn_graphene_junction(8, 8, 0.1, 2)          # 256 atoms = 8 slices
    indptr, idx, d = onb.neighbors(s.positions, s.box, s.pbc, 3.0)
    sp, col, _ = csr_to_sell(indptr, idx, np.zeros(idx.size), s.n)
    cnt = np.diff(indptr).astype(np.int32)
    rng = np.random.default_rng(0)
    E = int(sp[-1])
    y = rng.normal(size=(E, 2)).astype(np.float32)
    t = rng.normal(size=E).astype(np.float32)
    eps_t = rng.normal(size=s.n).astype(np.float32)
    eps0 = np.array([0.1, 0.5, -0.3], np.float32)
    pos_e = sell_positions(sp, cnt)
    valid = np.zeros(E, bool)
    valid[pos_e] = True
    t[~valid] = 0.0
    row_of = np.zeros(E, np.int64)
    row_of[pos_e] = np.repeat(np.arange(s.n), cnt)
    dy = torch.zeros((E, 2), dtype=torch.float32, device="cuda")
    dev = lambda a: torch.tensor(a, device="cuda")
    stats = g.mlp_loss(0, s.n, dev(sp), dev(cnt), dev(y), dev(t), dev(eps_t), dev(s.species), dev(eps0), dy)
    d_hop, d_on, _ = omlp.hamiltonian_residuals(y.astype(np.float64), row_of, valid, t, s.n, s.species,
                                                eps0.astype(np.float64), eps_t)
    loss, gh, go = omlp.loss_eq3(d_hop, d_on, valid)
    dy_ref = omlp.output_gradient(gh, go, row_of, valid)
    np.testing.assert_allclose(stats.cpu().numpy()[3], loss, rtol=1e-10)
    np.testing.assert_allclose(dy.cpu().numpy(), dy_ref, rtol=1e-5, atol=1e-9)
    # a batch of rows: only that batch's elements are written
    dy2 = torch.full((E, 2), 7.0, dtype=torch.float32, device="cuda")
    g.mlp_loss(64, 128, dev(sp), dev(cnt), dev(y), dev(t), dev(eps_t), dev(s.species), dev(eps0), dy2)
    dy2 = dy2.cpu().numpy()
    inside = np.zeros(E, bool)
    inside[int(sp[2]):int(sp[4])] = True
    assert np.all(dy2[~inside] == 7.0) and np.all(dy2[inside] != 7.0)


def test_adamw_matches_oracle(g):
    p, model = _model(g, 9)
    rng = np.random.default_rng(1)
    po = {k: np.asarray(v, np.float64) for k, v in p.items()}
    m = {k: np.zeros_like(v) for k, v in po.items()}
    v = {k: np.zeros_like(v) for k, v in po.items()}
    for t in range(1, 4):
        grads = {k: rng.normal(size=po[k].shape) for k in omlp.PARAM_NAMES}
        gflat = torch.tensor(g.pack_params({k: gv.astype(np.float32) for k, gv in grads.items()}), device="cuda")
        g.adamw_step(model, gflat, lr=1e-2, weight_decay=0.01)
        po, m, v = omlp.adamw_step(po, {k: grads[k].astype(np.float32).astype(np.float64) for k in grads}, m, v, t,
                                   lr=1e-2, wd=0.01)
    got = model.params_numpy()
    for k in omlp.PARAM_NAMES:
        np.testing.assert_allclose(got[k], po[k], rtol=1e-5, atol=1e-6)
    wb = model.wb.to(torch.float32).cpu().numpy()
    np.testing.assert_array_equal(wb[:2048], torch.tensor(got["W1"].reshape(-1)).to(torch.bfloat16).float().numpy())


@pytest.fixture(params=[0, 1], ids=["tcgen05", "mma_sync"])
def mlp_variant(request, g):
    """Forward kernel of the learned H: 5th-generation tensor cores (TMEM
    accumulators) or mma.sync tiles."""
    g.mlp_set_variant(request.param)
    yield request.param
    g.mlp_set_variant(0)


def test_learned_hamiltonian_matches_oracle(g, mlp_variant):
    s = synth.graphene_primitive(20, 20, 0.1, 8)
    cm = synth.descriptor_mixing("identity")
    p, model = _model(g, 4)
    pos = torch.tensor(s.positions, device="cuda")
    spc = torch.tensor(s.species, device="cuda")
    nb = g.build_neighbors(pos, s.box, s.pbc, 3.0, r_count=1.8)
    indptr, idx, d = onb.neighbors(s.positions, s.box, s.pbc, 3.0)
    _, _, x_ref = ode.descriptors(s.species, indptr, idx, d, cm.astype(np.float64), 3.0)
    mean, std = x_ref.mean(0), x_ref.std(0)
    model.set_normalisation(torch.tensor(mean, device="cuda"), torch.tensor(std, device="cuda"))
    H = g.build_hamiltonian(pos, spc, s.box, s.pbc, 3.0, nb, model, dtype=torch.float64)
    xn = bf16_round((x_ref - mean) / std)
    y_ref, _ = omlp.forward(_oracle_params_bf16(p), xn, np.zeros(32), np.ones(32))
    hop_ref, eps_ref = omlp.learned_hamiltonian(indptr, idx, y_ref, s.species, np.zeros(3))
    pos_e = sell_positions(nb.slice_ptr.cpu().numpy(), nb.cnt.cpu().numpy())
    hop = H.val.cpu().numpy()[pos_e]
    assert rel_l2(hop, hop_ref) <= 1e-2
    assert rel_l2(H.diag.cpu().numpy(), eps_ref) <= 1e-2
    # exactly symmetric
    lookup = {(int(i), int(j)): k for k, (i, j) in enumerate(zip(np.repeat(np.arange(s.n), np.diff(indptr)), idx))}
    for (i, j), k in list(lookup.items())[:2000]:
        assert hop[k] == hop[lookup[(j, i)]]


def test_tcgen05_and_mma_sync_forward_agree_on_many_tiles(g):
    """9600-atom junction-free sheet (75 x 32 tiles, ragged last chunks of
    each slice): both forward kernels give the same learned H up to the
    order of the FP32 sums (and the BF16 roundings that order can flip)."""
    s = synth.graphene_rect(60, 40, 0.1, 12)
    cm = synth.descriptor_mixing("identity")
    p, model = _model(g, 9)
    pos = torch.tensor(s.positions, device="cuda")
    spc = torch.tensor(s.species, device="cuda")
    nb = g.build_neighbors(pos, s.box, s.pbc, 3.0, r_count=1.8)
    out = []
    for variant in (0, 1):
        g.mlp_set_variant(variant)
        H = g.build_hamiltonian(pos, spc, s.box, s.pbc, 3.0, nb, model, dtype=torch.float32)
        out.append((H.val.cpu().numpy().astype(np.float64), H.diag.cpu().numpy().astype(np.float64)))
    g.mlp_set_variant(0)
    assert rel_l2(out[0][0], out[1][0]) <= 5e-3
    assert rel_l2(out[0][1], out[1][1]) <= 5e-3
    assert np.all(np.isfinite(out[0][0]))
