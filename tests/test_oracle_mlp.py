"""Pins for oracle.mlp: backward against central finite differences and
against torch.autograd (FP64), AdamW against torch.optim.AdamW, the Eq. 3
loss on closed-form residual sets, and the learned-H assembly."""
import numpy as np
import pytest
import torch

from oracle import mlp
from oracle import neighbors as nb
from oracle import descriptors as de
from paper_2509_06525_gb300 import synth


def _setup(E=37, seed=0):
    rng = np.random.default_rng(seed)
    params = {k: v.astype(np.float64) for k, v in synth.init_mlp(seed).items()}
    for k in ("b1", "b2", "b3"):
        params[k] = rng.normal(0, 0.1, size=params[k].shape)
    x = rng.normal(size=(E, 32))
    mean = rng.normal(size=32) * 0.1
    inv_std = rng.uniform(0.5, 2.0, size=32)
    return params, x, mean, inv_std


def _scalar_loss(params, x, mean, inv_std, wdy):
    y, _ = mlp.forward(params, x, mean, inv_std)
    return float(np.sum(y * wdy))


def test_backward_vs_finite_differences():
    params, x, mean, inv_std = _setup()
    rng = np.random.default_rng(1)
    wdy = rng.normal(size=(x.shape[0], 2))
    y, cache = mlp.forward(params, x, mean, inv_std)
    g = mlp.backward(params, cache, wdy)
    h = 1e-6
    for k in mlp.PARAM_NAMES:
        flat = params[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            pp = {kk: vv.copy() for kk, vv in params.items()}
            pm = {kk: vv.copy() for kk, vv in params.items()}
            pp[k].reshape(-1)[idx] += h
            pm[k].reshape(-1)[idx] -= h
            fd = (_scalar_loss(pp, x, mean, inv_std, wdy) - _scalar_loss(pm, x, mean, inv_std, wdy)) / (2 * h)
            an = g[k].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (k, idx, fd, an)


def test_forward_backward_vs_torch_autograd():
    params, x, mean, inv_std = _setup(E=50, seed=4)
    rng = np.random.default_rng(2)
    wdy = rng.normal(size=(50, 2))
    tp = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in params.items()}
    xn = (torch.tensor(x) - torch.tensor(mean)) * torch.tensor(inv_std)
    h1 = torch.nn.functional.silu(xn @ tp["W1"].T + tp["b1"])
    h2 = torch.nn.functional.silu(h1 @ tp["W2"].T + tp["b2"])
    yt = h2 @ tp["W3"].T + tp["b3"]
    (yt * torch.tensor(wdy)).sum().backward()
    y, cache = mlp.forward(params, x, mean, inv_std)
    np.testing.assert_allclose(y, yt.detach().numpy(), rtol=1e-13, atol=1e-13)
    g = mlp.backward(params, cache, wdy)
    for k in mlp.PARAM_NAMES:
        np.testing.assert_allclose(g[k], tp[k].grad.numpy(), rtol=1e-11, atol=1e-12)


def test_adamw_vs_torch():
    params, _, _, _ = _setup()
    rng = np.random.default_rng(5)
    tp = [torch.tensor(params[k], dtype=torch.float64, requires_grad=True) for k in mlp.PARAM_NAMES]
    opt = torch.optim.AdamW(tp, lr=1e-2, betas=(0.9, 0.999), eps=1e-8, weight_decay=0.03)
    p = dict(params)
    m = {k: np.zeros_like(v) for k, v in params.items()}
    v = {k: np.zeros_like(v) for k, v in params.items()}
    for t in range(1, 4):
        grads = {k: rng.normal(size=params[k].shape) for k in mlp.PARAM_NAMES}
        for tt, k in zip(tp, mlp.PARAM_NAMES):
            tt.grad = torch.tensor(grads[k])
        opt.step()
        p, m, v = mlp.adamw_step(p, grads, m, v, t, lr=1e-2, wd=0.03)
    for tt, k in zip(tp, mlp.PARAM_NAMES):
        np.testing.assert_allclose(p[k], tt.detach().numpy(), rtol=1e-13, atol=1e-14)


def test_loss_closed_form_and_gradient():
    valid = np.array([True, True, False, True])
    c = 0.3
    d_hop = np.array([c, -c, 7.0, c])        # padding entry must be ignored
    d_on = np.array([-c, c])
    loss, g_hop, g_on = mlp.loss_eq3(d_hop, d_on, valid)
    assert abs(loss - 2 * c * c) < 1e-15      # (mean|D|)^2 + mean D^2 with |D| = c
    assert g_hop[2] == 0.0
    # gradient against central differences of the loss in the residuals
    rng = np.random.default_rng(0)
    d_hop = rng.normal(size=9)
    d_on = rng.normal(size=4)
    valid = np.ones(9, bool)
    valid[3] = False
    _, g_hop, g_on = mlp.loss_eq3(d_hop, d_on, valid)
    h = 1e-7
    for k in range(9):
        if not valid[k]:
            continue
        dp, dm = d_hop.copy(), d_hop.copy()
        dp[k] += h
        dm[k] -= h
        fd = (mlp.loss_eq3(dp, d_on, valid)[0] - mlp.loss_eq3(dm, d_on, valid)[0]) / (2 * h)
        assert abs(fd - g_hop[k]) < 1e-7
    for k in range(4):
        dp, dm = d_on.copy(), d_on.copy()
        dp[k] += h
        dm[k] -= h
        fd = (mlp.loss_eq3(d_hop, dp, valid)[0] - mlp.loss_eq3(d_hop, dm, valid)[0]) / (2 * h)
        assert abs(fd - g_on[k]) < 1e-7


def test_output_gradient_chain_rule():
    """dL/dy from residuals + loss + output_gradient vs finite differences in y."""
    rng = np.random.default_rng(7)
    E, N = 12, 4
    edge_row = np.repeat(np.arange(N), 3)
    valid = np.ones(E, bool)
    valid[5] = False
    y = rng.normal(size=(E, 2))
    t_target = rng.normal(size=E)
    species = np.zeros(N, np.int64)
    eps0 = np.array([0.1, 0.0, 0.0])
    eps_t = rng.normal(size=N)

    def total(yy):
        dh, do, _ = mlp.hamiltonian_residuals(yy, edge_row, valid, t_target, N, species, eps0, eps_t)
        return mlp.loss_eq3(dh, do, valid)[0]

    dh, do, _ = mlp.hamiltonian_residuals(y, edge_row, valid, t_target, N, species, eps0, eps_t)
    _, gh, go = mlp.loss_eq3(dh, do, valid)
    dy = mlp.output_gradient(gh, go, edge_row, valid)
    h = 1e-7
    for e in range(E):
        for c in range(2):
            yp, ym = y.copy(), y.copy()
            yp[e, c] += h
            ym[e, c] -= h
            fd = (total(yp) - total(ym)) / (2 * h)
            assert abs(fd - dy[e, c]) < 1e-7, (e, c)


def test_learned_hamiltonian_symmetric():
    s = synth.graphene_rect(3, 3, sigma=0.1, seed=1)
    indptr, idx, d = nb.neighbors(s.positions, s.box, s.pbc, 3.0)
    rng = np.random.default_rng(0)
    y = rng.normal(size=(idx.size, 2))
    hop, eps = mlp.learned_hamiltonian(indptr, idx, y, s.species, np.zeros(3))
    lookup = {}
    for i in range(s.n):
        for k in range(indptr[i], indptr[i + 1]):
            lookup[(i, int(idx[k]))] = k
    for (i, j), k in lookup.items():
        kr = lookup[(j, i)]
        assert hop[k] == hop[kr]
        assert abs(hop[k] - 0.5 * (y[k, 0] + y[kr, 0])) < 1e-15
    rows = np.repeat(np.arange(s.n), np.diff(indptr))
    np.testing.assert_allclose(eps, np.bincount(rows, y[:, 1], minlength=s.n), atol=1e-14)
