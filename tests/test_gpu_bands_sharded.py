"""Band-energy training (Sec. 3, Eq. 3) in two situations the single-rank
tests do not reach.

* Cells of isolated atoms (no two closer than r_cut): the batch has no bond
  at all, H(k) is the diagonal of onsite energies, and the backward pass of
  the environment network runs with zero elements.  The parameter gradient
  must be exactly zero on every hopping-network entry and match the FP64
  oracle's onsite-only gradient on the onsite network.
* Cells sharded over two gloo ranks that share the one GPU (their kernels
  never wait on one another; the exchange is on the host): the loss and the
  gradient of the sharded step equal those of one rank over all cells, to
  FP32 rounding of the different summation order.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import env_bands as oe
from oracle import neighbors as onb
from paper_2509_06525_gb300 import synth

pytestmark = pytest.mark.gpu

CMIX = synth.descriptor_mixing("identity")


@pytest.fixture(scope="module")
def g():
    from paper_2509_06525_gb300 import build, gputb
    build.build()
    return gputb


def _isolated_cells():
    """Two 12 x 12 A cells of four atoms (B, N, C, C) 6 A apart."""
    out = []
    for k in range(2):
        pos = np.array([[0.5, 0.5, 0.0], [6.5, 0.5, 0.0], [0.5, 6.5, 0.0], [6.5, 6.5, 0.0]]) + 0.1 * k
        species = np.array([1, 2, 0, 0], np.int32)
        out.append(synth.Structure(pos, species, np.diag([12.0, 12.0, 20.0]), name=f"isolated-{k}"))
    return out


def _onsite_mask():
    """1 on the onsite network's entries of the flat parameter vector."""
    parts = {name: np.full(shape, 1.0 if name.startswith(("Wo", "bo")) else 0.0) for name, shape in oe.ENV_LAYOUT}
    return oe.pack(parts).astype(bool)


def test_isolated_atoms_give_an_onsite_only_gradient(g):
    from paper_2509_06525_gb300 import bands
    cells = _isolated_cells()
    p = synth.teacher_hbn_graphene()
    kpts = synth.band_kgrid(cells[0].box, 2, 1)
    batch = bands.build_cell_batch(cells, p, CMIX, kpts)
    assert batch.total == 0
    flat = synth.init_env_mlp(21, -1.0)
    eps0 = np.array([0.1, -0.2, 0.3])
    model = g.EnvModel(flat, CMIX, eps0)
    w = bands.band_weights(batch.n_atoms, (0, batch.n_atoms), len(cells) * len(kpts))
    tr = bands.BandTrainer(model, batch)
    stats, grad, evals = tr.loss_and_grad(w)
    gd = grad.cpu().numpy().astype(np.float64)
    mask = _onsite_mask()
    assert np.all(gd[~mask] == 0.0)
    cells_o = []
    for s in cells:
        indptr, idx, d = onb.neighbors(s.positions, s.box, s.pbc, p.rcut)
        assert idx.size == 0
        C, u, nz2, v = oe.edge_inputs(s.species, indptr, idx, d, CMIX.astype(float), p.rcut)
        cells_o.append(dict(n=s.n, species=s.species, indptr=indptr, indices=idx, dvec=d, C=C, u=u, nz2=nz2, v=v))
    E_ref = batch.e_ref.cpu().numpy().astype(np.float64)
    L, go, _ = oe.cell_loss_and_grad(flat.astype(np.float64), cells_o, kpts, E_ref,
                                     w.cpu().numpy().astype(np.float64), eps0)
    assert np.all(go[~mask] == 0.0)
    assert abs(float(stats[2].item()) - L) <= 1e-5 * L
    assert np.linalg.norm(gd - go) <= 1e-4 * np.linalg.norm(go)


N_CELLS = 6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    p = synth.teacher_graphene()
    cells = synth.band_training_cells(N_CELLS, 900)
    kpts = synth.band_kgrid(cells[0].box, 2, 2)
    return p, cells, kpts


def _sharded_worker(rank, world, port, out_path):
    from paper_2509_06525_gb300 import build, bands, gputb as gg
    from paper_2509_06525_gb300.distributed import block_shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    build.build()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, cells, kpts = _problem()
        first, count = block_shard(N_CELLS, rank, world)
        batch = bands.build_cell_batch(cells[first:first + count], p, CMIX, kpts)
        model = gg.EnvModel(synth.init_env_mlp(13, -1.0), CMIX, np.zeros(3))
        w = bands.band_weights(batch.n_atoms, (4, 20), N_CELLS * len(kpts))
        tr = bands.BandTrainer(model, batch, n_cells_total=N_CELLS)
        stats, grad, _ = tr.loss_and_grad(w)
        if rank == 0:
            np.save(out_path, np.concatenate([stats.cpu().numpy(), grad.cpu().numpy().astype(np.float64)]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_on_one_gpu_match_one_rank(g, tmp_path):
    from paper_2509_06525_gb300 import bands
    out = str(tmp_path / "sharded.npy")
    mp.start_processes(_sharded_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    p, cells, kpts = _problem()
    batch = bands.build_cell_batch(cells, p, CMIX, kpts)
    model = g.EnvModel(synth.init_env_mlp(13, -1.0), CMIX, np.zeros(3))
    w = bands.band_weights(batch.n_atoms, (4, 20), N_CELLS * len(kpts))
    stats, grad, _ = bands.BandTrainer(model, batch).loss_and_grad(w)
    st = stats.cpu().numpy()
    gd = grad.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got[:3], st, rtol=1e-6)
    assert np.linalg.norm(got[3:] - gd) <= 1e-5 * np.linalg.norm(gd)
