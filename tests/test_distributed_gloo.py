"""Multi-rank path on CPU: two gloo ranks split the random vectors of the
KPM trace estimate (Sec. 2.4) with vector_shard, each computes its block
with the FP64 oracle (vectors first .. first + count - 1), and
gather_moments must give the moments of the whole ensemble as one oracle
call over all vectors; max_over_ranks gives the slowest rank's time."""
import os
import socket

import numpy as np
import pytest
import scipy.sparse as sp
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import kpm as okpm
from paper_2509_06525_gb300.distributed import gather_moments, max_over_ranks, vector_shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _ring_hamiltonian(n=40, seed=3):
    rng = np.random.default_rng(seed)
    t = rng.uniform(-1.2, -0.8, n)
    rows = np.arange(n)
    H = sp.csr_matrix((t, (rows, (rows + 1) % n)), shape=(n, n))
    H = (H + H.T).tocsr()
    H.setdiag(rng.uniform(-0.3, 0.3, n))
    return H.tocsr()


@pytest.mark.parametrize("r_total,world", [(8, 2), (3, 2), (5, 3), (4, 4), (7, 1)])
def test_vector_shard_partitions_the_ensemble(r_total, world):
    seen = []
    for k in range(world):
        first, count = vector_shard(r_total, k, world)
        assert count >= 1
        seen.extend(range(first, first + count))
    assert seen == list(range(r_total))
    counts = [vector_shard(r_total, k, world)[1] for k in range(world)]
    assert max(counts) - min(counts) <= 1


def test_vector_shard_rejects_bad_arguments():
    with pytest.raises(ValueError):
        vector_shard(2, 0, 3)
    with pytest.raises(ValueError):
        vector_shard(4, 2, 2)


def test_oracle_vector_offset_selects_ensemble_members():
    """Vectors first .. first + R - 1 are the same columns of the full draw."""
    H = _ring_hamiltonian()
    full = okpm.random_phase_vectors(11, H.shape[0], 6)
    part = okpm.random_phase_vectors(11, H.shape[0], 2, first=3)
    assert np.array_equal(part, full[:, 3:5])
    _, mu_full = okpm.kpm_moments(H, 3.0, 0.0, 24, 6, 11)
    _, mu_part = okpm.kpm_moments(H, 3.0, 0.0, 24, 2, 11, first=3)
    np.testing.assert_allclose(mu_part, mu_full[3:5], rtol=0, atol=1e-15)


def _worker(rank, world, port, r_total, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        H = _ring_hamiltonian()
        first, count = vector_shard(r_total, rank, world)
        _, mu_local = okpm.kpm_moments(H, 3.0, 0.1, 32, count, 2024, first=first)
        mu_all = gather_moments(torch.tensor(mu_local), r_total)
        t_max = max_over_ranks(1.5 + rank, "cpu")
        if rank == 0:
            np.save(out_path, mu_all.numpy())
            with open(out_path + ".t", "w") as f:
                f.write(repr(t_max))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("r_total", [4, 3])
def test_two_gloo_ranks_reproduce_the_single_rank_ensemble(tmp_path, r_total):
    world = 2
    out = str(tmp_path / "mu.npy")
    mp.start_processes(_worker, args=(world, _free_port(), r_total, out), nprocs=world, join=True,
                       start_method="spawn")
    mu_all = np.load(out)
    _, mu_ref = okpm.kpm_moments(_ring_hamiltonian(), 3.0, 0.1, 32, r_total, 2024)
    assert mu_all.shape == mu_ref.shape
    np.testing.assert_allclose(mu_all, mu_ref, rtol=0, atol=1e-14)
    with open(out + ".t") as f:
        assert float(f.read()) == 2.5


# ---------------------------------------------------------------- band-energy training

def _band_cells(n_cells):
    from oracle import env_bands as oe
    from oracle import neighbors as onb
    from paper_2509_06525_gb300 import synth
    cm = synth.descriptor_mixing("identity").astype(float)
    cells = []
    for s in synth.band_training_cells(n_cells, 900):
        indptr, idx, d = onb.neighbors(s.positions, s.box, s.pbc, 3.0)
        C, u, nz2, v = oe.edge_inputs(s.species, indptr, idx, d, cm, 3.0)
        cells.append(dict(n=s.n, species=s.species, indptr=indptr, indices=idx, dvec=d, C=C, u=u, nz2=nz2, v=v))
    return cells


def _band_problem(n_cells):
    from paper_2509_06525_gb300 import synth
    cells = _band_cells(n_cells)
    kpts = synth.band_kgrid(synth.graphene_rect(2, 3).box, 2, 1)
    rng = np.random.default_rng(5)
    e_ref = rng.normal(0.0, 1.0, (n_cells, len(kpts), cells[0]["n"]))
    w = np.linspace(1.0, 0.5, cells[0]["n"]) / (n_cells * len(kpts))
    flat = synth.init_env_mlp(7, -1.0).astype(float)
    return cells, kpts, e_ref, w, flat


def _band_worker(rank, world, port, n_cells, out_path):
    """Each rank computes the model and bands of its cells with the oracle;
    band_step exchanges the band energies and the gradients."""
    from oracle import env_bands as oe
    from paper_2509_06525_gb300.distributed import band_step, block_shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cells, kpts, e_ref, w, flat = _band_problem(n_cells)
        first, count = block_shard(n_cells, rank, world)
        mine = cells[first:first + count]

        def forward_local():
            E, ctx = [], []
            for c in mine:
                t, hc = oe.hopping_forward(flat, c["C"], c["u"], c["nz2"])
                e, oc = oe.onsite_forward(flat, c["v"], c["species"], np.zeros(3))
                Ec, psi = oe.bands(c["n"], c["indptr"], c["indices"], c["dvec"], t, e, kpts)
                E.append(Ec)
                ctx.append((hc, oc, psi))
            return torch.tensor(np.stack(E)), ctx

        def loss_all(E_all, E_ref_all):
            L, dLdE = oe.band_loss(E_all.numpy(), E_ref_all.numpy(), w)
            return torch.tensor(dLdE), torch.tensor([L], dtype=torch.float64)

        def backward_local(ctx, dLdE):
            g = np.zeros(oe.ENV_NPARAM)
            for c, (hc, oc, psi), d in zip(mine, ctx, dLdE.numpy()):
                gt, ge = oe.band_gradient(c["indptr"], c["indices"], c["dvec"], kpts, psi, d)
                g += oe.hopping_backward(flat, hc, gt) + oe.onsite_backward(flat, oc, ge)
            return torch.tensor(g)

        stats, grad = band_step(forward_local, loss_all, backward_local, torch.tensor(e_ref), n_cells)
        if rank == 0:
            np.save(out_path, np.concatenate([stats.numpy(), grad.numpy()]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("n_cells,world", [(4, 2), (5, 2), (5, 3)])
def test_gloo_ranks_reproduce_the_single_process_band_step(tmp_path, n_cells, world):
    """Cells sharded over 2 or 3 gloo ranks (even and uneven shards): the
    loss of Eq. 3 and its parameter gradient equal one oracle evaluation
    over the whole batch."""
    from oracle import env_bands as oe
    out = str(tmp_path / "band.npy")
    mp.start_processes(_band_worker, args=(world, _free_port(), n_cells, out), nprocs=world, join=True,
                       start_method="spawn")
    got = np.load(out)
    cells, kpts, e_ref, w, flat = _band_problem(n_cells)
    L, grad, _ = oe.cell_loss_and_grad(flat, cells, kpts, e_ref, w, np.zeros(3))
    assert got[0] == pytest.approx(L, rel=1e-12)
    np.testing.assert_allclose(got[1:], grad, rtol=1e-10, atol=1e-12 * np.max(np.abs(grad)))


def _unsharded_worker(rank, world, port, out_path):
    from paper_2509_06525_gb300.bands import BandTrainer
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        try:
            BandTrainer(None, None)
            result = "accepted"
        except ValueError:
            result = "rejected"
        if rank == 0:
            with open(out_path, "w") as fh:
                fh.write(result)
    finally:
        dist.destroy_process_group()


def test_band_trainer_refuses_a_group_without_the_total_cell_count(tmp_path):
    """With several ranks and no n_cells_total, each rank would silently
    train on its own cells; the trainer must refuse."""
    out = str(tmp_path / "r.txt")
    mp.start_processes(_unsharded_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    assert open(out).read() == "rejected"
