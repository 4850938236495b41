"""Band-energy training of the environment-network model (Sec. 3: the
networks give H(R), the Bloch sum gives H(k), its eigenvalues E_pre enter
the loss of Eq. 3, AdamW updates the parameters; bands are brought in by a
band-expansion schedule).

Orchestration only: neighbours, descriptors, bond inputs, the model's H,
the Bloch bands, the loss, its Hellmann-Feynman gradient, the networks'
backward pass and AdamW are calls into libgputb.so.  The reference bands
are those of the analytic teacher's H of the same cells, through the same
Bloch kernel (there are no DFT bands here).

A batch of periodic cells with n atoms each is one block-diagonal SELL-32
structure: cell c owns rows [c P, c P + n) with P = 32 ceil(n / 32) (rows
n..P-1 of a cell carry no atom and no neighbours).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch

from . import gputb as g
from . import synth


@dataclass
class CellBatch:
    n_cells: int
    n_atoms: int
    rows_per_cell: int
    slice_ptr: torch.Tensor     # int64 [n_cells * P / 32 + 1]
    col: torch.Tensor           # int32, batch row indices
    cnt: torch.Tensor           # int32 [n_cells * P]
    species: torch.Tensor       # int32 [n_cells * P]
    v: torch.Tensor             # float32 [n_cells * P, 8]
    feat: torch.Tensor          # float32 [total, 20]
    t_teacher: torch.Tensor     # float32 [total]
    eps_teacher: torch.Tensor   # float32 [n_cells * P]
    kpts: torch.Tensor          # float32 [n_k, 3]
    total: int = 0              # SELL elements (the arrays hold at least one)
    e_ref: Optional[torch.Tensor] = None   # float32 [n_cells, n_k, n_atoms]
    flags: torch.Tensor = field(default=None)

    @property
    def n_rows(self) -> int:
        return self.n_cells * self.rows_per_cell


def build_cell_batch(structures: Sequence[synth.Structure], teacher, cmix, kpts: np.ndarray,
                     max_sweeps: int = 30) -> CellBatch:
    """Neighbours, bond inputs and teacher bands of equally sized periodic cells."""
    n = structures[0].n
    assert all(s.n == n for s in structures), "cells of one batch have the same atom count"
    P = 32 * ((n + 31) // 32)
    cm = torch.tensor(np.asarray(cmix, np.float32).reshape(-1), device="cuda")
    sp_all, col_all, cnt_all, spc_all, v_all, f_all, t_all, e_all = [], [], [], [], [], [], [], []
    base = 0
    for c, s in enumerate(structures):
        pos = torch.tensor(s.positions, device="cuda")
        spc = torch.tensor(s.species, device="cuda")
        nb = g.build_neighbors(pos, s.box, s.pbc, teacher.rcut, r_count=teacher.r_count, max_width=16)
        Ht = g.build_hamiltonian_teacher(pos, spc, s.box, s.pbc, nb, teacher, dtype=torch.float32, with_diag=True)
        v = g.compute_descriptors(pos, spc, s.box, s.pbc, teacher.rcut, nb, cm)
        feat = g.env_edge_inputs(pos, spc, s.box, s.pbc, teacher.rcut, nb, cm, v)
        pad = P - n
        sp_all.append(nb.slice_ptr[:-1] + base)
        col_all.append(nb.col + c * P)
        cnt_all.append(torch.nn.functional.pad(nb.cnt, (0, pad)))
        spc_all.append(torch.nn.functional.pad(spc, (0, pad)))
        v_all.append(torch.nn.functional.pad(v, (0, 0, 0, pad)))
        f_all.append(feat[:nb.total])
        t_all.append(Ht.val)
        e_all.append(torch.nn.functional.pad(Ht.diag, (0, pad)))
        base += nb.total
    sp_all.append(torch.tensor([base], dtype=torch.int64, device="cuda"))
    # one unreferenced element after the last so that no array is empty
    col_all.append(torch.zeros(1, dtype=torch.int32, device="cuda"))
    f_all.append(torch.zeros((1, g.ENV_NFEAT), dtype=torch.float32, device="cuda"))
    t_all.append(torch.zeros(1, dtype=torch.float32, device="cuda"))
    batch = CellBatch(len(structures), n, P, torch.cat(sp_all), torch.cat(col_all), torch.cat(cnt_all),
                      torch.cat(spc_all), torch.cat(v_all).contiguous(), torch.cat(f_all).contiguous(),
                      torch.cat(t_all), torch.cat(e_all),
                      torch.tensor(np.asarray(kpts, np.float32), device="cuda"), total=base,
                      flags=torch.zeros(1, dtype=torch.int32, device="cuda"))
    batch.e_ref, _ = bands_of(batch, batch.t_teacher, batch.eps_teacher, max_sweeps)
    return batch


def bands_of(batch: CellBatch, val, diag, max_sweeps: int = 30):
    return g.bloch_bands(batch.n_cells, batch.n_atoms, batch.rows_per_cell, batch.slice_ptr, batch.col, batch.cnt,
                         batch.feat, val, diag, batch.kpts, max_sweeps, flags=batch.flags)


def band_weights(n_bands: int, active: Tuple[int, int], n_spectra: int) -> torch.Tensor:
    """w_b = 1 / (number of weighted residuals) on bands [lo, hi), 0 elsewhere."""
    lo, hi = active
    w = np.zeros(n_bands, np.float32)
    w[lo:hi] = 1.0 / ((hi - lo) * n_spectra)
    return torch.tensor(w, device="cuda")


class BandTrainer:
    """One training step = model H -> bands -> Eq. 3 -> gradient -> AdamW.

    With a process group of several ranks and n_cells_total given, `batch`
    holds this rank's block of the cells (distributed.block_shard order) and
    each step exchanges the band energies and the gradients
    (distributed.band_step); the weights then count the residuals of the
    whole batch."""

    def __init__(self, model: g.EnvModel, batch: CellBatch, max_sweeps: int = 30, group=None,
                 n_cells_total: Optional[int] = None):
        import torch.distributed as dist
        several = dist.is_initialized() and dist.get_world_size(group) > 1
        if several and n_cells_total is None:
            raise ValueError("a process group of several ranks needs n_cells_total (the cells of all ranks); "
                             "without it each rank would train on its own cells with no exchange")
        self.model, self.batch, self.max_sweeps = model, batch, max_sweeps
        dev = batch.feat.device
        self.grad = torch.empty(g.ENV_NPARAM, dtype=torch.float32, device=dev)
        need = g.lib().tb_env_backward_workspace_size(batch.n_rows, batch.total)
        self.ws = torch.empty(max(int(need), 256), dtype=torch.uint8, device=dev)
        self.g_val = torch.zeros(max(batch.total, 1), dtype=torch.float32, device=dev)
        self.g_diag = torch.zeros(batch.n_rows, dtype=torch.float32, device=dev)
        self.stats = torch.zeros(3, dtype=torch.float64, device=dev)
        self.group = group
        self.n_cells_total = batch.n_cells if n_cells_total is None else int(n_cells_total)
        self.sharded = n_cells_total is not None and several
        if self.sharded:
            from .distributed import gather_blocks
            self.e_ref_all = gather_blocks(batch.e_ref, self.n_cells_total, group)

    def _loss_and_grad_sharded(self, weights: torch.Tensor):
        from .distributed import band_step
        b, m = self.batch, self.model

        def forward_local():
            val, diag = g.env_forward(b.n_rows, b.slice_ptr, b.cnt, b.feat, b.v, b.species, m, b.total)
            return bands_of(b, val, diag, self.max_sweeps)

        def loss_all(e_all, e_ref_all):
            dLdE, _ = g.band_loss(e_all, e_ref_all, weights, stats=self.stats)
            return dLdE, self.stats

        def backward_local(evecs, dLdE):
            g.band_gradient(b.n_cells, b.n_atoms, b.rows_per_cell, b.slice_ptr, b.col, b.cnt, b.feat, b.kpts, evecs,
                            dLdE, b.total, g_val=self.g_val, g_diag=self.g_diag)
            return g.env_backward(b.n_rows, b.slice_ptr, b.cnt, b.total, b.feat, b.v, b.species, m, self.g_val,
                                  self.g_diag, grad=self.grad, workspace=self.ws)

        stats, grad = band_step(forward_local, loss_all, backward_local, self.e_ref_all, self.n_cells_total,
                                self.group)
        return stats, grad, None

    def loss_and_grad(self, weights: torch.Tensor):
        if self.sharded:
            return self._loss_and_grad_sharded(weights)
        b, m = self.batch, self.model
        val, diag = g.env_forward(b.n_rows, b.slice_ptr, b.cnt, b.feat, b.v, b.species, m, b.total)
        evals, evecs = bands_of(b, val, diag, self.max_sweeps)
        dLdE, _ = g.band_loss(evals, b.e_ref, weights, stats=self.stats)
        g.band_gradient(b.n_cells, b.n_atoms, b.rows_per_cell, b.slice_ptr, b.col, b.cnt, b.feat, b.kpts, evecs,
                        dLdE, b.total, g_val=self.g_val, g_diag=self.g_diag)
        g.env_backward(b.n_rows, b.slice_ptr, b.cnt, b.total, b.feat, b.v, b.species, m, self.g_val, self.g_diag,
                       grad=self.grad, workspace=self.ws)
        return self.stats, self.grad, evals

    def step(self, weights: torch.Tensor, lr: float, weight_decay: float = 0.0):
        stats, grad, _ = self.loss_and_grad(weights)
        g.adamw_flat(self.model, grad, lr, weight_decay=weight_decay)
        return stats


def train_bands(model: g.EnvModel, batch: CellBatch, schedule: List[Tuple[int, Tuple[int, int]]],
                lr: float = 3e-3, lr_min: float = 3e-4, log_every: int = 25, group=None,
                n_cells_total: Optional[int] = None):
    """Band-expansion schedule: a list of (steps, (lo, hi)) stages, each
    fitting bands lo..hi-1 with a cosine-decayed learning rate.  Returns the
    loss history [(step, band window, L)].  group / n_cells_total: cells
    sharded over ranks (BandTrainer)."""
    tr = BandTrainer(model, batch, group=group, n_cells_total=n_cells_total)
    n_spec = tr.n_cells_total * batch.kpts.shape[0]
    hist = []
    k = 0
    for steps, window in schedule:
        w = band_weights(batch.n_atoms, window, n_spec)
        for s in range(steps):
            frac = s / max(steps - 1, 1)
            rate = lr_min + 0.5 * (lr - lr_min) * (1.0 + np.cos(np.pi * frac))
            stats = tr.step(w, rate)
            if s % log_every == 0 or s == steps - 1:
                hist.append((k, window, float(stats[2].item())))
            k += 1
    return hist


def band_mae(model: g.EnvModel, batch: CellBatch) -> float:
    """Mean |E_pre - E_ref| over all cells, k-points and bands (eV): the S
    term of tb_band_loss with every weight 1 / (number of residuals)."""
    val, diag = g.env_forward(batch.n_rows, batch.slice_ptr, batch.cnt, batch.feat, batch.v, batch.species, model,
                              batch.total)
    evals, _ = bands_of(batch, val, diag)
    n_spec = batch.n_cells * batch.kpts.shape[0]
    _, stats = g.band_loss(evals, batch.e_ref, band_weights(batch.n_atoms, (0, batch.n_atoms), n_spec))
    return float(stats[0].item())
