"""Training driver for the learned Hamiltonian (Sec. 2.1, Eq. 3 form).

Orchestration only: every numeric step (neighbours, teacher labels,
descriptors, edge features, feature statistics, forward, loss, backward,
AdamW) is a call into libgputb.so through the binding.  Training data are
the seeded finite-temperature snapshots of ``synth.training_snapshots``,
labelled by the analytic teacher.

Snapshots are concatenated into one block-diagonal SELL-32 structure (each
800-atom snapshot is exactly 25 slices), so a minibatch of snapshots is a
contiguous range of rows and of SELL elements.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Optional

import numpy as np
import torch

from . import gputb as g
from . import synth


@dataclass
class SnapshotSet:
    n_rows: int
    rows_per_snapshot: int
    slice_ptr: torch.Tensor     # int64, concatenated
    col: torch.Tensor           # int32, global row indices
    cnt: torch.Tensor
    species: torch.Tensor
    t_hop: torch.Tensor         # float32, SELL order (teacher hoppings)
    eps_t: torch.Tensor         # float32 [rows] (teacher onsite)
    x_raw: torch.Tensor         # float32 [elements][32]
    x_bf16: Optional[torch.Tensor] = None
    n_snapshots: int = 0
    parts: Optional[list] = None  # per snapshot: (structure, pos, spc, nb, v)
    rcut: float = 3.0

    def element_range(self, s0: int, s1: int):
        r0, r1 = s0 * self.rows_per_snapshot, s1 * self.rows_per_snapshot
        sp = self.slice_ptr
        return r0, r1, int(sp[r0 // 32].item()), int(sp[r1 // 32].item())


def build_snapshot_set(structures: List[synth.Structure], teacher, cmix: torch.Tensor) -> SnapshotSet:
    """Neighbours, teacher labels and raw edge features of every snapshot."""
    n0 = structures[0].n
    assert n0 % 32 == 0 and all(s.n == n0 for s in structures)
    sp_all, col_all, cnt_all, spc_all, t_all, eps_all, x_all, parts = [], [], [], [], [], [], [], []
    elem_base = 0
    for k, s in enumerate(structures):
        pos = torch.tensor(s.positions, device="cuda")
        spc = torch.tensor(s.species, device="cuda")
        nb = g.build_neighbors(pos, s.box, s.pbc, teacher.rcut, r_count=teacher.r_count, max_width=16)
        Ht = g.build_hamiltonian_teacher(pos, spc, s.box, s.pbc, nb, teacher, dtype=torch.float32)
        v = g.compute_descriptors(pos, spc, s.box, s.pbc, teacher.rcut, nb, cmix)
        xr, _ = g.edge_features(pos, spc, s.box, s.pbc, teacher.rcut, nb, cmix, v, raw=True, bf16=False)
        sp = nb.slice_ptr[:-1] + elem_base
        sp_all.append(sp)
        col_all.append(nb.col + k * n0)
        cnt_all.append(nb.cnt)
        spc_all.append(spc)
        t_all.append(Ht.val)
        eps_all.append(Ht.diag)
        x_all.append(xr)
        parts.append((s, pos, spc, nb, v))
        elem_base += nb.total
    sp_all.append(torch.tensor([elem_base], dtype=torch.int64, device="cuda"))
    return SnapshotSet(n_rows=n0 * len(structures), rows_per_snapshot=n0, slice_ptr=torch.cat(sp_all),
                       col=torch.cat(col_all), cnt=torch.cat(cnt_all), species=torch.cat(spc_all),
                       t_hop=torch.cat(t_all), eps_t=torch.cat(eps_all), x_raw=torch.cat(x_all).contiguous(),
                       n_snapshots=len(structures), parts=parts, rcut=teacher.rcut)


def fit_normalisation(model: g.MLPModel, ds: SnapshotSet, feature_mask: Optional[np.ndarray] = None):
    """Freeze the per-feature mean / std of the training inputs into the
    model (tb_feature_stats), then build the normalised BF16 inputs of every
    snapshot with tb_edge_features.  Features where feature_mask is 0 are
    switched off (inv_std = 0), e.g. the environment blocks for a
    radial-only model."""
    mask = None if feature_mask is None else np.asarray(feature_mask, np.float32)
    mean, _, inv_std = g.feature_stats(ds.x_raw, ds.n_rows, ds.slice_ptr, ds.cnt, mask=mask)
    model.mean = mean
    model.inv_std = inv_std
    xs = []
    for (s, pos, spc, nb, v) in ds.parts:
        _, xb = g.edge_features(pos, spc, s.box, s.pbc, ds.rcut, nb, model.cmix, v, model.mean,
                                model.inv_std, raw=False, bf16=True)
        xs.append(xb)
    ds.x_bf16 = torch.cat(xs).contiguous()


@dataclass
class TrainConfig:
    """Defaults measured on GB300 for the 200 x 800-atom graphene set: 800
    epochs of 50 minibatches (4 snapshots each) take ~6 s and reach held-out
    hopping / onsite RMSE of ~1 meV against the teacher."""
    epochs: int = 800
    batch_snapshots: int = 4
    lr: float = 3e-3
    lr_min: float = 1e-5
    seed: int = 0
    weight_decay: float = 0.0


def train(model: g.MLPModel, ds: SnapshotSet, cfg: TrainConfig, log=None):
    """AdamW on the Eq. 3-form loss with cosine learning-rate decay; returns
    the per-epoch mean loss history."""
    E_total = ds.x_raw.shape[0]
    y = torch.zeros((E_total, 2), dtype=torch.float32, device="cuda")
    dy = torch.zeros((E_total, 2), dtype=torch.float32, device="cuda")
    nb_batches = max(1, ds.n_snapshots // cfg.batch_snapshots)
    total_steps = cfg.epochs * nb_batches
    ranges = [ds.element_range(b * cfg.batch_snapshots, min(ds.n_snapshots, (b + 1) * cfg.batch_snapshots))
              for b in range(nb_batches)]
    ws = g._workspace(g.lib().tb_mlp_workspace_size(max(e1 - e0 for _, _, e0, e1 in ranges)), "cuda")
    rng = np.random.default_rng(cfg.seed)
    history = []
    step = 0
    for ep in range(cfg.epochs):
        losses = []
        for b in rng.permutation(nb_batches):
            r0, r1, e0, e1 = ranges[b]
            lr = cfg.lr_min + 0.5 * (cfg.lr - cfg.lr_min) * (1 + math.cos(math.pi * step / total_steps))
            xb = ds.x_bf16[e0:e1]
            st = g.lib().tb_mlp_forward(e1 - e0, g._ptr(xb), g._ptr(model.wb), g._ptr(model.p),
                                        g._ptr(y[e0:e1]), g._stream())
            g._check("tb_mlp_forward", st)
            stats = g.mlp_loss(r0, r1, ds.slice_ptr, ds.cnt, y, ds.t_hop, ds.eps_t, ds.species, model.eps0, dy)
            grad = g.mlp_backward(xb, model, dy[e0:e1], workspace=ws)
            g.adamw_step(model, grad, lr, weight_decay=cfg.weight_decay)
            losses.append(stats[3:4])
            step += 1
        history.append(float(torch.cat(losses).mean().item()))
        if log is not None:
            log(ep, history[-1])
    return history


def hamiltonian_errors(model: g.MLPModel, structures, teacher):
    """RMSE of learned vs teacher hoppings and onsite energies (eV) on the
    given snapshots, both in FP64."""
    se_h, se_o, nh, no = 0.0, 0.0, 0, 0
    for s in structures:
        pos = torch.tensor(s.positions, device="cuda")
        spc = torch.tensor(s.species, device="cuda")
        nb = g.build_neighbors(pos, s.box, s.pbc, teacher.rcut, r_count=teacher.r_count, max_width=16)
        Ht = g.build_hamiltonian_teacher(pos, spc, s.box, s.pbc, nb, teacher, dtype=torch.float64)
        Hl = g.build_hamiltonian(pos, spc, s.box, s.pbc, teacher.rcut, nb, model, dtype=torch.float64)
        se_h += float(((Hl.val - Ht.val) ** 2).sum())
        nh += int(nb.cnt.sum())
        se_o += float(((Hl.diag - Ht.diag) ** 2).sum())
        no += s.n
    return math.sqrt(se_h / max(nh, 1)), math.sqrt(se_o / max(no, 1))


def train_graphene_model(n_snapshots: int = synth.TRAIN_SNAPSHOTS, cfg: Optional[TrainConfig] = None,
                         feature_mask: Optional[np.ndarray] = None, init_seed: int = 0):
    """Train the learned pz model on the seeded 300 K graphene snapshots."""
    teacher = synth.teacher_graphene()
    model = g.MLPModel(synth.init_mlp(init_seed), synth.descriptor_mixing("identity"), np.zeros(3))
    ds = build_snapshot_set(synth.training_snapshots(n_snapshots), teacher, model.cmix)
    fit_normalisation(model, ds, feature_mask)
    history = train(model, ds, cfg or TrainConfig())
    return model, history
