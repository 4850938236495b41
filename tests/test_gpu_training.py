"""What the trained network gains (learned part of the method, Sec. 3).

The per-pair MLP is trained on the GPU by the library's own forward and
backward kernels on 200 seeded 300 K graphene snapshots labelled by the
teacher.  On held-out snapshots it is compared with two models without the
network's environment input:

* constant-parameter TB: one nearest-neighbour hopping, least-squares fitted
  to the teacher's bonds shorter than 1.8 A (the "empirical parameter
  fitting" the paper contrasts with, Sec. 1), onsite 0;
* radial-only learned model: the same MLP with the environment blocks
  (v_i, v_j, C*(v_i+v_j)) switched off.

Errors: hopping and onsite RMSE against the teacher H, and Jackson DOS
relative L1 against the FP64 teacher DOS computed with identical random
vectors and bounds (so the stochastic noise cancels)."""
import math

import numpy as np
import pytest
import torch

from oracle import hamiltonian as oha
from oracle import neighbors as onb
from oracle import teacher as ote
from paper_2509_06525_gb300 import synth
from tests.sell_helpers import sell_matrix

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    from paper_2509_06525_gb300 import build, gputb, train
    build.build()
    full, hist = train.train_graphene_model()
    radial, _ = train.train_graphene_model(feature_mask=np.r_[np.ones(8), np.zeros(24)])
    return gputb, train, full, radial, hist


def _constant_tb():
    t = []
    teacher = synth.teacher_graphene()
    for s in synth.training_snapshots(40):
        ip, idx, d = onb.neighbors(s.positions, s.box, s.pbc, 3.0)
        tt, _, _ = ote.teacher_elements(s.species, ip, idx, d, teacher)
        t.append(tt[ote.distances(d) < 1.8])
    return float(np.mean(np.concatenate(t)))


def test_training_converges(trained):
    g, train, full, radial, hist = trained
    assert hist[-1] < 1e-2 * hist[0]
    assert np.all(np.isfinite(hist))


def test_network_beats_models_without_it(trained):
    g, train, full, radial, _ = trained
    teacher = synth.teacher_graphene()
    held_out = synth.training_snapshots(8, seed_base=9000)
    eh_full, eo_full = train.hamiltonian_errors(full, held_out, teacher)
    eh_rad, eo_rad = train.hamiltonian_errors(radial, held_out, teacher)
    t_const = _constant_tb()
    se, n = 0.0, 0
    for s in held_out:
        ip, idx, d = onb.neighbors(s.positions, s.box, s.pbc, 3.0)
        t, _, _ = ote.teacher_elements(s.species, ip, idx, d, teacher)
        pred = np.where(ote.distances(d) < 1.8, t_const, 0.0)
        se += float(((pred - t) ** 2).sum())
        n += t.size
    eh_const = math.sqrt(se / n)
    print(f"hopping RMSE (eV): full {eh_full:.4g}, radial-only {eh_rad:.4g}, constant {eh_const:.4g}; "
          f"onsite RMSE: full {eo_full:.4g}, radial-only {eo_rad:.4g}")
    assert eh_full <= 3e-3 and eo_full <= 5e-3
    # the graphene teacher's environment factor almost never departs from 1
    # (n_i = 3 nearly everywhere at 300 K) and its onsite energy is one
    # constant, so on graphene the environment inputs can only tie with
    # radial-only (both ~1 meV; which one is ahead changes with rounding-level
    # changes of the labels).  The junction test below is where they must win.
    assert eh_full <= 1.1 * eh_rad and eo_full <= 1.5 * eo_rad
    assert eh_full < 0.05 * eh_const


def test_environment_inputs_matter_on_hbn_graphene_junction(trained):
    """On the h-BN/graphene junction the onsite energy depends on the atom's
    species and surroundings: the full model must clearly beat radial-only."""
    g, train, _, _, _ = trained
    teacher = synth.teacher_hbn_graphene()
    cm = synth.descriptor_mixing("species")
    snaps = [synth.hbn_graphene_junction(10, 20, 0.1, 5000 + k) for k in range(200)]
    held_out = [synth.hbn_graphene_junction(10, 20, 0.1, 9500 + k) for k in range(8)]
    errs = {}
    for name, mask in (("full", None), ("radial", np.r_[np.ones(8), np.zeros(24)])):
        model = g.MLPModel(synth.init_mlp(0), cm, np.zeros(3))
        ds = train.build_snapshot_set(snaps, teacher, model.cmix)
        train.fit_normalisation(model, ds, mask)
        train.train(model, ds, train.TrainConfig())
        errs[name] = train.hamiltonian_errors(model, held_out, teacher)
    print(f"junction hopping/onsite RMSE (eV): full {errs['full']}, radial-only {errs['radial']}")
    assert errs["full"][0] < errs["radial"][0]
    assert errs["full"][1] < 0.7 * errs["radial"][1]


def test_learned_fp32_dos_against_fp64_teacher(trained):
    """DOS L1 <= 1e-2 against the FP64 teacher on a held-out 24k-atom sheet,
    with the same random vectors and bounds; constant TB is far worse."""
    g, train, full, radial, _ = trained
    teacher = synth.teacher_graphene()
    s = synth.graphene_rect(100, 60, 0.1, 4242)
    pos = torch.tensor(s.positions, device="cuda")
    spc = torch.tensor(s.species, device="cuda")
    nb = g.build_neighbors(pos, s.box, s.pbc, 3.0, r_count=1.8)
    Ht = g.build_hamiltonian_teacher(pos, spc, s.box, s.pbc, nb, teacher, dtype=torch.float64)
    bd = g.spectral_bounds(Ht, 64, synth.LANCZOS_SEED)
    a, b = 1.05 * bd.a, bd.b
    M, R = 1024, 8
    E = torch.linspace(b - 0.95 * a, b + 0.95 * a, 2001, dtype=torch.float64, device="cuda")
    rho_t = g.kpm_dos(g.kpm_moments(Ht, a, b, M, R, 42), a, b, E).cpu().numpy()
    Hl = g.build_hamiltonian(pos, spc, s.box, s.pbc, 3.0, nb, full, dtype=torch.float32)
    rho_l = g.kpm_dos(g.kpm_moments(Hl, a, b, M, R, 42), a, b, E).cpu().numpy()
    l1_learned = np.sum(np.abs(rho_l - rho_t)) / np.sum(np.abs(rho_t))
    ip, idx, d = onb.neighbors(s.positions, s.box, s.pbc, 3.0)
    t_const = _constant_tb()
    hop = np.where(ote.distances(d) < 1.8, t_const, 0.0)
    Hc = sell_matrix(ip, idx, hop, None, s.n, torch.float64)
    rho_c = g.kpm_dos(g.kpm_moments(Hc, a, b, M, R, 42), a, b, E).cpu().numpy()
    l1_const = np.sum(np.abs(rho_c - rho_t)) / np.sum(np.abs(rho_t))
    print(f"DOS L1 vs FP64 teacher: learned FP32 {l1_learned:.3g}, constant TB {l1_const:.3g}")
    assert l1_learned <= 1e-2
    assert l1_learned < 0.2 * l1_const
