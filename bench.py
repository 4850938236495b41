#!/usr/bin/env python3
"""Benchmark of the GPUTB hot path on GB300: KPM atom*moments/s.

One step = one pass of the whole path over one synthetic structure:
cell-list neighbours -> Hamiltonian (learned MLP or analytic teacher) in
SELL-32 -> FP64 spectral bounds -> FP32 KPM moments (R random-phase vectors,
M moments) -> Jackson DOS.  value = N_atoms * M / (time per step), summed
over ranks.  Inputs are resident in HBM when the timed region starts; the
`e2e` figure repeats the step from pinned host buffers with the host<->device
copies inside the timed region.

--impl reference times the FP64 CPU oracle (the only other implementation of
this path) on a bounded sample of the same workload.

Launch: python bench.py [--gpus 1 --steps 3 --warmup 3]; for N > 1 under
torch.distributed.run, one rank per GPU, each rank runs its own replica of
the step on its own block of R random vectors (vectors rank*R .. rank*R+R-1
of one ensemble: the vectors are independent, so they shard across ranks
with no data-path collective); after the timed region the moments of all
ranks are gathered once into one ensemble.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2509_06525_gb300 import synth  # noqa: E402

METRIC = "KPM atom*moments/s on 1 GB300 (learned FP32 vs plain FP64), % HBM roofline"
UNIT = "atom*moments/s"
L2_BYTES = 126 * 1024 * 1024

# DRAM bytes (read + write) per launch of the timed Chebyshev kernel, per row
# of the matrix, from ncu captures (dram__bytes_read.sum +
# dram__bytes_write.sum) of the same kernel instantiation on a smaller sheet
# of the same structure (see profiles/); scaled to a full launch by the rows
# processed.  Keyed by (precision, R, mode, shape description); any kernel
# without an entry, or changed since its capture, reports null.
def _shape_key(pipelined, cpt, stages, minb, rows_per_tile, options=0, band_rows=0):
    return tuple(sorted(dict(pipelined=pipelined, complex_per_thread=cpt, stages=stages, min_blocks=minb,
                             rows_per_tile=rows_per_tile, rows_per_thread=1, staged_vectors=1, options=options,
                             band_rows=band_rows).items()))


MEASURED_TRAFFIC_PER_ROW = {
    # profiles/traffic_cheb_step_small_cases.md: 2M-row thermal sheet, 558.3 MB per launch
    ("f32", 8, "doubling", _shape_key(1, 2, 2, 4, 64)): 558_285_312 / 2_000_000,
    # 8M-row pristine sheet, 762.9 MB per launch
    ("f32", 1, "doubling", _shape_key(3, 1, 2, 3, 256, 0, 1024)): 762_949_376 / 8_000_000,
    # 2M-row thermal sheet, banded step without CTA barriers, 512.9 MB per launch
    ("f32", 8, "doubling", _shape_key(3, 2, 2, 3, 64, 1, 320)): 512_879_104 / 2_000_000,
}


def measured_traffic(workload, hamiltonian, mode, M, R, shape_desc, n_atoms=None, prec="f32"):
    key = (prec, R, mode, tuple(sorted(shape_desc.items())))
    per_row = MEASURED_TRAFFIC_PER_ROW.get(key)
    if per_row is None or n_atoms is None:
        return None
    return int(per_row * n_atoms)


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="graphene-10M-learned", choices=list(synth.WORKLOADS))
    p.add_argument("--hamiltonian", choices=["mlp", "teacher"], default="mlp")
    p.add_argument("--kpm", choices=["doubling", "direct"], default="doubling",
                   help="moment formation: doubling identities (about M/2 steps) or one step per moment")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 teacher comparison run")
    p.add_argument("--train-epochs", type=int, default=None,
                   help="epochs of the untimed model training (default: the training default); fewer for profiling")
    p.add_argument("--M", type=int, default=None, help="override the workload's moment count (profiling)")
    p.add_argument("--R", type=int, default=None, help="override the workload's vector count (profiling)")
    p.add_argument("--sk", type=int, default=1, help="measure the s, p, d Slater-Koster KPM (1) or skip it (0)")
    p.add_argument("--env", type=int, default=600,
                   help="environment-network model: band-training steps (0 skips the measurement)")
    p.add_argument("--batched", type=int, default=1,
                   help="measure the 64-snapshot h-BN/graphene junction batch in one graph (1) or skip it (0)")
    p.add_argument("--headline", type=int, default=1,
                   help="measure the 1e8-atom graphene step after the main line (1) or skip it (0); 1 GPU only")
    p.add_argument("--precision", type=int, default=1,
                   help="measure FP32 against FP64 vectors on the 1e6-atom sheet, M = 2048, R = 16 (1) or skip (0)")
    p.add_argument("--lsqt-steps", type=int, default=2,
                   help="VAC conductivity time steps of 0.1 fs measured after the main line (0: skip)")
    p.add_argument("--kernel-case", default=None, metavar="NXxNY",
                   help="profiling case only (prints no JSON): on an NX x NY-cell graphene sheet, "
                        "--case-kernel cheb: teacher FP32 H, two kpm_moments calls (M = 64, doubling) with one "
                        "forced step shape; env: three environment-network H builds (random model); mlp: "
                        "three learned-H builds (random per-pair MLP)")
    p.add_argument("--case-kernel", choices=["cheb", "env", "mlp"], default="cheb")
    p.add_argument("--case-sigma", type=float, default=0.1, help="kernel case: thermal displacement (A)")
    p.add_argument("--case-shape", type=int, default=-1, help="kernel case: forced shape (-1: autotuned)")
    p.add_argument("--case-diag", type=int, default=1, help="kernel case: H carries its onsite diagonal (1) or not (0)")
    return p.parse_args()


def run_kernel_case(args):
    """A small fixed case for ncu captures of one Chebyshev-step shape."""
    import torch
    from paper_2509_06525_gb300 import build, gputb as g
    build.build()
    nx, ny = (int(v) for v in args.kernel_case.lower().split("x"))
    R = args.R or 8
    s = synth.graphene_rect(nx, ny, args.case_sigma, 1003)
    p = synth.teacher_graphene()
    pos = torch.tensor(s.positions, device="cuda")
    spc = torch.tensor(s.species, device="cuda")
    nb = g.build_neighbors(pos, s.box, s.pbc, p.rcut, r_count=p.r_count, max_width=16)
    if args.case_kernel != "cheb":
        cm = synth.descriptor_mixing("identity")
        if args.case_kernel == "env":
            model = g.EnvModel(synth.init_env_mlp(11, -1.0), cm, np.zeros(3))
        else:
            model = g.MLPModel(synth.init_mlp(3), cm, np.zeros(3))
            model.set_normalisation(torch.zeros(32, device="cuda"), torch.ones(32, device="cuda"))
        v = g.compute_descriptors(pos, spc, s.box, s.pbc, p.rcut, nb, model.cmix)
        for _ in range(3):
            if args.case_kernel == "env":
                H = g.build_hamiltonian_env(pos, spc, s.box, s.pbc, p.rcut, nb, model, v=v)
            else:
                H = g.build_hamiltonian(pos, spc, s.box, s.pbc, p.rcut, nb, model, v=v, dtype=torch.float32)
        torch.cuda.synchronize()
        print("kernel case", args.case_kernel, s.n, "rows,", int(nb.total), "slots, val[0]", float(H.val[0]))
        return
    H = g.build_hamiltonian_teacher(pos, spc, s.box, s.pbc, nb, p, dtype=torch.float32,
                                    with_diag=bool(args.case_diag))
    bd = g.spectral_bounds(H, 64, synth.LANCZOS_SEED)
    if args.case_shape >= 0:
        g.kpm_force_shape(R, torch.float32, args.case_shape)
    else:
        g.kpm_autotune(H, bd.a, bd.b, R, doubling=True, record=False)
    for _ in range(2):
        mu = g.kpm_moments(H, bd.a, bd.b, args.M or 64, R, synth.KPM_SEED, doubling=True)
    torch.cuda.synchronize()
    info = g.kpm_shape_info(R, torch.float32, g.kpm_get_shape(s.n, R, torch.float32, doubling=True))
    print("kernel case", s.n, "rows, R =", R, "shape", info, "mu0", float(mu[:, 0].mean()))


# ---------------------------------------------------------------- structure

def make_structure(name, M=None, R=None):
    w = dict(synth.WORKLOADS[name])
    if M:
        w["M"] = M
    if R:
        w["R"] = R
    if w["kind"] == "rect":
        return synth.graphene_rect(w["nx"], w["ny"], w["sigma"], w["seed"]), w
    if w["kind"] == "prim":
        return synth.graphene_primitive(w["n1"], w["n2"], w["sigma"], w["seed"]), w
    raise SystemExit(f"workload {name} is not a single-structure workload")


def teacher_for(s):
    return synth.teacher_hbn_graphene() if np.any(s.species != 0) else synth.teacher_graphene()


# ---------------------------------------------------------------- clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}", "--format=csv,noheader",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in csv.reader(io.StringIO(out)):
            if len(row) < 9:
                continue
            try:
                sm.append(float(row[1].split()[0]))
                mx.append(float(row[2].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, row[5:9]):
                if "Active" in v and "Not" not in v:
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- peaks

def measured_peak(key, fallback):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)[key])
    except (OSError, KeyError, ValueError):
        return fallback


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ---------------------------------------------------------------- our arm

class Pipeline:
    """Holds the device-resident inputs and runs one step through the binding."""

    def __init__(self, s, w, hamiltonian, rank, torch, g, model=None, doubling=True):
        self.torch, self.g = torch, g
        self.s, self.w = s, w
        self.M, self.R = w["M"], w["R"]
        self.seed = synth.KPM_SEED
        self.first_vector = rank * w["R"]
        self.teacher = teacher_for(s)
        self.hamiltonian = hamiltonian
        self.model = model
        self.teacher_diag = bool(np.any(self.teacher.onsite[np.unique(s.species)] != 0.0))
        self.pos = torch.tensor(s.positions, device="cuda")
        self.spc = torch.tensor(s.species, device="cuda")
        self.pos_host = torch.tensor(s.positions).pin_memory()
        self.spc_host = torch.tensor(s.species).pin_memory()
        self.kpm_ms = []
        self.last = {}
        self.doubling = doubling

    def step(self, pos, spc, kind, dtype, record=True, energies=None):
        """One pass: neighbours -> H (learned or teacher) -> bounds -> KPM -> DOS."""
        g, torch, s = self.g, self.torch, self.s
        nb = g.build_neighbors(pos, s.box, s.pbc, self.teacher.rcut, r_count=self.teacher.r_count, max_width=16)
        if kind == "mlp":
            v = g.compute_descriptors(pos, spc, s.box, s.pbc, self.teacher.rcut, nb, self.model.cmix)
            H = g.build_hamiltonian(pos, spc, s.box, s.pbc, self.teacher.rcut, nb, self.model, v=v, dtype=dtype,
                                    with_diag=True)
        else:
            H = g.build_hamiltonian_teacher(pos, spc, s.box, s.pbc, nb, self.teacher, dtype=dtype,
                                            with_diag=self.teacher_diag)
        bd = g.spectral_bounds(H, 64, synth.LANCZOS_SEED)
        timing = self.kpm_ms if record else None
        mu = g.kpm_moments(H, bd.a, bd.b, self.M, self.R, self.seed, timing=timing, doubling=self.doubling,
                           first_vector=self.first_vector)
        E = energies if energies is not None else torch.linspace(bd.emin, bd.emax, self.w["K"],
                                                                 dtype=torch.float64, device="cuda")
        rho = g.kpm_dos(mu, bd.a, bd.b, E)
        self.last = dict(nb=nb, H=H, bd=bd, mu=mu, rho=rho, E=E)
        return mu, rho

    def step_e2e(self, kind, dtype):
        """The step from page-locked host arrays: positions and species enter
        through tb_copy_to_device, the moments and the DOS leave through
        tb_copy_to_host (the C ABI's host boundary)."""
        g = self.g
        if not hasattr(self, "pos_e2e"):
            self.pos_e2e = torch_empty_like_device(self.pos_host)
            self.spc_e2e = torch_empty_like_device(self.spc_host)
            self.mu_host = self.torch.empty((self.R, self.M), dtype=self.torch.float64).pin_memory()
            self.rho_host = self.torch.empty(self.w["K"], dtype=self.torch.float64).pin_memory()
        g.copy_to_device(self.pos_e2e, self.pos_host)
        g.copy_to_device(self.spc_e2e, self.spc_host)
        mu, rho = self.step(self.pos_e2e, self.spc_e2e, kind, dtype, record=False)
        g.copy_to_host(self.mu_host, mu)
        g.copy_to_host(self.rho_host, rho)
        return self.mu_host, self.rho_host


def step_bytes(nnz, n_atoms, R, sv, sc, has_diag, doubling, shape_desc):
    """Algorithmic bytes of one Chebyshev-step launch: the matrix in the
    format the chosen shape reads (4-byte columns, or the banded step's 2-byte
    tile-local indices plus one 128-byte record per tile), the diagonal, and
    the vector streams (x gathered once, v_{n-1}, v_{n+1}, plus v0 in direct
    mode)."""
    streams = 3 if doubling else 4
    if shape_desc.get("pipelined") == 3:
        tiles = -(-n_atoms // shape_desc["rows_per_tile"])
        matrix = nnz * (sv + 2) + tiles * 128
    else:
        matrix = nnz * (sv + 4)
    return matrix + (n_atoms * sv if has_diag else 0) + n_atoms * R * streams * sc


def torch_empty_like_device(host):
    import torch
    return torch.empty(host.shape, dtype=host.dtype, device="cuda")


def timed(torch, dist, fn, steps, warmup):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = e0.elapsed_time(e1) / steps
    if dist is not None:
        from paper_2509_06525_gb300.distributed import max_over_ranks
        ms = max_over_ranks(ms, "cuda")
    return ms


def batched_measurement(torch, g, rank):
    """The hbn-junction-64 workload: 64 uneven junction snapshots (teacher
    FP32 H, Lanczos bounds each) whose KPM moments run as one CUDA graph;
    CUDA-event time of the graph (after a warm-up launch)."""
    w = synth.WORKLOADS["hbn-junction-64"]
    snaps = synth.junction_snapshots(w["count"], w["seed"], w["sigma"])
    p = synth.teacher_hbn_graphene()
    mats, a, b, atoms, nnz = [], [], [], 0, 0
    for s in snaps:
        pos = torch.tensor(s.positions, device="cuda")
        spc = torch.tensor(s.species, device="cuda")
        nb = g.build_neighbors(pos, s.box, s.pbc, p.rcut, r_count=p.r_count, max_width=16)
        H = g.build_hamiltonian_teacher(pos, spc, s.box, s.pbc, nb, p, dtype=torch.float32)
        bd = g.spectral_bounds(H, 64, synth.LANCZOS_SEED)
        mats.append(H)
        a.append(bd.a)
        b.append(bd.b)
        atoms += s.n
        nnz += nb.total
    seed = synth.KPM_SEED + 1000 * rank
    best, shape_ms = g.kpm_moments_batched_autotune(mats, a, b, w["R"], doubling=True, reps=10)
    t0 = time.perf_counter()
    mu = g.kpm_moments_batched(mats, a, b, w["M"], w["R"], seed, doubling=True)   # captures the graph
    torch.cuda.synchronize()
    first_call_s = time.perf_counter() - t0
    ms = []
    mu = g.kpm_moments_batched(mats, a, b, w["M"], w["R"], seed, doubling=True, timing=ms, mu=mu)
    launches = (w["M"] - 1) // 2 + 1
    n_pad = sum(-(-s.n // 256) * 256 for s in snaps)
    desc = g.kpm_shape_info(w["R"], torch.float32, best)
    launch_bytes = step_bytes(nnz, atoms, w["R"], 4, 8, True, True, desc)
    sell_bytes = step_bytes(nnz, atoms, w["R"], 4, 8, True, True, {"pipelined": 0})
    per = ms[0] / launches
    peak, src = hbm_peak()
    return {"workload": "hbn-junction-64", "snapshots": len(snaps), "atoms": atoms, "padded_rows": n_pad,
            "moments": w["M"], "random_vectors": w["R"], "ms": ms[0],
            "atom_moments_per_s": atoms * w["M"] / (ms[0] * 1e-3),
            "first_call_s": first_call_s,
            "autotune": {"shape": best, "shape_desc": desc, "ms_per_step": shape_ms},
            "roofline": {"bound": "hbm", "kernel": "cheb_step (segmented), shape %d" % best,
                         "bytes_per_launch": launch_bytes, "ms_per_launch": per,
                         "achieved": launch_bytes / (per * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": launch_bytes / (per * 1e-3) / 1e9 / peak, "peak_source": src,
                         "sell_equivalent_frac": sell_bytes / (per * 1e-3) / 1e9 / peak,
                         "note": "ms = the cached graph's launch: the fold of the 64 snapshots, the random "
                                 "phases, every step and the reduction (the first call, which captures and "
                                 "instantiates the graph, is first_call_s); rows padded to 256 per snapshot"},
            "mu0_mean": float(mu[:, :, 0].mean().item())}


def sk_measurement(pipe, torch, g):
    """The s, p, d Slater-Koster model on the same structure (9 orbitals per
    atom, matrix-free): compressed SK form, Gershgorin bounds and the KPM
    moments of one random vector with the workload's M; CUDA-event time of the
    moments (after a warm-up call)."""
    s = pipe.s
    sk = synth.teacher_sk_graphene()
    nb = g.build_neighbors(pipe.pos, s.box, s.pbc, sk.rcut, r_count=0.0)
    geom = g.sk_geometry(pipe.pos, s.box, s.pbc, nb, sk)
    emin, emax, a, b = g.sk_bounds(nb, geom, sk)
    g.sk_kpm_moments(nb, geom, sk, a, b, 64, pipe.seed, first_vector=pipe.first_vector)
    ms = []
    mu = g.sk_kpm_moments(nb, geom, sk, a, b, pipe.M, pipe.seed, first_vector=pipe.first_vector, timing=ms)
    launches = (pipe.M - 1) // 2 + 1
    per = ms[0] / launches
    nnz = nb.total
    launch_bytes = nnz * (13 * 4 + 4) + 3 * s.n * 9 * 8    # compressed SK form + col, x gathered once, v_{n-1}, v_{n+1}
    flops = nnz * 700                                       # ~45 table entries + 81 complex MACs per pair
    peak, src = hbm_peak()
    achieved = launch_bytes / (per * 1e-3) / 1e9
    out = {"orbitals": 9 * s.n, "moments": pipe.M, "random_vectors": 1, "ms": ms[0],
           "orbital_moments_per_s": 9 * s.n * pipe.M / (ms[0] * 1e-3),
           "bounds": {"emin": emin, "emax": emax},
           "roofline": {"bound": "hbm", "kernel": "sk_step (matrix-free SK block SpMV + moment dots)",
                        "bytes_per_launch": launch_bytes, "ms_per_launch": per, "achieved": achieved,
                        "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_source": src,
                        "fp32_tflops": flops / (per * 1e-3) / 1e12},
           "mu1": float(mu[1].item())}
    del geom, nb
    torch.cuda.empty_cache()
    return out


def env_measurement(pipe, torch, g, train_steps):
    """The environment-network model (Eq. 2 edge feature, SK-form hopping and
    onsite networks): its H on the workload's structure straight from the
    positions (CUDA-event time after a warm-up call), then band-energy
    training (Eq. 3) of a fresh model on 64 disordered 24-atom cells x 16
    k-points against the teacher's bands, timed per step."""
    from paper_2509_06525_gb300 import bands as bands_mod
    s, nb = pipe.s, pipe.last["nb"]
    cm = synth.descriptor_mixing("identity")
    model = g.EnvModel(synth.init_env_mlp(11, -1.0), cm, np.zeros(3))
    v = g.compute_descriptors(pipe.pos, pipe.spc, s.box, s.pbc, pipe.teacher.rcut, nb, model.cmix)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def time_h(variant):
        g.env_set_variant(variant)
        try:
            g.build_hamiltonian_env(pipe.pos, pipe.spc, s.box, s.pbc, pipe.teacher.rcut, nb, model, v=v)
            torch.cuda.synchronize()
            e0.record()
            H = g.build_hamiltonian_env(pipe.pos, pipe.spc, s.box, s.pbc, pipe.teacher.rcut, nb, model, v=v)
            e1.record()
            torch.cuda.synchronize()
        finally:
            g.env_set_variant(0)
        return e0.elapsed_time(e1), H

    ms_fp32, H32 = time_h(1)
    ms_h, H = time_h(0)
    nnz = int(nb.cnt.sum().item())
    real = H32.val.abs().max().item()
    dev = (H.val - H32.val).abs().max().item()
    rel_l2 = ((H.val - H32.val).double().norm() / H32.val.double().norm()).item()
    del H32
    # network FMAs per bond: 8x32 + 32x8 (environment) + 8x32 + 32x32 + 32x2 (hopping); per atom 8x32 + 32
    flops = 2 * (nnz * 1856 + s.n * 288)
    # issued on the tensor cores per bond: K x N = 16x32 + 32x16 + 16x32 + 32x32 + 32x16 (padded operands)
    tc_flops = 2 * nnz * 3072
    bf16_peak = measured_peak("bf16_tflops", 1900.0)
    tc_tflops = tc_flops / (ms_h * 1e-3) / 1e12
    h_out = {"atoms": s.n, "bonds": nnz, "ms": ms_h, "bonds_per_s": nnz / (ms_h * 1e-3),
             "kernel": "env_hopping_tc_kernel (tcgen05, BF16 operands, FP32 accumulation) + env_onsite_kernel",
             "fp32_pipes_ms": ms_fp32,
             "vs_fp32_pipes": {"max_abs_diff": dev, "max_abs_t": real, "rel_l2": rel_l2},
             "roofline": {"bound": "tensor", "unit": "TFLOP/s", "achieved": tc_tflops, "peak": bf16_peak,
                          "frac": tc_tflops / bf16_peak, "peak_source": "measured (bf16 burst)",
                          "network_tflops": flops / (ms_h * 1e-3) / 1e12,
                          "note": "MMA flops of the padded operands; the kernel is limited by the per-bond "
                                  "geometry, descriptors and activations around the MMAs, not by the tensor pipe"}}
    del H, v
    cells = synth.band_training_cells(64, 5000)
    kpts = synth.band_kgrid(cells[0].box, 4, 4)
    batch = bands_mod.build_cell_batch(cells, pipe.teacher, cm, kpts)
    fresh = g.EnvModel(synth.init_env_mlp(12, -1.0), cm, np.zeros(3))
    mae0 = bands_mod.band_mae(fresh, batch)
    third = max(train_steps // 3, 1)
    schedule = [(third, (8, 16)), (third, (4, 20)), (train_steps - 2 * third, (0, 24))]
    torch.cuda.synchronize()
    e0.record()
    bands_mod.train_bands(fresh, batch, schedule, lr=3e-3, log_every=max(train_steps, 1))
    e1.record()
    torch.cuda.synchronize()
    ms_t = e0.elapsed_time(e1)
    mae1 = bands_mod.band_mae(fresh, batch)
    spectra = len(cells) * len(kpts)
    return {"hamiltonian": h_out,
            "band_training": {"cells": len(cells), "atoms_per_cell": cells[0].n, "k_points": len(kpts),
                              "steps": train_steps, "ms_per_step": ms_t / train_steps,
                              "spectra_per_s": spectra * train_steps / (ms_t * 1e-3),
                              "band_mae_ev": {"before": mae0, "after": mae1},
                              "schedule": [[n_, list(w_)] for n_, w_ in schedule]}}


def lsqt_measurement(pipe, n_steps, torch, g, dt=0.1):
    """VAC conductivity (Eq. 3 (sigma)) on the last step's Hamiltonian: x
    velocity, the workload's M and R, n_steps time steps of 0.1 fs; CUDA-event
    time of the whole loop (after one warm-up call with no time step)."""
    H, bd, s = pipe.last["H"], pipe.last["bd"], pipe.s
    vval = g.velocity_values(pipe.pos, s.box, s.pbc, pipe.teacher.rcut, H, (1.0, 0.0, 0.0))
    # the VAC moment recursion runs the Chebyshev step in direct mode: tune
    # that mode's shape on this matrix too (untimed)
    best, _ = g.kpm_autotune(H, bd.a, bd.b, pipe.R, doubling=False)
    g.lsqt_vac(H, vval, bd.a, bd.b, pipe.M, pipe.R, pipe.seed, 0, dt, first_vector=pipe.first_vector)
    ms = []
    mu = g.lsqt_vac(H, vval, bd.a, bd.b, pipe.M, pipe.R, pipe.seed, n_steps, dt, first_vector=pipe.first_vector,
                    timing=ms)
    E = torch.tensor([bd.b - 0.3 * bd.a, bd.b, bd.b + 0.3 * bd.a], dtype=torch.float64, device="cuda")
    C, S = g.lsqt_correlation(mu, bd.a, bd.b, E, dt)
    t = ms[0] * 1e-3
    pts = n_steps + 1
    # launches of the matrix: M - 1 moment steps per time point, and per time
    # step two propagations of K Chebyshev-Bessel terms (the library's cut:
    # |J_k(a dt / hbar)| < 1e-17 beyond k = a dt / hbar + 2)
    from scipy.special import jv
    x = bd.a * dt / g.HBAR_EV_FS
    K = 0
    while not (K > x + 2 and abs(jv(K, x)) < 1e-17):
        K += 1
    spmv = pts * (pipe.M - 1) + 2 * n_steps * K
    nnz = int(pipe.last["nb"].cnt.sum().item())
    sv, sc = (4, 8) if H.val.dtype == torch.float32 else (8, 16)
    launch_bytes = nnz * (sv + 4) + (s.n * sv if H.diag is not None else 0) + 4 * s.n * pipe.R * sc
    per_spmv_ms = ms[0] / spmv
    peak, peak_src = hbm_peak()
    return {"time_points": pts, "dt_fs": dt, "moments": pipe.M, "random_vectors": pipe.R, "direction": "x",
            "ms": ms[0], "ms_per_time_point": ms[0] / pts,
            "atom_moments_timepoints_per_s": s.n * pipe.M * pts / t,
            "matrix_launches": spmv, "bessel_terms": K, "direct_mode_shape": best,
            "roofline": {"bound": "hbm", "kernel": "Chebyshev step (direct mode, dot with V phi_L)",
                         "bytes_per_launch": launch_bytes, "ms_per_launch": per_spmv_ms,
                         "achieved": launch_bytes / (per_spmv_ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": launch_bytes / (per_spmv_ms * 1e-3) / 1e9 / peak, "peak_source": peak_src,
                         "note": "whole-loop time over all matrix launches (moment steps, propagation terms); "
                                 "bytes counted with 4-byte SELL columns whatever the step shape reads"},
            "C_at_E": [float(v) for v in C[0].cpu()], "S_end_at_E": [float(v) for v in S[-1].cpu()],
            "units": "C: A^2/fs^2/eV per orbital, S: A^2/fs/eV per orbital (sigma = 2 e^2 N / Omega * S)"}


def headline_measurement(torch, g, dist, steps, warmup):
    """The 1e8-atom pristine graphene sheet (graphene-100M: teacher FP32 H in
    SELL-32, complex FP32 vectors, R = 1, M = 1024, doubling mode, Jackson DOS
    on 4001 points): the whole step timed like the main line, after
    autotuning the Chebyshev step on this matrix; roofline of the step
    kernel from its CUDA-event time inside kpm_moments."""
    s, w = make_structure("graphene-100M")
    pipe = Pipeline(s, w, "teacher", 0, torch, g, None, doubling=True)
    pipe.step(pipe.pos, pipe.spc, "teacher", torch.float32, record=False)
    H, bd = pipe.last["H"], pipe.last["bd"]
    best, shape_ms = g.kpm_autotune(H, bd.a, bd.b, w["R"], doubling=True, reps=10)
    del H, bd
    pipe.kpm_ms.clear()
    sampler = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    for _ in range(warmup):
        pipe.step(pipe.pos, pipe.spc, "teacher", torch.float32, record=False)
    sampler.start()
    ms = timed(torch, dist, lambda: pipe.step(pipe.pos, pipe.spc, "teacher", torch.float32), steps, 0)
    clocks = sampler.stop()
    nb, H = pipe.last["nb"], pipe.last["H"]
    nnz = int(nb.cnt.sum().item())
    used = g.kpm_get_shape(s.n, w["R"], torch.float32, True)
    desc = g.kpm_shape_info(w["R"], torch.float32, used)
    launches = (w["M"] - 1) // 2 + 1
    launch_ms = sum(pipe.kpm_ms) / (len(pipe.kpm_ms) * launches)
    lb = step_bytes(nnz, s.n, w["R"], 4, 8, H.diag is not None, True, desc)
    lb_sell = step_bytes(nnz, s.n, w["R"], 4, 8, H.diag is not None, True, {"pipelined": 0})
    peak, src = hbm_peak()
    out = {"workload": "graphene-100M", "atoms": s.n, "moments": w["M"], "random_vectors": w["R"],
           "value": s.n * w["M"] / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
           "kpm_share_of_step": sum(pipe.kpm_ms) / (ms * steps),
           "roofline": {"bound": "hbm", "kernel": "cheb_step, shape %d" % used, "shape": desc,
                        "bytes_per_launch": lb, "launch_ms": launch_ms,
                        "achieved": lb / (launch_ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                        "frac": lb / (launch_ms * 1e-3) / 1e9 / peak, "peak_source": src,
                        "traffic": measured_traffic("graphene-100M", "teacher", "doubling", w["M"], w["R"], desc,
                                                    s.n),
                        "sell_equivalent_frac": lb_sell / (launch_ms * 1e-3) / 1e9 / peak,
                        "note": "sell_equivalent_frac counts the 4-byte-column SELL bytes of the same step"},
           "autotune": {"shape": best, "ms_per_step": shape_ms,
                        "shapes": [g.kpm_shape_info(w["R"], torch.float32, k) for k in range(len(shape_ms))]},
           "clocks": clocks, "mu0_mean": float(pipe.last["mu"][:, 0].mean().item())}
    del pipe, nb, H
    torch.cuda.empty_cache()
    return out


def million_atom_precision(torch, g):
    """The 1,000,000-atom 300 K graphene sheet (graphene-1M-300K: teacher H,
    M = 2048 moments, R = 16 vectors in one blocked SpMM, FP64 moment sums,
    Lanczos bounds), run with complex FP32 vectors (FP32 values) and with
    complex FP64 vectors (FP64 values) on the same GPU, both autotuned;
    CUDA-event time of the recursion; max |mu32_n - mu64_n| over the vectors
    per block of 256 moments (the FP64 path is pinned to the FP64 oracle at
    1e-12 by the parity tests)."""
    s, w = make_structure("graphene-1M-300K")
    p = teacher_for(s)
    pos = torch.tensor(s.positions, device="cuda")
    spc = torch.tensor(s.species, device="cuda")
    nb = g.build_neighbors(pos, s.box, s.pbc, p.rcut, r_count=p.r_count, max_width=16)
    nnz = int(nb.cnt.sum().item())
    peak, src = hbm_peak()
    res, mus = {}, {}
    for name, dt, sv, sc in (("fp32", torch.float32, 4, 8), ("fp64", torch.float64, 8, 16)):
        H = g.build_hamiltonian_teacher(pos, spc, s.box, s.pbc, nb, p, dtype=dt)
        bd = g.spectral_bounds(H, 64, synth.LANCZOS_SEED)
        best, shape_ms = g.kpm_autotune(H, bd.a, bd.b, w["R"], doubling=True, reps=20)
        g.kpm_moments(H, bd.a, bd.b, w["M"], w["R"], synth.KPM_SEED, doubling=True)
        ms = []
        mus[name] = g.kpm_moments(H, bd.a, bd.b, w["M"], w["R"], synth.KPM_SEED, doubling=True,
                                  timing=ms).cpu().numpy()
        launches = (w["M"] - 1) // 2 + 1
        desc = g.kpm_shape_info(w["R"], dt, best)
        lb = step_bytes(nnz, s.n, w["R"], sv, sc, H.diag is not None, True, desc)
        per = ms[0] / launches
        res[name] = {"ms": ms[0], "atom_moments_per_s": s.n * w["M"] / (ms[0] * 1e-3),
                     "shape": desc, "autotune_ms_per_step": shape_ms,
                     "roofline": {"bound": "hbm" if sv == 4 else "fp64 alu", "bytes_per_launch": lb,
                                  "ms_per_launch": per, "achieved": lb / (per * 1e-3) / 1e9, "peak": peak,
                                  "unit": "GB/s", "frac": lb / (per * 1e-3) / 1e9 / peak, "peak_source": src}}
        del H
    d = abs(mus["fp32"] - mus["fp64"]).max(axis=0)
    res["max_abs_dmu_per_256_moments"] = [float(d[k:k + 256].max()) for k in range(0, w["M"], 256)]
    res["max_abs_dmu"] = float(d.max())
    res["speedup_fp32_over_fp64"] = res["fp64"]["ms"] / res["fp32"]["ms"]
    del nb, pos, spc
    torch.cuda.empty_cache()
    return {"workload": "graphene-1M-300K", "atoms": s.n, "moments": w["M"], "random_vectors": w["R"], **res}


# ---------------------------------------------------------------- CPU oracle (baseline legs only)

_ORACLE_STATE = {}


def _oracle_sample(workload):
    """A 200k-atom sheet of the workload's structure (same lattice, sigma and
    seed), its oracle teacher Hamiltonian and bounds."""
    from oracle import bounds as obo, hamiltonian as oha, neighbors as onb, teacher as ote
    w = synth.WORKLOADS[workload]
    nx = min(w.get("nx", 250), 250)
    ny = min(w.get("ny", 200), 200)
    s = synth.graphene_rect(nx, ny, w["sigma"], w["seed"])
    p = teacher_for(s)
    indptr, idx, d = onb.neighbors(s.positions, s.box, s.pbc, p.rcut)
    t, eps, _ = ote.teacher_elements(s.species, indptr, idx, d, p)
    H = oha.csr_hamiltonian(s.n, indptr, idx, t, eps)
    _, _, a, b = obo.spectral_bounds(H, 64, synth.LANCZOS_SEED)
    return s, H, a, b


def _oracle_init(workload):
    from oracle import kpm as okpm
    s, H, a, b = _oracle_sample(workload)
    _ORACLE_STATE["Ht"] = okpm.rescale(H, a, b)
    _ORACLE_STATE["n"] = s.n


def _oracle_block(job):
    from oracle import kpm as okpm
    first, count, m = job
    v0 = okpm.random_phase_vectors(synth.KPM_SEED, _ORACLE_STATE["n"], count, first)
    t0 = time.perf_counter()
    okpm.chebyshev_moments(_ORACLE_STATE["Ht"], v0, m)
    return time.perf_counter() - t0


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


class OraclePool:
    """The FP64 oracle's KPM over blocks of random vectors in a pool of
    worker processes (spawned), one block per worker: the vectors of the
    stochastic trace are independent, so this runs the unmodified oracle on
    several host cores at once.  Each worker builds the sample Hamiltonian
    once, outside the timed calls."""

    def __init__(self, workload, R):
        import multiprocessing as mp
        self.R = R
        self.workers = max(1, min(R, os.cpu_count() or 1))
        per = -(-R // self.workers)
        self.blocks = [(f, min(per, R - f)) for f in range(0, R, per)]
        self.pool = mp.get_context("spawn").Pool(len(self.blocks), initializer=_oracle_init, initargs=(workload,))
        self.pool.map(_oracle_block, [(f, c, 2) for f, c in self.blocks])   # warm the workers

    def run(self, m):
        t0 = time.perf_counter()
        self.pool.map(_oracle_block, [(f, c, m) for f, c in self.blocks])
        return time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(workload, budget_s=12.0):
    """The FP64 oracle's KPM on a bounded sample of the same workload, on one
    host core and on several (a pool over vector blocks)."""
    from oracle import kpm as okpm
    w = synth.WORKLOADS[workload]
    s, H, a, b = _oracle_sample(workload)
    Ht = okpm.rescale(H, a, b)
    v0 = okpm.random_phase_vectors(synth.KPM_SEED, s.n, w["R"])
    # one core: double the moments until the budget is spent (the per-step cost is constant)
    m = 2
    while True:
        t0 = time.perf_counter()
        okpm.chebyshev_moments(Ht, v0, m)
        el = time.perf_counter() - t0
        if el > budget_s / 4 or m >= w["M"]:
            break
        m *= 2
    one = s.n * m / el
    pool = OraclePool(workload, w["R"])
    try:
        el_all = pool.run(m)
    finally:
        pool.close()
    many = s.n * m / el_all
    best_many = many >= one
    return {"value": max(one, many), "unit": UNIT, "cores": pool.workers if best_many else 1, "kind": "oracle",
            "value_1_core": one, "value_all_cores": many, "cores_all": pool.workers,
            "cores_on_host": os.cpu_count(), "cpu_model": cpu_model(),
            "sample": f"FP64 oracle KPM (SciPy CSR) on a {s.n}-atom sheet of the same graphene workload "
                      f"(sigma={w['sigma']} A), R={w['R']} vectors, {m} moments, teacher H; `value_1_core` in "
                      f"one process (all R vectors in one sparse product), `value_all_cores` with the vectors "
                      f"split over {pool.workers} worker processes; `value` is the faster of the two; not "
                      f"extrapolated"}


def run_ours(args):
    import torch
    import torch.distributed as dist_mod
    from paper_2509_06525_gb300 import build, gputb as g

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        torch.cuda.set_device(local)
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    build.build()
    s, w = make_structure(args.workload, args.M, args.R)
    model, training = None, None
    if args.hamiltonian == "mlp":
        from paper_2509_06525_gb300 import train as tr
        t0 = time.perf_counter()
        cfg = tr.TrainConfig() if args.train_epochs is None else tr.TrainConfig(epochs=args.train_epochs)
        model, hist = tr.train_graphene_model(cfg=cfg)
        torch.cuda.synchronize()
        training = {"snapshots": synth.TRAIN_SNAPSHOTS, "atoms_per_snapshot": 800,
                    "epochs": cfg.epochs, "seconds": time.perf_counter() - t0,
                    "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1]}
    pipe = Pipeline(s, w, args.hamiltonian, rank, torch, g, model, doubling=args.kpm == "doubling")
    kind = args.hamiltonian
    lib = g.lib()

    # autotune the Chebyshev step on this workload's own matrix (untimed),
    # then the warm-up steps with the chosen shape
    pipe.step(pipe.pos, pipe.spc, kind, torch.float32, record=False)
    H0, bd0 = pipe.last["H"], pipe.last["bd"]
    best, shape_ms = g.kpm_autotune(H0, bd0.a, bd0.b, w["R"], doubling=pipe.doubling, reps=20)
    autotune = {"shape": best, "shape_desc": g.kpm_shape_info(w["R"], torch.float32, best),
                "ms_per_step": shape_ms, "default_shape_ms": shape_ms[0],
                "shapes": [g.kpm_shape_info(w["R"], torch.float32, k) for k in range(len(shape_ms))]}
    del H0, bd0

    # device-resident timed region
    sampler = ClockSampler(local)
    pipe.kpm_ms.clear()
    for _ in range(args.warmup):
        pipe.step(pipe.pos, pipe.spc, kind, torch.float32, record=False)
    torch.cuda.synchronize()
    l0 = lib.tb_launch_count()
    sampler.start()
    ms = timed(torch, dist, lambda: pipe.step(pipe.pos, pipe.spc, kind, torch.float32), args.steps, 0)
    clocks = sampler.stop()
    launches = lib.tb_launch_count() - l0
    n_atoms, M, R = s.n, w["M"], w["R"]
    value = world * n_atoms * M / (ms * 1e-3)

    # roofline of the dominant kernel (the fused Chebyshev step)
    nb, H = pipe.last["nb"], pipe.last["H"]
    nnz = int(nb.cnt.sum().item())
    used_shape = g.kpm_get_shape(n_atoms, R, torch.float32, pipe.doubling)
    used_desc = g.kpm_shape_info(R, torch.float32, used_shape)
    launch_bytes = step_bytes(nnz, n_atoms, R, 4, 8, H.diag is not None, pipe.doubling, used_desc)
    sell_bytes = step_bytes(nnz, n_atoms, R, 4, 8, H.diag is not None, pipe.doubling, {"pipelined": 0})
    launches_per_kpm = (M - 1) // 2 + 1 if pipe.doubling else M - 1
    launch_ms = sum(pipe.kpm_ms) / (len(pipe.kpm_ms) * launches_per_kpm)
    achieved = launch_bytes / (launch_ms * 1e-3) / 1e9
    peak, peak_src = hbm_peak()
    kpm_frac_of_step = sum(pipe.kpm_ms) / (ms * args.steps)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "per_vector": {"value": value * R, "unit": "atom*moments*vectors/s",
                       "note": "N M R / t: the same step counted per random vector"},
        "config": {"workload": args.workload + ("" if (args.M is None and args.R is None) else "-override"),
                   "atoms": n_atoms, "moments": M, "random_vectors": R,
                   "hamiltonian": args.hamiltonian, "kpm_precision": "complex FP32, FP64 moment sums",
                   "kpm_moments": ("doubling identities, %d Chebyshev steps" % launches_per_kpm
                                   if pipe.doubling else "direct, %d Chebyshev steps" % launches_per_kpm),
                   "l2": "inputs larger than L2 (ELL and vector blocks >> 126 MB)",
                   "step": "neighbours + H build + FP64 bounds + KPM + Jackson DOS"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": measured_traffic(args.workload, args.hamiltonian, args.kpm, M, R, used_desc,
                                                 n_atoms),
                     "kernel": "cheb_step (fused Chebyshev step + moment dots), shape %d" % used_shape,
                     "shape": used_desc,
                     "bytes_per_launch": launch_bytes, "launch_ms": launch_ms, "peak_source": peak_src,
                     "kpm_share_of_step": kpm_frac_of_step,
                     "sell_equivalent_frac": sell_bytes / (launch_ms * 1e-3) / 1e9 / peak,
                     "note": "frac counts the bytes of the format the chosen shape reads; "
                             "sell_equivalent_frac the 4-byte-column SELL bytes of the same step"},
        "gpu_launches": launches,
        "clocks": clocks,
        "autotune": autotune,
    }

    if training is not None:
        out["training"] = training

    if dist is not None:
        # one ensemble from all ranks' vector blocks (outside the timed region)
        from paper_2509_06525_gb300.distributed import gather_moments
        mu_all = gather_moments(pipe.last["mu"], R * world)
        out["ensemble"] = {"random_vectors": int(mu_all.shape[0]), "ranks": world,
                           "mu0_mean": float(mu_all[:, 0].mean().item())}

    # the conductivity on the timed step's own (FP32) Hamiltonian, before the
    # FP64 comparison below replaces it
    if args.lsqt_steps > 0:
        out["lsqt"] = lsqt_measurement(pipe, args.lsqt_steps, torch, g)
    if args.sk:
        out["sk"] = sk_measurement(pipe, torch, g)
    if args.batched:
        out["batched"] = batched_measurement(torch, g, rank)
    if args.env > 0:
        out["env_model"] = env_measurement(pipe, torch, g, args.env)

    # plain FP64 teacher form on the same structure and GPU, and the DOS
    # error of the timed (learned FP32 by default) path against it
    if not args.no_fp64:
        rho32, E32 = pipe.last["rho"], pipe.last["E"]
        ms64 = timed(torch, dist, lambda: pipe.step(pipe.pos, pipe.spc, "teacher", torch.float64, record=False,
                                                    energies=E32), max(1, args.steps // 2), 1)
        rho64 = pipe.last["rho"]
        l1 = float((rho32 - rho64).abs().sum() / rho64.abs().sum())
        value64 = world * n_atoms * M / (ms64 * 1e-3)
        out["fp64_teacher"] = {"value": value64, "ms_per_step": ms64, "speedup_of_value": value / value64,
                               "dos_l1_vs_fp64_teacher": l1}

    if not args.no_e2e:
        ms_e2e = timed(torch, dist, lambda: pipe.step_e2e(kind, torch.float32), args.steps, 1)
        h2d = s.positions.nbytes + s.species.nbytes
        d2h = R * M * 8 + w["K"] * 8
        out["e2e"] = {"value": world * n_atoms * M / (ms_e2e * 1e-3), "unit": UNIT,
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e}

    if world == 1 and (args.headline or args.precision):
        # the other workloads, after this one's buffers are freed
        del pipe, nb, H
        torch.cuda.empty_cache()
        if args.precision:
            out["graphene_1M_fp32_vs_fp64"] = million_atom_precision(torch, g)
        if args.headline:
            out["graphene_100M_headline"] = headline_measurement(torch, g, dist, max(args.steps, 2), 2)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload)

    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = synth.WORKLOADS[args.workload]
    m = 64
    pool = OraclePool(args.workload, w["R"])
    try:
        s, _, _, _ = _oracle_sample(args.workload)
        for _ in range(args.warmup):
            pool.run(m)
        t = [pool.run(m) for _ in range(args.steps)]
    finally:
        pool.close()
    sec = sum(t) / len(t)
    value = s.n * m / sec
    sample = (f"FP64 oracle KPM (SciPy CSR) on a {s.n}-atom sheet of the same graphene workload, R={w['R']} "
              f"vectors split over {pool.workers} worker processes, {m} moments per step, teacher H")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "atoms": s.n, "moments": m, "random_vectors": w["R"],
                      "hamiltonian": "teacher"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.workers, "kind": "oracle",
                            "sample": sample, "cpu_model": cpu_model(), "cores_on_host": os.cpu_count()},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse_args()
    if args.kernel_case:
        run_kernel_case(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
