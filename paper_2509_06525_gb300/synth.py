"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module produces *inputs only*: lattice positions, species, boxes, Gaussian
thermal displacements, snapshot sizes, random MLP initial weights and model
constants.  It holds none of the method's arithmetic (no neighbour search, no
Hamiltonian, no KPM), so both the CUDA path and the independent FP64 oracle can
consume what it produces without sharing any computation.

Geometry follows the structures the paper computes on (graphene, h-BN/graphene
lateral junctions; Sec. 3, Fig. 4) with the finite-temperature MD snapshots of
Sec. 2.2 replaced by seeded Gaussian displacements of every Cartesian
component.

Conventions
-----------
* positions: float64 [N, 3] (Angstrom), C-contiguous.
* species:   int32 [N]; 0 = C, 1 = B, 2 = N.
* box:       float64 [3, 3]; row k is lattice vector a_k.  Rows have the
             lower-triangular form a1 = (ax, 0, 0), a2 = (bx, by, 0),
             a3 = (cx, cy, cz).
* pbc:       int32 [3]; graphene sheets are periodic in-plane only.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

A_CC = 1.42          # carbon-carbon bond length (Angstrom)
VACUUM_Z = 20.0      # height of the (non-periodic) box along z
SPECIES_C, SPECIES_B, SPECIES_N = 0, 1, 2
N_SPECIES = 3


@dataclass
class Structure:
    positions: np.ndarray            # float64 [N, 3]
    species: np.ndarray              # int32 [N]
    box: np.ndarray                  # float64 [3, 3]
    pbc: np.ndarray = field(default_factory=lambda: np.array([1, 1, 0], np.int32))
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.positions.shape[0])


def _displace(pos: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    if sigma > 0.0:
        rng = np.random.default_rng(seed)
        pos = pos + rng.normal(0.0, sigma, size=pos.shape)
    return np.ascontiguousarray(pos, dtype=np.float64)


def graphene_primitive(n1: int, n2: int, sigma: float = 0.0, seed: int = 0,
                       a_cc: float = A_CC) -> Structure:
    """Graphene on the 2-atom primitive (60-degree, triclinic) cell.

    a1 = a (1, 0, 0), a2 = a (1/2, sqrt(3)/2, 0) with a = sqrt(3) a_cc; basis
    (0, 0, 0) and (a1 + a2) / 3.  Atom index = ((c2 * n1) + c1) * 2 + b.
    """
    a = math.sqrt(3.0) * a_cc
    a1 = np.array([a, 0.0, 0.0])
    a2 = np.array([0.5 * a, 0.5 * math.sqrt(3.0) * a, 0.0])
    basis = np.stack([np.zeros(3), (a1 + a2) / 3.0])
    c2, c1, b = np.meshgrid(np.arange(n2), np.arange(n1), np.arange(2), indexing="ij")
    pos = (c1[..., None] * a1 + c2[..., None] * a2 + basis[b]).reshape(-1, 3)
    box = np.stack([n1 * a1, n2 * a2, np.array([0.0, 0.0, VACUUM_Z])])
    species = np.zeros(pos.shape[0], np.int32)
    return Structure(_displace(pos, sigma, seed), species, box,
                     name=f"graphene-prim-{n1}x{n2}")


def rect_cell_basis(a_cc: float = A_CC):
    """The 4-atom rectangular (armchair-along-x) graphene cell.

    Cell 3 a_cc by sqrt(3) a_cc; basis (0,0), (a_cc,0), (1.5a_cc, h),
    (2.5a_cc, h) with h = sqrt(3) a_cc / 2.  Basis atoms 0 and 2 lie on one
    sublattice (A), 1 and 3 on the other (B).
    """
    h = 0.5 * math.sqrt(3.0) * a_cc
    basis = np.array([[0.0, 0.0, 0.0], [a_cc, 0.0, 0.0],
                      [1.5 * a_cc, h, 0.0], [2.5 * a_cc, h, 0.0]])
    return 3.0 * a_cc, math.sqrt(3.0) * a_cc, basis


def graphene_rect(nx: int, ny: int, sigma: float = 0.0, seed: int = 0,
                  a_cc: float = A_CC) -> Structure:
    """Graphene on nx * ny rectangular 4-atom cells (N = 4 nx ny).

    Atom index = ((cy * nx) + cx) * 4 + b, so atoms are cell-ordered.
    """
    lx, ly, basis = rect_cell_basis(a_cc)
    cy, cx, b = np.meshgrid(np.arange(ny), np.arange(nx), np.arange(4), indexing="ij")
    pos = np.empty((cy.size, 3))
    pos[:, 0] = (cx * lx).reshape(-1) + basis[b.reshape(-1), 0]
    pos[:, 1] = (cy * ly).reshape(-1) + basis[b.reshape(-1), 1]
    pos[:, 2] = 0.0
    box = np.array([[nx * lx, 0.0, 0.0], [0.0, ny * ly, 0.0], [0.0, 0.0, VACUUM_Z]])
    species = np.zeros(pos.shape[0], np.int32)
    return Structure(_displace(pos, sigma, seed), species, box,
                     name=f"graphene-rect-{nx}x{ny}")


def sublattice_sign(nx: int, ny: int) -> np.ndarray:
    """+1 on sublattice A, -1 on sublattice B for graphene_rect ordering."""
    return np.tile(np.array([1.0, -1.0, 1.0, -1.0]), nx * ny)


def hbn_graphene_junction(nx: int, ny: int, sigma: float = 0.0, seed: int = 0,
                          a_cc: float = A_CC) -> Structure:
    """Lateral h-BN/graphene junction on a common honeycomb lattice.

    The left nx/2 cell columns are h-BN (B on sublattice A, N on sublattice
    B); the right columns are carbon.  Periodic in x and y, so the sheet has
    two interfaces.
    """
    s = graphene_rect(nx, ny, sigma, seed, a_cc)
    cx = (np.arange(s.n) // 4) % nx
    b = np.arange(s.n) % 4
    left = cx < nx // 2
    species = np.full(s.n, SPECIES_C, np.int32)
    species[left & ((b == 0) | (b == 2))] = SPECIES_B
    species[left & ((b == 1) | (b == 3))] = SPECIES_N
    s.species = species
    s.name = f"hbn-graphene-{nx}x{ny}"
    return s


def junction_snapshot_shapes(count: int, seed: int, n_min: int = 5000,
                             n_max: int = 200000):
    """Uneven snapshot sizes, log-uniform on [n_min, n_max] atoms.

    Returns a list of (nx, ny) rectangular-cell counts with
    nx = 2 ceil(sqrt(Ns/4)/2) and ny = max(3, round(Ns / (4 nx))).
    """
    rng = np.random.default_rng(seed)
    out = []
    for u in rng.uniform(math.log(n_min), math.log(n_max), size=count):
        ns = math.exp(u)
        nx = 2 * math.ceil(math.sqrt(ns / 4.0) / 2.0)
        ny = max(3, int(round(ns / (4.0 * nx))))
        out.append((nx, ny))
    return out


def junction_snapshots(count: int = 64, seed: int = 4000, sigma: float = 0.1):
    return [hbn_graphene_junction(nx, ny, sigma, seed + k)
            for k, (nx, ny) in enumerate(junction_snapshot_shapes(count, seed))]


# --------------------------------------------------------------------------
# Model constants (inputs to both sides; no arithmetic of the method here).
# --------------------------------------------------------------------------

@dataclass
class TeacherParams:
    """Analytic environment-dependent teacher TB model (pz, one orbital/atom).

    t_ij = P[Zi, Zj] exp(-beta (r/a_cc - 1)) (1 + gamma (n_i + n_j - 6)/6) f_c(r)
    eps_i = onsite[Zi], n_i = #neighbours closer than r_count.
    """
    hop_prefactor: np.ndarray       # float64 [3, 3] (eV), symmetric
    onsite: np.ndarray              # float64 [3] (eV)
    a_cc: float = A_CC
    beta: float = 3.0
    gamma: float = 0.05
    r_count: float = 1.8
    rcut: float = 3.0


def teacher_graphene() -> TeacherParams:
    p = np.full((3, 3), -2.7)
    return TeacherParams(p, np.zeros(3))


def teacher_hbn_graphene() -> TeacherParams:
    p = np.empty((3, 3))
    c, b, n = SPECIES_C, SPECIES_B, SPECIES_N
    p[c, c] = -2.7
    p[b, n] = p[n, b] = -2.3
    p[b, c] = p[c, b] = -2.0
    p[n, c] = p[c, n] = -2.5
    p[b, b] = p[n, n] = -2.3
    onsite = np.zeros(3)
    onsite[b], onsite[n] = 2.3, -2.1
    return TeacherParams(p, onsite)


@dataclass
class SKTeacher:
    """Synthetic s, p, d Slater-Koster teacher for carbon (no trained
    network here): the ten two-centre integrals (eV) in the order ss_sigma,
    sp_sigma, pp_sigma, pp_pi, sd_sigma, pd_sigma, pd_pi, dd_sigma, dd_pi,
    dd_delta, each with the distance form V0 exp(-beta (r/a_cc - 1)) f_c(r),
    and onsite energies E_s, E_p, E_d.  The numbers are synthetic."""
    v0: np.ndarray
    onsite: np.ndarray
    a_cc: float = 1.42
    beta: float = 3.0
    rcut: float = 3.0


def teacher_sk_graphene() -> SKTeacher:
    return SKTeacher(np.array([-5.0, 5.4, 6.2, -2.9, -2.0, -2.4, 1.2, -1.8, 1.0, -0.3]),
                     np.array([-7.5, 0.0, 14.0]))


N_BASIS = 8          # radial Chebyshev functions f_0..f_7
N_FEAT = 32          # per-edge MLP input width
N_HIDDEN = 64
N_OUT = 2            # (hopping, onsite share)


def descriptor_mixing(kind: str = "identity") -> np.ndarray:
    """Species-pair mixing matrices c^{Zi Zj}_{nk}, float32 [3, 3, 8, 8].

    'identity': c = I for every pair (single-species graphene).
    'species':  c = diag(s_p) with a distinct fixed positive scale vector per
                ordered pair p, so the network can tell bond types apart.
    """
    c = np.zeros((N_SPECIES, N_SPECIES, N_BASIS, N_BASIS), np.float32)
    for zi in range(N_SPECIES):
        for zj in range(N_SPECIES):
            if kind == "identity":
                c[zi, zj] = np.eye(N_BASIS)
            else:
                k = np.arange(N_BASIS)
                scale = 1.0 + 0.25 * zi + 0.125 * zj + 0.03125 * ((k * (zi + 1) + zj) % 5)
                c[zi, zj] = np.diag(scale)
    return c


def init_mlp(seed: int):
    """He-uniform initial weights of the 32-64-64-2 MLP (float32).

    Returns dict W1 [64,32], b1 [64], W2 [64,64], b2 [64], W3 [2,64], b3 [2].
    """
    rng = np.random.default_rng(seed)
    dims = [(N_HIDDEN, N_FEAT), (N_HIDDEN, N_HIDDEN), (N_OUT, N_HIDDEN)]
    out = {}
    for k, (o, i) in enumerate(dims, start=1):
        lim = math.sqrt(6.0 / i)
        out[f"W{k}"] = rng.uniform(-lim, lim, size=(o, i)).astype(np.float32)
        out[f"b{k}"] = np.zeros(o, np.float32)
    return out



# Shapes of the environment-network model, in the order of its flat
# parameter vector (weights [out][in] row-major, then biases): environment
# network 8-32-8, hopping network 8-32-32-2 (sigma, pi), onsite network 8-32-3.
ENV_SHAPES = ((32, 8), (32,), (8, 32), (8,),
              (32, 8), (32,), (32, 32), (32,), (2, 32), (2,),
              (32, 8), (32,), (3, 32), (3,))
ENV_NPARAM = sum(int(np.prod(s)) for s in ENV_SHAPES)


def init_env_mlp(seed: int, bias_pi: float = 0.0) -> np.ndarray:
    """He-uniform weights of the environment-network model as one flat
    float32 vector (biases zero except the pi output's, set to bias_pi)."""
    rng = np.random.default_rng(seed)
    out = []
    for s in ENV_SHAPES:
        if len(s) == 2:
            lim = math.sqrt(6.0 / s[1])
            out.append(rng.uniform(-lim, lim, size=s).reshape(-1))
        else:
            out.append(np.zeros(s))
    flat = np.concatenate(out).astype(np.float32)
    # the pi output bias sits after Wh3 in the hopping network's block
    off = sum(int(np.prod(s)) for s in ENV_SHAPES[:9]) + 1
    flat[off] = bias_pi
    return flat


def band_kgrid(box: np.ndarray, n1: int, n2: int) -> np.ndarray:
    """Shifted Monkhorst-Pack grid (k_z = 0) of an orthorhombic in-plane cell,
    Cartesian k in 1/Angstrom, [n1 * n2, 3] float64."""
    b1 = 2.0 * math.pi / box[0, 0]
    b2 = 2.0 * math.pi / box[1, 1]
    f1 = (np.arange(n1) + 0.5) / n1 - 0.5
    f2 = (np.arange(n2) + 0.5) / n2 - 0.5
    k1, k2 = np.meshgrid(f1, f2, indexing="ij")
    return np.stack([k1.reshape(-1) * b1, k2.reshape(-1) * b2, np.zeros(n1 * n2)], axis=1)


def band_training_cells(count: int, seed_base: int = 5000, nx: int = 2, ny: int = 3, sigma: float = 0.1):
    """Periodic graphene cells of nx * ny rectangular 4-atom cells (24 atoms
    at 2 x 3), displaced with sigma: the finite-temperature training cells
    of the band-energy fit."""
    return [graphene_rect(nx, ny, sigma, seed_base + s) for s in range(count)]

# --------------------------------------------------------------------------
# The five workloads (sizes and seeds).
# --------------------------------------------------------------------------

WORKLOADS = {
    "graphene-800-fp64": dict(kind="prim", n1=20, n2=20, sigma=0.05, seed=1001,
                              M=512, R=8, K=2001),
    "graphene-1M-300K": dict(kind="rect", nx=500, ny=500, sigma=0.1, seed=1002,
                             M=2048, R=16, K=2001),
    "graphene-10M-learned": dict(kind="rect", nx=2500, ny=1000, sigma=0.1, seed=1003,
                                 M=1024, R=8, K=2001),
    "hbn-junction-64": dict(kind="junction", count=64, sigma=0.1, seed=4000,
                            M=1024, R=8, K=2001),
    "graphene-100M": dict(kind="rect", nx=5000, ny=5000, sigma=0.0, seed=1005,
                          M=1024, R=1, K=4001),
}

KPM_SEED = 42
LANCZOS_SEED = 7
TRAIN_SNAPSHOTS = 200
TRAIN_SEED_BASE = 3000


def training_snapshots(count: int = TRAIN_SNAPSHOTS, seed_base: int = TRAIN_SEED_BASE,
                       sigma: float = 0.1):
    """800-atom graphene snapshots (20x20 primitive cells) at sigma = 0.1 A."""
    return [graphene_primitive(20, 20, sigma, seed_base + s) for s in range(count)]


def energy_grid(emin: float, emax: float, k: int) -> np.ndarray:
    return np.linspace(emin, emax, k)
