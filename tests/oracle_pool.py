"""The FP64 oracle's KPM moments of large structures, split over blocks of
random vectors in a pool of worker processes.  TEST INFRASTRUCTURE ONLY.

The vectors of the stochastic trace are independent (oracle.kpm draws vector
r from its own counter), so the moments of vectors first .. first + k - 1 can
be computed apart and concatenated.  Each worker rebuilds the oracle
Hamiltonian from the seeded structure description once (no large arrays are
pickled) and runs oracle.kpm.chebyshev_moments on its block.  The pool is
started with the 'spawn' method so that it is safe after CUDA has been
initialised in the calling process.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_STATE = {}


def build_structure(spec):
    """spec = (kind, nx, ny, sigma, seed) with kind 'rect' (graphene) or
    'junction' (h-BN/graphene); returns (structure, teacher parameters)."""
    from paper_2509_06525_gb300 import synth
    kind, nx, ny, sigma, seed = spec
    if kind == "rect":
        return synth.graphene_rect(nx, ny, sigma, seed), synth.teacher_graphene()
    if kind == "junction":
        return synth.hbn_graphene_junction(nx, ny, sigma, seed), synth.teacher_hbn_graphene()
    raise ValueError(kind)


def oracle_hamiltonian(spec):
    """(structure, teacher, CSR H, indptr, indices, hop, onsite) from the oracle."""
    from oracle import hamiltonian as oha
    from oracle import neighbors as onb
    from oracle import teacher as ote
    s, p = build_structure(spec)
    ip, idx, d = onb.neighbors(s.positions, s.box, s.pbc, p.rcut)
    t, eps, _ = ote.teacher_elements(s.species, ip, idx, d, p)
    return s, p, oha.csr_hamiltonian(s.n, ip, idx, t, eps), ip, idx, t, eps


def _init(spec, a, b):
    from oracle import kpm as okpm
    s, p, H, *_ = oracle_hamiltonian(spec)
    _STATE["Ht"] = okpm.rescale(H, a, b)
    _STATE["n"] = s.n


def _block(job):
    from oracle import kpm as okpm
    seed, first, count, M = job
    v0 = okpm.random_phase_vectors(seed, _STATE["n"], count, first)
    mu, _ = okpm.chebyshev_moments(_STATE["Ht"], v0, M)
    return first, mu


def kpm_moments_parallel(spec, a, b, M, R, seed, workers=None):
    """Per-vector oracle moments mu_r [R, M] of the structure `spec`."""
    workers = workers or max(1, min(R, os.cpu_count() or 1))
    per = (R + workers - 1) // workers
    jobs = [(seed, f, min(per, R - f), M) for f in range(0, R, per)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(jobs), initializer=_init, initargs=(spec, a, b)) as pool:
        parts = pool.map(_block, jobs)
    mu = np.zeros((R, M))
    for first, block in parts:
        mu[first:first + block.shape[0]] = block
    return mu
