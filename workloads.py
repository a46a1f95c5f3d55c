"""Seeded synthetic inputs for the MBL eigensolver hot path.

Shared by the tests and bench.py.  This module draws random numbers and names
workloads; it holds none of the method's arithmetic (no basis, no Hamiltonian,
no solver).  Fields follow Sec. 2.1: h_i drawn uniformly from [-W, W] per
disorder realisation; block vectors are standard normal.
"""
import numpy as np


def fields(L, W, seed):
    """h_i ~ Uniform[-W, W], i = 0..L-1, FP64, from numpy's default_rng(seed)."""
    return np.random.default_rng(seed).uniform(-W, W, L)


def batched_fields(L, W, seed):
    """Disorder-averaging batches reuse one draw per seed scaled by W:
    h = W * u, u ~ Uniform[-1, 1]^L from default_rng(seed)."""
    return W * np.random.default_rng(seed).uniform(-1.0, 1.0, L)


def block(n, k, seed, dtype=np.float64):
    """Row-major n x k block with N(0, 1) entries from default_rng(seed), cast once."""
    return np.random.default_rng(seed).standard_normal((n, k)).astype(dtype)


def initial_block(n, k, seed):
    """LOBPCG starting block X0 (n x k, N(0, 1), FP64) for the problem with this seed."""
    return np.random.default_rng([int(seed), 0x5EED]).standard_normal((n, k))


def sector_dim(L, n_up=None):
    """C(L, n_up) by exact integer arithmetic (for sizing buffers only)."""
    from math import comb
    return comb(L, L // 2 if n_up is None else n_up)


# Named workloads with their sizes (all Delta = 1, S^z = 0 sector, n_up = L/2).
SOLVE_L12 = dict(name="L12-open-W5-seed0", L=12, periodic=False, delta=1.0, W=5.0, seed=0,
                 nev=8, k=8)
SOLVE_L20 = dict(name="L20-periodic-W8-seed1", L=20, periodic=True, delta=1.0, W=8.0, seed=1,
                 nev=16, k=32)
SOLVE_L26 = dict(name="L26-periodic-W8-seed7", L=26, periodic=True, delta=1.0, W=8.0, seed=7,
                 nev=32, k=64)
MATVEC_SWEEP = [dict(L=L, periodic=False, delta=1.0, W=8.0, seed=0,
                     ks=(1, 8, 16) if L == 28 else (1, 8, 32, 64))
                for L in (22, 24, 26, 28)]


def batched_problems(W):
    """Disorder-averaging batch: 256 x L=16 (seeds 0..255), 64 x L=14 (256..319),
    32 x L=18 (320..351), open chains, nev = 8, fields scaled by W."""
    out = []
    for seed in range(352):
        L = 16 if seed < 256 else (14 if seed < 320 else 18)
        out.append(dict(L=L, periodic=False, delta=1.0, W=float(W), seed=seed, nev=8, k=8))
    return out
