"""Pins of the oracle's solver (Sec. 3.2, Sec. 6.2).

The folded LOBPCG is an iteration, so it is pinned by what fixes its answer
independently: dense LAPACK on the sector matrix (L <= 14), the delta = 0
free-fermion closed form (any L), residual certificates, and for the inner PCG
the exact solve of a small SPD system.
"""
import os

import numpy as np
import pytest

import workloads as wl
from oracle import closed_form as cf
from oracle import hamiltonian as ham
from oracle import solver

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    vals, evals = {}, []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, v = line.split()
            if key == "eval":
                evals.append(float(v))
            else:
                vals[key] = float(v)
    return vals, np.array(evals)


def test_golden_l12_is_dense_spectrum():
    cfg = wl.SOLVE_L12
    vals, ev8 = _read_golden("l12_open_w5_seed0_nearest8.txt")
    ch = ham.Chain(12, wl.fields(12, cfg["W"], cfg["seed"]), periodic=False)
    ev = np.linalg.eigvalsh(ham.dense_sector(ch))
    assert abs(ev[0] - vals["emin"]) < 1e-12 and abs(ev[-1] - vals["emax"]) < 1e-12
    assert ev8.size == 8 and np.all(np.isin(np.round(ev8, 10), np.round(ev, 10)))


@pytest.mark.parametrize("pcg_dtype", [np.float64, np.float32])
def test_lobpcg_l12_matches_dense(pcg_dtype):
    """Config L=12 open, nev = k = 8: eigenvalues within 1e-9 ||H|| of LAPACK and
    residuals within 1e-8 ||H||; the FP32 preconditioner gives the same answer
    (Sec. 6.2: single-precision PCG does not change the eigenvalue accuracy)."""
    cfg = wl.SOLVE_L12
    vals, ref = _read_golden("l12_open_w5_seed0_nearest8.txt")
    ch = ham.Chain(12, wl.fields(12, cfg["W"], cfg["seed"]), periodic=False)
    X0 = wl.initial_block(924, 8, cfg["seed"])
    r = solver.lobpcg_folded(ch, vals["sigma"], X0, 8, 1e-8, vals["norm_h"], max_iter=200,
                             pcg_iters=40, pcg_dtype=pcg_dtype)
    assert r.converged
    assert np.abs(r.evals - ref).max() <= 1e-9 * vals["norm_h"]
    assert r.resid.max() <= 1e-8 * vals["norm_h"]
    # residual certificate recomputed from the returned vectors
    Hy = ham.apply(ch, 0.0, r.evecs)
    res = np.linalg.norm(Hy - r.evecs * r.evals[None, :], axis=0)
    assert res.max() <= 1e-8 * vals["norm_h"]
    assert np.abs(r.evecs.T @ r.evecs - np.eye(8)).max() < 1e-10


def test_lobpcg_periodic_l14_with_guards_matches_dense():
    ch = ham.Chain(14, wl.fields(14, 8.0, 1), periodic=True)
    ev = np.linalg.eigvalsh(ham.dense_sector(ch))
    sigma = 0.5 * (ev[0] + ev[-1])
    nh = max(abs(ev[0]), abs(ev[-1]))
    ref = np.sort(ev[np.lexsort((ev, np.abs(ev - sigma)))[:16]])
    X0 = wl.initial_block(ev.size, 32, 1)
    r = solver.lobpcg_folded(ch, sigma, X0, 16, 1e-8, nh, max_iter=100, pcg_iters=20)
    assert r.converged
    assert np.abs(r.evals - ref).max() <= 1e-9 * nh


@pytest.mark.parametrize("L,periodic", [(14, False), (14, True)])
def test_lobpcg_delta0_matches_free_fermions(L, periodic):
    h = wl.fields(L, 3.0, 21)
    ch = ham.Chain(L, h, delta=0.0, periodic=periodic)
    n = ham.sector_dim(L, L // 2)
    allv = cf.free_fermion_energies(L, h, L // 2, periodic)
    sigma = 0.5 * (allv[0] + allv[-1]) + 0.0123
    nh = max(abs(allv[0]), abs(allv[-1]))
    ref = cf.free_fermion_nearest(L, h, L // 2, periodic, sigma, 6)
    r = solver.lobpcg_folded(ch, sigma, wl.initial_block(n, 12, 21), 6, 1e-8, nh,
                             max_iter=150, pcg_iters=80)
    assert r.converged
    assert np.abs(r.evals - ref).max() <= 1e-9 * nh


def test_pcg_solves_small_spd_system_exactly():
    """Jacobi-PCG terminates in n steps on an n x n SPD system (exact arithmetic);
    compare with a direct solve."""
    rng = np.random.default_rng(0)
    n = 40
    M = rng.standard_normal((n, n))
    A = M @ M.T + 0.5 * np.eye(n)
    B = rng.standard_normal((n, 3))
    W = solver.pcg_jacobi(lambda V: A @ V, 1.0 / np.diag(A), B, 3 * n)
    assert np.allclose(W, np.linalg.solve(A, B), rtol=1e-8, atol=1e-9)


def test_pcg_single_step_is_jacobi_scaled_steepest_descent():
    """One PCG step from 0: w = alpha z, z = M^-1 b, alpha = (b.z)/(z.Az)."""
    rng = np.random.default_rng(1)
    n = 12
    M = rng.standard_normal((n, n))
    A = M @ M.T + np.eye(n)
    b = rng.standard_normal((n, 1))
    z = b / np.diag(A)[:, None]
    alpha = (b.T @ z).item() / (z.T @ A @ z).item()
    W = solver.pcg_jacobi(lambda V: A @ V, 1.0 / np.diag(A), b, 1)
    assert np.allclose(W, alpha * z, rtol=1e-13, atol=1e-15)


def test_extreme_eigenvalues_match_dense():
    ch = ham.Chain(14, wl.fields(14, 8.0, 4), periodic=True)
    ev = np.linalg.eigvalsh(ham.dense_sector(ch))
    X0 = wl.block(ev.size, 4, 104)
    emin, _ = solver.lobpcg_extreme(ch, +1.0, X0, 1e-11)
    m_emax, _ = solver.lobpcg_extreme(ch, -1.0, X0, 1e-11)
    assert abs(emin - ev[0]) <= 1e-10 * abs(ev[0])
    assert abs(-m_emax - ev[-1]) <= 1e-10 * abs(ev[-1])
