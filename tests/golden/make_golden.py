"""Writes the stored expected values under tests/golden/ from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py [name ...]
(no names: every file).  Each file holds one seeded workload's spectrum bounds
E_min, E_max, sigma = (E_min + E_max) / 2, ||H|| = max(|E_min|, |E_max|) and the
eigenvalues nearest sigma, from the oracle's sector matrix by one of:
  * dense LAPACK (numpy.linalg.eigvalsh of the dense sector matrix), L <= 14;
  * shift-invert Lanczos (scipy eigsh on the oracle's sparse sector matrix, (H - sigma)^-1
    applied through a sparse LU with a minimum-degree ordering), L <= 18;
  * the oracle's own FP64 folded LOBPCG (Sec. 3.2) to a residual of 1e-10 ||H||, for
    L = 20, where the sparse LU no longer fits (its fill grows like n^3: 7.7 s and 19 M
    factor entries at L = 16, hours and tens of GB at L = 20); bounds there by Lanczos
    (scipy eigsh, which='SA'/'LA') on the same sparse matrix.
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as wl  # noqa: E402
from oracle import hamiltonian as ham  # noqa: E402


def _chain(cfg):
    return ham.Chain(cfg["L"], cfg.get("h", None) if cfg.get("h") is not None else
                     wl.fields(cfg["L"], cfg["W"], cfg["seed"]), delta=cfg["delta"], periodic=cfg["periodic"])


def _write(path, cfg, method, emin, emax, evals, extra=()):
    sigma = 0.5 * (emin + emax)
    norm_h = max(abs(emin), abs(emax))
    with open(path, "w") as f:
        f.write("# %s: L=%d %s delta=%g h%s seed %d; %s\n"
                % (cfg["name"], cfg["L"], "periodic" if cfg["periodic"] else "open", cfg["delta"],
                   cfg.get("hdesc", "~U[-%g,%g]" % (cfg["W"], cfg["W"])), cfg["seed"], method))
        for line in extra:
            f.write("# %s\n" % line)
        f.write("emin %.17g\nemax %.17g\nsigma %.17g\nnorm_h %.17g\n" % (emin, emax, sigma, norm_h))
        for v in evals:
            f.write("eval %.17g\n" % v)


def _nearest(ev, sigma, count):
    ev = np.asarray(ev)
    return np.sort(ev[np.lexsort((ev, np.abs(ev - sigma)))[:count]])


def dense_file(cfg, path):
    ch = _chain(cfg)
    ev = np.linalg.eigvalsh(ham.dense_sector(ch))
    emin, emax = float(ev[0]), float(ev[-1])
    _write(path, cfg, "dense eigh of the oracle sector matrix", emin, emax,
           _nearest(ev, 0.5 * (emin + emax), cfg["nev"]))


def _bounds_lanczos(Hs):
    import scipy.sparse.linalg as spla
    emin = float(spla.eigsh(Hs, 1, which="SA", tol=1e-14, return_eigenvectors=False)[0])
    emax = float(spla.eigsh(Hs, 1, which="LA", tol=1e-14, return_eigenvectors=False)[0])
    return emin, emax


def shift_invert_file(cfg, path, count):
    """The `count` eigenvalues nearest the midpoint (count >= nev, the rest a margin)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    ch = _chain(cfg)
    Hs = ham.sparse_sector(ch).tocsc()
    n = Hs.shape[0]
    emin, emax = _bounds_lanczos(Hs)
    sigma = 0.5 * (emin + emax)
    t0 = time.time()
    lu = spla.splu(Hs - sigma * sp.identity(n, format="csc"), permc_spec="MMD_AT_PLUS_A",
                   diag_pivot_thresh=0.0, options=dict(SymmetricMode=True))
    op = spla.LinearOperator((n, n), matvec=lu.solve, dtype=np.float64)
    ev = spla.eigsh(Hs, count, sigma=sigma, which="LM", OPinv=op, tol=0, return_eigenvectors=False)
    _write(path, cfg, "shift-invert Lanczos (scipy eigsh, sparse LU) on the oracle sparse sector matrix",
           emin, emax, _nearest(ev, sigma, count),
           extra=("%d nearest eigenvalues (nev = %d plus a margin); %.0f s" % (count, cfg["nev"], time.time() - t0),))


def oracle_lobpcg_file(cfg, path, pcg_iters, tol=1e-10):
    from oracle import solver
    ch = _chain(cfg)
    Hs = ham.sparse_sector(ch)
    emin, emax = _bounds_lanczos(Hs)
    sigma, norm_h = 0.5 * (emin + emax), max(abs(emin), abs(emax))
    n = Hs.shape[0]
    t0 = time.time()
    r = solver.lobpcg_folded(ch, sigma, wl.initial_block(n, cfg["k"], cfg["seed"]), cfg["nev"], tol, norm_h,
                             max_iter=200, pcg_iters=pcg_iters)
    if not r.converged:
        raise RuntimeError("oracle LOBPCG did not converge")
    # certificate from the sparse matrix (not the solver's own product)
    res = np.linalg.norm(Hs @ r.evecs - r.evecs * r.evals[None, :], axis=0)
    _write(path, cfg, "oracle FP64 folded LOBPCG (k=%d, %d PCG steps per iteration, FP64 PCG)" % (cfg["k"], pcg_iters),
           emin, emax, r.evals,
           extra=("%d iterations, %.0f s; max ||Hy - lambda y|| / ||H|| = %.3g (sparse-matrix certificate)"
                  % (r.iters, time.time() - t0, res.max() / norm_h),))


def _l18_headline():
    return dict(wl.SOLVE_L20, name="L18-periodic-W8-seed1", L=18)


def _batch(L, W, seed):
    return dict(name="batch-L%d-W%g-seed%d" % (L, W, seed), L=L, periodic=False, delta=1.0, W=W, seed=seed,
                nev=8, k=16, h=wl.batched_fields(L, W, seed), hdesc="=%g*U[-1,1]" % W)


JOBS = {
    "l12": lambda: dense_file(wl.SOLVE_L12, os.path.join(HERE, "l12_open_w5_seed0_nearest8.txt")),
    "l18": lambda: shift_invert_file(_l18_headline(), os.path.join(HERE, "l18_periodic_w8_seed1_nearest24.txt"), 24),
    "batch16": lambda: [shift_invert_file(_batch(16, W, s), os.path.join(HERE, "batch_l16_w%g_seed%d_nearest12.txt" % (W, s)), 12)
                        for (W, s) in ((2.0, 3), (8.0, 4))],
    "batch18": lambda: [shift_invert_file(_batch(18, W, s), os.path.join(HERE, "batch_l18_w%g_seed%d_nearest12.txt" % (W, s)), 12)
                        for (W, s) in ((4.0, 320), (8.0, 321))],
    "l20": lambda: oracle_lobpcg_file(wl.SOLVE_L20, os.path.join(HERE, "l20_periodic_w8_seed1_nearest16.txt"), 640),
}

if __name__ == "__main__":
    names = sys.argv[1:] or list(JOBS)
    for nm in names:
        t0 = time.time()
        JOBS[nm]()
        print("written", nm, "%.0f s" % (time.time() - t0), flush=True)
