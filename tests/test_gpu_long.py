"""Long GPU runs, opt-in: MBL_LONG_TESTS=1 (minutes of GPU time, not part of a default run).

The L = 26 periodic workload (n = 10,400,600, W = 8, seed 7, nev = 32, k = 64, mixed: FP32
PCG and Gram matrices, FP64 Cholesky-QR, Rayleigh-Ritz and residuals; Sec. 6.2 solves
this size with 20,000 PCG steps per LOBPCG iteration on up to 2048 nodes) is run for a
stated number of LOBPCG iterations and PCG steps (MBL_L26_ITERS, MBL_L26_PCG), to
convergence at ||r|| <= 1e-8 ||H|| or to the residual it reaches.  The returned vectors
are copied to the host and every residual ||H y - lambda y|| is recomputed with the
oracle's FP64 product; it must equal the library's own to within rounding, and the
vectors must be orthonormal.  The run's figures are printed as one JSON line.
"""
import json
import os
import time

import numpy as np
import pytest

import workloads as wl
from oracle import hamiltonian as ham

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("MBL_LONG_TESTS") != "1",
                                 reason="long L = 26 solve: set MBL_LONG_TESTS=1")]
DEV = "cuda:0"


@pytest.fixture(scope="module")
def mbl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2012_00217_gb300 as m
    m.binding.lib()
    return m


def test_l26_periodic_solve_residuals_recomputed_by_oracle(mbl):
    cfg = wl.SOLVE_L26
    L, k, nev = cfg["L"], cfg["k"], cfg["nev"]
    iters = int(os.environ.get("MBL_L26_ITERS", "30"))
    pcg = int(os.environ.get("MBL_L26_PCG", "1000"))
    h = wl.fields(L, cfg["W"], cfg["seed"])
    chain = mbl.make_chain(L, h, cfg["delta"], cfg["periodic"])
    n = mbl.basis_size(L, L // 2)
    opts = mbl.make_opts(nev, k, tol=1e-8, max_iter=iters, pcg_iters=pcg, mode=mbl.MODE_MIXED, use_graph=1)
    ws = torch.empty(max(mbl.lobpcg_workspace_size(chain, opts), mbl.bounds_workspace_size(chain, 4)),
                     dtype=torch.uint8, device=DEV)
    g = torch.Generator(device=DEV)
    g.manual_seed(cfg["seed"] + 100)
    Xb = torch.randn((n, 4), generator=g, device=DEV, dtype=torch.float64)
    X0 = torch.from_numpy(wl.initial_block(n, k, cfg["seed"])).to(DEV)
    for dt in (torch.float32, torch.float64):
        X = torch.randn((n, k), generator=g, device=DEV, dtype=dt)
        mbl.binding.autotune_product(chain, X, torch.empty_like(X), reps=2)
        del X
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    emin, emax, bit = mbl.spectrum_bounds(chain, Xb, ws, tol=1e-7, max_iter=1000)
    opts.norm_h = nh = max(abs(emin), abs(emax))
    vecs = torch.empty((n, nev), dtype=torch.float64, device=DEV)
    evals, resid, st, rc = mbl.lobpcg_solve(chain, 0.5 * (emin + emax), opts, X0, ws, vecs,
                                            allow_not_converged=True)
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    del ws, X0, Xb
    y = vecs.cpu().numpy()
    del vecs
    torch.cuda.empty_cache()
    ch = ham.Chain(L, h, delta=cfg["delta"], periodic=cfg["periodic"])
    t1 = time.perf_counter()
    r_oracle = np.linalg.norm(ham.apply(ch, 0.0, y) - y * evals[None, :], axis=0)
    t_oracle = time.perf_counter() - t1
    G = y.T @ y
    print(json.dumps(dict(workload=cfg["name"], n=n, nev=nev, k=k, lobpcg_iters=st["iters"], pcg_iters=pcg,
                          converged=st["converged"], seconds=seconds, bounds_iters=bit, sigma=0.5 * (emin + emax),
                          norm_h=nh, max_rel_resid_library=st["max_rel_resid"],
                          max_rel_resid_oracle=float(r_oracle.max() / nh), oracle_check_s=t_oracle,
                          evals=[float(v) for v in evals])))
    assert np.all(np.isfinite(evals))
    assert np.abs(G - np.eye(nev)).max() < 1e-8
    # the library's residuals (FP64, from its own product) are the oracle's to within rounding
    assert np.allclose(r_oracle, resid, rtol=1e-3, atol=1e-12 * nh)
