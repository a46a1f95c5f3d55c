"""Batched disorder averaging (Sec. 3.1: realisations are independent) against the
oracle: every problem of a mixed-L batch must give the dense-LAPACK eigenvalues nearest
its spectrum midpoint, both with sigmas supplied and with sigmas found by the batched
call itself, and the supplied-sigma results must equal the single-problem solve."""
import numpy as np
import pytest

import workloads as wl
from oracle import hamiltonian as ham

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def mbl():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2012_00217_gb300 as m
    m.binding.lib()
    return m


def _problems():
    out = []
    for seed, (L, W) in enumerate([(10, 2.0), (12, 4.0), (14, 8.0), (12, 8.0), (10, 4.0), (14, 2.0), (12, 2.0)]):
        h = wl.batched_fields(L, W, seed)
        ev = np.linalg.eigvalsh(ham.dense_sector(ham.Chain(L, h)))
        out.append(dict(L=L, h=h, ev=ev, seed=seed))
    return out


@pytest.mark.parametrize("given_sigma", [True, False])
def test_batched_matches_dense(mbl, given_sigma):
    probs = _problems()
    nev, k = 6, 12
    chains = [mbl.make_chain(p["L"], p["h"]) for p in probs]
    X0 = torch.cat([torch.from_numpy(wl.initial_block(p["ev"].size, k, p["seed"])) for p in probs]).to(DEV)
    sig = [0.5 * (p["ev"][0] + p["ev"][-1]) for p in probs]
    nh = max(max(abs(p["ev"][0]), abs(p["ev"][-1])) for p in probs)
    opts = mbl.make_opts(nev, k, tol=1e-8, max_iter=1000, pcg_iters=80, norm_h=nh if given_sigma else 0.0,
                         mode=mbl.MODE_MIXED)
    ws = torch.empty(mbl.binding.batched_workspace_size(chains, opts, 3), dtype=torch.uint8, device=DEV)
    evals, resid, stats, rc = mbl.binding.lobpcg_solve_batched(chains, opts, X0, ws, 3,
                                                               sigmas=sig if given_sigma else None)
    for i, p in enumerate(probs):
        assert stats[i]["converged"] == 1
        want = np.sort(p["ev"][np.lexsort((p["ev"], np.abs(p["ev"] - sig[i])))[:nev]])
        pn = max(abs(p["ev"][0]), abs(p["ev"][-1]))
        assert np.abs(evals[i] - want).max() <= 1e-9 * pn, (i, evals[i], want)
    if given_sigma:
        # the batched results are those of the single-problem entry point
        off = 0
        for i, p in enumerate(probs):
            n = p["ev"].size
            o1 = mbl.make_opts(nev, k, tol=1e-8, max_iter=1000, pcg_iters=80, norm_h=nh, mode=mbl.MODE_MIXED)
            w1 = torch.empty(mbl.lobpcg_workspace_size(chains[i], o1), dtype=torch.uint8, device=DEV)
            e1, _, _, _ = mbl.lobpcg_solve(chains[i], sig[i], o1, X0[off:off + n].contiguous(), w1)
            assert np.array_equal(e1, evals[i])
            off += n


def test_several_windows_and_sectors_per_realization(mbl):
    """Several spectral windows of one realization, and sectors other than S^z = 0, in one
    batched call: each (realization, sector, sigma) problem must give the dense-LAPACK
    eigenvalues of its sector nearest its own sigma, and the gap ratio of each window (on
    the GPU) must equal the oracle's on the same levels."""
    from oracle import observables as obs
    L, nev, k = 12, 6, 12
    h = wl.batched_fields(L, 3.0, 11)
    probs = []
    for n_up in (6, 5, 4):
        ev = np.linalg.eigvalsh(ham.dense_sector(ham.Chain(L, h, n_up=n_up)))
        for q in (0.2, 0.5, 0.8):  # three windows across the sector's spectrum
            probs.append(dict(n_up=n_up, ev=ev, sigma=float(np.quantile(ev, q))))
    chains = [mbl.make_chain(L, h, 1.0, False, p["n_up"]) for p in probs]
    X0 = torch.cat([torch.from_numpy(wl.initial_block(p["ev"].size, k, 40 + i)) for i, p in enumerate(probs)])
    nh = max(max(abs(p["ev"][0]), abs(p["ev"][-1])) for p in probs)
    opts = mbl.make_opts(nev, k, tol=1e-8, max_iter=1000, pcg_iters=80, norm_h=nh, mode=mbl.MODE_MIXED)
    ws = torch.empty(mbl.binding.batched_workspace_size(chains, opts, 4), dtype=torch.uint8, device=DEV)
    evals, resid, stats, rc = mbl.binding.lobpcg_solve_batched(chains, opts, X0.to(DEV), ws, 4,
                                                               sigmas=[p["sigma"] for p in probs])
    for i, p in enumerate(probs):
        assert stats[i]["converged"] == 1
        want = np.sort(p["ev"][np.lexsort((p["ev"], np.abs(p["ev"] - p["sigma"])))[:nev]])
        assert np.abs(evals[i] - want).max() <= 1e-9 * nh, (i, evals[i], want)
    r, c = mbl.gap_ratio(torch.from_numpy(np.ascontiguousarray(evals)).to(DEV))
    r, c = r.cpu().numpy(), c.cpu().numpy()
    for i in range(len(probs)):
        want, n = obs.gap_ratio_mean(evals[i])
        assert c[i] == n and abs(r[i] - want) <= 1e-13
