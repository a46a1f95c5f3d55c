"""GPU parity of the folded LOBPCG (Sec. 3.2, Sec. 6.2) and of the spectrum bounds.

Eigenvalues are compared with dense LAPACK on the oracle's sector matrix (L <= 14),
the delta = 0 free-fermion closed form, scipy's shift-invert Lanczos (L = 16), and the
oracle's own LOBPCG; tolerances are those of the method: |d lambda| <= 1e-9 ||H|| in
FP64 mode, <= 1e-6 ||H|| in mixed mode, residuals <= 1e-8 ||H|| (recomputed here from
the returned vectors with the oracle product).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import closed_form as cf
from oracle import hamiltonian as ham
from oracle import solver

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


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _solve(mbl, L, h, periodic, sigma, nev, k, mode, norm_h, pcg_iters, seed, delta=1.0, max_iter=300,
           use_graph=1):
    n = ham.sector_dim(L, L // 2)
    chain = mbl.make_chain(L, h, delta, periodic)
    opts = mbl.make_opts(nev, k, tol=1e-8, max_iter=max_iter, pcg_iters=pcg_iters, norm_h=norm_h, mode=mode,
                         use_graph=use_graph)
    ws = torch.empty(mbl.lobpcg_workspace_size(chain, opts), dtype=torch.uint8, device=DEV)
    X0 = _gpu(wl.initial_block(n, k, seed))
    evecs = torch.empty((n, nev), dtype=torch.float64, device=DEV)
    evals, resid, stats, rc = mbl.lobpcg_solve(chain, sigma, opts, X0, ws, evecs)
    return evals, resid, stats, evecs.cpu().numpy()


def _certify(L, h, periodic, evals, evecs, norm_h, delta=1.0):
    ch = ham.Chain(L, h, delta=delta, periodic=periodic)
    Hy = ham.apply(ch, 0.0, evecs)
    res = np.linalg.norm(Hy - evecs * evals[None, :], axis=0)
    assert res.max() <= 1e-8 * norm_h * 1.01, res.max() / norm_h
    G = evecs.T @ evecs
    assert np.abs(G - np.eye(G.shape[0])).max() < 1e-8


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("use_graph", [0, 1])
def test_l12_config_matches_dense(mbl, mode, use_graph):
    cfg = wl.SOLVE_L12
    L = cfg["L"]
    h = wl.fields(L, cfg["W"], cfg["seed"])
    ev = np.linalg.eigvalsh(ham.dense_sector(ham.Chain(L, h)))
    sigma = 0.5 * (ev[0] + ev[-1])
    nh = max(abs(ev[0]), abs(ev[-1]))
    want = np.sort(ev[np.lexsort((ev, np.abs(ev - sigma)))[:8]])
    evals, resid, stats, vecs = _solve(mbl, L, h, False, sigma, 8, 8, mode, nh, 40, cfg["seed"],
                                       use_graph=use_graph)
    assert stats["converged"] == 1
    tol = 1e-9 if mode == 0 else 1e-6
    assert np.abs(evals - want).max() <= tol * nh
    assert np.abs(evals - want).max() <= 1e-9 * nh  # both modes reach FP64 accuracy here
    _certify(L, h, False, evals, vecs, nh)


@pytest.mark.parametrize("mode", [0, 1])
def test_l14_periodic_guards_matches_dense(mbl, mode):
    L = 14
    h = wl.fields(L, 8.0, 1)
    ev = np.linalg.eigvalsh(ham.dense_sector(ham.Chain(L, h, periodic=True)))
    sigma = 0.5 * (ev[0] + ev[-1])
    nh = max(abs(ev[0]), abs(ev[-1]))
    want = np.sort(ev[np.lexsort((ev, np.abs(ev - sigma)))[:16]])
    evals, resid, stats, vecs = _solve(mbl, L, h, True, sigma, 16, 32, mode, nh, 20, 1)
    assert stats["converged"] == 1
    assert np.abs(evals - want).max() <= (1e-9 if mode == 0 else 1e-6) * nh
    _certify(L, h, True, evals, vecs, nh)


@pytest.mark.parametrize("periodic", [False, True])
def test_delta0_matches_free_fermions(mbl, periodic):
    L = 18
    h = wl.fields(L, 3.0, 21)
    allmin = cf.free_fermion_nearest(L, h, L // 2, periodic, -1e9, 1)[0]
    allmax = cf.free_fermion_nearest(L, h, L // 2, periodic, 1e9, 1)[0]
    sigma = 0.5 * (allmin + allmax) + 0.0123
    nh = max(abs(allmin), abs(allmax))
    want = cf.free_fermion_nearest(L, h, L // 2, periodic, sigma, 6)
    evals, resid, stats, vecs = _solve(mbl, L, h, periodic, sigma, 6, 16, 1, nh, 120, 21, delta=0.0,
                                       max_iter=400)
    assert stats["converged"] == 1
    assert np.abs(evals - want).max() <= 1e-6 * nh
    _certify(L, h, periodic, evals, vecs, nh, delta=0.0)


def test_l16_matches_shift_invert_lanczos(mbl):
    sp = pytest.importorskip("scipy.sparse")
    spla = pytest.importorskip("scipy.sparse.linalg")
    L = 16
    h = wl.fields(L, 8.0, 5)
    ch = ham.Chain(L, h)
    n = ham.sector_dim(L, 8)
    # sparse sector matrix assembled from the oracle product on unit vectors, in chunks
    rows, cols, vals = [], [], []
    for c0 in range(0, n, 2048):
        E = np.zeros((n, min(2048, n - c0)))
        E[np.arange(c0, c0 + E.shape[1]), np.arange(E.shape[1])] = 1.0
        Hc = ham.apply(ch, 0.0, E)
        r, c = np.nonzero(Hc)
        rows.append(r)
        cols.append(c + c0)
        vals.append(Hc[r, c])
    Hs = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    emin = spla.eigsh(Hs, 1, which="SA")[0][0]
    emax = spla.eigsh(Hs, 1, which="LA")[0][0]
    sigma = 0.5 * (emin + emax)
    nh = max(abs(emin), abs(emax))
    ev = spla.eigsh(Hs, 24, sigma=sigma, which="LM", return_eigenvectors=False)
    want = np.sort(ev[np.lexsort((ev, np.abs(ev - sigma)))[:10]])
    evals, resid, stats, vecs = _solve(mbl, L, h, False, sigma, 10, 20, 1, nh, 60, 5)
    assert stats["converged"] == 1
    assert np.abs(evals - want).max() <= 1e-6 * nh
    _certify(L, h, False, evals, vecs, nh)


def test_mixed_and_fp64_agree_l18(mbl):
    L = 18
    h = wl.fields(L, 8.0, 1)
    n = ham.sector_dim(L, 9)
    Xb = wl.block(n, 4, 101)
    chain = mbl.make_chain(L, h, 1.0, True)
    ws = torch.empty(mbl.bounds_workspace_size(chain, 4), dtype=torch.uint8, device=DEV)
    emin, emax, _ = mbl.spectrum_bounds(chain, _gpu(Xb), ws, tol=1e-10)
    sigma = 0.5 * (emin + emax)
    nh = max(abs(emin), abs(emax))
    e64, r64, s64, v64 = _solve(mbl, L, h, True, sigma, 16, 32, 0, nh, 160, 1)
    e32, r32, s32, v32 = _solve(mbl, L, h, True, sigma, 16, 32, 1, nh, 160, 1)
    assert s64["converged"] == 1 and s32["converged"] == 1
    assert np.abs(e64 - e32).max() <= 1e-6 * nh
    _certify(L, h, True, e32, v32, nh)
    # Sec. 6.2: single-precision PCG leaves the LOBPCG iteration count unchanged (within a few)
    assert abs(s64["iters"] - s32["iters"]) <= max(3, s64["iters"] // 5)


def test_spectrum_bounds_match_dense(mbl):
    """The FP64 Lanczos bounds (both ends from one recurrence) against dense LAPACK."""
    L = 14
    h = wl.fields(L, 8.0, 4)
    ev = np.linalg.eigvalsh(ham.dense_sector(ham.Chain(L, h, periodic=True)))
    n = ev.size
    X0 = _gpu(wl.block(n, 4, 104))
    chain = mbl.make_chain(L, h, 1.0, True)
    ws = torch.empty(mbl.bounds_workspace_size(chain, 4), dtype=torch.uint8, device=DEV)
    emin, emax, it = mbl.spectrum_bounds(chain, X0, ws, tol=1e-11)
    assert abs(emin - ev[0]) <= 1e-10 * abs(ev[0])
    assert abs(emax - ev[-1]) <= 1e-10 * abs(ev[-1])


def test_solver_rejects_bad_options(mbl):
    L = 12
    h = wl.fields(L, 5.0, 0)
    chain = mbl.make_chain(L, h)
    for bad in [dict(nev=9, k=8), dict(nev=0, k=8), dict(nev=4, k=400), dict(nev=4, k=8, tol=0.0)]:
        kw = dict(tol=1e-8)
        kw.update(bad)
        opts = mbl.make_opts(**kw)
        with pytest.raises(mbl.MBLError):
            mbl.lobpcg_workspace_size(chain, opts)


def test_not_converged_status(mbl):
    L = 12
    h = wl.fields(L, 5.0, 0)
    n = ham.sector_dim(L, 6)
    chain = mbl.make_chain(L, h)
    opts = mbl.make_opts(8, 8, tol=1e-12, max_iter=2, pcg_iters=5, norm_h=20.0)
    ws = torch.empty(mbl.lobpcg_workspace_size(chain, opts), dtype=torch.uint8, device=DEV)
    X0 = _gpu(wl.initial_block(n, 8, 0))
    evals, resid, stats, rc = mbl.lobpcg_solve(chain, -0.25, opts, X0, ws, allow_not_converged=True)
    assert rc == mbl.binding.MBL_ERR_NOT_CONVERGED
    assert stats["iters"] == 2 and stats["converged"] == 0
    assert np.all(np.isfinite(evals))


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("schedule", [3, 4, 5])
def test_bulk_copy_schedules_solve_matches_dense(mbl, mode, schedule):
    """The folded LOBPCG with every k = 32 product (PCG launches included) on schedule 3
    (staged tiles), 4 (streamed row blocks) or 5 (slab ring)."""
    L = 14
    h = wl.fields(L, 8.0, 1)
    ev = np.linalg.eigvalsh(ham.dense_sector(ham.Chain(L, h, periodic=True)))
    sigma = 0.5 * (ev[0] + ev[-1])
    nh = max(abs(ev[0]), abs(ev[-1]))
    want = np.sort(ev[np.lexsort((ev, np.abs(ev - sigma)))[:16]])
    try:
        for dt in (torch.float32, torch.float64):
            mbl.binding.set_product_schedule(32, dt, schedule)
        evals, resid, stats, vecs = _solve(mbl, L, h, True, sigma, 16, 32, mode, nh, 20, 1)
    finally:
        for dt in (torch.float32, torch.float64):
            mbl.binding.set_product_schedule(32, dt, 0)
    assert stats["converged"] == 1
    assert np.abs(evals - want).max() <= (1e-9 if mode == 0 else 1e-6) * nh
    _certify(L, h, True, evals, vecs, nh)


@pytest.mark.parametrize("L,k,nev", [(14, 32, 16), (16, 64, 24)])
def test_tensor_core_grams_solve_matches_dense(mbl, L, k, nev):
    """Mixed mode with its FP32 Grams and block updates on the tensor cores (tcgen05
    kind::tf32, two-term TF32 split): the eigenvalues nearest sigma still match dense
    LAPACK."""
    h = wl.fields(L, 8.0, 2)
    ev = np.linalg.eigvalsh(ham.dense_sector(ham.Chain(L, h, periodic=True)))
    sigma = 0.5 * (ev[0] + ev[-1])
    nh = max(abs(ev[0]), abs(ev[-1]))
    want = np.sort(ev[np.lexsort((ev, np.abs(ev - sigma)))[:nev]])
    try:
        mbl.binding.set_gram_engine(2)
        evals, resid, stats, vecs = _solve(mbl, L, h, True, sigma, nev, k, 1, nh, 40, 3)
    finally:
        mbl.binding.set_gram_engine(0)
    assert stats["converged"] == 1
    assert np.abs(evals - want).max() <= 1e-6 * nh
    _certify(L, h, True, evals, vecs, nh)
