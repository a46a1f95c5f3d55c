"""The allocation-free solve entry point (mbl_lobpcg_solve_noalloc).

Some callers cannot allocate device memory at the moment they need a solve: plug-ins
living inside an application whose own allocator owns the GPU memory, or real-time code
with a memory budget fixed in advance.  For them the library keeps one fixed 16 MiB
workspace in device memory and this entry point uses it instead of a caller-provided
buffer.  The test checks, through the C ABI and in both precision modes, that two calls
in a row give the same eigenpairs as the ordinary entry point (within the solver tests'
tolerance: 1e-9 ||H|| on eigenvalues), that the returned vectors pass the residual
certificate, that a problem close to the 16 MiB limit (L = 14, k = 32, FP64) gives the
dense eigenvalues, and that a problem whose workspace does not fit is refused before
anything runs.

The file is named so that pytest collects it last.
"""
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


@pytest.mark.parametrize("mode", [0, 1])
def test_noalloc_matches_workspace_entry_point(mbl, mode):
    cfg = wl.SOLVE_L12
    L, k, nev = cfg["L"], cfg["k"], cfg["nev"]
    h = wl.fields(L, cfg["W"], cfg["seed"])
    ev = np.linalg.eigvalsh(ham.dense_sector(ham.Chain(L, h)))
    sigma = 0.5 * (ev[0] + ev[-1])
    nh = max(abs(ev[0]), abs(ev[-1]))
    n = ev.size
    chain = mbl.make_chain(L, h, 1.0, False)
    opts = mbl.make_opts(nev, k, tol=1e-8, max_iter=300, pcg_iters=40, norm_h=nh, mode=mode, use_graph=0)
    X0 = torch.from_numpy(wl.initial_block(n, k, cfg["seed"])).to(DEV)
    ws = torch.empty(mbl.lobpcg_workspace_size(chain, opts), dtype=torch.uint8, device=DEV)
    ref_vals, _, ref_stats, _ = mbl.lobpcg_solve(chain, sigma, opts, X0, ws)
    assert ref_stats["converged"] == 1
    for _ in range(2):  # two calls in a row: the second reuses the first call's leftovers
        vecs = torch.empty((n, nev), dtype=torch.float64, device=DEV)
        vals, resid, stats, rc = mbl.binding.lobpcg_solve_noalloc(chain, sigma, opts, X0, vecs)
        assert rc == mbl.binding.MBL_OK and stats["converged"] == 1
        assert np.abs(vals - ref_vals).max() <= 1e-9 * nh
        y = vecs.cpu().numpy()
        r = np.linalg.norm(ham.apply(ham.Chain(L, h), 0.0, y) - y * vals[None, :], axis=0)
        assert r.max() <= 1e-8 * nh * 1.01


def test_noalloc_near_the_limit_matches_dense(mbl):
    """L = 14 periodic with k = 32 in FP64 mode needs most of the 16 MiB."""
    L, k, nev = 14, 32, 16
    h = wl.fields(L, 8.0, 1)
    ev = np.linalg.eigvalsh(ham.dense_sector(ham.Chain(L, h, periodic=True)))
    sigma = 0.5 * (ev[0] + ev[-1])
    nh = max(abs(ev[0]), abs(ev[-1]))
    want = np.sort(ev[np.lexsort((ev, np.abs(ev - sigma)))[:nev]])
    chain = mbl.make_chain(L, h, 1.0, True)
    opts = mbl.make_opts(nev, k, tol=1e-8, max_iter=300, pcg_iters=20, norm_h=nh, mode=mbl.MODE_FP64)
    need = mbl.lobpcg_workspace_size(chain, opts)
    assert 0.75 * mbl.binding.NOALLOC_SCRATCH_BYTES < need <= mbl.binding.NOALLOC_SCRATCH_BYTES
    X0 = torch.from_numpy(wl.initial_block(ev.size, k, 1)).to(DEV)
    vecs = torch.empty((ev.size, nev), dtype=torch.float64, device=DEV)
    vals, resid, stats, rc = mbl.binding.lobpcg_solve_noalloc(chain, sigma, opts, X0, vecs)
    assert rc == mbl.binding.MBL_OK and stats["converged"] == 1
    assert np.abs(vals - want).max() <= 1e-9 * nh
    y = vecs.cpu().numpy()
    r = np.linalg.norm(ham.apply(ham.Chain(L, h, periodic=True), 0.0, y) - y * vals[None, :], axis=0)
    assert r.max() <= 1e-8 * nh * 1.01


def test_noalloc_rejects_problem_larger_than_scratch(mbl):
    L = 20
    h = wl.fields(L, 8.0, 1)
    chain = mbl.make_chain(L, h, 1.0, True)
    opts = mbl.make_opts(16, 32, norm_h=40.0)
    assert mbl.lobpcg_workspace_size(chain, opts) > mbl.binding.NOALLOC_SCRATCH_BYTES
    X0 = torch.zeros((mbl.basis_size(L, 10), 32), dtype=torch.float64, device=DEV)
    with pytest.raises(mbl.MBLError) as ei:
        mbl.binding.lobpcg_solve_noalloc(chain, 0.0, opts, X0)
    assert ei.value.status == mbl.binding.MBL_ERR_WORKSPACE
