"""Thin ctypes binding of the C ABI in include/mbl.h (argument marshalling only).

Every function has the same name as its C entry point without the ``mbl_`` prefix.
Device buffers are torch CUDA tensors (passed by data pointer); the stream is
torch's current stream on the tensors' device.  Nothing here computes any part of
the method: it checks shapes and dtypes, forwards pointers and sizes, and raises
``MBLError`` on a non-zero status.  Loading fails loudly when the library has not
been built (there is no CPU fallback).
"""
import ctypes
import functools
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmbl_gb300.so")

MBL_OK = 0
MBL_ERR_ARG = -1
MBL_ERR_WORKSPACE = -2
MBL_ERR_CUDA = -3
MBL_ERR_NOT_CONVERGED = -4
MBL_ERR_BREAKDOWN = -5
MBL_ERR_NUMERIC = -6
MBL_F32 = 0
MBL_F64 = 1
MODE_FP64 = 0
MODE_MIXED = 1

EXPORTED = ("mbl_status_string", "mbl_basis_size", "mbl_basis_build", "mbl_basis_rank",
            "mbl_hamiltonian_apply", "mbl_lobpcg_workspace_size", "mbl_lobpcg_solve",
            "mbl_bounds_workspace_size", "mbl_spectrum_bounds", "mbl_lobpcg_solve_noalloc",
            "mbl_set_product_tile_bits", "mbl_set_product_lane_bytes", "mbl_batched_workspace_size",
            "mbl_lobpcg_solve_batched", "mbl_kernel_launch_count",
            "mbl_set_product_schedule", "mbl_autotune_product", "mbl_set_gram_engine",
            "mbl_gram_workspace_size", "mbl_gram", "mbl_product_tile_width", "mbl_gap_ratio",
            "mbl_entanglement_workspace_size", "mbl_entanglement_entropy", "mbl_update")
NOALLOC_SCRATCH_BYTES = 16 << 20


class MBLError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (what, status_string(status), status))


class Chain(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int), ("n_up", ctypes.c_int), ("periodic", ctypes.c_int),
                ("delta", ctypes.c_double), ("h_host", ctypes.POINTER(ctypes.c_double))]


class LobpcgOpts(ctypes.Structure):
    _fields_ = [("nev", ctypes.c_int), ("k", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("pcg_iters", ctypes.c_int), ("tol", ctypes.c_double), ("pcg_tol", ctypes.c_double),
                ("norm_h", ctypes.c_double), ("mode", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("timing", ctypes.c_int)]


class ProductChoice(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int), ("lane_bytes", ctypes.c_int), ("tile_bits", ctypes.c_int),
                ("microseconds", ctypes.c_double)]


class LobpcgStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("matvecs", ctypes.c_int64),
                ("seconds", ctypes.c_double), ("max_rel_resid", ctypes.c_double),
                ("norm_h", ctypes.c_double), ("t_setup", ctypes.c_double), ("t_resid", ctypes.c_double),
                ("t_pcg", ctypes.c_double), ("t_wp", ctypes.c_double), ("t_gram", ctypes.c_double),
                ("t_small", ctypes.c_double), ("t_update", ctypes.c_double), ("t_refresh", ctypes.c_double),
                ("t_hrr", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


@functools.lru_cache(maxsize=1)
def lib():
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("CUDA library %s is not built; run __graft_entry__.build()" % LIB_PATH)
    so = ctypes.CDLL(LIB_PATH)
    p, i32, i64, f64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    pch = ctypes.POINTER(Chain)
    popt = ctypes.POINTER(LobpcgOpts)
    so.mbl_status_string.restype = ctypes.c_char_p
    so.mbl_status_string.argtypes = [i32]
    so.mbl_kernel_launch_count.restype = i64
    so.mbl_kernel_launch_count.argtypes = []
    so.mbl_basis_size.restype = i64
    so.mbl_basis_size.argtypes = [i32, i32]
    so.mbl_basis_build.restype = i32
    so.mbl_basis_build.argtypes = [i32, i32, p, i64, p]
    so.mbl_basis_rank.restype = i32
    so.mbl_basis_rank.argtypes = [i32, i32, p, p, i64, p]
    so.mbl_hamiltonian_apply.restype = i32
    so.mbl_hamiltonian_apply.argtypes = [pch, f64, i32, p, i64, p, i64, i64, i32, p]
    so.mbl_batched_workspace_size.restype = i32
    so.mbl_batched_workspace_size.argtypes = [i32, pch, popt, i32, ctypes.POINTER(sz)]
    so.mbl_lobpcg_solve_batched.restype = i32
    so.mbl_lobpcg_solve_batched.argtypes = [i32, pch, p, popt, p, i32, p, sz, p, p, p,
                                            ctypes.POINTER(LobpcgStats), p]
    so.mbl_set_product_lane_bytes.restype = i32
    so.mbl_set_product_lane_bytes.argtypes = [i32, i32, i32]
    so.mbl_set_product_schedule.restype = i32
    so.mbl_set_product_schedule.argtypes = [i32, i32, i32]
    so.mbl_product_tile_width.restype = i32
    so.mbl_product_tile_width.argtypes = [i32, i32, i32, i32]
    so.mbl_gap_ratio.restype = i32
    so.mbl_gap_ratio.argtypes = [i32, i32, p, i64, p, p, p]
    so.mbl_entanglement_workspace_size.restype = i32
    so.mbl_entanglement_workspace_size.argtypes = [pch, i32, i32, ctypes.POINTER(sz)]
    so.mbl_entanglement_entropy.restype = i32
    so.mbl_entanglement_entropy.argtypes = [pch, i32, i32, p, i64, p, p, sz, p]
    so.mbl_set_gram_engine.restype = i32
    so.mbl_set_gram_engine.argtypes = [i32]
    so.mbl_gram_workspace_size.restype = i32
    so.mbl_gram_workspace_size.argtypes = [i64, i32, i32, ctypes.POINTER(sz)]
    so.mbl_update.restype = i32
    so.mbl_update.argtypes = [p, i64, i32, p, i64, i32, p, i64, p, i64, i64, f64, f64, i32, i32, p]
    so.mbl_gram.restype = i32
    so.mbl_gram.argtypes = [p, i64, i32, p, i64, i32, i64, p, i64, i32, i32, p, sz, p]
    so.mbl_autotune_product.restype = i32
    so.mbl_autotune_product.argtypes = [pch, i32, p, p, i64, i32, i32, ctypes.POINTER(ProductChoice), p]
    so.mbl_set_product_tile_bits.restype = i32
    so.mbl_set_product_tile_bits.argtypes = [i32, i32, i32]
    so.mbl_lobpcg_workspace_size.restype = i32
    so.mbl_lobpcg_workspace_size.argtypes = [pch, popt, ctypes.POINTER(sz)]
    so.mbl_lobpcg_solve.restype = i32
    so.mbl_lobpcg_solve.argtypes = [pch, f64, popt, p, p, sz, p, p, p, ctypes.POINTER(LobpcgStats), p]
    so.mbl_lobpcg_solve_noalloc.restype = i32
    so.mbl_lobpcg_solve_noalloc.argtypes = [pch, f64, popt, p, p, p, p, ctypes.POINTER(LobpcgStats), p]
    so.mbl_bounds_workspace_size.restype = i32
    so.mbl_bounds_workspace_size.argtypes = [pch, i32, ctypes.POINTER(sz)]
    so.mbl_spectrum_bounds.restype = i32
    so.mbl_spectrum_bounds.argtypes = [pch, i32, f64, i32, p, p, sz, p, p, p, p]
    return so


def status_string(status):
    return lib().mbl_status_string(int(status)).decode()


def kernel_launch_count():
    """Kernels the library has launched in this process (graph replays count their
    kernel nodes)."""
    return int(lib().mbl_kernel_launch_count())


def _check(rc, what, ok=(MBL_OK,)):
    if rc not in ok:
        raise MBLError(rc, what)
    return rc


def _torch():
    import torch
    return torch


def _stream_ptr(t):
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _dev(t, dtype, what):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % what)
    if t.dtype != dtype:
        raise TypeError("%s must have dtype %s" % (what, dtype))
    return ctypes.c_void_p(t.data_ptr())


def make_chain(L, h, delta=1.0, periodic=False, n_up=None):
    """Marshal one disorder realisation into the C struct (h copied to a host array
    kept alive on the returned object)."""
    hh = np.ascontiguousarray(np.asarray(h, dtype=np.float64))
    c = Chain(int(L), int(L) // 2 if n_up is None else int(n_up), int(bool(periodic)), float(delta),
              hh.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    c._keep = hh
    return c


def basis_size(L, n_up):
    return int(lib().mbl_basis_size(int(L), int(n_up)))


def basis_build(L, n_up, states):
    """states: int32/uint32-sized CUDA tensor (torch.int32) of basis_size(L, n_up) entries."""
    torch = _torch()
    ptr = _dev(states, torch.int32, "states")
    _check(lib().mbl_basis_build(int(L), int(n_up), ptr, states.numel(), _stream_ptr(states)),
           "mbl_basis_build")
    return states


def basis_rank(L, n_up, words, ranks):
    torch = _torch()
    wp = _dev(words, torch.int32, "words")
    rp = _dev(ranks, torch.int64, "ranks")
    if words.numel() != ranks.numel():
        raise ValueError("words and ranks differ in size")
    _check(lib().mbl_basis_rank(int(L), int(n_up), wp, rp, words.numel(), _stream_ptr(words)),
           "mbl_basis_rank")
    return ranks


def hamiltonian_apply(chain, sigma, X, Y):
    """Y = (H - sigma I) X for 2-D CUDA tensors (float32 or float64, row stride >= k,
    unit column stride)."""
    torch = _torch()
    if X.dim() != 2 or Y.dim() != 2 or X.shape != Y.shape:
        raise ValueError("X and Y must be 2-D with equal shapes")
    if X.dtype != Y.dtype or X.dtype not in (torch.float32, torch.float64):
        raise TypeError("X and Y must both be float32 or float64")
    if X.stride(1) != 1 or Y.stride(1) != 1:
        raise ValueError("columns must be contiguous")
    dt = MBL_F32 if X.dtype == torch.float32 else MBL_F64
    n, k = X.shape
    _check(lib().mbl_hamiltonian_apply(ctypes.byref(chain), float(sigma), dt, _dev(X, X.dtype, "X"),
                                       X.stride(0), _dev(Y, Y.dtype, "Y"), Y.stride(0), n, k,
                                       _stream_ptr(X)), "mbl_hamiltonian_apply")
    return Y


def set_product_tile_bits(k, dtype, bits):
    """Tile width of the product kernels for block width k and dtype (torch.float32 or
    torch.float64): 0 heuristic, -1 untiled, 2..16 low bits per tile."""
    torch = _torch()
    dt = MBL_F32 if dtype == torch.float32 else MBL_F64
    _check(lib().mbl_set_product_tile_bits(int(k), dt, int(bits)), "mbl_set_product_tile_bits")


def set_product_lane_bytes(k, dtype, nbytes):
    """Bytes per lane per neighbour row in the tiled product (16, 32, or 0 = default)."""
    torch = _torch()
    dt = MBL_F32 if dtype == torch.float32 else MBL_F64
    _check(lib().mbl_set_product_lane_bytes(int(k), dt, int(nbytes)), "mbl_set_product_lane_bytes")


def set_product_schedule(k, dtype, schedule):
    """mbl_set_product_schedule: 0 by size, 1 persistent, 2 ordered, 3 staged, 4 streamed,
    5 slab."""
    torch = _torch()
    dt = MBL_F32 if dtype == torch.float32 else MBL_F64
    _check(lib().mbl_set_product_schedule(int(k), dt, int(schedule)), "mbl_set_product_schedule")


def product_tile_width(L, dtype, k, schedule):
    """mbl_product_tile_width: the tile width B work order `schedule` uses (0: none)."""
    torch = _torch()
    dt = MBL_F32 if dtype == torch.float32 else MBL_F64
    w = lib().mbl_product_tile_width(int(L), dt, int(k), int(schedule))
    _check(w if w < 0 else MBL_OK, "mbl_product_tile_width")
    return w


def set_gram_engine(engine):
    """mbl_set_gram_engine: 0 default, 1 CUDA cores, 2 tensor cores (tcgen05 TF32 x3)."""
    _check(lib().mbl_set_gram_engine(int(engine)), "mbl_set_gram_engine")


def gram(A, B, precision="f32", engine=0):
    """mbl_gram: C = A^T B for contiguous FP64 CUDA tensors A (n x p), B (n x q); returns
    C as a new p x q FP64 CUDA tensor."""
    torch = _torch()
    if A.dim() != 2 or B.dim() != 2 or A.shape[0] != B.shape[0] or not (A.is_contiguous() and B.is_contiguous()):
        raise ValueError("A (n x p), B (n x q): contiguous, same n")
    n, p_ = A.shape
    q = B.shape[1]
    sz = ctypes.c_size_t(0)
    _check(lib().mbl_gram_workspace_size(int(n), int(p_), int(q), ctypes.byref(sz)), "mbl_gram_workspace_size")
    ws = torch.empty(sz.value, dtype=torch.uint8, device=A.device)
    C = torch.empty((p_, q), dtype=torch.float64, device=A.device)
    prec = MBL_F32 if precision == "f32" else MBL_F64
    _check(lib().mbl_gram(_dev(A, torch.float64, "A"), int(p_), int(p_), _dev(B, torch.float64, "B"), int(q), int(q),
                          int(n), _dev(C, torch.float64, "C"), int(q), prec, int(engine), _dev(ws, torch.uint8, "ws"),
                          ws.numel(), _stream_ptr(A)), "mbl_gram")
    return C


def update(A, M, C=None, alpha=1.0, beta=0.0, precision="f32", engine=0):
    """mbl_update: D = beta C + alpha A M for contiguous FP64 CUDA tensors A (n x p), M (p x q)
    and optional C (n x q); returns D as a new n x q FP64 CUDA tensor."""
    torch = _torch()
    if A.dim() != 2 or M.dim() != 2 or A.shape[1] != M.shape[0] or not (A.is_contiguous() and M.is_contiguous()):
        raise ValueError("A (n x p), M (p x q): contiguous")
    n, p_ = A.shape
    q = M.shape[1]
    if C is not None and (C.shape != (n, q) or not C.is_contiguous()):
        raise ValueError("C: contiguous n x q")
    D = torch.empty((n, q), dtype=torch.float64, device=A.device)
    prec = MBL_F32 if precision == "f32" else MBL_F64
    _check(lib().mbl_update(_dev(A, torch.float64, "A"), int(p_), int(p_), _dev(M, torch.float64, "M"), int(q), int(q),
                            _dev(C, torch.float64, "C") if C is not None else None, int(q),
                            _dev(D, torch.float64, "D"), int(q), int(n), float(alpha), float(beta), prec, int(engine),
                            _stream_ptr(A)), "mbl_update")
    return D


def autotune_product(chain, X, Y, reps=5):
    """mbl_autotune_product on the contiguous n x k CUDA tensors X (read) and Y
    (overwritten); returns the kept choice as a dict."""
    torch = _torch()
    if X.dtype not in (torch.float32, torch.float64) or Y.dtype != X.dtype or X.dim() != 2 or Y.shape != X.shape:
        raise ValueError("X, Y: equal n x k float32/float64 CUDA tensors")
    if not (X.is_contiguous() and Y.is_contiguous()):
        raise ValueError("X, Y must be contiguous (ld = k)")
    dt = MBL_F32 if X.dtype == torch.float32 else MBL_F64
    n, k = X.shape
    ch = ProductChoice()
    _check(lib().mbl_autotune_product(ctypes.byref(chain), dt, _dev(X, X.dtype, "X"), _dev(Y, Y.dtype, "Y"), int(n),
                                      int(k), int(reps), ctypes.byref(ch), _stream_ptr(X)), "mbl_autotune_product")
    return {f: getattr(ch, f) for f, _ in ch._fields_}


def make_opts(nev, k, tol=1e-8, max_iter=200, pcg_iters=50, pcg_tol=0.0, norm_h=0.0,
              mode=MODE_MIXED, use_graph=1, timing=0):
    return LobpcgOpts(int(nev), int(k), int(max_iter), int(pcg_iters), float(tol), float(pcg_tol),
                      float(norm_h), int(mode), int(use_graph), int(timing))


def lobpcg_workspace_size(chain, opts):
    out = ctypes.c_size_t(0)
    _check(lib().mbl_lobpcg_workspace_size(ctypes.byref(chain), ctypes.byref(opts), ctypes.byref(out)),
           "mbl_lobpcg_workspace_size")
    return int(out.value)


def lobpcg_solve(chain, sigma, opts, X0, workspace, evecs=None, allow_not_converged=False):
    """Returns (evals ndarray, resid ndarray, stats dict, status).  X0: n x k float64 CUDA
    tensor; workspace: uint8 CUDA tensor of >= lobpcg_workspace_size bytes; evecs:
    optional n x nev float64 CUDA tensor."""
    torch = _torch()
    nev = opts.nev
    evals = np.zeros(nev, dtype=np.float64)
    resid = np.zeros(nev, dtype=np.float64)
    stats = LobpcgStats()
    ev_ptr = _dev(evecs, torch.float64, "evecs") if evecs is not None else None
    if evecs is not None and (evecs.shape != (X0.shape[0], nev) or not evecs.is_contiguous()):
        raise ValueError("evecs must be a contiguous n x nev tensor")
    if not X0.is_contiguous() or X0.dim() != 2 or X0.shape[1] != opts.k:
        raise ValueError("X0 must be a contiguous n x k tensor")
    ok = (MBL_OK, MBL_ERR_NOT_CONVERGED) if allow_not_converged else (MBL_OK,)
    rc = lib().mbl_lobpcg_solve(ctypes.byref(chain), float(sigma), ctypes.byref(opts),
                                _dev(X0, torch.float64, "X0"), _dev(workspace, torch.uint8, "workspace"),
                                workspace.numel(), evals.ctypes.data_as(ctypes.c_void_p), ev_ptr,
                                resid.ctypes.data_as(ctypes.c_void_p), ctypes.byref(stats),
                                _stream_ptr(X0))
    _check(rc, "mbl_lobpcg_solve", ok)
    return evals, resid, stats.as_dict(), rc


def lobpcg_solve_noalloc(chain, sigma, opts, X0, evecs=None, allow_not_converged=False):
    """mbl_lobpcg_solve_noalloc: the same solve with the library's fixed in-device
    workspace (no allocation by the library or by this wrapper's callee).  Returns
    (evals, resid, stats dict, status)."""
    torch = _torch()
    nev = opts.nev
    evals = np.zeros(nev, dtype=np.float64)
    resid = np.zeros(nev, dtype=np.float64)
    stats = LobpcgStats()
    ev_ptr = _dev(evecs, torch.float64, "evecs") if evecs is not None else None
    if evecs is not None and (evecs.shape != (X0.shape[0], nev) or not evecs.is_contiguous()):
        raise ValueError("evecs must be a contiguous n x nev tensor")
    if not X0.is_contiguous() or X0.dim() != 2 or X0.shape[1] != opts.k:
        raise ValueError("X0 must be a contiguous n x k tensor")
    ok = (MBL_OK, MBL_ERR_NOT_CONVERGED) if allow_not_converged else (MBL_OK,)
    rc = lib().mbl_lobpcg_solve_noalloc(ctypes.byref(chain), float(sigma), ctypes.byref(opts),
                                        _dev(X0, torch.float64, "X0"), evals.ctypes.data_as(ctypes.c_void_p),
                                        ev_ptr, resid.ctypes.data_as(ctypes.c_void_p), ctypes.byref(stats),
                                        _stream_ptr(X0))
    _check(rc, "mbl_lobpcg_solve_noalloc", ok)
    return evals, resid, stats.as_dict(), rc


def chain_array(chains):
    """A contiguous C array of mbl_chain structs (keeps the field arrays alive)."""
    arr = (Chain * len(chains))(*chains)
    arr._keep = [c._keep for c in chains]
    return arr


def batched_workspace_size(chains, opts, nstreams):
    arr = chain_array(chains)
    out = ctypes.c_size_t(0)
    _check(lib().mbl_batched_workspace_size(len(chains), arr, ctypes.byref(opts), int(nstreams),
                                            ctypes.byref(out)), "mbl_batched_workspace_size")
    return int(out.value)


def lobpcg_solve_batched(chains, opts, X0, workspace, nstreams, sigmas=None, evecs=None,
                         allow_not_converged=False):
    """mbl_lobpcg_solve_batched.  X0: (sum n_i) x k float64 CUDA tensor (the problems'
    start blocks stacked); evecs: optional (sum n_i) x nev tensor.  Returns (evals
    nprob x nev, resid nprob x nev, list of stats dicts, status)."""
    torch = _torch()
    nprob, nev = len(chains), opts.nev
    arr = chain_array(chains)
    evals = np.zeros((nprob, nev), dtype=np.float64)
    resid = np.zeros((nprob, nev), dtype=np.float64)
    stats = (LobpcgStats * nprob)()
    sg = None
    if sigmas is not None:
        sg_arr = np.ascontiguousarray(np.asarray(sigmas, dtype=np.float64))
        sg = sg_arr.ctypes.data_as(ctypes.c_void_p)
    ev_ptr = _dev(evecs, torch.float64, "evecs") if evecs is not None else None
    ok = (MBL_OK, MBL_ERR_NOT_CONVERGED) if allow_not_converged else (MBL_OK,)
    rc = lib().mbl_lobpcg_solve_batched(nprob, arr, sg, ctypes.byref(opts), _dev(X0, torch.float64, "X0"),
                                        int(nstreams), _dev(workspace, torch.uint8, "workspace"),
                                        workspace.numel(), evals.ctypes.data_as(ctypes.c_void_p), ev_ptr,
                                        resid.ctypes.data_as(ctypes.c_void_p), stats, _stream_ptr(X0))
    _check(rc, "mbl_lobpcg_solve_batched", ok)
    return evals, resid, [st.as_dict() for st in stats], rc


def bounds_workspace_size(chain, k):
    out = ctypes.c_size_t(0)
    _check(lib().mbl_bounds_workspace_size(ctypes.byref(chain), int(k), ctypes.byref(out)),
           "mbl_bounds_workspace_size")
    return int(out.value)


def spectrum_bounds(chain, X0, workspace, tol=1e-10, max_iter=500):
    """(E_min, E_max, Lanczos steps): mbl_spectrum_bounds, one FP64 Lanczos recurrence on H
    started from column 0 of the n x k block X0."""
    torch = _torch()
    emin, emax, iters = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(lib().mbl_spectrum_bounds(ctypes.byref(chain), X0.shape[1], float(tol), int(max_iter),
                                     _dev(X0, torch.float64, "X0"), _dev(workspace, torch.uint8, "workspace"),
                                     workspace.numel(), ctypes.byref(emin), ctypes.byref(emax),
                                     ctypes.byref(iters), _stream_ptr(X0)), "mbl_spectrum_bounds")
    return emin.value, emax.value, iters.value


def gap_ratio(evals, m=None):
    """mbl_gap_ratio on the rows of a 2-D float64 CUDA tensor (one realization per row,
    its first m entries the levels): returns (r_mean float64, count int32) CUDA tensors."""
    torch = _torch()
    if evals.dim() != 2 or evals.dtype != torch.float64 or not evals.is_cuda or evals.stride(1) != 1:
        raise ValueError("evals: 2-D float64 CUDA tensor with unit column stride")
    nprob, ld = evals.shape[0], evals.stride(0) if evals.shape[0] > 1 else evals.shape[1]
    m = evals.shape[1] if m is None else int(m)
    r_mean = torch.empty(nprob, dtype=torch.float64, device=evals.device)
    count = torch.empty(nprob, dtype=torch.int32, device=evals.device)
    _check(lib().mbl_gap_ratio(int(nprob), m, ctypes.c_void_p(evals.data_ptr()), int(ld),
                               ctypes.c_void_p(r_mean.data_ptr()), ctypes.c_void_p(count.data_ptr()),
                               _stream_ptr(evals)), "mbl_gap_ratio")
    return r_mean, count


def entanglement_workspace_size(chain, l_a, nvec):
    sz = ctypes.c_size_t(0)
    _check(lib().mbl_entanglement_workspace_size(ctypes.byref(chain), int(l_a), int(nvec), ctypes.byref(sz)),
           "mbl_entanglement_workspace_size")
    return sz.value


def entanglement_entropy(chain, l_a, V, workspace=None):
    """mbl_entanglement_entropy of the columns of the n x nvec float64 CUDA tensor V (unit
    column stride); returns a float64 CUDA tensor of nvec entropies."""
    torch = _torch()
    if V.dim() != 2 or V.dtype != torch.float64 or not V.is_cuda or V.stride(1) != 1:
        raise ValueError("V: 2-D float64 CUDA tensor with unit column stride")
    nvec = V.shape[1]
    ldv = V.stride(0) if V.shape[0] > 1 else nvec
    need = entanglement_workspace_size(chain, l_a, nvec)
    if workspace is None:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=V.device)
    S = torch.empty(nvec, dtype=torch.float64, device=V.device)
    _check(lib().mbl_entanglement_entropy(ctypes.byref(chain), int(l_a), int(nvec), ctypes.c_void_p(V.data_ptr()),
                                          int(ldv), ctypes.c_void_p(S.data_ptr()),
                                          _dev(workspace, torch.uint8, "workspace"), workspace.numel(),
                                          _stream_ptr(V)), "mbl_entanglement_entropy")
    return S
