"""Oracle: S^z-sector basis and Hamiltonian products (Sec. 2.1).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The model is Eq. (model): H = sum_<ij> S_i.S_j + sum_i h_i S^z_i, with S = sigma/2,
generalised by an anisotropy ``delta`` on the Z_iZ_j part (delta = 1 is the paper's
model).  Eq. (Hmatrix) writes it as a sum of one 4x4 bond matrix per bond plus one
2x2 field term per site.  The sector with ``n_up`` up spins has dimension
C(L, n_up) (Sec. 2.1, Table 1).  States are L-bit words, bit i = site i, bit 1 = up,
listed in ascending integer order.

The C part (``mbl_oracle.c``) does the row loops; this module adds the ctypes
wrappers and two brute-force builders that pin it:
  * ``dense_full_pauli`` -- the full 2^L x 2^L matrix assembled from Kronecker
    products of Pauli matrices exactly as Eq. (Hmatrix) states it;
  * ``dense_sector``     -- the sector block obtained by applying the C product to
    the identity, column by column.
"""
import ctypes
import functools

import numpy as np

from . import build as _build


class Chain:
    """One disorder realisation: L sites, open or periodic, anisotropy delta,
    fields h (length L, FP64).  Eq. (model)."""

    def __init__(self, L, h, delta=1.0, periodic=False, n_up=None):
        self.L = int(L)
        self.h = np.ascontiguousarray(np.asarray(h, dtype=np.float64))
        if self.h.shape != (self.L,):
            raise ValueError("h must have length L")
        self.delta = float(delta)
        self.periodic = bool(periodic)
        self.n_up = self.L // 2 if n_up is None else int(n_up)

    def num_bonds(self):
        return (self.L - 1) + (1 if (self.periodic and self.L > 2) else 0)


@functools.lru_cache(maxsize=1)
def lib():
    path = _build.build()
    so = ctypes.CDLL(path)
    i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    p = ctypes.c_void_p
    so.orc_binomial.restype = i64
    so.orc_binomial.argtypes = [i32, i32]
    so.orc_sector_dim.restype = i64
    so.orc_sector_dim.argtypes = [i32, i32]
    so.orc_basis_enumerate.restype = i64
    so.orc_basis_enumerate.argtypes = [i32, i32, p, i64]
    so.orc_rank_many.restype = i32
    so.orc_rank_many.argtypes = [p, i64, p, p, i64]
    so.orc_diag.restype = i32
    so.orc_diag.argtypes = [i32, i32, f64, p, p, i64, p]
    so.orc_fold_diag.restype = i32
    so.orc_fold_diag.argtypes = [i32, i32, f64, p, f64, p, i64, p]
    so.orc_flippable.restype = i32
    so.orc_flippable.argtypes = [i32, i32, ctypes.c_uint32]
    for name in ("orc_apply_f64", "orc_apply_f32"):
        fn = getattr(so, name)
        fn.restype = i32
        fn.argtypes = [i32, i32, f64, p, f64, p, i64, i32, p, i64, p, i64]
    so.orc_apply_rows_f64.restype = i32
    so.orc_apply_rows_f64.argtypes = [i32, i32, f64, p, f64, p, i64, i32, p, i64, p, i64, p]
    return so


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def sector_dim(L, n_up):
    return int(lib().orc_sector_dim(L, n_up))


@functools.lru_cache(maxsize=8)
def _basis_cached(L, n_up):
    n = sector_dim(L, n_up)
    if n < 0:
        raise ValueError("bad (L, n_up)")
    states = np.empty(n, dtype=np.uint32)
    cnt = lib().orc_basis_enumerate(L, n_up, _ptr(states), n)
    if cnt != n:
        raise RuntimeError("enumeration count %d != C(L,n_up) %d" % (cnt, n))
    states.setflags(write=False)
    return states


def basis(L, n_up=None):
    """Ascending list of the L-bit words with popcount n_up (default L/2)."""
    return _basis_cached(int(L), int(L) // 2 if n_up is None else int(n_up))


def rank(states, query):
    """Position of each query word in ``states`` (-1 when absent), by bisection."""
    q = np.ascontiguousarray(np.asarray(query, dtype=np.uint32))
    out = np.empty(q.shape, dtype=np.int64)
    lib().orc_rank_many(_ptr(states), states.size, _ptr(q), _ptr(out), q.size)
    return out


def diag(chain):
    """d(s) for every sector state (FP64)."""
    st = basis(chain.L, chain.n_up)
    d = np.empty(st.size, dtype=np.float64)
    rc = lib().orc_diag(chain.L, int(chain.periodic), chain.delta, _ptr(chain.h), _ptr(st),
                        st.size, _ptr(d))
    if rc != 0:
        raise ValueError("orc_diag failed")
    return d


def flippable(chain):
    """f(s): number of bonds whose spins differ, for every sector state."""
    st = basis(chain.L, chain.n_up)
    so = lib()
    return np.array([so.orc_flippable(chain.L, int(chain.periodic), int(s)) for s in st],
                    dtype=np.int64)


def fold_diag(chain, sigma):
    """diag((H - sigma)^2) = (d - sigma)^2 + f/4: the Jacobi preconditioner of the
    PCG inner solve (Sec. 3.2)."""
    st = basis(chain.L, chain.n_up)
    out = np.empty(st.size, dtype=np.float64)
    rc = lib().orc_fold_diag(chain.L, int(chain.periodic), chain.delta, _ptr(chain.h),
                             float(sigma), _ptr(st), st.size, _ptr(out))
    if rc != 0:
        raise ValueError("orc_fold_diag failed")
    return out


def apply(chain, sigma, X):
    """Y = (H - sigma I) X for a row-major n x k block; FP64 in and out, or
    FP32 in and out (FP32 accumulation) when X is float32."""
    st = basis(chain.L, chain.n_up)
    X = np.asarray(X)
    vec = X.ndim == 1
    if vec:
        X = X[:, None]
    if X.dtype == np.float32:
        fn, dt = lib().orc_apply_f32, np.float32
    else:
        fn, dt = lib().orc_apply_f64, np.float64
    X = np.ascontiguousarray(X, dtype=dt)
    n, k = X.shape
    if n != st.size:
        raise ValueError("row count %d != sector dimension %d" % (n, st.size))
    Y = np.empty((n, k), dtype=dt)
    rc = fn(chain.L, int(chain.periodic), chain.delta, _ptr(chain.h), float(sigma), _ptr(st),
            n, k, _ptr(X), k, _ptr(Y), k)
    if rc != 0:
        raise ValueError("oracle apply failed (%d)" % rc)
    return Y[:, 0] if vec else Y


def apply_rows(chain, sigma, X, rows):
    """Rows ``rows`` of (H - sigma I) X, without the full product (FP64)."""
    st = basis(chain.L, chain.n_up)
    X = np.ascontiguousarray(X, dtype=np.float64)
    n, k = X.shape
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    out = np.empty((rows.size, k), dtype=np.float64)
    rc = lib().orc_apply_rows_f64(chain.L, int(chain.periodic), chain.delta, _ptr(chain.h),
                                  float(sigma), _ptr(st), n, k, _ptr(X), k, _ptr(rows),
                                  rows.size, _ptr(out))
    if rc != 0:
        raise ValueError("oracle apply_rows failed")
    return out


def dense_sector(chain):
    """The sector block of H as a dense FP64 matrix, by applying H to the identity."""
    n = sector_dim(chain.L, chain.n_up)
    return apply(chain, 0.0, np.eye(n))


def sparse_sector(chain):
    """The sector block of H as a scipy CSR matrix, from the matrix elements of
    Eq. (Hmatrix) entry by entry: d(s) on the diagonal, and for every bond (i, j) and
    every state s whose spins i and j differ, 1/2 at (rank(s'), rank(s)) with s' = s
    with those two spins exchanged (ranks by bisection in the enumerated basis).
    For the shift-invert Lanczos reference at sizes where the dense matrix does not fit."""
    import scipy.sparse as sp
    st = basis(chain.L, chain.n_up)
    n = st.size
    L = chain.L
    bonds = [(i, i + 1) for i in range(L - 1)]
    if chain.periodic and L > 2:
        bonds.append((L - 1, 0))
    rows, cols, vals = [np.arange(n)], [np.arange(n)], [diag(chain)]
    for (i, j) in bonds:
        differ = ((st >> np.uint32(i)) ^ (st >> np.uint32(j))) & np.uint32(1)
        src = np.nonzero(differ)[0]
        dst = rank(st, st[src] ^ np.uint32((1 << i) | (1 << j)))
        if np.any(dst < 0):
            raise RuntimeError("an exchanged state left the sector")
        rows.append(dst)
        cols.append(src)
        vals.append(np.full(src.size, 0.5))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


# Pauli matrices written in the single-site basis (index 0 = bit 0 = spin down,
# index 1 = bit 1 = spin up), so that Z|up> = +|up>, X|up> = |down> and
# Y|up> = i|down>, Y|down> = -i|up>.
_PAULI = {
    "I": np.eye(2),
    "X": np.array([[0.0, 1.0], [1.0, 0.0]]),
    "Y": np.array([[0.0, 1.0j], [-1.0j, 0.0]]),
    "Z": np.array([[-1.0, 0.0], [0.0, 1.0]]),
}


def _site_op(L, ops):
    """Kronecker product over sites with ``ops[i]`` on site i and I elsewhere.
    Site i is bit i of the basis index, so site L-1 is the leftmost factor."""
    m = np.ones((1, 1), dtype=complex)
    for i in reversed(range(L)):
        m = np.kron(m, _PAULI[ops.get(i, "I")])
    return m


def dense_full_pauli(chain):
    """Full 2^L x 2^L matrix of Eq. (Hmatrix) built from Pauli Kronecker products:
    sum over bonds of (X X + Y Y + delta Z Z)/4 on the two bond sites, plus
    sum_i h_i Z_i / 2.  Brute force; for L <= 12."""
    L = chain.L
    if L > 12:
        raise ValueError("dense_full_pauli is for L <= 12")
    H = np.zeros((2 ** L, 2 ** L), dtype=complex)
    bonds = [(i, i + 1) for i in range(L - 1)]
    if chain.periodic and L > 2:
        bonds.append((L - 1, 0))
    for (i, j) in bonds:
        H += 0.25 * _site_op(L, {i: "X", j: "X"})
        H += 0.25 * _site_op(L, {i: "Y", j: "Y"})
        H += 0.25 * chain.delta * _site_op(L, {i: "Z", j: "Z"})
    for i in range(L):
        H += 0.5 * chain.h[i] * _site_op(L, {i: "Z"})
    return H


def total_sz_full(L):
    """sum_i Z_i / 2 in the full space (its eigenvalue labels the sectors)."""
    return sum(0.5 * _site_op(L, {i: "Z"}) for i in range(L))
