"""Pins of the oracle's Hamiltonian product (Sec. 2.1, Eq. (model), Eq. (Hmatrix)).

The C product is checked against things it does not compute itself:
  * the full 2^L matrix assembled from Pauli Kronecker products (Eq. (Hmatrix)),
    restricted to the sector, element by element;
  * S^z conservation of that full matrix (Sec. 2.1: H commutes with total S^z);
  * symmetry, the closed-form trace, and the delta = 0 free-fermion spectrum.
"""
from math import comb

import numpy as np
import pytest

import workloads as wl
from oracle import closed_form as cf
from oracle import hamiltonian as ham


def _chain(L, periodic, delta, W=3.0, seed=3, n_up=None):
    return ham.Chain(L, wl.fields(L, W, seed), delta=delta, periodic=periodic, n_up=n_up)


@pytest.mark.parametrize("L", [4, 6, 8, 10])
@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("delta", [0.0, 0.7, 1.0])
def test_sector_block_equals_pauli_build(L, periodic, delta):
    ch = _chain(L, periodic, delta, seed=L)
    full = ham.dense_full_pauli(ch)
    assert np.abs(full.imag).max() == 0.0
    for n_up in range(L + 1):
        ch.n_up = n_up
        st = ham.basis(L, n_up).astype(np.int64)
        ref = full.real[np.ix_(st, st)]
        got = ham.dense_sector(ch)
        assert np.array_equal(got, ref) or np.abs(got - ref).max() <= 1e-14 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("L", [4, 6, 8, 10])
@pytest.mark.parametrize("periodic", [False, True])
def test_sparse_sector_equals_pauli_build(L, periodic):
    """The entry-by-entry sparse sector matrix (used by the shift-invert references) is
    the Pauli-Kronecker matrix of Eq. (Hmatrix) restricted to each sector."""
    pytest.importorskip("scipy.sparse")
    ch = _chain(L, periodic, 0.8, seed=20 + L)
    full = ham.dense_full_pauli(ch).real
    for n_up in range(L + 1):
        ch.n_up = n_up
        st = ham.basis(L, n_up).astype(np.int64)
        got = ham.sparse_sector(ch).toarray()
        assert np.abs(got - full[np.ix_(st, st)]).max() <= 1e-14 * max(1.0, np.abs(full).max())


def test_sparse_sector_product_matches_c_product_l16():
    pytest.importorskip("scipy.sparse")
    ch = _chain(16, True, 1.0, W=8.0, seed=5)
    X = wl.block(ham.sector_dim(16, 8), 3, 7)
    d = ham.sparse_sector(ch) @ X - ham.apply(ch, 0.0, X)
    assert np.abs(d).max() <= 1e-12 * np.abs(X).max()


@pytest.mark.parametrize("periodic", [False, True])
def test_full_hamiltonian_conserves_total_sz(periodic):
    L = 8
    ch = _chain(L, periodic, 1.0)
    full = ham.dense_full_pauli(ch)
    sz = ham.total_sz_full(L)
    assert np.abs(full @ sz - sz @ full).max() < 1e-12
    # no element couples words of different popcount
    pc = np.array([bin(s).count("1") for s in range(2 ** L)])
    rows, cols = np.nonzero(np.abs(full) > 0)
    assert np.all(pc[rows] == pc[cols])


@pytest.mark.parametrize("L,periodic", [(10, False), (12, True), (12, False)])
def test_sector_matrix_is_symmetric(L, periodic):
    Hd = ham.dense_sector(_chain(L, periodic, 1.0))
    assert np.array_equal(Hd, Hd.T)


def test_adjoint_identity_large():
    ch = _chain(18, True, 1.0, W=8.0, seed=11)
    n = ham.sector_dim(18, 9)
    x = wl.block(n, 2, 1)
    y = wl.block(n, 2, 2)
    lhs = np.sum(y * ham.apply(ch, 0.3, x), axis=0)
    rhs = np.sum(ham.apply(ch, 0.3, y) * x, axis=0)
    scale = np.linalg.norm(x, axis=0) * np.linalg.norm(y, axis=0) * 20.0
    assert np.all(np.abs(lhs - rhs) <= 1e-13 * scale)


@pytest.mark.parametrize("L,n_up,periodic", [(10, 5, False), (12, 6, False), (12, 6, True),
                                             (11, 4, True), (9, 2, False)])
def test_trace_closed_form(L, n_up, periodic):
    ch = _chain(L, periodic, 0.8, n_up=n_up)
    n = comb(L, n_up)
    tr = float(np.sum(ham.diag(ch)))
    assert abs(tr - cf.trace_h(L, ch.h, 0.8, n_up, periodic, n)) <= 1e-11 * n


def test_trace_l12_open_value():
    """At n_up = L/2 the fields trace to zero and Tr H = -delta n / 4 (open chain):
    L = 12 gives -924/4 = -231 for delta = 1."""
    ch = ham.Chain(12, wl.fields(12, 5.0, 0), delta=1.0, periodic=False)
    assert abs(float(np.sum(ham.diag(ch))) + 231.0) < 1e-11


@pytest.mark.parametrize("L,n_up,periodic", [(8, 4, False), (8, 4, True), (10, 5, True),
                                             (10, 3, True), (10, 4, False), (9, 4, True)])
def test_free_fermion_spectrum_at_delta0(L, n_up, periodic):
    ch = _chain(L, periodic, 0.0, W=2.0, seed=L + n_up, n_up=n_up)
    ev = np.linalg.eigvalsh(ham.dense_sector(ch))
    ff = cf.free_fermion_energies(L, ch.h, n_up, periodic)
    assert np.abs(ev - ff).max() < 1e-12 * max(1.0, np.abs(ev).max())


def test_free_fermion_nearest_matches_full_list():
    L, n_up = 12, 6
    h = wl.fields(L, 4.0, 9)
    allv = cf.free_fermion_energies(L, h, n_up, True)
    sigma = 0.1
    near = cf.free_fermion_nearest(L, h, n_up, True, sigma, 10)
    idx = np.lexsort((allv, np.abs(allv - sigma)))[:10]
    assert np.allclose(near, np.sort(allv[idx]), atol=1e-13)


@pytest.mark.parametrize("periodic", [False, True])
def test_fold_diag_is_diagonal_of_square(periodic):
    ch = _chain(10, periodic, 1.0)
    sigma = -0.4
    Hs = ham.dense_sector(ch) - sigma * np.eye(ham.sector_dim(10, 5))
    ref = np.diag(Hs @ Hs)
    assert np.allclose(ham.fold_diag(ch, sigma), ref, rtol=1e-14, atol=1e-13)


def test_apply_is_linear_in_sigma_and_rows_agree():
    ch = _chain(14, True, 1.0, W=8.0)
    n = ham.sector_dim(14, 7)
    X = wl.block(n, 3, 5)
    Y0 = ham.apply(ch, 0.0, X)
    Y1 = ham.apply(ch, 1.25, X)
    assert np.allclose(Y0 - Y1, 1.25 * X, rtol=0, atol=1e-13)
    rows = np.array([0, 1, n // 3, n - 2, n - 1])
    assert np.allclose(ham.apply_rows(ch, 1.25, X, rows), Y1[rows], rtol=0, atol=1e-14)


def test_apply_f32_close_to_f64():
    ch = _chain(14, False, 1.0, W=8.0)
    n = ham.sector_dim(14, 7)
    X = wl.block(n, 4, 6, np.float32)
    y32 = ham.apply(ch, 0.5, X)
    y64 = ham.apply(ch, 0.5, X.astype(np.float64))
    # each output is at most 1 + 13 rounded terms: (d - sigma) x plus up to 13 halves
    scale = np.abs(ham.diag(ch) - 0.5)[:, None] * np.abs(X) + 0.5 * 13 * np.abs(X).max()
    bound = 16 * np.finfo(np.float32).eps * scale
    assert np.all(np.abs(y32 - y64) <= bound)
