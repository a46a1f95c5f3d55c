"""Pins of the oracle's sector basis and ranks (Sec. 2.1, Table 1).

The oracle enumerates states by brute force and ranks by bisection; these tests
tie both to facts fixed outside the oracle: the dimensions printed in Table 1,
the binomial count C(L, n_up), and the combinatorial number system identity
rank(s) = sum_j C(p_j, j) (p_1 < ... < p_m the up-spin sites), which is the
closed form the GPU ranker evaluates.
"""
import os
from math import comb

import numpy as np
import pytest

from oracle import hamiltonian as ham

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_sector_dims.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                L, n = line.split()
                rows.append((int(L), int(n)))
    return rows


@pytest.mark.parametrize("L,n", _table1())
def test_sector_dim_matches_table1(L, n):
    assert ham.sector_dim(L, L // 2) == n


@pytest.mark.parametrize("L", [2, 5, 8, 11, 14, 16])
def test_enumeration_is_every_popcount_word_ascending(L):
    for n_up in range(L + 1):
        st = ham.basis(L, n_up)
        assert st.size == comb(L, n_up)
        assert np.all(np.diff(st.astype(np.int64)) > 0)
        pc = np.array([bin(int(s)).count("1") for s in st])
        assert np.all(pc == n_up)
        assert np.all(st < (1 << L))


def test_enumeration_large_sector_count_and_ends():
    st = ham.basis(22, 11)
    assert st.size == 705432
    assert int(st[0]) == (1 << 11) - 1
    assert int(st[-1]) == ((1 << 11) - 1) << 11


def _cns_rank(s):
    r, j = 0, 0
    for p in range(32):
        if (s >> p) & 1:
            j += 1
            r += comb(p, j)
    return r


@pytest.mark.parametrize("L,n_up", [(10, 5), (12, 6), (12, 3), (13, 7), (16, 8)])
def test_rank_equals_combinatorial_number_system(L, n_up):
    st = ham.basis(L, n_up)
    ranks = ham.rank(st, st)
    assert np.array_equal(ranks, np.arange(st.size))
    cns = np.array([_cns_rank(int(s)) for s in st])
    assert np.array_equal(cns, np.arange(st.size))


def test_rank_of_absent_word_is_minus_one():
    st = ham.basis(10, 5)
    q = np.array([0, 1, (1 << 10) - 1, 0b1111], dtype=np.uint32)
    assert np.all(ham.rank(st, q) == -1)


@pytest.mark.parametrize("L", [10, 12])
def test_open_bond_rank_delta(L):
    """Exchanging the spins of bond (i, i+1) moves the rank by +C(i, c) when the up
    spin moves right and by -C(i, c) when it moves left, c = up spins below site i."""
    st = ham.basis(L, L // 2)
    for r, s in enumerate(st):
        s = int(s)
        for i in range(L - 1):
            bi, bj = (s >> i) & 1, (s >> (i + 1)) & 1
            if bi == bj:
                continue
            c = bin(s & ((1 << i) - 1)).count("1")
            r2 = int(ham.rank(st, [s ^ (3 << i)])[0])
            assert r2 == (r + comb(i, c) if bi else r - comb(i, c))
