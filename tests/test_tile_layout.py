"""The tile decomposition of the sector that every tiled product kernel relies on, checked on
the CPU against the oracle (no GPU, no library).

A state s of L sites splits into B low bits u and H = L - B high bits t; the states with the
same t are one tile of C(B, p) consecutive rows (p = n_up - popc(t)), in colex order of u.
Every term of a tile's product is then one contiguous block of rows (Sec. 4.1's MATVEC,
restated for this layout):
- the joining bond (B - 1, B): the rows whose two spins differ form one range, and their
  partners are that range moved by one rank shift;
- the wrap bond (L - 1, 0) of a periodic chain: the partners lie in tile t ^ 2^(H-1), at the
  colex rank of u ^ 1;
- a low bond: the partner is in the same tile, at the colex rank of the flipped pattern;
- a high bond (B + b, B + b + 1) whose spins differ in t: every row of the tile moves to the
  same in-tile row of tile t ^ (3 << b), a shift of +-C(B + b, p + popc(t mod 2^b)).
This test rebuilds (H - sigma) X from exactly those blocks and compares it with the oracle's
product element by element."""
from math import comb

import numpy as np
import pytest

from oracle import hamiltonian as ham


def _rank(s):
    r, j = 0, 0
    while s:
        p = (s & -s).bit_length() - 1
        s &= s - 1
        j += 1
        r += comb(p, j)
    return r


def _unrank(nbits, m, r):
    s, p = 0, nbits - 1
    for j in range(m, 0, -1):
        while comb(p, j) > r:
            p -= 1
        s |= 1 << p
        r -= comb(p, j)
        p -= 1
    return s


def tiled_apply(L, n_up, periodic, B, delta, h, sigma, X):
    """(H - sigma) X assembled tile by tile from the contiguous row blocks above."""
    n = comb(L, n_up)
    H = L - B
    Y = np.full_like(X, np.nan)
    wrap_bond = periodic and L > 2
    for t in range(1 << H):
        p = n_up - bin(t).count("1")
        if p < 0 or p > B:
            continue
        R = comb(B, p)
        off = _rank((t << B) | ((1 << p) - 1))
        assert off + R <= n
        # joining bond: rows with bit B-1 of u != bit 0 of t form [jbase, jbase + jcnt)
        c0 = comb(B - 1, p)
        if t & 1:
            jbase, jcnt, jsrc = 0, c0, off - c0
        else:
            jbase, jcnt, jsrc = c0, R - c0, off + c0 + (comb(B - 1, p - 1) if p >= 1 else 0)
        # high bonds: one shift per antiparallel pair of high bits
        shifts = []
        for b in range(H - 1):
            if ((t >> b) ^ (t >> (b + 1))) & 1:
                d = comb(B + b, p + bin(t & ((1 << b) - 1)).count("1"))
                shifts.append(d if (t >> b) & 1 else -d)
        # wrap partner tile
        t2 = t ^ (1 << (H - 1))
        p2 = n_up - bin(t2).count("1")
        offper = _rank((t2 << B) | ((1 << p2) - 1)) if 0 <= p2 <= B else None
        thi = (t >> (H - 1)) & 1
        for j in range(R):
            u = _unrank(B, p, j)
            s = (t << B) | u
            acc = np.zeros(X.shape[1])
            if 0 <= j - jbase < jcnt:
                assert 0 <= jsrc + j - jbase < n
                acc += X[jsrc + j - jbase]
            if wrap_bond and (u & 1) != thi:
                assert offper is not None
                jr = _rank(u ^ 1)
                assert jr < comb(B, p2)
                acc += X[offper + jr]
            for i in range(B - 1):
                if ((u >> i) ^ (u >> (i + 1))) & 1:
                    jn = _rank(u ^ (3 << i))
                    assert jn < R
                    acc += X[off + jn]
            for sh in shifts:
                assert 0 <= off + sh + j < n
                acc += X[off + sh + j]
            a = bin((s ^ (s >> 1)) & ((1 << (L - 1)) - 1)).count("1")
            if wrap_bond:
                a += ((s >> (L - 1)) ^ s) & 1
            nbond = L if wrap_bond else L - 1
            d = delta * nbond / 4 - delta / 2 * a + sum(h[i] * (((s >> i) & 1) - 0.5) for i in range(L)) - sigma
            Y[off + j] = d * X[off + j] + 0.5 * acc
    return Y


@pytest.mark.parametrize("L", [4, 5, 6, 7, 8, 9, 10])
def test_tile_blocks_rebuild_the_product(L):
    rng = np.random.default_rng(100 + L)
    for n_up in range(L + 1):
        for periodic in (False, True):
            h = rng.uniform(-3.0, 3.0, L)
            chain = ham.Chain(L, h, delta=0.8, periodic=periodic, n_up=n_up)
            X = rng.standard_normal((comb(L, n_up), 2))
            ref = ham.apply(chain, 0.3, X)
            for B in range(2, L - 1):
                got = tiled_apply(L, n_up, periodic, B, 0.8, h, 0.3, X)
                assert np.allclose(got, ref, rtol=0, atol=1e-12), (L, n_up, periodic, B)
