"""Closed forms that pin the oracle (Sec. 2.1 model, Table 1 dimensions).

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``free_fermion_energies`` -- at delta = 0 the chain of Eq. (model) maps by the
  Jordan-Wigner transformation onto free fermions: S^+_iS^-_j + h.c. becomes a
  hopping of amplitude 1/2 and h_i S^z_i = h_i (n_i - 1/2).  Every eigenvalue in the
  sector with N up spins is a sum of N distinct eigenvalues of the L x L hopping
  matrix T (T_ii = h_i, T_{i,i+1} = T_{i+1,i} = 1/2), minus sum_i h_i / 2.  On a
  periodic chain the wrap-around hop carries the fermion-parity sign (-1)^(N-1).
* ``trace_h`` -- Tr H over the sector: the field terms average to h_i (2N-L)/L and a
  bond's z_i z_j averages to 1 - 4N(L-N)/(L(L-1)) over the C(L, N) states.
* ``free_fermion_entropy`` -- the entanglement entropy of the first l_a sites in an
  eigenstate of the open delta = 0 chain, from its single-particle modes alone (the
  correlation-matrix method of Peschel, 2003): with C_ij = sum over occupied modes k of
  phi_k(i) phi_k(j) restricted to the first l_a sites and its eigenvalues nu,
  S = -sum [nu ln nu + (1 - nu) ln (1 - nu)].  The Jordan-Wigner string of a site in the
  left block only involves sites of that block, so the spin and fermion reduced states
  agree.
"""
import itertools

import numpy as np


def hopping_matrix(L, h, n_up, periodic):
    T = np.diag(np.asarray(h, dtype=np.float64)).copy()
    for i in range(L - 1):
        T[i, i + 1] = T[i + 1, i] = 0.5
    if periodic and L > 2:
        sign = 1.0 if (n_up - 1) % 2 == 0 else -1.0
        T[0, L - 1] += 0.5 * sign
        T[L - 1, 0] += 0.5 * sign
    return T


def free_fermion_energies(L, h, n_up, periodic, limit=None):
    """All sector eigenvalues at delta = 0 (sorted), by enumerating the N-subsets of
    single-particle levels.  ``limit`` caps the subset count for safety."""
    eps = np.linalg.eigvalsh(hopping_matrix(L, h, n_up, periodic))
    shift = -0.5 * float(np.sum(h))
    subsets = itertools.combinations(range(L), n_up)
    out = []
    for cnt, q in enumerate(subsets):
        if limit is not None and cnt >= limit:
            raise ValueError("too many subsets")
        out.append(sum(eps[list(q)]) + shift)
    return np.sort(np.array(out))


def free_fermion_nearest(L, h, n_up, periodic, sigma, nev):
    """The nev sector eigenvalues nearest sigma at delta = 0, sorted ascending.
    Vectorised subset sums so that L = 26 (10.4 M subsets) stays cheap."""
    eps = np.linalg.eigvalsh(hopping_matrix(L, h, n_up, periodic))
    shift = -0.5 * float(np.sum(h))
    # Subset sums by dynamic programming over levels, grouped by subset size.
    sums = [np.array([0.0])]
    for e in eps:
        new = [None] * (len(sums) + 1)
        for size, arr in enumerate(sums):
            new[size] = arr if new[size] is None else np.concatenate([new[size], arr])
            plus = arr + e
            new[size + 1] = plus if new[size + 1] is None else np.concatenate([new[size + 1], plus])
        sums = [a for a in new[: n_up + 1]]
    energies = sums[n_up] + shift
    dist = np.abs(energies - sigma)
    idx = np.lexsort((energies, dist))[:nev]
    return np.sort(energies[idx])


def trace_h(L, h, delta, n_up, periodic, n):
    """Tr H over the sector of dimension n = C(L, n_up)."""
    nb = (L - 1) + (1 if (periodic and L > 2) else 0)
    zz = 1.0 - 4.0 * n_up * (L - n_up) / (L * (L - 1.0))
    z = (2.0 * n_up - L) / L
    return n * (0.25 * delta * nb * zz + 0.5 * float(np.sum(h)) * z)


def free_fermion_entropy(L, h, occupied, l_a):
    """(energy, entropy of sites 0..l_a-1) of the open delta = 0 eigenstate that fills the
    single-particle modes ``occupied`` (indices into the ascending single-particle levels)."""
    T = hopping_matrix(L, h, len(occupied), False)
    eps, phi = np.linalg.eigh(T)
    occ = list(occupied)
    energy = float(np.sum(eps[occ]) - 0.5 * np.sum(h))
    C = phi[:l_a, occ] @ phi[:l_a, occ].T
    nu = np.clip(np.linalg.eigvalsh(C), 0.0, 1.0)
    ent = 0.0
    for v in nu:
        for q in (v, 1.0 - v):
            if q > 1e-300:
                ent -= q * np.log(q)
    return energy, float(ent)
