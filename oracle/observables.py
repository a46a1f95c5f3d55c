"""Oracle: localization indicators computed from converged eigenpairs (Sec. 2.2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Half-chain entanglement entropy (Sec. 2.2).  Cut the chain after the first l_a sites.  A
sector vector psi (rows in ascending integer order of the states, bit i = site i) is, for
each number p of up spins on the left, a matrix M_p whose rows are the left patterns with p
up spins and whose columns are the right patterns with n_up - p; the reduced density
matrix of the left block is the direct sum of M_p M_p^T.  With sigma the singular values of
all M_p of the normalised vector, S = -sum sigma^2 ln sigma^2 (terms with sigma = 0 are 0).

Adjacent gap ratio.  Sec. 2.2 names it as an indicator that needs only eigenvalues and
defers its form to the cited work of Oganesyan and Huse. Written out: for the levels
E_0 <= E_1 <= ... <= E_{m-1} of one realization, the gaps are delta_j = E_{j+1} - E_j, and
for each interior level j = 1 .. m-2

    r_j = min(delta_{j-1}, delta_j) / max(delta_{j-1}, delta_j),

a number in [0, 1].  A level whose two gaps are both zero has no ratio and is skipped (an
exact double degeneracy carries no spacing information).  A realization's value is the
mean of its ratios, and a set of realizations is averaged ratio by ratio (each
realization weighted by its count of ratios).  Levels may come in any order; they are
sorted first.  For Poisson levels (localized) the mean is 2 ln 2 - 1 = 0.3863; for the
3 x 3 Gaussian orthogonal ensemble it is 4 - 2 sqrt(3) = 0.5359, the Wigner-like surmise
of Atas et al. (2013) for thermal Hamiltonians.
"""
import numpy as np


def gap_ratios(levels):
    """The ratios r_j of one realization's levels (1-D array, any order), skipping
    levels whose two gaps are both zero."""
    E = np.sort(np.asarray(levels, dtype=np.float64))
    if E.size < 3:
        return np.zeros(0)
    if not np.all(np.isfinite(E)):
        raise ValueError("non-finite level")
    d = np.diff(E)
    lo = np.minimum(d[:-1], d[1:])
    hi = np.maximum(d[:-1], d[1:])
    keep = hi > 0.0
    return lo[keep] / hi[keep]


def gap_ratio_mean(levels):
    """(mean ratio, number of ratios) of one realization; mean NaN when it has none."""
    r = gap_ratios(levels)
    return (float(np.mean(r)) if r.size else float("nan")), int(r.size)


def gap_ratio_average(realizations):
    """Mean over every ratio of every realization (each weighted by its count)."""
    rs = [gap_ratios(e) for e in realizations]
    n = sum(r.size for r in rs)
    return float(sum(r.sum() for r in rs) / n) if n else float("nan")


def entanglement_entropy(states, psi, l_a):
    """S of the first l_a sites for the sector vector psi (FP64, one entry per state of
    ``states``, the sector's words in ascending order), by the SVD of each M_p."""
    states = np.asarray(states, dtype=np.uint64)
    v = np.asarray(psi, dtype=np.float64)
    v = v / np.linalg.norm(v)
    left = states & np.uint64((1 << l_a) - 1)
    right = states >> np.uint64(l_a)
    pc = np.array([bin(int(a)).count("1") for a in left])
    ent = 0.0
    for p in np.unique(pc):
        sel = pc == p
        la, ia = np.unique(left[sel], return_inverse=True)
        rb, ib = np.unique(right[sel], return_inverse=True)
        M = np.zeros((la.size, rb.size))
        M[ia, ib] = v[sel]
        s2 = np.linalg.svd(M, compute_uv=False) ** 2
        s2 = s2[s2 > 0.0]
        ent -= float(np.sum(s2 * np.log(s2)))
    return ent
