"""Oracle: folded-spectrum LOBPCG with a Jacobi-PCG preconditioner (Sec. 3.2, Sec. 6.2).

TEST INFRASTRUCTURE ONLY (see the package docstring).

What the paper fixes (Sec. 3.2): LOBPCG (Knyazev 2001; Duersch et al. 2018) applied
to the spectral fold A = (H - sigma I)^2, whose smallest eigenvalues belong to the
eigenvalues of H nearest sigma; the preconditioner is Jacobi-preconditioned CG on
A.  Sec. 6.2 runs the PCG in single precision and LOBPCG in double precision, with
a fixed number of PCG iterations per LOBPCG iteration (5,000 at L = 24, 20,000 at
L = 26).  What it leaves to the companion paper, and the reading taken here:

  * PCG: independent CG per column on A w = r, zero initial guess, Jacobi
    M = diag(A) = (d - sigma)^2 + f/4, ``pcg_iters`` steps, optionally frozen once
    r^T M^-1 r falls below ``pcg_tol^2`` times its initial value.  The right-hand
    sides are the LOBPCG residual columns scaled to unit norm.
  * LOBPCG: block X (n x k, orthonormal), search block W (preconditioned residuals,
    made orthogonal to X twice), previous-direction block P (made orthogonal to X);
    the basis [X, W, P] is orthonormalised by SVQB (Stathopoulos & Wu: scale to unit
    columns, eigendecompose the Gram, drop directions whose Gram eigenvalue is below
    ``svqb_tau`` times the largest); Rayleigh-Ritz with A keeps the k smallest;
    X <- S C_X, P <- [W, P] C_[W,P]; X is re-orthonormalised by Cholesky-QR and
    (H - sigma)X and AX are recomputed from it every iteration.
  * Fold degeneracy and stopping: every iteration a Rayleigh-Ritz with H itself on
    span(X) gives Ritz pairs (lambda_j, y_j); the nev nearest sigma (ties: lower
    lambda first) are accepted when each has ||H y - lambda y||_2 <= tol * norm_h.
    The same Rayleigh-Ritz is the final extraction.

Library primitives used as single steps: numpy matmul and numpy.linalg.eigh /
cholesky on the small dense matrices.
"""
import time

import numpy as np

from . import hamiltonian as ham


def _sym(G):
    return 0.5 * (G + G.T)


def cholqr(X):
    """X <- X R^-1 with X^T X = R^T R (Cholesky-QR)."""
    G = _sym(X.T @ X)
    Lc = np.linalg.cholesky(G)
    return np.linalg.solve(Lc, X.T).T


def pcg_jacobi(apply_A, dinv, B, iters, tol=0.0, dtype=np.float64):
    """Column-wise Jacobi-PCG on A W = B from W = 0 (Sec. 3.2).  Arithmetic in
    ``dtype`` (float32 restates the single-precision preconditioner of Sec. 6.2)."""
    B = np.asarray(B, dtype=dtype)
    dinv = np.asarray(dinv, dtype=dtype)[:, None]
    W = np.zeros_like(B)
    R = B.copy()
    Z = dinv * R
    P = Z.copy()
    rz = np.sum(R * Z, axis=0)
    rz0 = rz.copy()
    active = rz > 0
    for _ in range(int(iters)):
        Q = apply_A(P)
        pq = np.sum(P * Q, axis=0)
        ok = active & (pq > 0)
        alpha = np.where(ok, rz / np.where(ok, pq, 1), 0).astype(dtype)
        W += alpha * P
        R -= alpha * Q
        Z = dinv * R
        rz_new = np.sum(R * Z, axis=0)
        if tol > 0:
            active = active & (rz_new > (tol * tol) * rz0)
        okb = active & (rz > 0)
        beta = np.where(okb, rz_new / np.where(okb, rz, 1), 0).astype(dtype)
        P = Z + beta * P
        rz = rz_new
    return W


def _nearest(mu, nev):
    """Indices of the nev values of mu = lambda - sigma nearest 0; ties -> lower first."""
    return np.lexsort((mu, np.abs(mu)))[:nev]


class Result:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def h_rayleigh_ritz(X, T):
    """Rayleigh-Ritz with H - sigma on span(X), X orthonormal, T = (H - sigma)X.
    Returns mu (ascending), V, and the residual norms ||(H - sigma)y - mu y|| of
    y = X v, formed from the explicit block E = T - X M."""
    M = _sym(X.T @ T)
    mu, V = np.linalg.eigh(M)
    E = T - X @ M
    res = np.linalg.norm(E @ V, axis=0)
    return mu, V, res


def lobpcg_folded(chain, sigma, X0, nev, tol, norm_h, max_iter=200, pcg_iters=50,
                  pcg_tol=0.0, pcg_dtype=np.float64, svqb_tau=1e-14, verbose=False):
    """The nev eigenpairs of H nearest sigma by LOBPCG on (H - sigma)^2.

    Returns a Result with evals (ascending), evecs (n x nev), resid (absolute
    ||Hy - lambda y||_2), iters, converged, matvecs (single-column applications of
    H), history (max relative residual of the accepted pairs per iteration)."""
    t0 = time.perf_counter()
    X = np.array(X0, dtype=np.float64, copy=True)
    n, k = X.shape
    if not (1 <= nev <= k <= n):
        raise ValueError("need 1 <= nev <= k <= n")
    napply = [0]

    def shifted(V):
        napply[0] += V.shape[1]
        return ham.apply(chain, sigma, V)

    def fold(V):
        # float32 blocks go through the FP32 product (FP32 storage and sums)
        return shifted(shifted(V))

    dinv = 1.0 / ham.fold_diag(chain, sigma)

    X = cholqr(X)
    T = shifted(X)
    AX = shifted(T)
    th, C = np.linalg.eigh(_sym(X.T @ AX))
    X, T, AX = X @ C, T @ C, AX @ C
    P = None
    history = []
    converged = False
    it = 0
    while True:
        mu, V, res = h_rayleigh_ritz(X, T)
        sel = _nearest(mu, nev)
        rel = res[sel] / norm_h
        history.append(float(np.max(rel)))
        if verbose:
            print("it %3d  max rel resid %.3e" % (it, history[-1]))
        if np.all(rel <= tol):
            converged = True
            break
        if it >= max_iter:
            break
        it += 1
        # folded residual and preconditioned search directions
        Theta = _sym(X.T @ AX)
        R = AX - X @ Theta
        rn = np.linalg.norm(R, axis=0)
        Rn = R / np.where(rn > 0, rn, 1.0)
        W = pcg_jacobi(fold, dinv, Rn, pcg_iters, pcg_tol, pcg_dtype).astype(np.float64)
        W -= X @ (X.T @ W)
        W -= X @ (X.T @ W)
        AW = fold(W)
        blocks, ablocks = [X, W], [AX, AW]
        if P is not None:
            P -= X @ (X.T @ P)
            P -= X @ (X.T @ P)
            AP = fold(P)
            blocks.append(P)
            ablocks.append(AP)
        S = np.hstack(blocks)
        AS = np.hstack(ablocks)
        # SVQB orthonormalisation of the basis
        G = _sym(S.T @ S)
        dg = np.diag(G).copy()
        live = dg > 0
        Dm = np.where(live, 1.0 / np.sqrt(np.where(live, dg, 1.0)), 0.0)
        Gs = Dm[:, None] * G * Dm[None, :]
        ls, U = np.linalg.eigh(Gs)
        keep = ls > svqb_tau * ls.max()
        Cs = Dm[:, None] * U[:, keep] / np.sqrt(ls[keep])[None, :]
        # Rayleigh-Ritz with A, keep the k smallest
        GA = _sym(Cs.T @ (S.T @ AS) @ Cs)
        thA, Z = np.linalg.eigh(GA)
        coef = Cs @ Z[:, :k]
        Xn = S @ coef
        P = S[:, k:] @ coef[k:]
        pn = np.linalg.norm(P, axis=0)
        P = P / np.where(pn > 0, pn, 1.0)
        X = cholqr(Xn)
        T = shifted(X)
        AX = shifted(T)
    Y = X @ V[:, sel]
    lam = sigma + mu[sel]
    order = np.argsort(lam)
    return Result(evals=lam[order], evecs=Y[:, order], resid=res[sel][order], iters=it,
                  converged=converged, matvecs=napply[0], history=history,
                  seconds=time.perf_counter() - t0)


def lobpcg_extreme(chain, sign, X0, tol, max_iter=500, svqb_tau=1e-14):
    """Smallest eigenvalue of sign * H (sign = +1: E_min, sign = -1: -E_max) by
    unpreconditioned LOBPCG with the same orthonormalisation (spectrum bounds used to
    place sigma at the middle of the spectrum and to scale tolerances).  The first
    column is accepted when ||sign H x - theta x|| <= tol * |theta|."""
    X = cholqr(np.array(X0, dtype=np.float64, copy=True))
    n, k = X.shape

    def op(V):
        return sign * ham.apply(chain, 0.0, V)

    AX = op(X)
    th, C = np.linalg.eigh(_sym(X.T @ AX))
    X, AX = X @ C, AX @ C
    P = AP = None
    it = 0
    theta = th[0]
    while True:
        Theta = _sym(X.T @ AX)
        th, C = np.linalg.eigh(Theta)
        X, AX = X @ C, AX @ C
        R = AX - X * th[None, :]
        theta = th[0]
        if np.linalg.norm(R[:, 0]) <= tol * abs(theta) or it >= max_iter:
            break
        it += 1
        W = R - X @ (X.T @ R)
        W -= X @ (X.T @ W)
        AW = op(W)
        blocks, ablocks = [X, W], [AX, AW]
        if P is not None:
            Cp = X.T @ P
            P = P - X @ Cp
            AP = AP - AX @ Cp
            blocks.append(P)
            ablocks.append(AP)
        S = np.hstack(blocks)
        AS = np.hstack(ablocks)
        G = _sym(S.T @ S)
        dg = np.diag(G).copy()
        live = dg > 0
        Dm = np.where(live, 1.0 / np.sqrt(np.where(live, dg, 1.0)), 0.0)
        ls, U = np.linalg.eigh(Dm[:, None] * G * Dm[None, :])
        keep = ls > svqb_tau * ls.max()
        Cs = Dm[:, None] * U[:, keep] / np.sqrt(ls[keep])[None, :]
        thA, Z = np.linalg.eigh(_sym(Cs.T @ (S.T @ AS) @ Cs))
        coef = Cs @ Z[:, :k]
        Xn = S @ coef
        P = S[:, k:] @ coef[k:]
        AP = AS[:, k:] @ coef[k:]
        X = cholqr(Xn)
        AX = op(X)
    return float(theta), it


def spectrum_bounds(chain, X0, tol=1e-10, max_iter=500):
    """(E_min, E_max) of the sector Hamiltonian.  Dense eigvalsh for n <= 4000,
    otherwise LOBPCG on +H and -H from the block X0."""
    n = ham.sector_dim(chain.L, chain.n_up)
    if n <= 4000:
        ev = np.linalg.eigvalsh(ham.dense_sector(chain))
        return float(ev[0]), float(ev[-1])
    emin, _ = lobpcg_extreme(chain, +1.0, X0, tol, max_iter)
    memax, _ = lobpcg_extreme(chain, -1.0, X0, tol, max_iter)
    return emin, -memax
