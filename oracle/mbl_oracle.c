/*
 * mbl_oracle.c -- plain, slow, FP64 CPU oracle for the S^z-sector Hamiltonian
 * of the disordered Heisenberg chain (Sec. 2.1, Eq. (model), Eq. (Hmatrix)).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may load this file:
 * only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py do.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Conventions (the reading of the paper used throughout):
 *   - site i of an L-site chain is bit i of a state word s (bit 0 = site 0);
 *     bit = 1 is spin up, z_i = +1; bit = 0 is spin down, z_i = -1.
 *   - the sector with n_up up spins holds every L-bit word of popcount n_up,
 *     listed in ascending integer order; its size is C(L, n_up) (Sec. 2.1,
 *     the sector dimension formula and Table 1).
 *   - bonds: (i, i+1) for i = 0..L-2; a periodic chain adds (L-1, 0) when L > 2
 *     (Sec. 2.1 uses open chains; the periodic bond is the usual wrap-around).
 *   - H = sum_bonds [ (X_iX_j + Y_iY_j)/4 + delta Z_iZ_j/4 ] + sum_i h_i Z_i/2,
 *     i.e. Eq. (model) with S = sigma/2 and an anisotropy delta on the ZZ part
 *     (delta = 1 is Eq. (model) itself).  Its matrix elements:
 *       diagonal      d(s) = sum_bonds delta/4 z_i z_j + sum_i h_i/2 z_i,
 *       off-diagonal  <s'|H|s> = 1/2 when s' = s with the two differing spins
 *                     of one bond exchanged (the flip-flop S^+S^- + S^-S^+ over 2).
 *
 * Every function here follows those definitions literally: states are found
 * by brute-force enumeration, ranks by binary search in that list, and the
 * product y = (H - sigma I) x by looping over rows and bonds.
 */
#include <stdint.h>
#include <stdlib.h>

#define ORC_OK 0
#define ORC_ERR_ARG -1

static int bit_of(uint32_t s, int i) { return (int)((s >> i) & 1u); }

static int popcount_plain(uint32_t s)
{
    int c = 0;
    while (s) {
        c += (int)(s & 1u);
        s >>= 1;
    }
    return c;
}

/* Binomial coefficient by Pascal's rule; exact in int64 for n <= 62. */
int64_t orc_binomial(int n, int k)
{
    if (n < 0 || k < 0 || k > n || n > 62) return 0;
    int64_t row[64];
    for (int j = 0; j <= k; ++j) row[j] = 0;
    row[0] = 1;
    for (int m = 1; m <= n; ++m)
        for (int j = (m < k ? m : k); j >= 1; --j) row[j] += row[j - 1];
    return row[k];
}

/* Sector dimension n = C(L, n_up) (Sec. 2.1; Table 1 lists it for L = 16..26). */
int64_t orc_sector_dim(int L, int n_up)
{
    if (L < 1 || L > 32 || n_up < 0 || n_up > L) return -1;
    return orc_binomial(L, n_up);
}

/* Enumerate the sector by brute force: every L-bit word with popcount n_up,
 * ascending.  Returns the count written, or -1 on bad arguments / short buffer. */
int64_t orc_basis_enumerate(int L, int n_up, uint32_t *states, int64_t cap)
{
    if (L < 1 || L > 32 || n_up < 0 || n_up > L) return -1;
    uint64_t end = (uint64_t)1 << L;
    int64_t cnt = 0;
    for (uint64_t s = 0; s < end; ++s) {
        if (popcount_plain((uint32_t)s) != n_up) continue;
        if (cnt >= cap) return -1;
        states[cnt++] = (uint32_t)s;
    }
    return cnt;
}

/* Rank = position of s in the ascending state list; -1 when s is absent. */
int64_t orc_rank(const uint32_t *states, int64_t n, uint32_t s)
{
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (states[mid] == s) return mid;
        if (states[mid] < s) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

int orc_rank_many(const uint32_t *states, int64_t n, const uint32_t *query,
                  int64_t *out, int64_t cnt)
{
    for (int64_t q = 0; q < cnt; ++q) out[q] = orc_rank(states, n, query[q]);
    return ORC_OK;
}

static int num_bonds(int L, int periodic) { return (L - 1) + ((periodic && L > 2) ? 1 : 0); }

static void bond_sites(int L, int b, int *i, int *j)
{
    if (b < L - 1) {
        *i = b;
        *j = b + 1;
    } else {
        *i = L - 1;
        *j = 0;
    }
}

/* d(s) = sum_bonds delta/4 z_i z_j + sum_i h_i/2 z_i  (Eq. (model), S^z = z/2). */
double orc_diag_elem(int L, int periodic, double delta, const double *h, uint32_t s)
{
    double e = 0.0;
    int nb = num_bonds(L, periodic);
    for (int b = 0; b < nb; ++b) {
        int i, j;
        bond_sites(L, b, &i, &j);
        double zi = bit_of(s, i) ? 1.0 : -1.0;
        double zj = bit_of(s, j) ? 1.0 : -1.0;
        e += 0.25 * delta * zi * zj;
    }
    for (int i = 0; i < L; ++i) {
        double zi = bit_of(s, i) ? 1.0 : -1.0;
        e += 0.5 * h[i] * zi;
    }
    return e;
}

/* Number of bonds whose two spins differ: the off-diagonal entries of row s. */
int orc_flippable(int L, int periodic, uint32_t s)
{
    int f = 0, nb = num_bonds(L, periodic);
    for (int b = 0; b < nb; ++b) {
        int i, j;
        bond_sites(L, b, &i, &j);
        if (bit_of(s, i) != bit_of(s, j)) ++f;
    }
    return f;
}

int orc_diag(int L, int periodic, double delta, const double *h, const uint32_t *states,
             int64_t n, double *d)
{
    if (L < 2 || L > 32 || n < 0) return ORC_ERR_ARG;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n; ++r) d[r] = orc_diag_elem(L, periodic, delta, h, states[r]);
    return ORC_OK;
}

/* Diagonal of the folded operator A = (H - sigma)^2:
 * A[s,s] = sum_t (H - sigma)[s,t]^2 = (d(s) - sigma)^2 + f(s) * (1/2)^2. */
int orc_fold_diag(int L, int periodic, double delta, const double *h, double sigma,
                  const uint32_t *states, int64_t n, double *out)
{
    if (L < 2 || L > 32 || n < 0) return ORC_ERR_ARG;
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n; ++r) {
        double dd = orc_diag_elem(L, periodic, delta, h, states[r]) - sigma;
        out[r] = dd * dd + 0.25 * (double)orc_flippable(L, periodic, states[r]);
    }
    return ORC_OK;
}

/* y = (H - sigma I) x for a row-major n x k block, pulling every neighbour.
 * Each row: diagonal term first, then one 1/2 x[r'] per flippable bond in
 * bond order (0,1), (1,2), ..., then the wrap bond.  Neighbour ranks come from
 * binary search in the state list. */
int orc_apply_f64(int L, int periodic, double delta, const double *h, double sigma,
                  const uint32_t *states, int64_t n, int k, const double *X, int64_t ldx,
                  double *Y, int64_t ldy)
{
    if (L < 2 || L > 32 || n < 0 || k < 1 || ldx < k || ldy < k) return ORC_ERR_ARG;
    int nb = num_bonds(L, periodic);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t r = 0; r < n; ++r) {
        uint32_t s = states[r];
        double dd = orc_diag_elem(L, periodic, delta, h, s) - sigma;
        for (int c = 0; c < k; ++c) Y[r * ldy + c] = dd * X[r * ldx + c];
        for (int b = 0; b < nb; ++b) {
            int i, j;
            bond_sites(L, b, &i, &j);
            if (bit_of(s, i) == bit_of(s, j)) continue;
            uint32_t s2 = s ^ ((1u << i) | (1u << j));
            int64_t r2 = orc_rank(states, n, s2);
            if (r2 < 0) {
                bad = 1;
                continue;
            }
            for (int c = 0; c < k; ++c) Y[r * ldy + c] += 0.5 * X[r2 * ldx + c];
        }
    }
    return bad ? ORC_ERR_ARG : ORC_OK;
}

/* Same product with FP32 storage and FP32 accumulation (the diagonal element is
 * formed in FP64 and rounded once).  Used only to restate the paper's
 * single-precision preconditioner (Sec. 6.2) inside the oracle. */
int orc_apply_f32(int L, int periodic, double delta, const double *h, double sigma,
                  const uint32_t *states, int64_t n, int k, const float *X, int64_t ldx,
                  float *Y, int64_t ldy)
{
    if (L < 2 || L > 32 || n < 0 || k < 1 || ldx < k || ldy < k) return ORC_ERR_ARG;
    int nb = num_bonds(L, periodic);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t r = 0; r < n; ++r) {
        uint32_t s = states[r];
        float dd = (float)(orc_diag_elem(L, periodic, delta, h, s) - sigma);
        for (int c = 0; c < k; ++c) Y[r * ldy + c] = dd * X[r * ldx + c];
        for (int b = 0; b < nb; ++b) {
            int i, j;
            bond_sites(L, b, &i, &j);
            if (bit_of(s, i) == bit_of(s, j)) continue;
            uint32_t s2 = s ^ ((1u << i) | (1u << j));
            int64_t r2 = orc_rank(states, n, s2);
            if (r2 < 0) {
                bad = 1;
                continue;
            }
            for (int c = 0; c < k; ++c) Y[r * ldy + c] += 0.5f * X[r2 * ldx + c];
        }
    }
    return bad ? ORC_ERR_ARG : ORC_OK;
}

/* Selected rows only: y[q] = ((H - sigma) x)[rows[q]] -- lets tests check a few
 * sampled outputs of a full-size product without the full product. */
int orc_apply_rows_f64(int L, int periodic, double delta, const double *h, double sigma,
                       const uint32_t *states, int64_t n, int k, const double *X, int64_t ldx,
                       const int64_t *rows, int64_t nrows, double *Yrows)
{
    if (L < 2 || L > 32 || n < 0 || k < 1 || ldx < k) return ORC_ERR_ARG;
    int nb = num_bonds(L, periodic);
    for (int64_t q = 0; q < nrows; ++q) {
        int64_t r = rows[q];
        if (r < 0 || r >= n) return ORC_ERR_ARG;
        uint32_t s = states[r];
        double dd = orc_diag_elem(L, periodic, delta, h, s) - sigma;
        for (int c = 0; c < k; ++c) Yrows[q * k + c] = dd * X[r * ldx + c];
        for (int b = 0; b < nb; ++b) {
            int i, j;
            bond_sites(L, b, &i, &j);
            if (bit_of(s, i) == bit_of(s, j)) continue;
            int64_t r2 = orc_rank(states, n, s ^ ((1u << i) | (1u << j)));
            if (r2 < 0) return ORC_ERR_ARG;
            for (int c = 0; c < k; ++c) Yrows[q * k + c] += 0.5 * X[r2 * ldx + c];
        }
    }
    return ORC_OK;
}
