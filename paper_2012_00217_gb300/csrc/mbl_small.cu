// mbl_small.cu -- small dense kernels of the LOBPCG iteration (Sec. 3.2), each run by
// one block: symmetric eigendecomposition by parallel cyclic Jacobi, Cholesky with
// triangular inverse, the SVQB + Rayleigh-Ritz step on S = [X W P], and the selection
// of the Ritz pairs nearest sigma.
//
// Precision.  GB300 executes FP64 at about 1/64 of its FP32 rate, so in mixed mode
// the (3k x 3k) eigenproblems run in FP32 and only a k-dimensional refinement runs in
// FP64: the k Ritz directions picked in FP32 are re-orthonormalised (Cholesky, FP64)
// and a k x k Rayleigh-Ritz with the FP64 projection of A finishes the step.  The
// convergence test (H Rayleigh-Ritz and residuals) is always FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mbl_dense.h"
#include "mbl_device.cuh"
#include "mbl_internal.h"

namespace mbl {

constexpr int kSmallThreads = 512;
constexpr int kMaxSweeps = 20;
constexpr int kMaxK = 64;        // block width limit of the solver
constexpr int kMaxW = 3 * kMaxK;  // width of S = [X W P]

template <typename T>
struct Eps;
template <>
struct Eps<float> {
    static __device__ __forceinline__ float v() { return 1.2e-7f; }
};
template <>
struct Eps<double> {
    static __device__ __forceinline__ double v() { return 2.3e-16; }
};

// Odd row stride for matrices in shared memory: walking down a column then touches a
// different bank in every lane.
__host__ __device__ inline int pad_ld(int n) { return n | 1; }

// Parallel cyclic Jacobi on the symmetric n x n matrix A (row stride ld): the
// round-robin (circle) ordering rotates n/2 disjoint pairs per round.  A rotation zeroes
// a_pq with t = sign(tau)/(|tau| + sqrt(1 + tau^2)), tau = (a_qq - a_pp)/(2 a_pq); pairs
// with |a_pq| <= eps sqrt(|a_pp a_qq|) are skipped (the relative test keeps the small
// eigenvalues of graded matrices accurate); sweeps stop when one rotates nothing or after
// max_sweeps.  On exit diag(A) holds the eigenvalues and the columns of V (stride ld)
// the eigenvectors (WANT_V = false: eigenvalues only, V not touched).  Each warp rotates
// whole rows / columns of its pairs, lanes striding the other index.  cs, pairs: n + 2
// entries (shared or global memory of this block).
template <typename T, bool WANT_V = true>
__device__ void dev_jacobi(int n, int ld, T *A, T *V, T *cs, int *pairs, int *s_rot, int max_sweeps)
{
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    if (WANT_V)
        for (int i = warp; i < n; i += nwarps)
            for (int j = lane; j < n; j += 32) V[i * ld + j] = (i == j) ? (T)1 : (T)0;
    __syncthreads();
    if (n < 2) return;
    const int np = (n + 1) & ~1;
    const int half = np / 2;
    const T eps = Eps<T>::v();
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (tid == 0) *s_rot = 0;
        __syncthreads();
        for (int round = 0; round < np - 1; ++round) {
            for (int i = tid; i < half; i += nt) {
                int p, q;
                if (i == 0) {
                    p = round;
                    q = np - 1;
                } else {
                    p = (round + i) % (np - 1);
                    q = (round - i + (np - 1)) % (np - 1);
                }
                if (p > q) {
                    const int t = p;
                    p = q;
                    q = t;
                }
                T c = (T)1, s = (T)0;
                if (q < n) {
                    const T apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
                    if (apq != (T)0 && fabs(apq) > eps * sqrt(fabs(app * aqq))) {
                        const T tau = (aqq - app) / ((T)2 * apq);
                        const T t = (tau >= (T)0 ? (T)1 : (T)-1) / (fabs(tau) + sqrt((T)1 + tau * tau));
                        c = (T)1 / sqrt((T)1 + t * t);
                        s = t * c;
                        *s_rot = 1;
                    }
                }
                pairs[2 * i] = p;
                pairs[2 * i + 1] = q;
                cs[2 * i] = c;
                cs[2 * i + 1] = s;
            }
            __syncthreads();
            for (int i = warp; i < half; i += nwarps) {  // rows p, q
                const T s = cs[2 * i + 1];
                if (s == (T)0) continue;
                const T c = cs[2 * i];
                T *Ap = A + pairs[2 * i] * ld, *Aq = A + pairs[2 * i + 1] * ld;
                for (int j = lane; j < n; j += 32) {
                    const T ap = Ap[j], aq = Aq[j];
                    Ap[j] = c * ap - s * aq;
                    Aq[j] = s * ap + c * aq;
                }
            }
            __syncthreads();
            for (int i = warp; i < half; i += nwarps) {  // columns p, q of A and V
                const T s = cs[2 * i + 1];
                if (s == (T)0) continue;
                const T c = cs[2 * i];
                const int p = pairs[2 * i], q = pairs[2 * i + 1];
                for (int j = lane; j < n; j += 32) {
                    T *Aj = A + j * ld;
                    const T ap = Aj[p], aq = Aj[q];
                    Aj[p] = c * ap - s * aq;
                    Aj[q] = s * ap + c * aq;
                    if (WANT_V) {
                        T *Vj = V + j * ld;
                        const T vp = Vj[p], vq = Vj[q];
                        Vj[p] = c * vp - s * vq;
                        Vj[q] = s * vp + c * vq;
                    }
                }
            }
            __syncthreads();
        }
        const int rot = *s_rot;
        __syncthreads();
        if (!rot) break;
    }
}

// Ascending sort of the eigenpairs left by dev_jacobi: w[rank] = A[j][j],
// Vs[:, rank] = V[:, j] (Vs row stride ldo).
template <typename T, typename TO>
__device__ void dev_sort_eig(int n, int ld, const T *A, const T *V, TO *w, TO *Vs, int ldo)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = tid; j < n; j += nt) {
        const T lj = A[j * ld + j];
        int rank = 0;
        for (int i = 0; i < n; ++i) {
            const T li = A[i * ld + i];
            if (li < lj || (li == lj && i < j)) ++rank;
        }
        w[rank] = (TO)lj;
        for (int i = 0; i < n; ++i) Vs[i * ldo + rank] = (TO)V[i * ld + j];
    }
    __syncthreads();
}

// Upper Cholesky G = R^T R of the symmetric part of G (n x n, ld ldg) and Rinv = R^-1.
// Returns 1 (in every thread) when a pivot is not positive and finite; Rinv is then I.
__device__ int dev_chol_inv(int n, const double *G, int ldg, double *R, double *Rinv, int *s_flag)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) *s_flag = 0;
    for (int e = tid; e < n * n; e += nt) {
        const int i = e / n, j = e % n;
        R[e] = (j >= i) ? 0.5 * (G[i * ldg + j] + G[j * ldg + i]) : 0.0;
    }
    __syncthreads();
    for (int kk = 0; kk < n; ++kk) {
        if (tid == 0) {
            const double d = R[kk * n + kk];
            double pv = 1.0;
            if (!(d > 0.0) || !isfinite(d)) *s_flag = 1;
            else pv = sqrt(d);
            R[kk * n + kk] = pv;
        }
        __syncthreads();
        const double piv = R[kk * n + kk];
        for (int j = kk + 1 + tid; j < n; j += nt) R[kk * n + j] /= piv;
        __syncthreads();
        const int m = n - kk - 1;
        for (int e = tid; e < m * m; e += nt) {
            const int i = kk + 1 + e / m, j = kk + 1 + e % m;
            if (j >= i) R[i * n + j] -= R[kk * n + i] * R[kk * n + j];
        }
        __syncthreads();
    }
    for (int j = tid; j < n; j += nt) {
        for (int i = n - 1; i >= 0; --i) {
            double s = (i == j) ? 1.0 : 0.0;
            for (int m = i + 1; m <= j; ++m) s -= R[i * n + m] * Rinv[m * n + j];
            Rinv[i * n + j] = (i <= j) ? s / R[i * n + i] : 0.0;
        }
    }
    __syncthreads();
    const int bad = *s_flag;
    if (bad)
        for (int e = tid; e < n * n; e += nt) Rinv[e] = (e / n == e % n) ? 1.0 : 0.0;
    __syncthreads();
    return bad;
}

// In-place upper Cholesky R^T R = A of the symmetric n x n matrix A (row stride ld, both
// triangles on entry; the upper one holds R on exit) when every pivot exceeds tol (A has a
// unit diagonal here, so tol bounds its conditioning); returns false (in every thread) as
// soon as one does not.
template <typename T>
__device__ bool dev_chol_upper(int n, T *A, int ld, T tol, int *s_flag)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) *s_flag = 0;
    __syncthreads();
    for (int kk = 0; kk < n; ++kk) {
        if (tid == 0) {
            const T d = A[kk * ld + kk];
            if (!(d > tol) || !isfinite(d)) *s_flag = 1;
            else A[kk * ld + kk] = sqrt(d);
        }
        __syncthreads();
        if (*s_flag) return false;
        const T piv = A[kk * ld + kk];
        for (int j = kk + 1 + tid; j < n; j += nt) A[kk * ld + j] /= piv;
        __syncthreads();
        const int m = n - kk - 1;
        for (int e = tid; e < m * m; e += nt) {
            const int i = kk + 1 + e / m, j = kk + 1 + e % m;
            if (j >= i) A[i * ld + j] -= A[kk * ld + i] * A[kk * ld + j];
        }
        __syncthreads();
    }
    return true;
}

// Ri = R^-1 for the upper-triangular R (row strides ldr, ldi), one column per thread.
template <typename T>
__device__ void dev_tri_inv_upper(int n, const T *R, int ldr, T *Ri, int ldi)
{
    for (int j = threadIdx.x; j < n; j += blockDim.x)
        for (int i = n - 1; i >= 0; --i) {
            T s = (i == j) ? (T)1 : (T)0;
            if (i < j)
                for (int m = i + 1; m <= j; ++m) s -= R[i * ldr + m] * Ri[m * ldi + j];
            Ri[i * ldi + j] = (i <= j) ? s / R[i * ldr + i] : (T)0;
        }
    __syncthreads();
}

// C (rows x cols, stride ldc) = op(A) op(B) in precision TA, one output per thread step.
// transA: A stored (inner x rows), else (rows x inner); B stored (inner x cols).
template <typename TC, typename TA, typename TB>
__device__ void dev_matmul(int rows, int cols, int inner, const TA *A, int lda, bool transA, const TB *B, int ldb,
                           TC *C, int ldc)
{
    for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
        const int i = e / cols, j = e - (e / cols) * cols;
        TC acc = (TC)0;
        if (transA)
            for (int m = 0; m < inner; ++m) acc += (TC)A[m * lda + i] * (TC)B[m * ldb + j];
        else
            for (int m = 0; m < inner; ++m) acc += (TC)A[i * lda + m] * (TC)B[m * ldb + j];
        C[i * ldc + j] = acc;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------------
// Symmetric eigendecomposition (FP64 Jacobi) of G (n x n, ld ldg): w ascending, Z
// (n x n, stride n) eigenvectors in columns.  A and V live in shared memory for n <= 64.
__global__ void __launch_bounds__(kSmallThreads) k_small_eig(int n, const double *G, int64_t ldg, double *w,
                                                             double *Z, double *work, int in_smem)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_rot;
    __shared__ double cs[kMaxW + 2];
    __shared__ int pairs[kMaxW + 2];
    const int ld = pad_ld(n);
    double *A = in_smem ? reinterpret_cast<double *>(smem_raw) : work;
    double *V = A + n * ld;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, j = e % n;
        A[i * ld + j] = 0.5 * (G[i * ldg + j] + G[j * ldg + i]);
    }
    __syncthreads();
    dev_jacobi<double>(n, ld, A, V, cs, pairs, &s_rot, kMaxSweeps);
    dev_sort_eig<double, double>(n, ld, A, V, w, Z, n);
}

static size_t eig_smem_bytes(int n) { return (size_t)2 * n * pad_ld(n) * sizeof(double); }

size_t small_eig_work_doubles(int n) { return (size_t)2 * n * pad_ld(n) + 8; }

int small_eig(int n, const double *G, int64_t ldg, double *w, double *Z, double *work, cudaStream_t st)
{
    static const bool attr_once = [&]() {
        cudaFuncSetAttribute(k_small_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)eig_smem_bytes(64));
        return true;
    }();
    (void)attr_once;
    const int in_smem = n <= 64;
    note_launch();
    k_small_eig<<<1, kSmallThreads, in_smem ? eig_smem_bytes(n) : 0, st>>>(n, G, ldg, w, Z, work, in_smem);
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

__global__ void __launch_bounds__(kSmallThreads) k_small_chol_inv(int n, const double *G, int64_t ldg, double *Rinv,
                                                                  double *work, int *flag)
{
    __shared__ int s_flag;
    const int bad = dev_chol_inv(n, G, (int)ldg, work, Rinv, &s_flag);
    if (threadIdx.x == 0) *flag = bad;
}

int small_chol_inv(int n, const double *G, int64_t ldg, double *Rinv, double *work, int *flag, cudaStream_t st)
{
    note_launch();
    k_small_chol_inv<<<1, kSmallThreads, 0, st>>>(n, G, ldg, Rinv, work, flag);
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

// ---------------------------------------------------------------------------------
// Rayleigh-Ritz on span(S), S = [X W P] with w columns, in an S-orthonormal basis C_S:
//   D = diag(G_S)^-1/2; Cholesky D G_S D = R^T R when every pivot is well above zero,
//   C_S = D R^-1; else SVQB (Stathopoulos & Wu): eig(D G_S D) = U L U^T, keep
//   L_i > tau max L, C_S = D U_keep L_keep^-1/2.  Then eig(C_S^T G_A C_S) = Z theta,
//   coef = C_S Z[:, first k]  (the k smallest; the k largest, descending, if 'largest').
// T is the precision of the two w x w eigensolves.  With T = float a k-dimensional FP64
// refinement follows: Y = C_S Z_k R^-1 (R^T R = Z_k^T Z_k), M = Y^T G_A Y, eig(M) = Q mu
// (FP64), coef = Y Q.  info[0] = kept directions, info[1] = 1 on NaN/Inf or a failed
// refinement.

size_t small_rr_work_doubles(int w) { return (size_t)16 * w * w + 16 * w + 256; }

template <typename T>
__device__ void rr_body(int w, int k, int largest, const double *GS, const double *GA, double tau, double *coef,
                        double *theta, double *work, int *info, T *As, T *Vs, int use_smem)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    __shared__ int s_rot, s_keep, s_first, s_flag;
    __shared__ T csb[kMaxW + 2];
    __shared__ int pairs[kMaxW + 2];
    __shared__ double cs64[kMaxK + 2];
    __shared__ int pairs64[kMaxK + 2];
    const int ld = pad_ld(w);
    // FP64 workspace
    double *dsc = work;                       // w
    double *GAs = dsc + w;                    // w x w, symmetrised G_A
    double *Cs = GAs + w * w;                 // w x w (keep columns used)
    double *Zk = Cs + w * w;                  // w x k
    double *ZR = Zk + w * k;                  // w x k
    double *Y = ZR + w * k;                   // w x k
    double *Bm = Y + w * k;                   // w x k
    double *M = Bm + w * k;                   // k x k
    double *R = M + k * k;                    // k x k
    double *Ri = R + k * k;                   // k x k
    double *Q = Ri + k * k;                   // k x k
    double *mu = Q + k * k;                   // k
    T *lam = reinterpret_cast<T *>(mu + k);   // w
    T *GAt = lam + w + 2;                     // w x w
    T *Cst = GAt + w * w;                     // w x w
    T *U = Cst + w * w;                       // w x w
    T *T2 = U + w * w;                        // w x w
    T *Z = T2 + w * w;                        // w x w
    T *Ag = reinterpret_cast<T *>(((uintptr_t)(Z + w * w) + 15) & ~(uintptr_t)15);
    T *A = use_smem ? As : Ag;
    T *V = use_smem ? Vs : Ag + w * ld;

    for (int i = tid; i < w; i += nt) {
        const double d = GS[i * w + i];
        dsc[i] = (d > 0.0 && isfinite(d)) ? 1.0 / sqrt(d) : 0.0;
    }
    __syncthreads();
    for (int e = tid; e < w * w; e += nt) {
        const int i = e / w, j = e - (e / w) * w;
        const double g = 0.5 * (GA[i * w + j] + GA[j * w + i]);
        GAs[e] = g;
        GAt[e] = (T)g;
        A[i * ld + j] = (T)(dsc[i] * 0.5 * (GS[i * w + j] + GS[j * w + i]) * dsc[j]);
    }
    __syncthreads();
    // An S-orthonormal basis: from the Cholesky factor of D G_S D when that is well
    // conditioned (every pivot of the unit-diagonal matrix above chol_tol), C_S = D R^-1,
    // all w directions kept; otherwise SVQB, which drops the nearly dependent directions.
    const T chol_tol = sizeof(T) == sizeof(float) ? (T)1e-3 : (T)1e-8;
    // the factor and its inverse in shared memory when the w x w tiles are there (V is free
    // until the SVQB fallback sets it, A until the projection overwrites it): the column
    // loops of both are latency chains
    T *Rm = use_smem ? V : T2, *Ui = use_smem ? A : U;
    const int ldr = use_smem ? ld : w;
    for (int e = tid; e < w * w; e += nt) Rm[(e / w) * ldr + (e % w)] = A[(e / w) * ld + (e % w)];
    const bool chol = dev_chol_upper<T>(w, Rm, ldr, chol_tol, &s_flag);
    if (chol) {
        dev_tri_inv_upper<T>(w, Rm, ldr, Ui, ldr);
        for (int e = tid; e < w * w; e += nt) {
            const int i = e / w, j = e - i * w;
            const double c = dsc[i] * (double)Ui[i * ldr + j];
            Cs[e] = c;
            Cst[e] = (T)c;
        }
        if (tid == 0) {
            s_first = 0;
            s_keep = w;
        }
        __syncthreads();
    } else {
        dev_jacobi<T>(w, ld, A, V, csb, pairs, &s_rot, kMaxSweeps);
        dev_sort_eig<T, T>(w, ld, A, V, lam, U, w);
        if (tid == 0) {
            const double lmax = (double)lam[w - 1];
            int first = w;
            for (int i = 0; i < w; ++i)
                if ((double)lam[i] > tau * lmax) {
                    first = i;
                    break;
                }
            s_first = first;
            s_keep = w - first;
        }
        __syncthreads();
        const int first = s_first, keep = s_keep;
        for (int e = tid; e < w * keep; e += nt) {
            const int i = e / keep, j = e - (e / keep) * keep;
            const double c = dsc[i] * (double)U[i * w + first + j] / sqrt((double)lam[first + j]);
            Cs[i * w + j] = c;
            Cst[i * w + j] = (T)c;
        }
        __syncthreads();
    }
    const int keep = s_keep;
    // projected G_A in precision T: T2 = G_A Cs, A = Cs^T T2 (keep x keep, stride ldk)
    const int ldk = pad_ld(keep);
    dev_matmul<T, T, T>(w, keep, w, GAt, w, false, Cst, w, T2, w);
    dev_matmul<T, T, T>(keep, keep, w, Cst, w, true, T2, w, A, ldk);
    for (int e = tid; e < keep * keep; e += nt) {
        const int i = e / keep, j = e - (e / keep) * keep;
        if (i < j) {
            const T a = (T)0.5 * (A[i * ldk + j] + A[j * ldk + i]);
            A[i * ldk + j] = a;
            A[j * ldk + i] = a;
        }
    }
    __syncthreads();
    dev_jacobi<T>(keep, ldk, A, V, csb, pairs, &s_rot, kMaxSweeps);
    dev_sort_eig<T, T>(keep, ldk, A, V, lam, Z, keep);
    const int kk = k < keep ? k : keep;
    if (sizeof(T) == sizeof(double)) {
        for (int e = tid; e < w * k; e += nt) {
            const int i = e / k, j = e - (e / k) * k;
            double s = 0.0;
            if (j < kk) {
                const int col = largest ? keep - 1 - j : j;
                for (int m = 0; m < keep; ++m) s += Cs[i * w + m] * (double)Z[m * keep + col];
            }
            coef[e] = s;
        }
        for (int j = tid; j < k; j += nt) theta[j] = j < kk ? (double)lam[largest ? keep - 1 - j : j] : 0.0;
        if (tid == 0) {
            info[0] = keep;
            int bad = 0;
            for (int j = 0; j < kk; ++j)
                if (!isfinite((double)lam[j])) bad = 1;
            info[1] = bad;
        }
        return;
    }
    // FP64 refinement of the k-dimensional Ritz subspace
    for (int e = tid; e < keep * kk; e += nt) {
        const int i = e / kk, j = e - (e / kk) * kk;
        Zk[e] = (double)Z[i * keep + (largest ? keep - 1 - j : j)];
    }
    __syncthreads();
    dev_matmul<double, double, double>(kk, kk, keep, Zk, kk, true, Zk, kk, M, kk);
    const int bad_chol = dev_chol_inv(kk, M, kk, R, Ri, &s_flag);
    dev_matmul<double, double, double>(keep, kk, kk, Zk, kk, false, Ri, kk, ZR, kk);
    dev_matmul<double, double, double>(w, kk, keep, Cs, w, false, ZR, kk, Y, kk);
    dev_matmul<double, double, double>(w, kk, w, GAs, w, false, Y, kk, Bm, kk);
    // the k x k projection reuses the shared region (the w x w solves are done)
    const int ldkk = pad_ld(kk);
    const bool ref_smem = use_smem && (size_t)2 * kk * ldkk * sizeof(double) <= (size_t)2 * w * ld * sizeof(T);
    double *A64 = ref_smem ? reinterpret_cast<double *>(As) : reinterpret_cast<double *>(Ag);
    double *V64 = A64 + kk * ldkk;
    dev_matmul<double, double, double>(kk, kk, w, Y, kk, true, Bm, kk, A64, ldkk);
    for (int e = tid; e < kk * kk; e += nt) {
        const int i = e / kk, j = e - (e / kk) * kk;
        if (i < j) {
            const double a = 0.5 * (A64[i * ldkk + j] + A64[j * ldkk + i]);
            A64[i * ldkk + j] = a;
            A64[j * ldkk + i] = a;
        }
    }
    __syncthreads();
    dev_jacobi<double>(kk, ldkk, A64, V64, cs64, pairs64, &s_rot, kMaxSweeps);
    dev_sort_eig<double, double>(kk, ldkk, A64, V64, mu, Q, kk);
    for (int e = tid; e < w * k; e += nt) {  // coef = Y Q (descending for 'largest')
        const int i = e / k, j = e - (e / k) * k;
        double s = 0.0;
        if (j < kk) {
            const int col = largest ? kk - 1 - j : j;
            for (int m = 0; m < kk; ++m) s += Y[i * kk + m] * Q[m * kk + col];
        }
        coef[e] = s;
    }
    for (int j = tid; j < k; j += nt) theta[j] = j < kk ? mu[largest ? kk - 1 - j : j] : 0.0;
    if (tid == 0) {
        info[0] = keep;
        int bad = bad_chol;
        for (int j = 0; j < kk; ++j)
            if (!isfinite(mu[j])) bad = 1;
        info[1] = bad;
    }
}

template <typename T>
__global__ void __launch_bounds__(kSmallThreads) k_small_rr(int w, int k, int largest, const double *GS,
                                                            const double *GA, double tau, double *coef,
                                                            double *theta, double *work, int *info, int use_smem)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *As = reinterpret_cast<T *>(smem_raw);
    T *Vs = As + w * pad_ld(w);
    rr_body<T>(w, k, largest, GS, GA, tau, coef, theta, work, info, As, Vs, use_smem);
}

int small_svqb_rr(int w, int k, int largest, int mixed, const double *GS, const double *GA, double tau,
                  double *coef, double *theta, double *work, int *info, cudaStream_t st)
{
    const int cap = 160 * 1024;
    static const bool attr_once = [&]() {
        cudaFuncSetAttribute(k_small_rr<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
        cudaFuncSetAttribute(k_small_rr<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
        return true;
    }();
    (void)attr_once;
    const size_t es = mixed ? sizeof(float) : sizeof(double);
    const size_t sm = 2 * (size_t)w * pad_ld(w) * es;
    const int use_smem = sm <= (size_t)cap;
    note_launch();
    if (mixed)
        k_small_rr<float><<<1, kSmallThreads, use_smem ? sm : 0, st>>>(w, k, largest, GS, GA, tau, coef, theta,
                                                                       work, info, use_smem);
    else
        k_small_rr<double><<<1, kSmallThreads, use_smem ? sm : 0, st>>>(w, k, largest, GS, GA, tau, coef, theta,
                                                                        work, info, use_smem);
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

// ---------------------------------------------------------------------------------
// Rayleigh-Ritz with H on span(X) for the convergence test and the final extraction.
// In: mu, V = eig(M), M = X^T (H - sigma) X; EtE = E^T E, E = (H - sigma)X - X M.
// Residual of pair j: sqrt(v_j^T EtE v_j).  Selects the nev values of mu nearest 0
// (ties: lower first), writes sel (ascending mu), res_sel, st[0] = converged,
// st[1] = NaN/Inf seen, dst[0] = max relative residual of the selection.
// res_all[j] = sqrt(v_j^T sym(EtE) v_j), one block per column j: thread a forms
// (sym(EtE) v_j)_a, the block sums v_j[a] times it in a fixed shape (warp shuffles, then
// the warps in order).
__global__ void __launch_bounds__(64) k_hrr_resid(int k, const double *V, const double *EtE, double *res_all)
{
    __shared__ double s_w[2];
    const int j = blockIdx.x, a = threadIdx.x;
    double s = 0.0;
    if (a < k) {
        double t = 0.0;
        for (int b = 0; b < k; ++b) t += 0.5 * (EtE[a * k + b] + EtE[b * k + a]) * V[b * k + j];
        s = V[a * k + j] * t;
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((a & 31) == 0) s_w[a >> 5] = s;
    __syncthreads();
    if (a == 0) res_all[j] = sqrt(fmax(s_w[0] + s_w[1], 0.0));
}

// The nev Ritz values nearest 0 (|mu| ascending, ties: lower mu, then lower index), in
// ascending index order: thread j ranks its own value against all k, and the chosen
// ones are compacted by ballot.
__global__ void __launch_bounds__(64) k_hrr_pick(int k, int nev, const double *mu, const double *res_all,
                                                 double tol_abs, double norm_h, int *sel, double *res_sel, int *st,
                                                 double *dst)
{
    __shared__ unsigned s_ball[2];
    __shared__ int s_conv[2], s_bad[2];
    __shared__ double s_mx[2];
    const int j = threadIdx.x, lane = j & 31, w = j >> 5;
    bool pick = false;
    if (j < k) {
        const double mj = mu[j], aj = fabs(mj);
        int rank = 0;
        for (int i = 0; i < k; ++i) {
            const double mi = mu[i], ai = fabs(mi);
            if (ai < aj || (ai == aj && (mi < mj || (mi == mj && i < j)))) ++rank;
        }
        pick = rank < nev;
    }
    const unsigned ball = __ballot_sync(0xffffffffu, pick);
    if (lane == 0) s_ball[w] = ball;
    __syncthreads();
    int conv = 1, bad = 0;
    double mx = 0.0;
    if (pick) {
        const int pos = __popc(ball & ((1u << lane) - 1u)) + (w ? __popc(s_ball[0]) : 0);
        const double r = res_all[j];
        sel[pos] = j;
        res_sel[pos] = r;
        if (!isfinite(r) || !isfinite(mu[j])) bad = 1;
        if (!(r <= tol_abs)) conv = 0;
        mx = r / norm_h;
    }
    conv = __all_sync(0xffffffffu, conv);
    bad = __any_sync(0xffffffffu, bad);
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0) {
        s_conv[w] = conv;
        s_bad[w] = bad;
        s_mx[w] = mx;
    }
    __syncthreads();
    if (j == 0) {
        st[0] = s_conv[0] && s_conv[1];
        st[1] = s_bad[0] || s_bad[1];
        dst[0] = fmax(s_mx[0], s_mx[1]);
    }
}

int hrr_select(int k, int nev, const double *mu, const double *V, const double *EtE, double tol_abs, double norm_h,
               double *res_all, int *sel, double *res_sel, int *st, double *dst, cudaStream_t s)
{
    note_launch();
    k_hrr_resid<<<k, 64, 0, s>>>(k, V, EtE, res_all);
    note_launch();
    k_hrr_pick<<<1, 64, 0, s>>>(k, nev, mu, res_all, tol_abs, norm_h, sel, res_sel, st, dst);
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

// Csel (k x nev) = V[:, sel]
__global__ void k_gather_cols(int k, int nev, const double *V, const int *sel, double *Csel)
{
    for (int e = threadIdx.x; e < k * nev; e += blockDim.x) {
        const int i = e / nev, j = e % nev;
        Csel[e] = V[i * k + sel[j]];
    }
}

int gather_cols(int k, int nev, const double *V, const int *sel, double *Csel, cudaStream_t st)
{
    note_launch();
    k_gather_cols<<<1, 256, 0, st>>>(k, nev, V, sel, Csel);
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

// ---------------------------------------------------------------------------------
// Half-chain entanglement entropy (Sec. 2.2) of sector vectors.  Cut after the first la
// sites.  With p up spins on the left, a vector's entries form the R x T matrix
// M_p[i][c] = v[off_c + i]: i the colex rank of the left pattern among those with p ones,
// c the colex rank of the right pattern among those with n_up - p ones, off_c the row of
// the first state with that right pattern (the left p spins lowest).  The reduced density
// matrix of the left block is the direct sum of the M_p M_p^T.  One block per
// (vector, p): M_p gathered densely into its workspace, the smaller Gram (M M^T or
// M^T M, with the same nonzero eigenvalues), its eigenvalues by Jacobi (FP64), and the
// sums s0 = sum lambda, s1 = sum lambda ln lambda over lambda > 0, in a fixed order.  A
// second launch forms S = ln N - (sum_p s1) / N with N = sum_p s0 = ||v||^2, so v need
// not be normalised.

EntanglementPlan entanglement_plan(int L, int n_up, int la)
{
    EntanglementPlan pl{};
    const int lb = L - la;
    for (int p = 0; p <= la; ++p) {
        const int q = n_up - p;
        if (q < 0 || q > lb) continue;
        const int64_t R = host_binom(la, p), T = host_binom(lb, q);
        const int64_t d = R < T ? R : T;
        if (d > pl.dmax) pl.dmax = d;
        if (T > pl.tmax) pl.tmax = T;
        if (R * T > pl.mmax) pl.mmax = R * T;
    }
    // M (mmax), A (dmax x pad_ld(dmax)), cs (dmax + 2), pairs and offsets (as doubles)
    pl.block_doubles = pl.mmax + pl.dmax * (int64_t)pad_ld((int)pl.dmax) + 2 * (pl.dmax + 2) + pl.tmax + 8;
    pl.blocks_per_vector = la + 1;
    return pl;
}

__global__ void __launch_bounds__(kSmallThreads)
    k_ent_block(int L, int n_up, int la, const double *__restrict__ V, int64_t ldv, double *work,
                int64_t block_doubles, int64_t mmax, int64_t dmax, double *parts)
{
    __shared__ uint32_t sb[kBinomDim * kBinomDim];
    __shared__ int s_rot;
    __shared__ double s_r0[kSmallThreads / 32], s_r1[kSmallThreads / 32];
    load_binom(sb);
    __syncthreads();
    const int e = blockIdx.x / (la + 1), p = blockIdx.x % (la + 1);
    const int lb = L - la, q = n_up - p;
    double *out = parts + 2 * (int64_t)blockIdx.x;
    if (q < 0 || q > lb) {  // no state has p up spins on the left
        if (threadIdx.x == 0) {
            out[0] = 0.0;
            out[1] = 0.0;
        }
        return;
    }
    const int R = (int)binom(sb, la, p), T = (int)binom(sb, lb, q);
    const bool left = R <= T;  // Gram over the left patterns (d = R), else over the right ones
    const int d = left ? R : T, ld = pad_ld(d);
    double *M = work + (int64_t)blockIdx.x * block_doubles;  // R x T, row-major
    double *A = M + mmax;
    double *cs = A + dmax * (int64_t)pad_ld((int)dmax);
    int *pairs = reinterpret_cast<int *>(cs + dmax + 2);
    uint32_t *off = reinterpret_cast<uint32_t *>(cs + 2 * (dmax + 2));
    for (int c = threadIdx.x; c < T; c += blockDim.x) {
        const uint32_t b = cns_unrank(sb, lb, q, (uint32_t)c);
        off[c] = cns_rank(sb, (b << la) | ((1u << p) - 1u));
    }
    __syncthreads();
    const double *v = V + e;
    for (int64_t x = threadIdx.x; x < (int64_t)R * T; x += blockDim.x) {
        const int i = (int)(x % R), c = (int)(x / R);  // consecutive threads: consecutive rows of a tile
        M[(int64_t)i * T + c] = v[((int64_t)off[c] + i) * ldv];
    }
    __syncthreads();
    for (int64_t x = threadIdx.x; x < (int64_t)d * d; x += blockDim.x) {
        const int i = (int)(x / d), j = (int)(x % d);
        if (j < i) continue;
        double acc = 0.0;
        if (left) {
            const double *mi = M + (int64_t)i * T, *mj = M + (int64_t)j * T;
            for (int c = 0; c < T; ++c) acc += mi[c] * mj[c];
        } else {
            for (int r = 0; r < R; ++r) acc += M[(int64_t)r * T + i] * M[(int64_t)r * T + j];
        }
        A[(int64_t)i * ld + j] = acc;
        A[(int64_t)j * ld + i] = acc;
    }
    __syncthreads();
    dev_jacobi<double, false>(d, ld, A, nullptr, cs, pairs, &s_rot, kMaxSweeps);
    double s0 = 0.0, s1 = 0.0;
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        const double lam = A[(int64_t)i * ld + i];
        if (lam > 0.0) {
            s0 += lam;
            s1 += lam * log(lam);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s_r0[threadIdx.x >> 5] = s0;
        s_r1[threadIdx.x >> 5] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0;
        for (int w = 0; w < kSmallThreads / 32; ++w) {
            a0 += s_r0[w];
            a1 += s_r1[w];
        }
        out[0] = a0;
        out[1] = a1;
    }
}

__global__ void k_ent_combine(int nvec, int per, const double *parts, double *S)
{
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nvec) return;
    double n2 = 0.0, a1 = 0.0;
    for (int p = 0; p < per; ++p) {
        n2 += parts[2 * ((int64_t)e * per + p)];
        a1 += parts[2 * ((int64_t)e * per + p) + 1];
    }
    S[e] = n2 > 0.0 ? log(n2) - a1 / n2 : NAN;
}

int entanglement_launch(int L, int n_up, int la, int nvec, const double *V, int64_t ldv, double *S, void *work,
                        size_t work_bytes, cudaStream_t st)
{
    const EntanglementPlan pl = entanglement_plan(L, n_up, la);
    const int64_t nblk = (int64_t)nvec * pl.blocks_per_vector;
    const size_t need = entanglement_work_bytes(pl, nvec);
    if (work_bytes < need) return MBL_ERR_WORKSPACE;
    double *w = (double *)(((uintptr_t)work + 255) & ~(uintptr_t)255);
    double *parts = w + nblk * pl.block_doubles;
    note_launch();
    k_ent_block<<<(unsigned)nblk, kSmallThreads, 0, st>>>(L, n_up, la, V, ldv, w, pl.block_doubles, pl.mmax,
                                                          pl.dmax, parts);
    if (cudaGetLastError() != cudaSuccess) return MBL_ERR_CUDA;
    note_launch();
    k_ent_combine<<<(nvec + 127) / 128, 128, 0, st>>>(nvec, pl.blocks_per_vector, parts, S);
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

size_t entanglement_work_bytes(const EntanglementPlan &pl, int nvec)
{
    const int64_t nblk = (int64_t)nvec * pl.blocks_per_vector;
    return (size_t)(nblk * pl.block_doubles + 2 * nblk + 64) * sizeof(double) + 256;
}


}  // namespace mbl
