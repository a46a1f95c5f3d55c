// mbl_dense.cu -- dense linear algebra of the LOBPCG iteration (Sec. 3.2: LOBPCG is a
// block method whose Gram matrices and updates are matrix-matrix operations; they
// replace the paper's allreduce reductions, Sec. 6.2).
//
//  * tall-skinny Gram  C = A^T B      (A: n x p, B: n x q, p, q <= 192), deterministic:
//    fixed row slabs -> per-slab partial tiles -> fixed-order sum;
//  * tall-skinny update D = beta C + alpha A M   (M: p x q small);
//  * per-column dot products, casts between FP64 storage and the PCG precision;
//  (the small dense kernels on one block are in mbl_small.cu).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mbl_dense.h"
#include "mbl_internal.h"

namespace mbl {

// ---------------------------------------------------------------------------------
// Gram: partial tiles.  Block (tp, tq, slab) computes the TS x TS output tile (tp, tq)
// over rows [slab * rows_per_slab, ...).  256 threads (16 x 16), MT x MT outputs each
// (MT = TS / 16); threads whose outputs all lie outside p x q only help with staging, so
// small Grams cost what they compute.
constexpr int kGR = 16;  // rows staged per step

template <typename CT, int TS>
__global__ void __launch_bounds__(256) k_gram_partial(const double *__restrict__ A, int64_t lda, int p,
                                                      const double *__restrict__ B, int64_t ldb, int q,
                                                      int64_t n, int64_t rows_per_slab, double *__restrict__ part)
{
    constexpr int MT = TS / 16;
    __shared__ CT As[kGR][TS + 1];
    __shared__ CT Bs[kGR][TS + 1];
    const int tp = blockIdx.x, tq = blockIdx.y, slab = blockIdx.z;
    const int p0 = tp * TS, q0 = tq * TS;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const bool active = (p0 + ty < p) && (q0 + tx < q);
    CT acc[MT][MT];
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < MT; ++j) acc[i][j] = (CT)0;
    const int64_t r_begin = (int64_t)slab * rows_per_slab;
    int64_t r_end = r_begin + rows_per_slab;
    if (r_end > n) r_end = n;
    const int pw = min(TS, p - p0), qw = min(TS, q - q0);
    for (int64_t r0 = r_begin; r0 < r_end; r0 += kGR) {
        for (int e = threadIdx.x; e < kGR * TS; e += 256) {
            const int rr = e / TS, cc = e % TS;
            const int64_t row = r0 + rr;
            const bool in = row < r_end;
            As[rr][cc] = (in && cc < pw) ? (CT)A[row * lda + p0 + cc] : (CT)0;
            Bs[rr][cc] = (in && cc < qw) ? (CT)B[row * ldb + q0 + cc] : (CT)0;
        }
        __syncthreads();
        if (active) {
#pragma unroll 4
            for (int rr = 0; rr < kGR; ++rr) {
                CT a[MT], b[MT];
#pragma unroll
                for (int i = 0; i < MT; ++i) a[i] = As[rr][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < MT; ++j) b[j] = Bs[rr][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < MT; ++i)
#pragma unroll
                    for (int j = 0; j < MT; ++j) acc[i][j] += a[i] * b[j];
            }
        }
        __syncthreads();
    }
    double *out = part + (int64_t)slab * p * q;
#pragma unroll
    for (int i = 0; i < MT; ++i)
#pragma unroll
        for (int j = 0; j < MT; ++j) {
            const int pi = p0 + ty + 16 * i, qj = q0 + tx + 16 * j;
            if (pi < p && qj < q) out[(int64_t)pi * q + qj] = (double)acc[i][j];
        }
}

// C[i][j] (ldc) = sum over slabs of part[slab][i][j] (part[slab][j][i] when colmajor, the
// tensor-core Gram's layout); optionally the symmetric part (C + C^T)/2 when p == q and
// sym != 0.  A block takes 32 outputs consecutive in the partials' order; its 8 warps split
// the slabs (warp g sums slabs g, g + 8, ...), and one thread per output adds the 8 group
// sums in group order, so the result is the same on every run.
constexpr int kRedGroups = 8;

__global__ void __launch_bounds__(256) k_gram_reduce(const double *__restrict__ part, int nslab, int p, int q,
                                                     double *__restrict__ C, int64_t ldc, int sym, int colmajor)
{
    __shared__ double s_sum[kRedGroups][32], s_tr[kRedGroups][32];
    const int o = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int e = blockIdx.x * 32 + o;
    const int pq = p * q;
    const int i = colmajor ? e % p : e / q, j = colmajor ? e / p : e % q;
    double s = 0.0, t = 0.0;
    if (e < pq) {
        const int64_t et = colmajor ? (int64_t)i * p + j : (int64_t)j * q + i;
        for (int b = g; b < nslab; b += kRedGroups) {
            s += part[(int64_t)b * pq + e];
            if (sym) t += part[(int64_t)b * pq + et];
        }
    }
    s_sum[g][o] = s;
    s_tr[g][o] = t;
    __syncthreads();
    if (g == 0 && e < pq) {
        double a = 0.0, c = 0.0;
        for (int h = 0; h < kRedGroups; ++h) {
            a += s_sum[h][o];
            c += s_tr[h][o];
        }
        C[(int64_t)i * ldc + j] = sym ? 0.5 * (a + c) : a;
    }
}

// Output tile edge: 64 when both sizes are multiples of 64, 16 for tiny outputs, else 32.
static int gram_tile(int p, int q)
{
    if (p % 64 == 0 && q % 64 == 0) return 64;
    if (p <= 16 && q <= 16) return 16;
    return 32;
}

static int gram_slabs(int64_t n, int p, int q)
{
    const int ts = gram_tile(p, q);
    const int tiles = ((p + ts - 1) / ts) * ((q + ts - 1) / ts);
    int want = (2 * num_sms() + tiles - 1) / tiles;
    int64_t max_by_rows = (n + 255) / 256;  // at least 256 rows per slab
    if (want > max_by_rows) want = (int)max_by_rows;
    if (want < 1) want = 1;
    return want;
}

size_t gram_partial_doubles(int64_t n, int p, int q)
{
    const size_t cuda = (size_t)gram_slabs(n, p, q), tc = gram_tc_supported(p, q) ? (size_t)gram_tc_slabs(n, p) : 0;
    return (cuda > tc ? cuda : tc) * p * q;
}

static int g_gram_engine = 0;
static thread_local int t_gram_engine = 0;  // per-call choice (mbl_gram), overrides the switch
void set_gram_engine(int engine) { g_gram_engine = engine; }
void set_gram_engine_local(int engine) { t_gram_engine = engine; }

// FP32 Grams go to the tensor cores when selected and the shape fits (p, q <= 256).  By
// default when both sides are >= 64 (measured with the TMA-fed kernel at n = 184,756:
// S^T S 96 x 96 in 96 us against 576 us on the CUDA cores, 64 x 64 in 89 us against 147 us;
// at n = 705,432, 192 x 192 in 1.0 ms against 4.1 ms; 32 x 32 is a tie).
static bool use_tensor_cores(int p, int q)
{
    const int e = t_gram_engine ? t_gram_engine : g_gram_engine;
    if (e == 1 || !gram_tc_supported(p, q)) return false;
    return e == 2 || (p >= 64 && q >= 64);
}

// FP32 block updates on the tensor cores: when asked for (engine 2) or by default from
// MBL_UPDATE_TC_MIN_ROWS rows on (a grid of at least 128 row tiles; measured on GB300 at
// n = 184,756 and 705,432 the TMA-fed kernel takes 0.2-0.8x the CUDA-core kernel's time).
#ifndef MBL_UPDATE_TC_MIN_ROWS
#define MBL_UPDATE_TC_MIN_ROWS 16384
#endif
static bool update_on_tensor_cores(const double *A, int64_t lda, int p, int q, const double *C, int64_t ldc,
                                   const double *D, int64_t ldd, double beta, int64_t n)
{
    const int e = t_gram_engine ? t_gram_engine : g_gram_engine;
    if (e == 1 || (e == 0 && n < MBL_UPDATE_TC_MIN_ROWS)) return false;
    return update_tc_supported(A, lda, p, q, C, ldc, D, ldd, beta);
}

template <typename CT, int TS>
static void launch_gram(const double *A, int64_t lda, int p, const double *B, int64_t ldb, int q, int64_t n,
                        int64_t rps, int nslab, double *part, cudaStream_t st)
{
    dim3 grid((p + TS - 1) / TS, (q + TS - 1) / TS, nslab);
    note_launch();
    k_gram_partial<CT, TS><<<grid, 256, 0, st>>>(A, lda, p, B, ldb, q, n, rps, part);
}

int gram(const double *A, int64_t lda, int p, const double *B, int64_t ldb, int q, int64_t n, double *C,
         int64_t ldc, int sym, int compute_f32, double *part, cudaStream_t st)
{
    if (compute_f32 && use_tensor_cores(p, q) && gram_tc_eligible(A, lda, p, B, ldb, q)) {
        const int nslab = gram_tc_slabs(n, p);
        const int rc = gram_tc_partial(A, lda, p, B, ldb, q, n, nslab, part, st);
        if (rc != MBL_OK) return rc;
        note_launch();
        k_gram_reduce<<<(p * q + 31) / 32, 256, 0, st>>>(part, nslab, p, q, C, ldc, sym, 1);
        return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
    }
    const int nslab = gram_slabs(n, p, q);
    const int64_t rps = (n + nslab - 1) / nslab;
    const int ts = gram_tile(p, q);
    if (compute_f32) {
        if (ts == 64) launch_gram<float, 64>(A, lda, p, B, ldb, q, n, rps, nslab, part, st);
        else if (ts == 32) launch_gram<float, 32>(A, lda, p, B, ldb, q, n, rps, nslab, part, st);
        else launch_gram<float, 16>(A, lda, p, B, ldb, q, n, rps, nslab, part, st);
    } else {
        if (ts == 64) launch_gram<double, 64>(A, lda, p, B, ldb, q, n, rps, nslab, part, st);
        else if (ts == 32) launch_gram<double, 32>(A, lda, p, B, ldb, q, n, rps, nslab, part, st);
        else launch_gram<double, 16>(A, lda, p, B, ldb, q, n, rps, nslab, part, st);
    }
    note_launch();
    k_gram_reduce<<<(p * q + 31) / 32, 256, 0, st>>>(part, nslab, p, q, C, ldc, sym, 0);
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

// ---------------------------------------------------------------------------------
// Update: D = beta * C + alpha * A M.  Block: 32 rows; M (p x q) and the 32 rows of A
// staged in shared memory; thread (row, 4-column group).
template <typename CT>
__global__ void __launch_bounds__(256) k_update(const double *__restrict__ A, int64_t lda, int p,
                                                const double *__restrict__ M, int64_t ldm, int q,
                                                const double *C, int64_t ldc, double *D, int64_t ldd,
                                                int64_t n, double alpha, double beta)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CT *Ms = reinterpret_cast<CT *>(smem_raw);  // p x q
    CT *As = Ms + p * q;                        // 32 x p
    for (int e = threadIdx.x; e < p * q; e += blockDim.x) Ms[e] = (CT)M[(int64_t)(e / q) * ldm + (e % q)];
    const int groups = (q + 3) / 4;              // 4-column groups per row
    const int rows_per_pass = 256 / groups;      // >= 4 for q <= 256
    for (int64_t r0 = (int64_t)blockIdx.x * 32; r0 < n; r0 += (int64_t)gridDim.x * 32) {
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * p; e += blockDim.x) {
            const int rr = e / p, cc = e % p;
            const int64_t row = r0 + rr;
            As[e] = row < n ? (CT)A[row * lda + cc] : (CT)0;
        }
        __syncthreads();
        for (int rr = threadIdx.x / groups; rr < 32; rr += rows_per_pass) {
            if (threadIdx.x / groups >= rows_per_pass) break;
            const int64_t row = r0 + rr;
            if (row >= n) break;
            const int c0 = (threadIdx.x % groups) * 4;
            CT acc[4] = {(CT)0, (CT)0, (CT)0, (CT)0};
            const CT *arow = As + rr * p;
            for (int i = 0; i < p; ++i) {
                const CT a = arow[i];
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (c0 + j < q) acc[j] += a * Ms[i * q + c0 + j];
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (c0 + j >= q) break;
                double v = alpha * (double)acc[j];
                if (beta != 0.0) v += beta * C[row * ldc + c0 + j];
                D[row * ldd + c0 + j] = v;
            }
        }
    }
}

int update(const double *A, int64_t lda, int p, const double *M, int64_t ldm, int q, const double *C, int64_t ldc,
           double *D, int64_t ldd, int64_t n, double alpha, double beta, int compute_f32, cudaStream_t st)
{
    if (n <= 0) return MBL_OK;
    if (compute_f32 && update_on_tensor_cores(A, lda, p, q, C, ldc, D, ldd, beta, n))
        return update_tc(A, lda, p, M, ldm, q, C, ldc, D, ldd, n, alpha, beta, st);
    int64_t blocks = (n + 31) / 32;
    const int64_t cap = (int64_t)num_sms() * 4;
    if (blocks > cap) blocks = cap;
    static const bool attr_set_once = [&]() {
        // largest use: p = 192, q = 64 -> (192 * 64 + 32 * 192) doubles = 144 KB
        const int mx = (192 * 64 + 32 * 192) * (int)sizeof(double);
        cudaFuncSetAttribute(k_update<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        cudaFuncSetAttribute(k_update<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
        return true;
    }();
    (void)attr_set_once;
    if (compute_f32) {
        const size_t sm = (size_t)(p * q + 32 * p) * sizeof(float);
        note_launch();
        k_update<float><<<(int)blocks, 256, sm, st>>>(A, lda, p, M, ldm, q, C, ldc, D, ldd, n, alpha, beta);
    } else {
        const size_t sm = (size_t)(p * q + 32 * p) * sizeof(double);
        note_launch();
        k_update<double><<<(int)blocks, 256, sm, st>>>(A, lda, p, M, ldm, q, C, ldc, D, ldd, n, alpha, beta);
    }
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

// ---------------------------------------------------------------------------------
// Per-column sums of squares: out[c] = sum_r A[r, c]^2 (deterministic two-pass).
__global__ void __launch_bounds__(256) k_colsq_partial(const double *__restrict__ A, int64_t lda, int k, int64_t n,
                                                       int64_t rows_per_block, double *__restrict__ part)
{
    __shared__ double s[256];
    const int per = 256 / k;
    const int c = threadIdx.x % k, ro = threadIdx.x / k;
    double acc = 0.0;
    const int64_t r_begin = (int64_t)blockIdx.x * rows_per_block;
    int64_t r_end = r_begin + rows_per_block;
    if (r_end > n) r_end = n;
    if (ro < per)
        for (int64_t r = r_begin + ro; r < r_end; r += per) {
            const double v = A[r * lda + c];
            acc += v * v;
        }
    s[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < k) {
        double t = 0.0;
        for (int j = 0; j < per; ++j) t += s[j * k + threadIdx.x];
        part[(int64_t)blockIdx.x * k + threadIdx.x] = t;
    }
}

__global__ void k_colsq_reduce(const double *__restrict__ part, int nb, int k, double *__restrict__ out, int take_sqrt)
{
    const int c = threadIdx.x;
    if (c >= k) return;
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += part[(int64_t)b * k + c];
    out[c] = take_sqrt ? sqrt(t) : t;
}

int colnorms(const double *A, int64_t lda, int k, int64_t n, double *out, int take_sqrt, double *part,
             cudaStream_t st)
{
    int nb = 2 * num_sms();
    if ((int64_t)nb * 256 > n) nb = (int)((n + 255) / 256);
    if (nb < 1) nb = 1;
    const int64_t rpb = (n + nb - 1) / nb;
    note_launch();
    k_colsq_partial<<<nb, 256, 0, st>>>(A, lda, k, n, rpb, part);
    note_launch();
    k_colsq_reduce<<<1, 64, 0, st>>>(part, nb, k, out, take_sqrt);
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

size_t colnorm_partial_doubles(int k) { return (size_t)2 * num_sms() * k; }

// dst (FP64, ldd) = (double) src (T, lds), n x k
template <typename T>
__global__ void k_widen(const T *__restrict__ src, int64_t lds, double *__restrict__ dst, int64_t ldd, int k, int64_t n)
{
    const int64_t total = n * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / k;
        const int c = (int)(e % k);
        dst[r * ldd + c] = (double)src[r * lds + c];
    }
}

int widen(int src_f32, const void *src, int64_t lds, double *dst, int64_t ldd, int k, int64_t n, cudaStream_t st)
{
    const int grid = num_sms() * 8;
    note_launch();
    if (src_f32)
        k_widen<float><<<grid, 256, 0, st>>>((const float *)src, lds, dst, ldd, k, n);
    else
        k_widen<double><<<grid, 256, 0, st>>>((const double *)src, lds, dst, ldd, k, n);
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

// column scaling in place: A[r, c] *= scale[c] (scale given as norms: multiply by 1/norm)
__global__ void k_scale_cols_inv(double *__restrict__ A, int64_t lda, int k, int64_t n, const double *__restrict__ norms)
{
    const int64_t total = n * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / k;
        const int c = (int)(e % k);
        const double nv = norms[c];
        A[r * lda + c] = nv > 0.0 ? A[r * lda + c] / nv : 0.0;
    }
}

int scale_cols_inv(double *A, int64_t lda, int k, int64_t n, const double *norms, cudaStream_t st)
{
    note_launch();
    k_scale_cols_inv<<<num_sms() * 8, 256, 0, st>>>(A, lda, k, n, norms);
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

// D (n x k, ldd) = S (n x k, lds): strided block copy
__global__ void k_copy_block(const double *__restrict__ S, int64_t lds, double *__restrict__ D, int64_t ldd, int k, int64_t n)
{
    const int64_t total = n * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / k;
        const int c = (int)(e % k);
        D[r * ldd + c] = S[r * lds + c];
    }
}

int copy_block(const double *S, int64_t lds, double *D, int64_t ldd, int k, int64_t n, cudaStream_t st)
{
    note_launch();
    k_copy_block<<<num_sms() * 8, 256, 0, st>>>(S, lds, D, ldd, k, n);
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

}  // namespace mbl
