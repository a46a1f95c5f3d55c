// mbl_gram_tc.cu -- the tall-skinny Gram C = A^T B of the LOBPCG Rayleigh-Ritz step
// (Sec. 3.2: the block method's dense contraction) on the 5th-generation tensor cores of
// sm_103a: tcgen05.mma kind::tf32 with the accumulator in tensor memory (TMEM).
//
// FP32 accuracy from TF32 operands: every FP64 input x is rounded once to FP32, then
// split x = hi + lo with hi = tf32(x) and lo = tf32(x - hi) (x - hi is exact in FP32), and
// D += Ahi Bhi + Ahi Blo + Alo Bhi; the dropped Alo Blo and the rounding of lo are below
// 2^-21 relative, the order of FP32's own rounding.
//
// Work split: block (m_tile, slab) owns the 128 x Np accumulator of columns
// [128 m_tile, +128) of A against all Np (>= q, multiple of 16) columns of B over a slab
// of rows, and writes it as one slab partial (FP64) for the fixed-order slab reduction
// of mbl_dense.cu.  Rows are staged 32 at a time (four MMA k-steps of 8), converted and
// split by all 256 threads into two shared-memory buffers (K-major, no swizzle: 8-row x
// 16-byte core matrices, 128 B apart along K, 1024 B apart along M/N); one thread issues
// the MMAs of a chunk and commits them to the buffer's mbarrier, which the next use of
// that buffer waits on, so staging of chunk i+1 overlaps the MMAs of chunk i.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mbl_dense.h"
#include "mbl_internal.h"

namespace mbl {

namespace {

constexpr int kTcM = 128;        // accumulator rows (M of the MMA)
constexpr int kTcKC = 32;        // rows of A and B staged per chunk
constexpr int kTcThreads = 256;  // 8 warps
constexpr long long kTcWaitCycles = 2000000000ll;  // ~1 s at 2 GHz

// Operand tile of R rows (R a multiple of 8) and kTcKC K-elements: byte offset of the
// 4-element K quad kq of row r.  Core matrices (8 rows x 16 B) are 128 B apart along K
// and 1024 B apart along the rows.
__device__ __forceinline__ uint32_t tile_offset(int r, int kq) { return (uint32_t)((r >> 3) * 1024 + kq * 128 + (r & 7) * 16); }

__host__ __device__ constexpr uint32_t tile_bytes(int rows) { return (uint32_t)rows * kTcKC * 4u; }

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading byte offset (between
// core matrices along K), stride byte offset (between 8-row groups), descriptor version
// 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::tf32: D in FP32, A and B in TF32, both K-major,
// N = n_cols (multiple of 16), M = 128.
__host__ __device__ constexpr uint32_t instr_desc_tf32(int n_cols)
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n_cols >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *m, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(m)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t *m, unsigned parity)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(saddr(m)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > kTcWaitCycles) return false;
    }
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *m)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(m))
                 : "memory");
}

// Stage rows [r0, r0 + kTcKC) of columns [c0, c0 + cols) of X (row-major, ld) as the hi
// and lo TF32 parts of an R-row operand tile; rows past n and columns past cols are 0.
__device__ __forceinline__ void stage(const double *__restrict__ X, int64_t ld, int64_t n, int64_t r0, int c0,
                                      int cols, int R, float *hi, float *lo)
{
    for (int task = threadIdx.x; task < R * (kTcKC / 4); task += kTcThreads) {
        const int r = task % R, kq = task / R;
        float h[4], l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int64_t row = r0 + 4 * kq + i;
            const float x = (row < n && r < cols) ? (float)__ldg(X + row * ld + c0 + r) : 0.0f;
            h[i] = to_tf32(x);
            l[i] = to_tf32(x - h[i]);
        }
        const uint32_t off = tile_offset(r, kq) / 4;
        *reinterpret_cast<float4 *>(hi + off) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4 *>(lo + off) = make_float4(l[0], l[1], l[2], l[3]);
    }
}

__global__ void __launch_bounds__(kTcThreads, 1)
    k_gram_tc(const double *__restrict__ A, int64_t lda, int p, const double *__restrict__ B, int64_t ldb, int q,
              int np, int64_t n, int64_t rows_per_slab, double *__restrict__ part, uint32_t tmem_cols)
{
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    __shared__ __align__(8) uint64_t s_mbar[2];
    __shared__ uint32_t s_tmem;
    const int m_tile = blockIdx.x, slab = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t a_bytes = tile_bytes(kTcM), b_bytes = tile_bytes(np);
    const uint32_t buf_bytes = 2 * a_bytes + 2 * b_bytes;  // A hi, A lo, B hi, B lo
    if (threadIdx.x == 0) {
        mbar_init(&s_mbar[0], 1);
        mbar_init(&s_mbar[1], 1);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&s_tmem)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = instr_desc_tf32(np);
    const int c0 = m_tile * kTcM, acols = min(kTcM, p - c0);
    const int64_t r_begin = (int64_t)slab * rows_per_slab;
    const int64_t r_end = min(n, r_begin + rows_per_slab);
    const int nchunks = r_end > r_begin ? (int)((r_end - r_begin + kTcKC - 1) / kTcKC) : 0;
    bool ok = true;
    for (int i = 0; i < nchunks; ++i) {
        const int b = i & 1;
        if (i >= 2) ok = ok && mbar_wait(&s_mbar[b], (unsigned)(((i - 2) >> 1) & 1));
        if (!__syncthreads_and(ok)) break;
        unsigned char *base = tc_raw + b * buf_bytes;
        float *ahi = reinterpret_cast<float *>(base), *alo = reinterpret_cast<float *>(base + a_bytes);
        float *bhi = reinterpret_cast<float *>(base + 2 * a_bytes);
        float *blo = reinterpret_cast<float *>(base + 2 * a_bytes + b_bytes);
        const int64_t r0 = r_begin + (int64_t)i * kTcKC;
        stage(A, lda, r_end, r0, c0, acols, kTcM, ahi, alo);
        stage(B, ldb, r_end, r0, 0, q, np, bhi, blo);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = saddr(ahi), a1 = saddr(alo), b0 = saddr(bhi), b1 = saddr(blo);
#pragma unroll
            for (int s = 0; s < kTcKC / 8; ++s) {
                const uint32_t ks = (uint32_t)s * 256u;  // two core matrices along K per step
                mma_tf32(tmem, smem_desc(a0 + ks), smem_desc(b0 + ks), idesc, (i > 0 || s > 0) ? 1 : 0);
                mma_tf32(tmem, smem_desc(a0 + ks), smem_desc(b1 + ks), idesc, 1);
                mma_tf32(tmem, smem_desc(a1 + ks), smem_desc(b0 + ks), idesc, 1);
            }
            mma_commit(&s_mbar[b]);
        }
    }
    // the last commit covers every MMA of the block
    if (nchunks > 0) {
        const int last = nchunks - 1;
        const bool done = mbar_wait(&s_mbar[last & 1], (unsigned)((last >> 1) & 1));
        ok = ok && done;
        if (!done && nchunks > 1) mbar_wait(&s_mbar[(last - 1) & 1], (unsigned)(((last - 1) >> 1) & 1));
    }
    ok = __syncthreads_and(ok);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // accumulator -> slab partial: warp w reads TMEM lanes 32 (w % 4) .. +31 and every
    // other 8-column group (w / 4 picks which)
    double *out = part + (int64_t)slab * p * q;
    const int quad = warp & 3, half = warp >> 2;
    const int row = c0 + quad * 32 + lane;
    for (int cg = half; cg * 8 < np; cg += 2) {
        uint32_t v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (nchunks > 0) {
            const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(cg * 8);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        }
        if (row < p) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int col = cg * 8 + j;
                if (col < q) out[(int64_t)row * q + col] = ok ? (double)__uint_as_float(v[j]) : (double)NAN;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

}  // namespace

bool gram_tc_supported(int p, int q) { return p >= 1 && q >= 1 && p <= 256 && q <= 256; }

int gram_tc_slabs(int64_t n, int p)
{
    const int mtiles = (p + kTcM - 1) / kTcM;
    int want = num_sms() / mtiles;
    const int64_t by_rows = (n + 4 * kTcKC - 1) / (4 * kTcKC);  // at least 128 rows per slab
    if (want > by_rows) want = (int)by_rows;
    return want < 1 ? 1 : want;
}

int gram_tc_partial(const double *A, int64_t lda, int p, const double *B, int64_t ldb, int q, int64_t n, int nslab,
                    double *part, cudaStream_t st)
{
    if (!gram_tc_supported(p, q)) return MBL_ERR_ARG;
    const int np = (q + 15) / 16 * 16;
    const uint32_t tmem_cols = np <= 32 ? 32u : (np <= 64 ? 64u : (np <= 128 ? 128u : 256u));
    const size_t smem = 2 * (size_t)(2 * tile_bytes(kTcM) + 2 * tile_bytes(np));
    static const bool attr = []() {
        cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2 * (2 * tile_bytes(kTcM) + 2 * tile_bytes(256))));
        return true;
    }();
    (void)attr;
    const int64_t rps = ((n + nslab - 1) / nslab + kTcKC - 1) / kTcKC * kTcKC;
    dim3 grid((p + kTcM - 1) / kTcM, nslab);
    note_launch();
    k_gram_tc<<<grid, kTcThreads, smem, st>>>(A, lda, p, B, ldb, q, np, n, rps, part, tmem_cols);
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

}  // namespace mbl
