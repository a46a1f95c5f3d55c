// mbl_gram_tc.cu -- the dense contractions of the LOBPCG step (Sec. 3.2: the block method's
// Grams and block updates) on the 5th-generation tensor cores of sm_103a: tcgen05.mma
// kind::tf32 with the accumulators in tensor memory (TMEM), operands moved by TMA.
//
// FP32 accuracy from TF32 operands: every FP64 input x is cut to FP32 and split into
// x = hi + lo, hi and lo TF32 (by bit operations: conversions and arithmetic on GB300's FP64
// pipe would bind these HBM-bound kernels), and D += Ahi Bhi + Ahi Blo + Alo Bhi; the dropped
// Alo Blo and the rounding of lo are below 2^-21 relative, the order of FP32's own rounding.
//
// Both kernels are persistent (one CTA per SM) with warp roles joined by mbarriers: a TMA
// producer fills a ring of 128-byte-swizzled FP64 boxes, converter warps write the TF32
// operand tiles (no-swizzle K-major core matrices: 8 rows x 16 bytes, 128 B apart along K),
// one thread issues the MMAs, and epilogue warps read the accumulators with tcgen05.ld.
// Every ring and mbarrier has one waiting role that waits on each of its phases in turn.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mbl_dense.h"
#include "mbl_internal.h"

namespace mbl {

namespace {

constexpr int kTcM = 128;        // accumulator rows (M of the MMA)
constexpr int kTcKC = 32;        // K per staged chunk of the update's M operand
constexpr long long kTcWaitCycles = 2000000000ll;  // ~1 s at 2 GHz

// Operand tile of R rows (R a multiple of 8) and kTcKC K-elements (the update's staged M):
// byte offset of the 4-element K quad kq of row r.  Core matrices (8 rows x 16 B) are 128 B
// apart along K and 1024 B apart along the rows.
__device__ __forceinline__ uint32_t tile_offset(int r, int kq) { return (uint32_t)((r >> 3) * 1024 + kq * 128 + (r & 7) * 16); }

__host__ __device__ constexpr uint32_t tile_bytes(int rows) { return (uint32_t)rows * kTcKC * 4u; }

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ float to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
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

// ---------------------------------------------------------------------------------
// Block update D = beta C + alpha A M (A: n x p, M: p x q, C, D: n x q, all FP64 in memory) of
// the LOBPCG step (Sec. 3.2) with FP32 accuracy on the tensor cores: A and M rounded to FP32
// and split into two TF32 parts (file header), D_acc = Ahi Mhi + Ahi Mlo + Alo Mhi per
// k-step.  Here M of the MMA is a tile of 128 rows of A, N = q (padded to 16), K = p (padded
// to 16).
//
// The kernel is HBM-bound (p + 2q doubles per row against ~6 p q tensor-core flops), so every
// byte moves by TMA and the arithmetic is spread over warp roles of one persistent CTA per SM:
//   warp 24      A producer: cp.async.bulk.tensor loads of 128-row x 16-column FP64 boxes of A
//                (128-byte swizzle) into a ring of kUpdMaxStages-at-most 16 KB slots,
//   warps 8-23   converters: FP64 -> hi/lo TF32 (bit operations, not the FP64 pipe) in the
//                no-swizzle K-major core-matrix layout of the MMA, into a ring of (up to four)
//                operand buffers, deep enough to cover the MMA-to-commit round trip,
//   warp 25      MMA issuer (one thread): two k-steps of three kind::tf32 MMAs per box into
//                one of two tensor-memory accumulators,
//   warp 26      C producer: the tile's C (q/16 boxes) into one of one or two C/D slots,
//   warps 0-7    epilogue: tcgen05.ld of the accumulator (warp w reads lanes 32 (w % 4) .. +31,
//                thread = row, w / 4 picks alternate 16-column groups), D = beta C + alpha acc
//                in FP32 (C rounded to FP32 like the other inputs; FP64 arithmetic here would be
//                bound by GB300's narrow FP64 pipe), widened in place in the slot, then
//                cp.async.bulk.tensor stores of the D tile.
// Each ring and mbarrier has one waiting role that waits on every phase in turn (a parity
// wait cannot tell phase u from u - 2).  M (both TF32 parts) is staged once per CTA.  Every
// wait is bounded; on a timeout the CTA stops, waits (bounded) for its own copies and MMAs,
// writes NaN into its tiles of D (the solver's finiteness check reports it) and returns.
constexpr int kUpdMaxP = 192, kUpdMaxQ = 64;
constexpr int kUpdThreads = 864;       // 27 warps
constexpr int kUpdEpiThreads = 256;    // warps 0-7
constexpr int kUpdConvThreads = 512;   // warps 8-23
constexpr int kUpdOpBufs = 4;          // at most this many [hi, lo] operand buffers between converters and MMA
constexpr int kUpdBoxBytes = 16384;    // 128 rows x 16 FP64 columns, one ring slot
constexpr int kUpdKC = 16;             // K columns per ring slot
constexpr int kUpdOpBytes = 8192;      // one TF32 operand part of a slot: 128 rows x 16 K
constexpr int kUpdMaxStages = 8;
constexpr int kUpdSmemMax = 230400;    // dynamic shared memory asked for (227 KB less the static part)

struct UpdBars {
    uint64_t full[kUpdMaxStages], empty[kUpdMaxStages];
    uint64_t afull[kUpdOpBufs], aempty[kUpdOpBufs], accfull[2], accempty[2], cfull[2], cempty[2], done;
};

__device__ __forceinline__ void mbar_arrive1(uint64_t *m)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(m)) : "memory");
}

__device__ __forceinline__ void mbar_expect(uint64_t *m, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(m)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_box(uint32_t dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(saddr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_store_box(const CUtensorMap *map, int x, int y, uint32_t src)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     (uint64_t)map),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
}

// AND of v over the 256 epilogue threads (named barrier 1): their branches stay uniform, so
// the named barrier below never waits for a thread that has left
__device__ __forceinline__ bool epi_all(bool v)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\tbar.red.and.pred po, 1, 256, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

// FP64 <-> FP32 without the FP64 pipe (a few integer ops per element on GB300, where F2F
// runs on the narrow FP64 unit).
// x = hi + lo in TF32 parts for the MMA, from the FP64 bits: x32 = x with its mantissa cut to
// the top 23 bits (truncation: relative error below 2^-23), hi = x32 with its low 13 mantissa
// bits cleared (a TF32 value), lo = tf32(x32 - hi) (x32 - hi is exact).  Four elements at a
// time, branch-free on the common path; the rare operand outside the normal FP32 range goes
// through the conversion instruction after one warp vote.
__device__ __forceinline__ void split_tf32x4(const double (&x)[4], float (&h)[4], float (&l)[4])
{
    uint32_t u[4];
    bool odd = false;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const unsigned long long bits = (unsigned long long)__double_as_longlong(x[e]);
        const uint32_t hi = (uint32_t)(bits >> 32), lo = (uint32_t)bits;
        const uint32_t ex = (hi >> 20) & 0x7FFu;
        const bool normal = ex - 897u <= 253u;  // FP32-normal range
        u[e] = normal ? ((hi & 0x80000000u) | ((ex - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29))
                      : (hi & 0x80000000u);  // zero and FP64 subnormals: signed zero
        odd |= !normal && ex != 0u;
    }
    if (__any_sync(0xffffffffu, odd)) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const uint32_t ex = (uint32_t)((unsigned long long)__double_as_longlong(x[e]) >> 52) & 0x7FFu;
            if (ex - 897u > 253u && ex != 0u) u[e] = __float_as_uint((float)x[e]);
        }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        h[e] = __uint_as_float(u[e] & 0xFFFFE000u);
        l[e] = to_tf32(__uint_as_float(u[e]) - h[e]);
    }
}

// x cut to FP32 by its bits (top 23 mantissa bits); zero and FP64 subnormals give a signed
// zero, values outside the normal FP32 range take the conversion instruction
__device__ __forceinline__ float narrow_f32(double x)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(bits >> 32), lo = (uint32_t)bits;
    const uint32_t ex = (hi >> 20) & 0x7FFu;
    if (ex - 897u <= 253u)
        return __uint_as_float((hi & 0x80000000u) | ((ex - 896u) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
    if (ex == 0u) return __uint_as_float(hi & 0x80000000u);
    return (float)x;
}

// widening is exact: the FP32 fields moved into FP64 position
__device__ __forceinline__ double f32_to_f64_fast(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t ex = (u >> 23) & 0xFFu;
    if (ex - 1u <= 253u)
        return __hiloint2double((int)((u & 0x80000000u) | ((ex + 896u) << 20) | ((u & 0x7FFFFFu) >> 3)),
                                (int)(u << 29));
    if ((u & 0x7FFFFFFFu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
    return (double)f;
}

// byte offset of the 16-byte unit `unit` (FP64 columns 2 unit, 2 unit + 1) of row r inside
// one 128-byte-swizzled box
__device__ __forceinline__ uint32_t swz_off(int r, int unit) { return (uint32_t)(r * 128 + ((unit ^ (r & 7)) << 4)); }

// operand part of one 16-wide K slot: 8-row x 16-byte core matrices, 128 B apart along K and
// 512 B apart along the rows
__device__ __forceinline__ uint32_t tile16_offset(int r, int kq) { return (uint32_t)((r >> 3) * 512 + kq * 128 + (r & 7) * 16); }

__device__ __forceinline__ uint64_t smem_desc_sbo(uint32_t addr, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((128u >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// 16 accumulator columns of this thread's TMEM lane; the wait names the registers so no use
// of them is scheduled before the load has landed
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                   "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]),
                   "+r"(v[15])
                 :
                 : "memory");
}

// 8 accumulator columns, as tmem_ld16
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7])
                 :
                 : "memory");
}

__global__ void __launch_bounds__(kUpdThreads, 1)
    k_update_tma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmC,
                 const __grid_constant__ CUtensorMap tmD, const double *__restrict__ M, int64_t ldm, int p, int q,
                 int np, double *D, int64_t ldd, int64_t n, double alpha, double beta, int nstages, int ncs,
                 int nab, uint32_t acc_cols)
{
    extern __shared__ unsigned char upd_raw[];
    __shared__ __align__(8) UpdBars bars;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_err;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nck = (p + kUpdKC - 1) / kUpdKC;  // 16-wide K slots of A per tile
    const int nm = (p + kTcKC - 1) / kTcKC;     // 32-wide K chunks of the staged M
    const int ncb = (q + 15) / 16;              // 16-column boxes of C / D per tile
    const uint32_t b_bytes = tile_bytes(np);
    // 1024-byte aligned carve-up: A ring | ncs C/D slots | two [hi, lo] operand buffers | [hi, lo] x nm of M
    const uint32_t raw0 = saddr(upd_raw);
    const uint32_t pad = ((raw0 + 1023u) & ~1023u) - raw0;
    unsigned char *ring = upd_raw + pad;
    unsigned char *cslot = ring + (size_t)nstages * kUpdBoxBytes;
    unsigned char *abuf = cslot + (size_t)ncs * ncb * kUpdBoxBytes;
    unsigned char *mbuf = abuf + (size_t)2 * nab * kUpdOpBytes;
    const int64_t ntiles = (n + kTcM - 1) / kTcM;
    const int my_tiles = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    const bool use_c = beta != 0.0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < nstages; ++s) {
            mbar_init(&bars.full[s], 1);
            mbar_init(&bars.empty[s], kUpdConvThreads);
        }
        for (int b = 0; b < nab; ++b) {
            mbar_init(&bars.afull[b], kUpdConvThreads);
            mbar_init(&bars.aempty[b], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bars.accfull[b], 1);
            mbar_init(&bars.accempty[b], kUpdEpiThreads);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bars.cfull[b], 1);
            mbar_init(&bars.cempty[b], 1);
        }
        mbar_init(&bars.done, 1);
        s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 25) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&s_tmem)),
                     "r"(2 * acc_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // M^T as the B operand: row nn of the tile = column nn of M, K = rows of M (32 per chunk)
    for (int task = threadIdx.x; task < nm * np * (kTcKC / 4); task += kUpdThreads) {
        const int c = task / (np * (kTcKC / 4)), rem = task % (np * (kTcKC / 4));
        const int nn = rem % np, kq = rem / np;
        float h[4], l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int kk = c * kTcKC + 4 * kq + i;
            const float x = (kk < p && nn < q) ? (float)M[(int64_t)kk * ldm + nn] : 0.0f;
            h[i] = to_tf32(x);
            l[i] = to_tf32(x - h[i]);
        }
        const uint32_t off = tile_offset(nn, kq) / 4;
        *reinterpret_cast<float4 *>(reinterpret_cast<float *>(mbuf + (size_t)(2 * c) * b_bytes) + off) =
            make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4 *>(reinterpret_cast<float *>(mbuf + (size_t)(2 * c + 1) * b_bytes) + off) =
            make_float4(l[0], l[1], l[2], l[3]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const int total = my_tiles * nck;  // ring positions of this CTA: tile i, slot c -> i nck + c

    if (warp == 24) {
        // ---------------- A producer ----------------
        if (lane == 0) {
            int issued = 0;
            for (; issued < total && !s_err; ++issued) {
                const int s = issued % nstages, u = issued / nstages;
                if (u >= 1 && !mbar_wait(&bars.empty[s], (unsigned)((u - 1) & 1))) {
                    s_err = 1;
                    break;
                }
                const int i = issued / nck, c = issued % nck;
                const int y = (int)((blockIdx.x + (int64_t)i * gridDim.x) * kTcM);
                mbar_expect(&bars.full[s], (unsigned)kUpdBoxBytes);
                tma_load_box(saddr(ring + (size_t)s * kUpdBoxBytes), &tmA, c * kUpdKC, y, &bars.full[s]);
            }
            // no copy may still be landing in shared memory when the CTA ends
            for (int pos = issued > nstages ? issued - nstages : 0; pos < issued; ++pos)
                if (!mbar_wait(&bars.full[pos % nstages], (unsigned)((pos / nstages) & 1))) s_err = 1;
        }
        __syncwarp();
    } else if (warp == 26) {
        // ---------------- C producer: tile i's C into C/D slot i % ncs ----------------
        if (lane == 0) {
            int issued = 0;
            for (; issued < my_tiles && !s_err; ++issued) {
                const int cs = issued % ncs, uc = issued / ncs;
                if (uc >= 1 && !mbar_wait(&bars.cempty[cs], (unsigned)((uc - 1) & 1))) {
                    s_err = 1;
                    break;
                }
                if (!use_c) {
                    mbar_arrive1(&bars.cfull[cs]);
                    continue;
                }
                const int y = (int)((blockIdx.x + (int64_t)issued * gridDim.x) * kTcM);
                unsigned char *dst = cslot + (size_t)cs * ncb * kUpdBoxBytes;
                mbar_expect(&bars.cfull[cs], (unsigned)(ncb * kUpdBoxBytes));
                for (int bx = 0; bx < ncb; ++bx)
                    tma_load_box(saddr(dst + (size_t)bx * kUpdBoxBytes), &tmC, 16 * bx, y, &bars.cfull[cs]);
            }
            for (int t = issued > ncs ? issued - ncs : 0; t < issued; ++t)
                if (!mbar_wait(&bars.cfull[t % ncs], (unsigned)((t / ncs) & 1))) s_err = 1;
        }
        __syncwarp();
    } else if (warp == 25) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = instr_desc_tf32(np);
            for (int i = 0; i < my_tiles && !s_err; ++i) {
                const int a = i & 1, ua = i >> 1;
                if (ua >= 1 && !mbar_wait(&bars.accempty[a], (unsigned)((ua - 1) & 1))) {
                    s_err = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d_tmem = tmem + (uint32_t)a * acc_cols;
                bool bad = false;
                for (int c = 0; c < nck; ++c) {
                    const int g = i * nck + c, b = g % nab, ub = g / nab;
                    if (!mbar_wait(&bars.afull[b], (unsigned)(ub & 1))) {
                        bad = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a0 = saddr(abuf + (size_t)(2 * b) * kUpdOpBytes), a1 = a0 + kUpdOpBytes;
                    const uint32_t b0 = saddr(mbuf + (size_t)(2 * (c >> 1)) * b_bytes) + (uint32_t)(c & 1) * 512u;
                    const uint32_t b1 = b0 + b_bytes;
#pragma unroll
                    for (int s2 = 0; s2 < kUpdKC / 8; ++s2) {
                        const uint32_t ks = (uint32_t)s2 * 256u;
                        const uint64_t dA0 = smem_desc_sbo(a0 + ks, 512u), dA1 = smem_desc_sbo(a1 + ks, 512u);
                        const uint64_t dB0 = smem_desc_sbo(b0 + ks, 1024u), dB1 = smem_desc_sbo(b1 + ks, 1024u);
                        mma_tf32(d_tmem, dA0, dB0, idesc, (c > 0 || s2 > 0) ? 1 : 0);
                        mma_tf32(d_tmem, dA0, dB1, idesc, 1);
                        mma_tf32(d_tmem, dA1, dB0, idesc, 1);
                    }
                    mma_commit(&bars.aempty[b]);
                }
                if (bad) {
                    s_err = 1;
                    break;
                }
                mma_commit(&bars.accfull[a]);
            }
            // every MMA of this CTA has completed before the tensor memory is released
            mma_commit(&bars.done);
            if (!mbar_wait(&bars.done, 0u)) s_err = 1;
        }
        __syncwarp();
    } else if (warp >= 8) {
        // ---------------- converters: 512 threads, warp cw owns rows 8 cw .. 8 cw + 7 ----------------
        const int cw = warp - 8;
        const int kq = lane >> 3;  // 4-column quad of the 16-column slot
        for (int g = 0; g < total && !s_err; ++g) {
            const int s = g % nstages, u = g / nstages;
            const int b = g % nab, ub = g / nab;
            if (!mbar_wait(&bars.full[s], (unsigned)(u & 1)) ||
                (ub >= 1 && !mbar_wait(&bars.aempty[b], (unsigned)((ub - 1) & 1)))) {
                s_err = 1;
                break;
            }
            const unsigned char *slot = ring + (size_t)s * kUpdBoxBytes;
            float *ahi = reinterpret_cast<float *>(abuf + (size_t)(2 * b) * kUpdOpBytes);
            float *alo = reinterpret_cast<float *>(abuf + (size_t)(2 * b + 1) * kUpdOpBytes);
            {
                const int r = 8 * cw + (lane & 7);
                // columns past p and rows past n were zero-filled by the copy
                const double2 v0 = *reinterpret_cast<const double2 *>(slot + swz_off(r, 2 * kq));
                const double2 v1 = *reinterpret_cast<const double2 *>(slot + swz_off(r, 2 * kq + 1));
                const double x[4] = {v0.x, v0.y, v1.x, v1.y};
                float h[4], l[4];
                split_tf32x4(x, h, l);
                const uint32_t off = tile16_offset(r, kq) / 4;
                *reinterpret_cast<float4 *>(ahi + off) = make_float4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<float4 *>(alo + off) = make_float4(l[0], l[1], l[2], l[3]);
            }
            mbar_arrive1(&bars.empty[s]);  // this thread's reads of the slot are done
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive1(&bars.afull[b]);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: 256 threads, thread = row of the tile x column half ----------------
        const int quad = warp & 3, half = warp >> 2;
        const int r = 32 * quad + lane;
        const float alpha32 = (float)alpha, beta32 = (float)beta;
        for (int i = 0; i < my_tiles; ++i) {
            const int a = i & 1, ua = i >> 1;
            const int y = (int)((blockIdx.x + (int64_t)i * gridDim.x) * kTcM);
            const int cs = i % ncs, uc = i / ncs;
            unsigned char *tslot = cslot + (size_t)cs * ncb * kUpdBoxBytes;
            bool ok = !s_err && mbar_wait(&bars.accfull[a], (unsigned)(ua & 1));
            ok = ok && mbar_wait(&bars.cfull[cs], (unsigned)(uc & 1));
            __syncwarp();
            if (!epi_all(ok)) {
                s_err = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int g16 = half; g16 * 16 < np; g16 += 2) {
                uint32_t v[16];
                tmem_ld16(tmem + (uint32_t)a * acc_cols + ((uint32_t)(32 * quad) << 16) + (uint32_t)(16 * g16), v);
                unsigned char *bx = tslot + (size_t)g16 * kUpdBoxBytes;
#pragma unroll
                for (int uu = 0; uu < 8; ++uu) {
                    double2 *cell = reinterpret_cast<double2 *>(bx + swz_off(r, uu));
                    float d0 = alpha32 * __uint_as_float(v[2 * uu]), d1 = alpha32 * __uint_as_float(v[2 * uu + 1]);
                    if (use_c) {
                        const double2 cv = *cell;
                        d0 = fmaf(beta32, narrow_f32(cv.x), d0);
                        d1 = fmaf(beta32, narrow_f32(cv.y), d1);
                    }
                    *cell = make_double2(f32_to_f64_fast(d0), f32_to_f64_fast(d1));
                }
            }
            // the accumulator may be overwritten by the tile after next
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive1(&bars.accempty[a]);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("bar.sync 1, 256;" ::: "memory");
            if (threadIdx.x == 0) {
                for (int bxi = 0; bxi < ncb; ++bxi)
                    tma_store_box(&tmD, 16 * bxi, y, saddr(tslot + (size_t)bxi * kUpdBoxBytes));
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                // a slot is handed back once its store has read it: with two slots the previous
                // tile's store, with one this tile's
                if (ncs == 2) {
                    asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                    if (i >= 1) mbar_arrive1(&bars.cempty[(i - 1) % 2]);
                } else {
                    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                    mbar_arrive1(&bars.cempty[0]);
                }
            }
            __syncwarp();
        }
        if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        __syncwarp();
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (s_err) {
        for (int i = 0; i < my_tiles; ++i) {
            const int64_t r0 = (blockIdx.x + (int64_t)i * gridDim.x) * kTcM;
            for (int e = threadIdx.x; e < kTcM * q; e += kUpdThreads) {
                const int64_t row = r0 + e / q;
                if (row < n) D[row * ldd + e % q] = (double)NAN;
            }
        }
    }
    __syncwarp();
    if (warp == 25)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * acc_cols)
                     : "memory");
}

// ---------------------------------------------------------------------------------
// Gram C = A^T B (A: n x p, B: n x q, FP64 in memory; p, q <= 256) with FP32 accuracy on the
// tensor cores, fed by TMA: the same ring protocol, bit-level TF32 split and warp roles as
// the block update above, with the contraction now over the rows.  One persistent CTA per
// SM owns a slab of rows (a multiple of 16) and accumulates the p x q Gram of its slab in
// tensor memory (M = 128 columns of A per accumulator tile, N = q padded to 16); the slab
// partials are summed in a fixed order by the reduction kernel of mbl_dense.cu.  The tensor
// core rounds its FP32 accumulator once per MMA (toward zero, as measured: a 1,216-row slab of
// same-sign terms, the diagonal of S^T S, drifted by 2.5e-5), so
//   - the small products Ahi Blo + Alo Bhi go to an accumulator of their own, leaving one
//     rounding of the full-size accumulator per k-step,
//   - the accumulators are drained every 16 chunks (256 rows; 8 when the correction
//     accumulators do not fit in tensor memory) into the slab partial, kept as a float-float
//     pair (TwoSum, no FP64 pipe) and widened to FP64 at the end,
//   - two accumulator sets, where they fit, let the MMAs run on while one is drained.
//   warp 24      producer: per 16-row chunk, the 16-column boxes of A (and of B when B is
//                not A) into one ring slot,
//   warps 8-23   converters: each chunk transposed into K-major TF32 hi/lo operand tiles (the
//                K index is the row of A): lanes read 16 consecutive columns of one row of a
//                swizzled box, write 8 consecutive 16-byte core-matrix rows,
//   warp 25      MMA issuer: per chunk and accumulator tile, two k-steps of three MMAs,
//   warps 0-7    epilogue: per drain, tcgen05.ld of the accumulators (warp w: lanes
//                32 (w % 4) .. +31, alternate 16-column groups by w / 4) into the partial.
// When B is A (S^T S) the B operand is the A tile itself.
constexpr int kGrKC = 16;                          // rows (K) per chunk
constexpr int kGrBoxBytes = kGrKC * 16 * 8;        // 16 rows x 16 FP64 columns
constexpr int kGrThreads = 832;                    // 26 warps
constexpr int kGrConvThreads = 512;                // warps 8-23
constexpr int kGrEpiThreads = 256;                 // warps 0-7
constexpr int kGrMaxStages = 8;

struct GrBars {
    uint64_t full[kGrMaxStages], empty[kGrMaxStages], afull[2], aempty[2], accfull[2], accempty[2], done;
};

// (hi, lo) += v exactly up to the rounding of lo (Knuth's TwoSum on hi)
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float v)
{
    const float s = hi + v, bb = s - hi;
    const float e = (hi - (s - bb)) + (v - bb);
    hi = s;
    lo += e;
}

__global__ void __launch_bounds__(kGrThreads, 1)
    k_gram_tma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int p, int q,
               int same, int ma, int np, int64_t n, int64_t rows_per_slab, double *__restrict__ part, int nstages,
               int nacc, int split, int drain, uint32_t tmem_cols)
{
    extern __shared__ unsigned char gr_raw[];
    __shared__ __align__(8) GrBars bars;
    __shared__ uint32_t s_tmem;
    __shared__ volatile int s_err;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nba = (p + 15) / 16, nbb = same ? 0 : (q + 15) / 16;  // boxes per chunk
    const int nrows_b = same ? 0 : np;                             // rows of a separate B tile
    const uint32_t slot_bytes = (uint32_t)(nba + nbb) * kGrBoxBytes;
    const uint32_t buf_bytes = (uint32_t)(ma + nrows_b) * kGrKC * 4u * 2u;  // [A hi, A lo, B hi, B lo]
    const uint32_t raw0 = saddr(gr_raw);
    const uint32_t pad = ((raw0 + 1023u) & ~1023u) - raw0;
    unsigned char *ring = gr_raw + pad;
    unsigned char *obuf = ring + (size_t)nstages * slot_bytes;
    const int mtiles = ma / kTcM;
    const int64_t r_begin = (int64_t)blockIdx.x * rows_per_slab;
    const int64_t r_end = min(n, r_begin + rows_per_slab);
    const int total = r_end > r_begin ? (int)((r_end - r_begin + kGrKC - 1) / kGrKC) : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < nstages; ++s) {
            mbar_init(&bars.full[s], 1);
            mbar_init(&bars.empty[s], kGrConvThreads);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bars.afull[b], kGrConvThreads);
            mbar_init(&bars.aempty[b], 1);
            mbar_init(&bars.accfull[b], 1);
            mbar_init(&bars.accempty[b], kGrEpiThreads);
        }
        mbar_init(&bars.done, 1);
        s_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const int nper = (total + drain - 1) / drain;  // accumulator periods
    const int nsub = split ? 2 : 1;                 // accumulators per tile: full-size [, correction]
    if (warp == 25) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&s_tmem)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    if (warp == 24) {
        // ---------------- producer ----------------
        if (lane == 0) {
            int issued = 0;
            for (; issued < total && !s_err; ++issued) {
                const int s = issued % nstages, u = issued / nstages;
                if (u >= 1 && !mbar_wait(&bars.empty[s], (unsigned)((u - 1) & 1))) {
                    s_err = 1;
                    break;
                }
                const int y = (int)(r_begin + (int64_t)issued * kGrKC);
                const uint32_t dst = saddr(ring + (size_t)s * slot_bytes);
                mbar_expect(&bars.full[s], slot_bytes);
                for (int b = 0; b < nba; ++b) tma_load_box(dst + b * kGrBoxBytes, &tmA, 16 * b, y, &bars.full[s]);
                for (int b = 0; b < nbb; ++b)
                    tma_load_box(dst + (nba + b) * kGrBoxBytes, &tmB, 16 * b, y, &bars.full[s]);
            }
            for (int pos = issued > nstages ? issued - nstages : 0; pos < issued; ++pos)
                if (!mbar_wait(&bars.full[pos % nstages], (unsigned)((pos / nstages) & 1))) s_err = 1;
        }
        __syncwarp();
    } else if (warp == 25) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = instr_desc_tf32(np);
            for (int g = 0; g < total && !s_err; ++g) {
                const int b = g & 1, ub = g >> 1;
                const int per = g / drain, a = per % nacc, ua = per / nacc;
                const bool first = g % drain == 0;
                if (first && ua >= 1 && !mbar_wait(&bars.accempty[a], (unsigned)((ua - 1) & 1))) {
                    s_err = 1;
                    break;
                }
                if (!mbar_wait(&bars.afull[b], (unsigned)(ub & 1))) {
                    s_err = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t base = saddr(obuf + (size_t)b * buf_bytes);
                const uint32_t a_hi = base, a_lo = base + (uint32_t)ma * kGrKC * 4u;
                const uint32_t b_hi = same ? a_hi : base + (uint32_t)ma * kGrKC * 8u;
                const uint32_t b_lo = same ? a_lo : b_hi + (uint32_t)nrows_b * kGrKC * 4u;
                for (int m = 0; m < mtiles; ++m) {
                    const uint32_t d_tmem = tmem + (uint32_t)(((a * mtiles + m) * nsub) * np);
                    const uint32_t c_tmem = d_tmem + (uint32_t)((nsub - 1) * np);  // = d_tmem without split
                    const uint32_t mo = (uint32_t)m * (kTcM / 8) * 512u;  // 128 rows of the A tile
#pragma unroll
                    for (int s2 = 0; s2 < kGrKC / 8; ++s2) {
                        const uint32_t ks = (uint32_t)s2 * 256u;
                        const uint64_t dA0 = smem_desc_sbo(a_hi + mo + ks, 512u), dA1 = smem_desc_sbo(a_lo + mo + ks, 512u);
                        const uint64_t dB0 = smem_desc_sbo(b_hi + ks, 512u), dB1 = smem_desc_sbo(b_lo + ks, 512u);
                        mma_tf32(d_tmem, dA0, dB0, idesc, (!first || s2 > 0) ? 1 : 0);
                        mma_tf32(c_tmem, dA0, dB1, idesc, (!first || s2 > 0 || !split) ? 1 : 0);
                        mma_tf32(c_tmem, dA1, dB0, idesc, 1);
                    }
                }
                mma_commit(&bars.aempty[b]);
                if (g % drain == drain - 1 || g == total - 1) mma_commit(&bars.accfull[a]);
            }
            mma_commit(&bars.done);
            if (!mbar_wait(&bars.done, 0u)) s_err = 1;
        }
        __syncwarp();
    } else if (warp >= 8) {
        // ---------------- converters: chunk -> K-major TF32 tiles (K = row of A / B) ----------------
        const int cw = warp - 8;
        const int wa = (ma / 16) * 2, wb = (nrows_b / 16) * 2;  // warp items: 16 columns x 2 K-quads
        const int col16 = lane & 15, kqo = lane >> 4;
        for (int g = 0; g < total && !s_err; ++g) {
            const int s = g % nstages, u = g / nstages, b = g & 1, ub = g >> 1;
            if (!mbar_wait(&bars.full[s], (unsigned)(u & 1)) ||
                (ub >= 1 && !mbar_wait(&bars.aempty[b], (unsigned)((ub - 1) & 1)))) {
                s_err = 1;
                break;
            }
            const unsigned char *slot = ring + (size_t)s * slot_bytes;
            unsigned char *base = obuf + (size_t)b * buf_bytes;
            for (int wi = cw; wi < wa + wb; wi += 16) {
                const bool is_a = wi < wa;
                const int wl = is_a ? wi : wi - wa;
                const int c = 16 * (wl >> 1) + col16;           // column of A (or B) = tile row
                const int kq = 2 * (wl & 1) + kqo;              // rows 4 kq .. 4 kq + 3 of the chunk
                const int nb = is_a ? nba : (q + 15) / 16;
                const unsigned char *box = slot + (size_t)((is_a ? 0 : nba) + c / 16) * kGrBoxBytes;
                double x[4] = {0.0, 0.0, 0.0, 0.0};
                if (c < 16 * nb) {  // columns past p (q) inside the last box were zero-filled
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int r = 4 * kq + i;
                        x[i] = *reinterpret_cast<const double *>(box + swz_off(r, col16 >> 1) + (col16 & 1) * 8);
                    }
                }
                float h[4], l[4];
                split_tf32x4(x, h, l);
                const int rows = is_a ? ma : nrows_b;
                float *hi = reinterpret_cast<float *>(base + (is_a ? 0 : (size_t)ma * kGrKC * 8));
                float *lo = hi + rows * kGrKC;
                const uint32_t off = tile16_offset(c, kq) / 4;
                *reinterpret_cast<float4 *>(hi + off) = make_float4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<float4 *>(lo + off) = make_float4(l[0], l[1], l[2], l[3]);
            }
            mbar_arrive1(&bars.empty[s]);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive1(&bars.afull[b]);
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: drain each accumulator period into the partial ----------------
        const int quad = warp & 3, half = warp >> 2;
        // the slab partial is column-major (element (i, j) at j p + i): a warp's 32 rows of one
        // column are 32 consecutive elements; (hi, lo) pairs live in its own storage until the end
        double *out = part + (int64_t)blockIdx.x * p * q;
        float2 *acc2 = reinterpret_cast<float2 *>(out);
        bool ok = !s_err;
        for (int per = 0; per < nper; ++per) {
            const int a = per % nacc, ua = per / nacc;
            ok = ok && !s_err && mbar_wait(&bars.accfull[a], (unsigned)(ua & 1));
            __syncwarp();
            if (!__all_sync(0xffffffffu, ok)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            for (int m = 0; m < mtiles; ++m) {
                const int row = m * kTcM + 32 * quad + lane;
                for (int g8 = half; g8 * 8 < np; g8 += 2) {
                    const uint32_t t0 = tmem + (uint32_t)(((a * mtiles + m) * nsub) * np + 8 * g8) +
                                        ((uint32_t)(32 * quad) << 16);
                    // the partial's 8 (hi, lo) pairs first, so their loads fly during the TMEM reads
                    float2 c2[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int col = 8 * g8 + e;
                        c2[e] = make_float2(0.0f, 0.0f);
                        if (per > 0 && row < p && col < q) c2[e] = acc2[(int64_t)col * p + row];
                    }
                    uint32_t v[8], w[8];
                    __syncwarp();
                    tmem_ld8(t0, v);
                    if (split) {
                        tmem_ld8(t0 + (uint32_t)np, w);
                    } else {
#pragma unroll
                        for (int e = 0; e < 8; ++e) w[e] = 0u;
                    }
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int col = 8 * g8 + e;
                        two_sum_acc(c2[e].x, c2[e].y, __uint_as_float(v[e]));
                        two_sum_acc(c2[e].x, c2[e].y, __uint_as_float(w[e]));
                        if (row < p && col < q) acc2[(int64_t)col * p + row] = c2[e];
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive1(&bars.accempty[a]);
        }
        // widen the pairs in place: each thread the elements it drained (its row, its 8-column groups)
        for (int m = 0; m < mtiles && ok; ++m) {
            const int row = m * kTcM + 32 * quad + lane;
            if (row < p)
                for (int col = 8 * half; col < q; col += (col % 8 == 7) ? 9 : 1) {
                    const int64_t e = (int64_t)col * p + row;
                    const float2 c2 = nper > 0 ? acc2[e] : make_float2(0.0f, 0.0f);
                    out[e] = f32_to_f64_fast(c2.x) + f32_to_f64_fast(c2.y);
                }
        }
        if (!ok) s_err = 1;
        __syncwarp();
    }

    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (s_err) {  // the reduction's finiteness reports it
        double *out = part + (int64_t)blockIdx.x * p * q;
        for (int e = threadIdx.x; e < p * q; e += kGrThreads) out[e] = (double)NAN;
    }
    __syncwarp();
    if (warp == 25)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// ---------------------------------------------------------------------------------
// Host side of the tensor maps: the driver's encoder, looked up once through the runtime.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn tensor_map_encoder()
{
    static EncodeTiledFn fn = []() -> EncodeTiledFn {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &qr) !=
                cudaSuccess ||
            qr != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// An FP64 row-major matrix (rows x cols, leading dimension ld) as a 2-D tensor map with
// 16-column x box_rows-row boxes and 128-byte swizzle.
bool fp64_box_map(CUtensorMap *m, const double *base, int64_t rows, int cols, int64_t ld, int box_rows = kTcM)
{
    const EncodeTiledFn enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(double)};
    const cuuint32_t box[2] = {16, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double *>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool tma_addressable(const double *base, int64_t ld) { return base && ((uintptr_t)base & 15u) == 0 && (ld & 1) == 0; }

// shared memory of everything but the A ring, with ncs C/D slots and nab operand buffers
size_t update_fixed_smem(int p, int q, int ncs, int nab)
{
    const int np = (q + 15) / 16 * 16, nm = (p + kTcKC - 1) / kTcKC;
    return 1024 + (size_t)ncs * ((q + 15) / 16) * kUpdBoxBytes + (size_t)2 * nab * kUpdOpBytes +
           (size_t)2 * nm * tile_bytes(np);
}

struct UpdConfig {
    int ncs, nab, ns;  // C/D slots, operand buffers, A ring slots (0: does not fit)
};

// the deepest buffering that fits: two C/D slots and four operand buffers with an A ring of
// at least four slots, else one C/D slot, else two operand buffers (an A ring of two slots
// already keeps the loads ahead; the operand buffers cover the MMA round trip)
UpdConfig update_config(int p, int q)
{
    const int cfg[3][3] = {{2, 4, 4}, {1, 4, 2}, {1, 2, 2}};
    for (const auto &c : cfg) {
        const size_t fixed = update_fixed_smem(p, q, c[0], c[1]);
        if (fixed >= (size_t)kUpdSmemMax) continue;
        int ns = (int)(((size_t)kUpdSmemMax - fixed) / kUpdBoxBytes);
        if (ns > kUpdMaxStages) ns = kUpdMaxStages;
        if (ns >= c[2]) return UpdConfig{c[0], c[1], ns};
    }
    return UpdConfig{1, 2, 0};
}

}  // namespace

bool gram_tc_supported(int p, int q) { return p >= 1 && q >= 1 && p <= 256 && q <= 256; }

namespace {

// A ring of at least two chunks next to two operand buffers; 0 if it does not fit
int gram_stages(int p, int q, bool same)
{
    const int ma = (p + kTcM - 1) / kTcM * kTcM, np = (q + 15) / 16 * 16;
    const size_t slot = (size_t)((p + 15) / 16 + (same ? 0 : (q + 15) / 16)) * kGrBoxBytes;
    const size_t fixed = 1024 + (size_t)2 * (ma + (same ? 0 : np)) * kGrKC * 4 * 2;
    if (fixed >= (size_t)kUpdSmemMax) return 0;
    const int ns = (int)(((size_t)kUpdSmemMax - fixed) / slot);
    return ns > kGrMaxStages ? kGrMaxStages : ns;
}

bool gram_same(const double *A, int64_t lda, int p, const double *B, int64_t ldb, int q)
{
    return A == B && lda == ldb && p == q;
}

}  // namespace

bool gram_tc_eligible(const double *A, int64_t lda, int p, const double *B, int64_t ldb, int q)
{
    if (!gram_tc_supported(p, q) || !tensor_map_encoder()) return false;
    if (!tma_addressable(A, lda) || !tma_addressable(B, ldb)) return false;
    return gram_stages(p, q, gram_same(A, lda, p, B, ldb, q)) >= 2;
}

int gram_tc_slabs(int64_t n, int p)
{
    (void)p;
    int64_t want = num_sms();
    const int64_t by_rows = (n + 8 * kGrKC - 1) / (8 * kGrKC);  // at least 128 rows per slab
    if (want > by_rows) want = by_rows;
    return want < 1 ? 1 : (int)want;
}

int gram_tc_partial(const double *A, int64_t lda, int p, const double *B, int64_t ldb, int q, int64_t n, int nslab,
                    double *part, cudaStream_t st)
{
    if (!gram_tc_eligible(A, lda, p, B, ldb, q) || n > ((int64_t)1 << 31) || nslab < 1) return MBL_ERR_ARG;
    const bool same = gram_same(A, lda, p, B, ldb, q);
    CUtensorMap ta, tb;
    if (!fp64_box_map(&ta, A, n > 0 ? n : 1, p, lda, kGrKC) || !fp64_box_map(&tb, B, n > 0 ? n : 1, q, ldb, kGrKC))
        return MBL_ERR_ARG;
    const int ma = (p + kTcM - 1) / kTcM * kTcM, np = (q + 15) / 16 * 16;
    // accumulator layout: with a correction accumulator per tile when it fits, two sets when
    // those fit too
    const int tile_cols = (ma / kTcM) * np;
    int split = 1, nacc = 2, drain = 16;
    if (4 * tile_cols > 512) nacc = 1;
    if (2 * tile_cols > 512) {
        split = 0;
        nacc = 2 * tile_cols <= 512 ? 2 : 1;
        drain = 8;
    }
    const int cols = nacc * (split ? 2 : 1) * tile_cols;
    const uint32_t tmem_cols = cols <= 32 ? 32u : (cols <= 64 ? 64u : (cols <= 128 ? 128u : (cols <= 256 ? 256u : 512u)));
    const int ns = gram_stages(p, q, same);
    const size_t slot = (size_t)((p + 15) / 16 + (same ? 0 : (q + 15) / 16)) * kGrBoxBytes;
    const size_t smem = 1024 + (size_t)2 * (ma + (same ? 0 : np)) * kGrKC * 4 * 2 + (size_t)ns * slot;
    static const bool attr = []() {
        cudaFuncSetAttribute(k_gram_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, kUpdSmemMax);
        return true;
    }();
    (void)attr;
    const int64_t rps = ((n + nslab - 1) / nslab + kGrKC - 1) / kGrKC * kGrKC;
    note_launch();
    k_gram_tma<<<nslab, kGrThreads, smem, st>>>(ta, tb, p, q, same ? 1 : 0, ma, np, n, rps, part, ns, nacc, split,
                                                 drain, tmem_cols);
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

bool update_tc_supported(const double *A, int64_t lda, int p, int q, const double *C, int64_t ldc, const double *D,
                         int64_t ldd, double beta)
{
    if (p < 1 || q < 1 || p > kUpdMaxP || q > kUpdMaxQ || update_config(p, q).ns < 2) return false;
    if (!tensor_map_encoder()) return false;
    return tma_addressable(A, lda) && tma_addressable(D, ldd) && (beta == 0.0 || tma_addressable(C, ldc));
}

int update_tc(const double *A, int64_t lda, int p, const double *M, int64_t ldm, int q, const double *C, int64_t ldc,
              double *D, int64_t ldd, int64_t n, double alpha, double beta, cudaStream_t st)
{
    if (!update_tc_supported(A, lda, p, q, C, ldc, D, ldd, beta) || n > ((int64_t)1 << 31)) return MBL_ERR_ARG;
    if (n <= 0) return MBL_OK;
    const bool use_c = beta != 0.0;
    CUtensorMap ta, tc, td;
    if (!fp64_box_map(&ta, A, n, p, lda) || !fp64_box_map(&td, D, n, q, ldd) ||
        !fp64_box_map(&tc, use_c ? C : D, n, q, use_c ? ldc : ldd))
        return MBL_ERR_ARG;
    const int np = (q + 15) / 16 * 16;
    const uint32_t acc_cols = np <= 32 ? 32u : 64u;
    const UpdConfig cfg = update_config(p, q);
    const size_t smem = update_fixed_smem(p, q, cfg.ncs, cfg.nab) + (size_t)cfg.ns * kUpdBoxBytes;
    static const bool attr = []() {
        cudaFuncSetAttribute(k_update_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, kUpdSmemMax);
        return true;
    }();
    (void)attr;
    const int64_t ntiles = (n + kTcM - 1) / kTcM;
    int grid = num_sms();
    if (grid > ntiles) grid = (int)ntiles;
    note_launch();
    k_update_tma<<<grid, kUpdThreads, smem, st>>>(ta, tc, td, M, ldm, p, q, np, D, ldd, n, alpha, beta, cfg.ns,
                                                   cfg.ncs, cfg.nab, acc_cols);
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

}  // namespace mbl
