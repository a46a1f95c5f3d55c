// mbl_apply.cu -- the block product Y = (H - sigma I) X on one S^z sector (Sec. 4.1,
// the MATVEC that dominates the solver's cost, Sec. 3.2) and the Jacobi-PCG kernels
// built around it (Sec. 3.2 preconditioner; Sec. 6.2 runs it in single precision).
//
// Gather (pull) form: each output row is produced by one group of lanes that reads
// its own row of X and the rows of its flip-flop neighbours, so no atomics are
// needed and results are bitwise reproducible.  Index arithmetic uses the
// combinatorial number system: exchanging the spins of open bond (i, i+1) moves the
// rank by +C(i, c) (up spin moves right) or -C(i, c) (moves left), c = number of up
// spins below site i; the wrap bond of a periodic chain is re-ranked.
//
// Work split inside a warp (k wide enough for several lanes per row): every lane
// first ranks one of 32 consecutive rows (state, diagonal, neighbour list into
// shared memory); then groups of G lanes stream the rows, each lane moving 16 bytes
// of every neighbour row.  For k * sizeof(T) <= 16 one lane owns a whole row.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <atomic>
#include <mutex>
#include <vector>

#include "mbl_device.cuh"
#include "mbl_internal.h"

namespace mbl {

template <typename T, int V>
struct alignas(sizeof(T) * V) Vec {
    T v[V];
};

template <typename T, int K>
struct RowLayout {
    static constexpr int kBytes = K * (int)sizeof(T);
    static constexpr int V = kBytes >= 16 ? 16 / (int)sizeof(T) : K;  // elements per lane
    static constexpr int G = K / V;                                    // lanes per row
    static_assert(G >= 1 && G <= 32 && (G & (G - 1)) == 0, "unsupported row width");
};

// Tiled kernels move up to LB bytes per lane (LB = 16 or 32) of every neighbour row.
#ifndef MBL_CH_PASSES
#define MBL_CH_PASSES 4
#endif
#ifndef MBL_CH_MIN
#define MBL_CH_MIN 32
#endif

template <typename T, int K, int LB = 32>
struct WideRowLayout {
    static constexpr int kBytes = K * (int)sizeof(T);
    static constexpr int V = kBytes >= LB ? LB / (int)sizeof(T) : K;
    static constexpr int G = K / V;
    static_assert(G >= 1 && G <= 32 && (G & (G - 1)) == 0, "unsupported row width");
    // rows per work item of the tiled product: at least MBL_CH_PASSES row-passes of the
    // warp (32 / G rows each) and at least MBL_CH_MIN rows, so the per-tile setup of an
    // item (tile offset, high-bond shifts) is spread over enough rows
    static constexpr int CH = (MBL_CH_PASSES * (32 / G) > MBL_CH_MIN) ? MBL_CH_PASSES * (32 / G) : MBL_CH_MIN;
};

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxNb = 32;  // at most |B| <= 32 neighbours per row

// What the product kernel does with each finished output row.
enum ApplyMode {
    kPlain = 0,    // Y = (H - sigma) X
    kPcgT = 1,     // t = (H - sigma) p; accumulate t.t per column; finish alpha = rz / t.t
    kPcgQ = 2,     // q = (H - sigma) t; r -= alpha q; accumulate r.(dinv r); finish beta
};

// Per-column PCG scalars (FP64), laid out as arrays of kMaxK.
struct PcgScalars {
    double *rz, *rz0, *alpha, *beta;
    int *active;
    double tol2;  // pcg_tol^2 (0: never freeze)
    // when set (tiled kernels), the q-launch also does w += alpha p for its rows
    void *w = nullptr;
    const void *p = nullptr;
};

struct Reduce {
    double *partials;   // [gridDim.x][k]
    unsigned *counter;  // zero on entry; the last block resets it
};

// ---------------------------------------------------------------------------------
// Per-row index work: state, shifted diagonal and neighbour ranks.
template <typename T>
__device__ __forceinline__ int row_neighbours(const uint32_t *sb, const ChainParams &cp, uint32_t r,
                                              uint32_t s, uint32_t *nb)
{
    int f = 0;
    uint32_t fm = (s ^ (s >> 1)) & cp.open_mask;
    while (fm) {
        int i = __ffs(fm) - 1;
        fm &= fm - 1;
        int c = __popc(s & ((1u << i) - 1u));
        uint32_t d = binom(sb, i, c);
        nb[f++] = ((s >> i) & 1u) ? r + d : r - d;
    }
    if (cp.periodic && (((s >> (cp.L - 1)) ^ s) & 1u)) {
        nb[f++] = cns_rank(sb, s ^ (1u | (1u << (cp.L - 1))));
    }
    return f;
}

template <typename T, int V>
__device__ __forceinline__ Vec<T, V> ldv(const T *p)
{
    return *reinterpret_cast<const Vec<T, V> *>(p);
}

template <typename T, int V>
__device__ __forceinline__ void stv(T *p, const Vec<T, V> &x)
{
    *reinterpret_cast<Vec<T, V> *>(p) = x;
}

// Store with the evict-first hint: a product's output is not read again by the same
// launch, so it should not push the input's rows out of L2.
template <typename T, int V>
__device__ __forceinline__ void stv_stream(T *p, const Vec<T, V> &x)
{
    if constexpr ((V * sizeof(T)) % 16 == 0) {
        const float4 *src = reinterpret_cast<const float4 *>(&x);
        float4 *dst = reinterpret_cast<float4 *>(p);
#pragma unroll
        for (int i = 0; i < (int)(V * sizeof(T) / 16); ++i) __stcs(dst + i, src[i]);
    } else {
        stv<T, V>(p, x);
    }
}

// Products that must not be fused with a neighbouring add: the tiled kernels round
// d * x and delta/2 * count on their own, so every variant adds the same rounded terms
// in the same order and their results agree bit for bit.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// Gather the neighbour rows listed in nbl[0..f) into acc: chunks of 8 independent
// 16-byte loads are issued before any of them is consumed.
template <typename T, int V>
__device__ __forceinline__ void gather_add(T (&acc)[V], const T *__restrict__ X, int64_t ldx, int col, int f,
                                           const uint32_t *nbl)
{
    const T half = (T)0.5;
    for (int u = 0; u < f; u += 8) {
        Vec<T, V> a[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
#pragma unroll
            for (int v = 0; v < V; ++v) a[j].v[v] = (T)0;
            if (u + j < f) a[j] = ldv<T, V>(X + (int64_t)nbl[u + j] * ldx + col);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] += half * a[j].v[v];
    }
}

// Two rows at once (16 loads in flight per lane).
template <typename T, int V>
__device__ __forceinline__ void gather_add2(T (&acc0)[V], T (&acc1)[V], const T *__restrict__ X, int64_t ldx, int col,
                                            int f0, const uint32_t *nb0, int f1, const uint32_t *nb1)
{
    const T half = (T)0.5;
    const int fm = f0 > f1 ? f0 : f1;
    for (int u = 0; u < fm; u += 8) {
        Vec<T, V> a[8], b[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                a[j].v[v] = (T)0;
                b[j].v[v] = (T)0;
            }
            if (u + j < f0) a[j] = ldv<T, V>(X + (int64_t)nb0[u + j] * ldx + col);
            if (u + j < f1) b[j] = ldv<T, V>(X + (int64_t)nb1[u + j] * ldx + col);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int v = 0; v < V; ++v) {
                acc0[v] += half * a[j].v[v];
                acc1[v] += half * b[j].v[v];
            }
    }
}

// Epilogue of one output row: store (and accumulate t.t), or fold into the PCG
// residual update r -= alpha q (and accumulate r.(M^-1 r)).
template <typename T, int V, int MODE>
__device__ __forceinline__ void finish_row(const T (&acc)[V], int f, uint32_t r, T *__restrict__ Y, int64_t ldy,
                                           T *__restrict__ R, const T *__restrict__ dinv, int col, const T (&alpha)[V],
                                           T (&part)[V], T *__restrict__ Wf = nullptr,
                                           const T *__restrict__ Pf = nullptr)
{
    if (f < 0) return;
    if (MODE == 0 || MODE == 1) {
        Vec<T, V> y;
#pragma unroll
        for (int v = 0; v < V; ++v) y.v[v] = acc[v];
        if (MODE == 0)
            stv_stream<T, V>(Y + (int64_t)r * ldy + col, y);
        else
            stv<T, V>(Y + (int64_t)r * ldy + col, y);
        if (MODE == 1) {
#pragma unroll
            for (int v = 0; v < V; ++v) part[v] += acc[v] * acc[v];
        }
    } else {
        Vec<T, V> rr = ldv<T, V>(R + (int64_t)r * ldy + col);
        const T di = dinv[r];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            rr.v[v] -= alpha[v] * acc[v];
            part[v] += rr.v[v] * (di * rr.v[v]);
        }
        stv<T, V>(R + (int64_t)r * ldy + col, rr);
        if (Wf) {  // the solution update of the same PCG step, row by row
            Vec<T, V> wv = ldv<T, V>(Wf + (int64_t)r * ldy + col);
            const Vec<T, V> pv = ldv<T, V>(Pf + (int64_t)r * ldy + col);
#pragma unroll
            for (int v = 0; v < V; ++v) wv.v[v] += alpha[v] * pv.v[v];
            stv<T, V>(Wf + (int64_t)r * ldy + col, wv);
        }
    }
}

// Shared-memory scratch of one product block.
template <typename T>
struct ApplySmem {
    uint32_t binom[kBinomDim * kBinomDim];
    T tab[1024];
    uint32_t nb[kWarps][32][kMaxNb + 1];  // neighbour lists, stride 33 words
    T dsig[kWarps][32];
    int cnt[kWarps][32];
    T red[kWarps][64];
};

// Reduce per-lane column partials (lanes with equal lane % G share columns) over the
// block, write this block's k partials, and let the last block finish.  Returns true
// in the last block (after a __syncthreads, with the block's partial visible).
template <typename T, int V, int G, int NT = kThreads>
__device__ __forceinline__ bool block_column_reduce(T (*red)[64], T (&part)[V], int k, const Reduce &rd)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < V; ++v)
        for (int off = G; off < 32; off <<= 1) part[v] += __shfl_xor_sync(0xffffffffu, part[v], off);
    if (lane < G) {
#pragma unroll
        for (int v = 0; v < V; ++v) red[warp][lane * V + v] = part[v];
    }
    __syncthreads();
    if (threadIdx.x < k) {
        double acc = 0.0;
        for (int w = 0; w < NT / 32; ++w) acc += (double)red[w][threadIdx.x];
        rd.partials[(int64_t)blockIdx.x * k + threadIdx.x] = acc;
    }
    __threadfence();
    __shared__ unsigned s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned ticket = atomicAdd(rd.counter, 1u);
        s_last = (ticket == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    return true;
}

// In the last block: total[c] = sum over blocks (fixed order) of partials, using
// kThreads / k threads per column and a fixed-shape tree.
template <int NT = kThreads>
__device__ __forceinline__ void finish_column_sums(const Reduce &rd, int k, double *total)
{
    __shared__ double s_tree[NT];
    const int per = NT / k;  // threads per column (k divides 256 or per >= 1)
    const int c = threadIdx.x / per, j = threadIdx.x % per;
    double acc = 0.0;
    if (c < k) {
        // blocks j, j + per, ... in that order, eight requested at a time
        constexpr int kBatch = 8;
        for (int b0 = j; b0 < (int)gridDim.x; b0 += kBatch * per) {
            double q[kBatch];
#pragma unroll
            for (int i = 0; i < kBatch; ++i) {
                const int b = b0 + i * per;
                q[i] = b < (int)gridDim.x ? rd.partials[(int64_t)b * k + c] : 0.0;
            }
#pragma unroll
            for (int i = 0; i < kBatch; ++i) {
                if (b0 + i * per >= (int)gridDim.x) break;
                acc += q[i];
            }
        }
    }
    s_tree[threadIdx.x] = acc;
    __syncthreads();
    if (c < k && j == 0) {
        double t = 0.0;
        for (int q = 0; q < per; ++q) t += s_tree[threadIdx.x + q];
        total[c] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) *rd.counter = 0u;
}

// PCG epilogue of a product launch: block partials of t.t (kPcgT) or r.(M^-1 r)
// (kPcgQ), then in the last block alpha = rz / t.t, or beta = rz_new / rz with the
// freeze rule (a column stops once rz_new <= tol^2 rz0, or on NaN/Inf).
// FP32 variant of the two reductions, for the FP32 kernels: block partials and the
// last block's sum over blocks are compensated FP32 pairs (s + c, TwoSum), stored as
// float2 in the partial slots, and only the k final totals are widened to FP64.  The
// FP64 pipe (about 1/64 of the FP32 rate) would otherwise set a serial tail of
// several microseconds per launch in the last block.
template <int V, int G, int NT = kThreads>
__device__ __forceinline__ bool block_column_reduce_f32(float (*red)[64], float (&part)[V], int k, const Reduce &rd)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < V; ++v)
        for (int off = G; off < 32; off <<= 1) part[v] += __shfl_xor_sync(0xffffffffu, part[v], off);
    if (lane < G) {
#pragma unroll
        for (int v = 0; v < V; ++v) red[warp][lane * V + v] = part[v];
    }
    __syncthreads();
    if (threadIdx.x < k) {
        float sum = 0.0f, cmp = 0.0f;
        for (int w = 0; w < NT / 32; ++w) {
            float hi, e;
            two_sum(sum, red[w][threadIdx.x], hi, e);
            sum = hi;
            cmp += e;
        }
        reinterpret_cast<float2 *>(rd.partials)[(int64_t)blockIdx.x * k + threadIdx.x] = make_float2(sum, cmp);
    }
    __threadfence();
    __shared__ unsigned s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned ticket = atomicAdd(rd.counter, 1u);
        s_last = (ticket == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    return true;
}

template <int NT = kThreads>
__device__ __forceinline__ void finish_column_sums_f32(const Reduce &rd, int k, double *total)
{
    __shared__ float2 s_tree2[NT];
    const int per = NT / k;
    const int c = threadIdx.x / per, j = threadIdx.x % per;
    float sum = 0.0f, cmp = 0.0f;
    if (c < k) {
        // the partials of blocks j, j + per, j + 2 per, ... in that order, requested eight at
        // a time so that the serial tail waits for few memory round trips
        const float2 *pp = reinterpret_cast<const float2 *>(rd.partials);
        constexpr int kBatch = 8;
        for (int b0 = j; b0 < (int)gridDim.x; b0 += kBatch * per) {
            float2 q[kBatch];
#pragma unroll
            for (int i = 0; i < kBatch; ++i) {
                const int b = b0 + i * per;
                q[i] = b < (int)gridDim.x ? pp[(int64_t)b * k + c] : make_float2(0.0f, 0.0f);
            }
#pragma unroll
            for (int i = 0; i < kBatch; ++i) {
                if (b0 + i * per >= (int)gridDim.x) break;
                float hi, e;
                two_sum(sum, q[i].x, hi, e);
                sum = hi;
                cmp += e + q[i].y;
            }
        }
    }
    s_tree2[threadIdx.x] = make_float2(sum, cmp);
    __syncthreads();
    if (c < k && j == 0) {
        float S = 0.0f, C = 0.0f;
        for (int q = 0; q < per; ++q) {
            const float2 v = s_tree2[threadIdx.x + q];
            float hi, e;
            two_sum(S, v.x, hi, e);
            S = hi;
            C += e + v.y;
        }
        total[c] = (double)S + (double)C;
    }
    __syncthreads();
    if (threadIdx.x == 0) *rd.counter = 0u;
}

template <typename T, int V, int G, int MODE, int NT = kThreads>
__device__ __forceinline__ void pcg_block_finish(T (*red)[64], T (&part)[V], int K, const PcgScalars &ps,
                                                 const Reduce &rd)
{
    __shared__ double s_tot[64];
    if constexpr (sizeof(T) == 4) {
        if (!block_column_reduce_f32<V, G, NT>(red, part, K, rd)) return;
        finish_column_sums_f32<NT>(rd, K, s_tot);
    } else {
        if (!block_column_reduce<T, V, G, NT>(red, part, K, rd)) return;
        finish_column_sums<NT>(rd, K, s_tot);
    }
    if (threadIdx.x < K) {
        const int c = threadIdx.x;
        if (MODE == kPcgT) {
            const double tt = s_tot[c];
            const bool ok = ps.active[c] && tt > 0.0 && isfinite(tt);
            ps.alpha[c] = ok ? ps.rz[c] / tt : 0.0;
        } else {
            const double rzn = s_tot[c];
            int act = ps.active[c];
            if (!isfinite(rzn)) act = 0;
            if (ps.tol2 > 0.0 && rzn <= ps.tol2 * ps.rz0[c]) act = 0;
            ps.beta[c] = (act && ps.rz[c] > 0.0) ? rzn / ps.rz[c] : 0.0;
            if (!act) ps.alpha[c] = 0.0;
            ps.active[c] = act;
            ps.rz[c] = rzn;
        }
    }
}

// ---------------------------------------------------------------------------------
// The product kernel.  K = compile-time block width (row-major rows of K elements at
// stride ldx / ldy).  Grid-stride loop over batches of 32 consecutive rows per warp.
template <typename T, int K, int MODE>
__global__ void __launch_bounds__(kThreads) k_apply(ChainParams cp, const T *__restrict__ X, int64_t ldx,
                                                    T *__restrict__ Y, int64_t ldy, uint32_t n,
                                                    T *__restrict__ R, const T *__restrict__ dinv,
                                                    PcgScalars ps, Reduce rd)
{
    using Lay = RowLayout<T, K>;
    constexpr int V = Lay::V, G = Lay::G, RPW = 32 / G;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ApplySmem<T> &sm = *reinterpret_cast<ApplySmem<T> *>(smem_raw);
    load_binom(sm.binom);
    build_field_tables<T>(sm.tab, cp);
    __syncthreads();

    const T dconst = (T)cp.diag_const, hdelta = (T)cp.half_delta;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int col = (lane % G) * V;
    T part[V];
#pragma unroll
    for (int v = 0; v < V; ++v) part[v] = (T)0;
    T alpha[V];
    if (MODE == kPcgQ) {
#pragma unroll
        for (int v = 0; v < V; ++v) alpha[v] = (T)ps.alpha[col + v];
    }

    const uint32_t nbatch = (n + 31u) / 32u;
    for (uint32_t b = blockIdx.x * kWarps + warp; b < nbatch; b += gridDim.x * kWarps) {
        const uint32_t base = b * 32u;
        if constexpr (G == 1) {
            const uint32_t r = base + lane;
            if (r < n) {
                uint32_t s = state_of(sm.binom, cp, r);
                T d = diag_shifted<T>(sm.tab, dconst, hdelta, cp, s);
                uint32_t *nbl = sm.nb[warp][lane];
                int f = row_neighbours<T>(sm.binom, cp, r, s, nbl);
                Vec<T, V> x = ldv<T, V>(X + (int64_t)r * ldx);
                T acc[V];
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] = d * x.v[v];
                gather_add<T, V>(acc, X, ldx, 0, f, nbl);
                if (MODE == kPlain || MODE == kPcgT) {
                    Vec<T, V> y;
#pragma unroll
                    for (int v = 0; v < V; ++v) y.v[v] = acc[v];
                    stv<T, V>(Y + (int64_t)r * ldy, y);
                    if (MODE == kPcgT) {
#pragma unroll
                        for (int v = 0; v < V; ++v) part[v] += acc[v] * acc[v];
                    }
                } else {
                    Vec<T, V> rr = ldv<T, V>(R + (int64_t)r * ldy);
                    T di = dinv[r];
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        rr.v[v] -= alpha[v] * acc[v];
                        part[v] += rr.v[v] * (di * rr.v[v]);
                    }
                    stv<T, V>(R + (int64_t)r * ldy, rr);
                }
            }
        } else {
            // phase 1: lane t ranks row base + t
            {
                const uint32_t r = base + lane;
                int f = 0;
                T d = (T)0;
                if (r < n) {
                    uint32_t s = state_of(sm.binom, cp, r);
                    d = diag_shifted<T>(sm.tab, dconst, hdelta, cp, s);
                    f = row_neighbours<T>(sm.binom, cp, r, s, sm.nb[warp][lane]);
                }
                sm.dsig[warp][lane] = d;
                sm.cnt[warp][lane] = (r < n) ? f : -1;
            }
            __syncwarp();
            // phase 2: groups of G lanes stream the rows, two rows per group at a time
#pragma unroll 1
            for (int sub = 0; sub < G; sub += 2) {
                const int ri0 = sub * RPW + lane / G;
                const int ri1 = ri0 + RPW;  // sub + 1 < G because G is even here
                const int f0 = sm.cnt[warp][ri0], f1 = sm.cnt[warp][ri1];
                const uint32_t r0 = base + ri0, r1 = base + ri1;
                T acc0[V], acc1[V];
                {
                    Vec<T, V> x0, x1;
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        x0.v[v] = (T)0;
                        x1.v[v] = (T)0;
                    }
                    if (f0 >= 0) x0 = ldv<T, V>(X + (int64_t)r0 * ldx + col);
                    if (f1 >= 0) x1 = ldv<T, V>(X + (int64_t)r1 * ldx + col);
                    const T d0 = sm.dsig[warp][ri0], d1 = sm.dsig[warp][ri1];
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        acc0[v] = d0 * x0.v[v];
                        acc1[v] = d1 * x1.v[v];
                    }
                }
                gather_add2<T, V>(acc0, acc1, X, ldx, col, f0, sm.nb[warp][ri0], f1, sm.nb[warp][ri1]);
                finish_row<T, V, MODE>(acc0, f0, r0, Y, ldy, R, dinv, col, alpha, part);
                finish_row<T, V, MODE>(acc1, f1, r1, Y, ldy, R, dinv, col, alpha, part);
            }
            __syncwarp();
        }
    }

    if (MODE == kPlain) return;
    pcg_block_finish<T, V, G, MODE>(sm.red, part, K, ps, rd);
}


// ---------------------------------------------------------------------------------
// Tile-structured product.  Split a state s into a high part t (bits B..L-1, H = L - B
// bits) and a low part u (bits 0..B-1).  All states with the same t are consecutive
// rows -- a tile of C(B, p) rows, p = n_up - popc(t), ordered by the colex rank j of u --
// so the rank-shift rule of a bond exchange (+C(i, c) when the up spin moves from i to
// i + 1, -C(i, c) the other way, c = up spins below site i) takes these forms:
//   * bonds inside the low part: in-tile neighbours that depend only on (B, p, j);
//   * bonds inside the high part (i = B + b): c = p + popc(t mod 2^b), the same shift for
//     every row of the tile -- the neighbour rows are the tile's rows moved as a block;
//   * the joining bond (B-1, B): shift +C(B-1, p-1) or -C(B-1, p), also per tile;
//   * the wrap bond of a periodic chain: rank = offset of tile t ^ 2^(H-1) plus the rank
//     of u ^ 1 in its class.
// Everything that depends on the low pattern alone comes from a small table built once
// per tile width (LowRec); each warp processes a chunk of rows of one tile.

constexpr uint32_t kNoRow = 0xffffffffu;

struct LowRec {
    uint16_t u;      // low pattern
    uint8_t cnt;     // flippable bonds inside the low part
    uint8_t alow;    // antiparallel bonds inside the low part
    uint16_t jper;   // colex rank of u ^ 1 among the words of its popcount
    uint16_t pad;
    uint16_t nb[12];  // in-tile ranks of the low-part neighbours
};
static_assert(sizeof(LowRec) == 32, "LowRec layout");

constexpr int kLowMaxB = 13;  // at most 12 low bonds, C(13, 6) = 1716 rows per tile
// records for B = 2..13 at offsets 2^B - 4 (the sizes 2^B, B < current, summed)
constexpr int kLowRecords = (1 << (kLowMaxB + 1)) - 4;
static __device__ __align__(16) LowRec g_lowtab[kLowRecords];

__host__ __device__ inline int lowtab_base(int B) { return (1 << B) - 4; }

// Resident blocks per SM the tiled kernel is compiled for (register budget 65536 /
// (256 * this)); 3 keeps every variant free of spills.
#ifndef MBL_TILED_MIN_BLOCKS
#define MBL_TILED_MIN_BLOCKS 3
#endif
// Bytes per lane of rows from the rest of the vector requested before a row's in-tile work
#ifndef MBL_ROW_EARLY_BYTES
#define MBL_ROW_EARLY_BYTES 64
#endif
// 1: the PCG solution update w += alpha p runs in the direction-update launch (a streaming
// kernel), 0: in the epilogue of the q-launch
#ifndef MBL_PCG_W_IN_UPDATE
#define MBL_PCG_W_IN_UPDATE 1
#endif

// Per-tile values of a tile t (p = n_up - popc(t) up spins in its low part), computed
// by one warp, one lane each: the tile's first row (lane 0), the diagonal constant of
// its high bits, the rank shift of every high bond whose two spins differ (lane b + 1
// for bond (B + b, B + b + 1): C(B + b, p + popc(t mod 2^b)), + when the up spin moves
// up, - when it moves down; compacted in bond order), and the first row of the tile
// across the wrap bond (lane 31).
template <typename T>
struct TileMeta {
    uint32_t off, offper;
    int nh;
    T ct;
    uint32_t shift[32];
};

template <typename T>
__device__ __forceinline__ void tile_meta_warp(const uint32_t *sbin, const T *tab, const ChainParams &cp, int B,
                                               uint32_t t, int p, TileMeta<T> &tm)
{
    const int lane = threadIdx.x & 31, m = cp.n_up, H = cp.L - B;
    uint32_t v32 = 0;
    bool flip = false;
    if (lane == 0) {
        v32 = cns_rank(sbin, (t << B) | ((1u << p) - 1u));
        const uint32_t ahigh = __popc((t ^ (t >> 1)) & ((1u << (H - 1)) - 1u));
        tm.ct = (cp_diag_const<T>(cp) + field_sum(tab, t << B)) - mul_rn(cp_half_delta<T>(cp), (T)ahigh);
    } else if (lane <= H - 1) {
        const int b = lane - 1;
        if (((t >> b) ^ (t >> (b + 1))) & 1u) {
            flip = true;
            const uint32_t dlt = binom(sbin, B + b, p + __popc(t & ((1u << b) - 1u)));
            v32 = ((t >> b) & 1u) ? dlt : (0u - dlt);  // modulo 2^32, applied as int32
        }
    } else if (lane == 31 && cp.periodic) {
        const uint32_t t2 = t ^ (1u << (H - 1));
        const int p2 = m - __popc(t2);
        v32 = (p2 >= 0 && p2 <= B) ? cns_rank(sbin, (t2 << B) | ((1u << p2) - 1u)) : kNoRow;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, flip);
    if (flip) tm.shift[__popc(bal & ((1u << lane) - 1u))] = v32;
    if (lane == 0) {
        tm.off = v32;
        tm.nh = __popc(bal);
    }
    if (lane == 31) tm.offper = v32;
}

// Packed FP32 pair arithmetic (FADD2 / FMUL2 / FFMA2 on sm_100 and later): each is two
// independent, correctly rounded operations, so the results equal those of the scalar
// instructions bit for bit; the FP64 kernels use the scalar forms.
template <typename T, int V>
__device__ __forceinline__ void vadd(T (&s)[V], const Vec<T, V> &a)
{
    if constexpr (sizeof(T) == 4 && V % 2 == 0) {
#pragma unroll
        for (int v = 0; v < V; v += 2) {
            const float2 r = __fadd2_rn(make_float2(s[v], s[v + 1]), make_float2(a.v[v], a.v[v + 1]));
            s[v] = r.x;
            s[v + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) s[v] += a.v[v];
    }
}

// acc = 1/2 nb + (d x), with d x rounded on its own (exact 1/2: one rounding for the fma).
template <typename T, int V>
__device__ __forceinline__ void half_sum_plus_dx(T (&acc)[V], const T (&nb)[V], T d, const Vec<T, V> &x)
{
    if constexpr (sizeof(T) == 4 && V % 2 == 0) {
        const float2 d2 = make_float2(d, d), h2 = make_float2(0.5f, 0.5f);
#pragma unroll
        for (int v = 0; v < V; v += 2) {
            const float2 dx = __fmul2_rn(d2, make_float2(x.v[v], x.v[v + 1]));
            const float2 r = __ffma2_rn(h2, make_float2(nb[v], nb[v + 1]), dx);
            acc[v] = r.x;
            acc[v + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = fma_rn((T)0.5, nb[v], mul_rn(d, x.v[v]));
    }
}

// One pass of a warp over RPW rows of a tile (row j of this lane group, `valid` when it
// is a row of the work item; otherwise j is some other row of the same tile and only the
// output is dropped).  Own row and in-tile neighbours come from Xt (row stride ldt: the
// tile in shared memory, or X itself from the tile's first row); the joining, wrap and
// high-bond rows from X.  y = (d - sigma) x + 1/2 (sum of neighbour rows), the
// neighbours summed first in a fixed order (low bonds, joining, wrap, high bonds):
// scaling by 1/2 is exact, so only the order of the additions is a choice, and every
// work order (persistent, ordered, staged, streamed) makes the same one.  The rows from
// the rest of the vector (joining and wrap partners, the first high-bond rows) are
// requested before the in-tile work so that their latency overlaps it.  Every load reads
// a row of the chain's vector (the own row where a bond does not apply, row 0 of the
// tile in an unused low-bond slot, the last shift past a tile's high bonds); only the
// additions are conditional, so no register has to be cleared before a load.
template <typename T, int V, int NB, int MODE>
__device__ __forceinline__ void tile_row_pass(const ChainParams &cp, int B, const T *__restrict__ X, int64_t ldx,
                                              const T *__restrict__ Xt, int64_t ldt, const LowRec *__restrict__ rp,
                                              uint32_t j, bool valid, const TileMeta<T> &tm, const T *tab, T hdelta,
                                              uint32_t t0, uint32_t thi, uint32_t sup, uint32_t sdn, int col,
                                              T *__restrict__ Y, int64_t ldy, T *__restrict__ R,
                                              const T *__restrict__ dinv, const T *s_alpha, T (&part)[V],
                                              void *ps_w, const void *ps_p)
{
    constexpr int kVecBytes = V * (int)sizeof(T);
    // early global rows: joining + wrap + kEarly high-bond rows, MBL_ROW_EARLY_BYTES per lane
    constexpr int kEarly = MBL_ROW_EARLY_BYTES / kVecBytes - 2 > 0 ? MBL_ROW_EARLY_BYTES / kVecBytes - 2 : 0;
    // in-tile rows requested together (64 bytes per lane)
    constexpr int NBL = 64 / kVecBytes > 1 ? 64 / kVecBytes : 1;
    const uint32_t r = tm.off + j;
    const T *__restrict__ xr = X + (int64_t)r * ldx + col;
    const uint4 w0 = __ldg(reinterpret_cast<const uint4 *>(rp + j));
    const uint4 w1 = __ldg(reinterpret_cast<const uint4 *>(rp + j) + 1);
    const uint32_t u = w0.x & 0xffffu, cnt = (w0.x >> 16) & 0xffu, alow = w0.x >> 24;
    const uint32_t ub = (u >> (B - 1)) & 1u;
    const bool join = ub != t0;
    const bool wrap = cp.periodic && (u & 1u) != thi;
    const int nh = tm.nh;
    // the joining and wrap partners apply to about half of the rows each: loaded only there
    Vec<T, V> ja, wb;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        ja.v[v] = (T)0;
        wb.v[v] = (T)0;
    }
    if (join) ja = ldv<T, V>(xr + (ub ? (int64_t)sup : -(int64_t)sdn) * ldx);
    if (wrap) wb = ldv<T, V>(X + (int64_t)(tm.offper + (w0.y & 0xffffu)) * ldx + col);
    // the q-launch's own rows of r and M^-1, needed after the sum
    Vec<T, V> rq;
    T dq = (T)0;
    if constexpr (MODE == kPcgQ) {
        rq = ldv<T, V>(R + (int64_t)r * ldy + col);
        dq = dinv[r];
    }
    Vec<T, V> hb[kEarly > 0 ? kEarly : 1];
#pragma unroll
    for (int e = 0; e < kEarly; ++e) {
        const int hh = e < nh ? e : (nh > 0 ? nh - 1 : 0);
        hb[e] = ldv<T, V>(nh > 0 ? xr + (int64_t)(int32_t)tm.shift[hh] * ldx : xr);
    }
    T nb[V];
#pragma unroll
    for (int v = 0; v < V; ++v) nb[v] = (T)0;
    {
        // in-tile neighbours; the loop runs to the warp's largest count
        const uint32_t nbw[6] = {w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
        const int cmax = (int)__reduce_max_sync(0xffffffffu, valid ? cnt : 0u);
#pragma unroll
        for (int q0 = 0; q0 < 12; q0 += NBL) {
            if (q0 >= cmax) break;
            Vec<T, V> a[NBL];
#pragma unroll
            for (int e = 0; e < NBL; ++e) {
                const int q = q0 + e;
                const int qq = q < 12 ? q : 11;
                const uint32_t jn = (nbw[qq >> 1] >> (16 * (qq & 1))) & 0xffffu;
                a[e] = ldv<T, V>(Xt + (int64_t)jn * ldt + col);
            }
#pragma unroll
            for (int e = 0; e < NBL; ++e)
                if (q0 + e < (int)cnt) vadd<T, V>(nb, a[e]);
        }
    }
    if (join) vadd<T, V>(nb, ja);
    if (wrap) vadd<T, V>(nb, wb);
#pragma unroll
    for (int e = 0; e < kEarly; ++e)
        if (e < nh) vadd<T, V>(nb, hb[e]);
    for (int h0 = kEarly; h0 < nh; h0 += NB) {
        // the remaining high-bond neighbours: the tile's rows moved as a block, one shift
        // per bond
        Vec<T, V> a[NB];
#pragma unroll
        for (int e = 0; e < NB; ++e) {
            const int hh = h0 + e < nh ? h0 + e : nh - 1;
            a[e] = ldv<T, V>(xr + (int64_t)(int32_t)tm.shift[hh] * ldx);
        }
#pragma unroll
        for (int e = 0; e < NB; ++e)
            if (h0 + e < nh) vadd<T, V>(nb, a[e]);
    }
    const Vec<T, V> x = ldv<T, V>(Xt + (int64_t)j * ldt + col);
    const T d = (tm.ct + (tab[u & 255u] + tab[256 + (u >> 8)])) -
                mul_rn(hdelta, (T)(alow + (join ? 1u : 0u) + (wrap ? 1u : 0u)));
    T acc[V];
    half_sum_plus_dx<T, V>(acc, nb, d, x);
    if (valid) {
        T alpha[V];
#pragma unroll
        for (int v = 0; v < V; ++v) alpha[v] = (MODE == kPcgQ) ? s_alpha[col + v] : (T)0;
        if constexpr (MODE == kPcgQ) {
            if (ps_w == nullptr) {
                // r -= alpha q and r.(M^-1 r) on the prefetched row (as finish_row does)
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    rq.v[v] -= alpha[v] * acc[v];
                    part[v] += rq.v[v] * (dq * rq.v[v]);
                }
                stv<T, V>(R + (int64_t)r * ldy + col, rq);
                return;
            }
        }
        finish_row<T, V, MODE>(acc, 0, r, Y, ldy, R, dinv, col, alpha, part, (T *)ps_w, (const T *)ps_p);
    }
}

template <typename T, int K, int MODE, int LB>
__global__ void __launch_bounds__(kThreads, MBL_TILED_MIN_BLOCKS) k_apply_tiled(ChainParams cp, int B,
                                                                               const T *__restrict__ X, int64_t ldx,
                                                                               T *__restrict__ Y, int64_t ldy,
                                                                               T *__restrict__ R,
                                                                               const T *__restrict__ dinv,
                                                                               PcgScalars ps, Reduce rd)
{
    using Lay = WideRowLayout<T, K, LB>;
    constexpr int V = Lay::V, G = Lay::G, RPW = 32 / G, CH = Lay::CH;
    // neighbour loads issued together: 128 bytes per lane (two to eight vectors)
    constexpr int NBr = 128 / (V * (int)sizeof(T));
    constexpr int NB = NBr < 2 ? 2 : (NBr > 8 ? 8 : NBr);
    if (MODE == kPlain) {
        // ordered schedule (at most one item per warp): a block whose items hold no rows
        // leaves before any setup
        const uint32_t nch = (__ldg(&g_binom.v[B * kBinomDim + B / 2]) + CH - 1) / CH;
        const uint32_t tot = (1u << (cp.L - B)) * nch;
        if ((uint64_t)gridDim.x * kWarps >= tot) {
            int any = 0;
            if (threadIdx.x < kWarps) {
                const uint32_t item = blockIdx.x * kWarps + threadIdx.x;
                if (item < tot) {
                    const uint32_t t = item / nch, c = item % nch;
                    const int p = cp.n_up - __popc(t);
                    any = (p >= 0 && p <= B && c * CH < __ldg(&g_binom.v[B * kBinomDim + p])) ? 1 : 0;
                }
            }
            if (!__syncthreads_or(any)) return;
        }
    }
    __shared__ uint32_t sbin[kBinomDim * kBinomDim];
    __shared__ T tab[1024];
    __shared__ T red[kWarps][64];
    __shared__ uint32_t spref[kLowMaxB + 2];  // spref[p] = sum_{q < p} C(B, q)
    __shared__ T s_alpha[64];
    __shared__ TileMeta<T> s_meta[kWarps];
    load_binom(sbin);
    build_field_tables<T>(tab, cp);
    if (MODE == kPcgQ && threadIdx.x < K) s_alpha[threadIdx.x] = (T)ps.alpha[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int q = 0; q <= B + 1 && q <= kLowMaxB + 1; ++q) {
            spref[q] = acc;
            acc += binom(sbin, B, q);
        }
    }
    __syncthreads();

    const int L = cp.L, m = cp.n_up, H = L - B;
    const uint32_t ntile = 1u << H;
    const uint32_t nchunk = (binom(sbin, B, B / 2) + CH - 1) / CH;
    const uint32_t total = ntile * nchunk;
    const T hdelta = cp_half_delta<T>(cp);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / G;
    const int col = (lane % G) * V;
    const LowRec *__restrict__ tbl = g_lowtab + lowtab_base(B);
    TileMeta<T> &tm = s_meta[warp];
    T part[V];
#pragma unroll
    for (int v = 0; v < V; ++v) part[v] = (T)0;
    const uint32_t gw = blockIdx.x * kWarps + warp, nw = gridDim.x * kWarps;
    for (uint32_t item = gw; item < total; item += nw) {
        // tile-major: the warps in flight cover a run of consecutive tiles, so in-tile
        // neighbours and the tiles reached by the low high-part bonds stay in L2
        const uint32_t t = item / nchunk, c = item % nchunk;
        const int p = m - __popc(t);
        if (p < 0 || p > B) continue;  // warp-uniform
        const uint32_t Rt = binom(sbin, B, p);
        const uint32_t j_begin = c * CH;
        if (j_begin >= Rt) continue;
        const uint32_t j_end = min(Rt, j_begin + CH);
        __syncwarp();
        tile_meta_warp<T>(sbin, tab, cp, B, t, p, tm);
        __syncwarp();
        const uint32_t t0 = t & 1u, thi = (t >> (H - 1)) & 1u;
        const uint32_t sup = p >= 1 ? binom(sbin, B - 1, p - 1) : 0u;  // joining bond, up spin moves up
        const uint32_t sdn = binom(sbin, B - 1, p);                     // joining bond, moves down
        const LowRec *__restrict__ rp = tbl + spref[p];
        const T *__restrict__ Xt = X + (int64_t)tm.off * ldx;
        for (uint32_t j0 = j_begin; j0 < j_end; j0 += RPW) {
            const uint32_t j = j0 + grp;
            tile_row_pass<T, V, NB, MODE>(cp, B, X, ldx, Xt, ldx, rp, min(j, j_end - 1u), j < j_end, tm, tab, hdelta,
                                          t0, thi, sup,
                                          sdn, col, Y, ldy, R, dinv, s_alpha, part, ps.w, ps.p);
        }
    }
    if (MODE == kPlain) return;
    pcg_block_finish<T, V, G, MODE>(red, part, K, ps, rd);
}

// ---------------------------------------------------------------------------------
// Staged tiled product: a block takes whole tiles (B chosen so a tile fits in 48 KB of
// shared memory), copies the tile's rows into shared memory with one bulk asynchronous
// copy (the tile is contiguous in X), and serves the in-tile (low-bond) neighbours from
// there; the own row too.  Only the high-bond rows (own row + per-tile shift), the joining
// row and the wrap row come from L2/HBM.  Requires ldx = ldy = K and rows of a multiple of
// 16 bytes.  Same arithmetic, in the same order, as k_apply_tiled with the same tile width.

constexpr int kStageBytes = 48 * 1024;
constexpr long long kWaitCycles = 2000000000ll;  // ~1 s at 2 GHz: bounded mbarrier wait

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *mbar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *mbar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete, for at most kWaitCycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, unsigned parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(mbar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

// One bulk copy global -> shared (addresses 16-byte aligned, size a multiple of 16),
// completing on mbar.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, uint64_t *mbar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(mbar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

#ifndef MBL_STAGED_MIN_BLOCKS
#define MBL_STAGED_MIN_BLOCKS 3
#endif

template <typename T, int K, int MODE, int LB>
__global__ void __launch_bounds__(kThreads, MBL_STAGED_MIN_BLOCKS)
    k_apply_staged(ChainParams cp, int B, const T *__restrict__ X, T *__restrict__ Y, T *__restrict__ R,
                   const T *__restrict__ dinv, PcgScalars ps, Reduce rd)
{
    using Lay = WideRowLayout<T, K, LB>;
    constexpr int V = Lay::V, G = Lay::G, RPW = 32 / G, RPB = kWarps * RPW;
    constexpr int NBr = 128 / (V * (int)sizeof(T));
    constexpr int NB = NBr < 2 ? 2 : (NBr > 8 ? 8 : NBr);
    static_assert((K * sizeof(T)) % 16 == 0, "staged rows must be multiples of 16 bytes");
    extern __shared__ __align__(128) unsigned char stage_raw[];
    T *__restrict__ s_tile = reinterpret_cast<T *>(stage_raw);
    __shared__ uint32_t sbin[kBinomDim * kBinomDim];
    __shared__ T tab[1024];
    __shared__ T red[kWarps][64];
    __shared__ uint32_t spref[kLowMaxB + 2];
    __shared__ T s_alpha[64];
    __shared__ TileMeta<T> s_meta;
    __shared__ __align__(8) uint64_t s_mbar;
    load_binom(sbin);
    build_field_tables<T>(tab, cp);
    if (MODE == kPcgQ && threadIdx.x < K) s_alpha[threadIdx.x] = (T)ps.alpha[threadIdx.x];
    if (threadIdx.x == 0) mbar_init(&s_mbar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int q = 0; q <= B + 1 && q <= kLowMaxB + 1; ++q) {
            spref[q] = acc;
            acc += binom(sbin, B, q);
        }
    }
    __syncthreads();

    const int L = cp.L, m = cp.n_up, H = L - B;
    const uint32_t ntile = 1u << H;
    const T hdelta = cp_half_delta<T>(cp);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / G;
    const int col = (lane % G) * V;
    const LowRec *__restrict__ tbl = g_lowtab + lowtab_base(B);
    T part[V];
#pragma unroll
    for (int v = 0; v < V; ++v) part[v] = (T)0;
    unsigned parity = 0;
    for (uint32_t t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int p = m - __popc(t);
        if (p < 0 || p > B) continue;  // block-uniform
        const uint32_t Rt = binom(sbin, B, p);
        if (warp == 0) {
            tile_meta_warp<T>(sbin, tab, cp, B, t, p, s_meta);
            __syncwarp();
            if (lane == 0) {
                const unsigned bytes = Rt * (unsigned)(K * sizeof(T));
                mbar_arrive_expect_tx(&s_mbar, bytes);
                bulk_copy_g2s(s_tile, X + (int64_t)s_meta.off * K, bytes, &s_mbar);
            }
        }
        __syncthreads();
        const bool got = mbar_wait_bounded(&s_mbar, parity);
        parity ^= 1u;
        if (!__syncthreads_and(got)) {
            // the copy did not complete in time: wait once more (bounded) so no copy is
            // left in flight, mark this tile's rows NaN, and stop
            mbar_wait_bounded(&s_mbar, parity ^ 1u);
            for (uint32_t j = threadIdx.x / G; j < Rt; j += kThreads / G) {
                Vec<T, V> nanv;
#pragma unroll
                for (int v = 0; v < V; ++v) nanv.v[v] = (T)NAN;
                T *dst = (MODE == kPcgQ) ? R : Y;
                stv<T, V>(dst + (int64_t)(s_meta.off + j) * K + col, nanv);
            }
#pragma unroll
            for (int v = 0; v < V; ++v) part[v] = (T)NAN;
            break;
        }
        const uint32_t t0 = t & 1u, thi = (t >> (H - 1)) & 1u;
        const uint32_t sup = p >= 1 ? binom(sbin, B - 1, p - 1) : 0u;
        const uint32_t sdn = binom(sbin, B - 1, p);
        const LowRec *__restrict__ rp = tbl + spref[p];
        for (uint32_t j0 = warp * RPW; j0 < Rt; j0 += RPB) {
            const uint32_t j = j0 + grp;
            tile_row_pass<T, V, NB, MODE>(cp, B, X, K, s_tile, K, rp, min(j, Rt - 1u), j < Rt, s_meta, tab, hdelta,
                                          t0, thi, sup,
                                          sdn, col, Y, K, R, dinv, s_alpha, part, ps.w, ps.p);
        }
        // every read of this tile is done before the next copy overwrites it
        __syncthreads();
        if (threadIdx.x == 0) fence_proxy_async_smem();
    }
    if (MODE == kPlain) return;
    pcg_block_finish<T, V, G, MODE>(red, part, K, ps, rd);
}

// ---------------------------------------------------------------------------------
// Streamed tiled product: a few blocks per SM take whole tiles, and every row block the
// product of a tile reads reaches shared memory by a bulk asynchronous copy.  Each term
// of a tile's rows is one contiguous block of X: the tile itself (own rows and in-tile
// neighbours), the joining-bond partners (the tile's rows whose boundary spins differ,
// moved by one rank shift), the wrap partner tile, and one block per antiparallel high
// bond (the tile's rows moved by that bond's rank shift).  The last warp of the block
// is the producer: it walks the block's tiles and issues the copies, in that order, into
// a ring of tile-sized slots (one full and one empty mbarrier per slot), so up to a ring
// of data is in flight per SM without holding registers.  The other warps consume the
// slots in the same order, adding each block into per-row accumulators: the sums are
// formed in the order of the other work orders (low bonds, joining, wrap, high bonds)
// and the result is bitwise that of k_apply_tiled at the same tile width.  PCG launches
// also stream the rows of r (and w, p) their epilogue reads.  Rows of 32 to 512 bytes
// (one 32-byte vector per lane), ld = K, 16-byte aligned bases.  Every mbarrier wait is
// bounded; on a timeout the block stops copying, waits for the copies it issued, and
// writes NaN to the rest of its output rows (and its PCG partials).

constexpr int kMaxSlots = 12;
#ifndef MBL_STREAM_PASSES
#define MBL_STREAM_PASSES 3  // row groups of a consumer lane per tile
#endif
#ifndef MBL_STREAM_BLOCKS
#define MBL_STREAM_BLOCKS 2  // resident blocks per SM (each with its own ring)
#endif
constexpr int kStreamPasses = MBL_STREAM_PASSES;
constexpr int kStreamBlocks = MBL_STREAM_BLOCKS;

#ifndef MBL_STREAM_MIN_SLOTS
#define MBL_STREAM_MIN_SLOTS 6
#endif

__device__ __forceinline__ void mbar_arrive(uint64_t *mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(mbar)) : "memory");
}

// Bounded wait that also gives up once another warp of the block has flagged a failure.
__device__ __forceinline__ bool ring_wait(uint64_t *mbar, unsigned parity, volatile int *fail)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(mbar, parity)) {
        if (*fail) return false;
        if (clock64() - t0 > kWaitCycles) {
            *fail = 1;
            return false;
        }
    }
    return true;
}

template <typename T, int K>
struct StreamLayout {
    static constexpr int RB = K * (int)sizeof(T);  // row bytes
    static constexpr int V = 32 / (int)sizeof(T);  // one 32-byte vector per lane
    static constexpr int G = RB / 32;              // lanes per row
    static constexpr int RPW = 32 / G;             // rows per warp and pass
    static constexpr int NCW = kWarps - 1;         // consumer warps
    static constexpr int RPP = NCW * RPW;          // rows per pass of the block
    static constexpr int CAP = kStreamPasses * RPP;  // largest tile the consumers cover
    static constexpr bool ok = RB >= 32 && RB <= 512 && (RB % 32) == 0 && (32 % G) == 0;
};

// Position in the ring: slot index and the parity of its current use.
struct RingPos {
    uint32_t s, ph;
    __device__ __forceinline__ void next(uint32_t nbuf)
    {
        if (++s == nbuf) {
            s = 0;
            ph ^= 1u;
        }
    }
};

template <typename T, int K, int MODE>
__global__ void __launch_bounds__(kThreads, kStreamBlocks)
    k_apply_streamed(ChainParams cp, int B, int nbuf, const T *__restrict__ X, T *__restrict__ Y,
                     T *__restrict__ R, const T *__restrict__ dinv, PcgScalars ps, Reduce rd)
{
    using SL = StreamLayout<T, K>;
    constexpr int V = SL::V, G = SL::G, RPW = SL::RPW, RPP = SL::RPP, P = kStreamPasses;
    static_assert(SL::ok, "streamed rows: 32 to 512 bytes");
    extern __shared__ __align__(128) unsigned char ring_raw[];
    __shared__ uint32_t sbin[kBinomDim * kBinomDim];
    __shared__ T tab[1024];
    __shared__ T red[kWarps][64];
    __shared__ uint32_t spref[kLowMaxB + 2];
    __shared__ T s_alpha[64];
    __shared__ TileMeta<T> s_meta[kWarps];
    __shared__ __align__(8) uint64_t s_full[kMaxSlots], s_empty[kMaxSlots];
    __shared__ int s_fail;
    load_binom(sbin);
    build_field_tables<T>(tab, cp);
    if (MODE == kPcgQ && threadIdx.x < K) s_alpha[threadIdx.x] = (T)ps.alpha[threadIdx.x];
    if (threadIdx.x == 0) {
        for (int s = 0; s < nbuf; ++s) {
            mbar_init(&s_full[s], 1);
            mbar_init(&s_empty[s], SL::NCW);
        }
        s_fail = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int q = 0; q <= B + 1 && q <= kLowMaxB + 1; ++q) {
            spref[q] = acc;
            acc += binom(sbin, B, q);
        }
    }
    __syncthreads();

    const int L = cp.L, m = cp.n_up, H = L - B;
    const uint32_t ntile = 1u << H;
    const uint32_t rmax = binom(sbin, B, B / 2);
    const uint32_t slot_elems = rmax * K;
    T *__restrict__ ring = reinterpret_cast<T *>(ring_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int *fail = &s_fail;
    T part[V];
#pragma unroll
    for (int v = 0; v < V; ++v) part[v] = (T)0;
    TileMeta<T> &tm = s_meta[warp];
    const bool fused_w = (MODE == kPcgQ) && ps.w != nullptr;

    if (warp == kWarps - 1) {
        // producer
        RingPos pos{0u, 0u};
        uint32_t k = 0;
        bool ok = true;
        for (uint32_t t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
            const int p = m - __popc(t);
            if (p < 0 || p > B) continue;  // warp-uniform
            __syncwarp();
            tile_meta_warp<T>(sbin, tab, cp, B, t, p, tm);
            __syncwarp();
            if (lane == 0) {
                const uint32_t Rt = binom(sbin, B, p), c0 = binom(sbin, B - 1, p);
                const uint32_t sup = p >= 1 ? binom(sbin, B - 1, p - 1) : 0u;
                const uint32_t t0 = t & 1u;
                const uint32_t jcnt = t0 ? c0 : Rt - c0;
                const int64_t jsrc = t0 ? (int64_t)tm.off - (int64_t)c0 : (int64_t)tm.off + c0 + sup;
                auto issue = [&](const T *src, uint32_t rows) {
                    if (!ok) return;
                    const uint32_t s = pos.s;
                    // the slot's previous use (one lap ago) must have been released
                    if (k >= (uint32_t)nbuf && !ring_wait(&s_empty[s], pos.ph ^ 1u, fail)) {
                        ok = false;
                        return;
                    }
                    fence_proxy_async_smem();
                    const unsigned bytes = rows * (unsigned)SL::RB;
                    mbar_arrive_expect_tx(&s_full[s], bytes);
                    bulk_copy_g2s(ring + (size_t)s * slot_elems, src, bytes, &s_full[s]);
                    ++k;
                    pos.next((uint32_t)nbuf);
                };
                issue(X + (int64_t)tm.off * K, Rt);
                if (jcnt) issue(X + jsrc * K, jcnt);
                if (cp.periodic && tm.offper != kNoRow) {
                    const int p2 = m - __popc(t ^ (1u << (H - 1)));
                    issue(X + (int64_t)tm.offper * K, binom(sbin, B, p2));
                }
                for (int h = 0; h < tm.nh; ++h) issue(X + ((int64_t)tm.off + (int32_t)tm.shift[h]) * K, Rt);
                if (MODE == kPcgQ) {
                    issue(R + (int64_t)tm.off * K, Rt);
                    if (fused_w) {
                        issue((const T *)ps.w + (int64_t)tm.off * K, Rt);
                        issue((const T *)ps.p + (int64_t)tm.off * K, Rt);
                    }
                }
            }
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        }
        if (!ok && lane == 0) {
            // leave no copy in flight: wait (bounded) for the last ring of issued copies
            const uint32_t k0 = k > (uint32_t)nbuf ? k - (uint32_t)nbuf : 0u;
            for (uint32_t kk = k0; kk < k; ++kk)
                mbar_wait_bounded(&s_full[kk % (uint32_t)nbuf], (kk / (uint32_t)nbuf) & 1u);
        }
    } else {
        // consumers: warp w covers rows pp * RPP + w * RPW + lane / G of every tile
        const int grp = lane / G, col = (lane % G) * V;
        const T hdelta = cp_half_delta<T>(cp);
        const LowRec *__restrict__ tbl = g_lowtab + lowtab_base(B);
        RingPos pos{0u, 0u};
        bool ok = true;
        for (uint32_t t = blockIdx.x; t < ntile; t += gridDim.x) {
            const int p = m - __popc(t);
            if (p < 0 || p > B) continue;  // warp-uniform
            __syncwarp();
            tile_meta_warp<T>(sbin, tab, cp, B, t, p, tm);
            __syncwarp();
            const uint32_t Rt = binom(sbin, B, p), c0 = binom(sbin, B - 1, p);
            const uint32_t t0 = t & 1u, thi = (t >> (H - 1)) & 1u;
            const uint32_t jbase = t0 ? 0u : c0, jcnt = t0 ? c0 : Rt - c0;
            const bool has_wrap = cp.periodic && tm.offper != kNoRow;
            const uint32_t off = tm.off;
            const int nh = tm.nh;
            const T ct = tm.ct;
            uint32_t jrow[P];
#pragma unroll
            for (int pp = 0; pp < P; ++pp) jrow[pp] = (uint32_t)(pp * RPP + warp * RPW + grp);
            if (ok) {
                const LowRec *__restrict__ rp = tbl + spref[p];
                uint4 w0[P], w1[P];
#pragma unroll
                for (int pp = 0; pp < P; ++pp) {
                    w0[pp] = make_uint4(0, 0, 0, 0);
                    w1[pp] = make_uint4(0, 0, 0, 0);
                    if (jrow[pp] < Rt) {
                        w0[pp] = __ldg(reinterpret_cast<const uint4 *>(rp + jrow[pp]));
                        w1[pp] = __ldg(reinterpret_cast<const uint4 *>(rp + jrow[pp]) + 1);
                    }
                }
                T nb[P][V], dx[P][V];
                T di[P];
#pragma unroll
                for (int pp = 0; pp < P; ++pp) {
                    di[pp] = (T)0;
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        nb[pp][v] = (T)0;
                        dx[pp][v] = (T)0;
                    }
                }
                // wait for the item at ring position q; false for the whole warp (and the
                // block flagged) once any lane gave up
                auto take_at = [&](const RingPos &q, const T *&slot) -> bool {
                    slot = ring + (size_t)q.s * slot_elems;
                    return __all_sync(0xffffffffu, ring_wait(&s_full[q.s], q.ph, fail)) != 0;
                };
                auto take = [&](const T *&slot) -> bool { return take_at(pos, slot); };
                auto give = [&]() {
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&s_empty[pos.s]);
                    pos.next((uint32_t)nbuf);
                };
                const T *slot = nullptr;
                {
                    if ((ok = take(slot))) {
#pragma unroll
                        for (int pp = 0; pp < P; ++pp) {
                            if (jrow[pp] >= Rt) continue;
                            const uint32_t j = jrow[pp];
                            const uint32_t u = w0[pp].x & 0xffffu, cnt = (w0[pp].x >> 16) & 0xffu,
                                           alow = w0[pp].x >> 24;
                            const bool join = j - jbase < jcnt;
                            const bool wrap = has_wrap && (u & 1u) != thi;
                            const Vec<T, V> x = ldv<T, V>(slot + (int64_t)j * K + col);
                            const T d = (ct + (tab[u & 255u] + tab[256 + (u >> 8)])) -
                                        mul_rn(hdelta, (T)(alow + (join ? 1u : 0u) + (wrap ? 1u : 0u)));
#pragma unroll
                            for (int v = 0; v < V; ++v) dx[pp][v] = mul_rn(d, x.v[v]);
                            const uint32_t nbw[6] = {w0[pp].z, w0[pp].w, w1[pp].x, w1[pp].y, w1[pp].z, w1[pp].w};
#pragma unroll
                            for (int q = 0; q < 12; ++q) {
                                if (q >= (int)cnt) break;
                                const uint32_t jn = (nbw[q >> 1] >> (16 * (q & 1))) & 0xffffu;
                                const Vec<T, V> a = ldv<T, V>(slot + (int64_t)jn * K + col);
#pragma unroll
                                for (int v = 0; v < V; ++v) nb[pp][v] += a.v[v];
                            }
                            if (MODE == kPcgQ) di[pp] = dinv[off + j];
                        }
                        give();
                    }
                }
                if (ok && jcnt) {
                    if ((ok = take(slot))) {
#pragma unroll
                        for (int pp = 0; pp < P; ++pp)
                            if (jrow[pp] < Rt && jrow[pp] - jbase < jcnt) {
                                const Vec<T, V> a = ldv<T, V>(slot + (int64_t)(jrow[pp] - jbase) * K + col);
#pragma unroll
                                for (int v = 0; v < V; ++v) nb[pp][v] += a.v[v];
                            }
                        give();
                    }
                }
                if (ok && has_wrap) {
                    if ((ok = take(slot))) {
#pragma unroll
                        for (int pp = 0; pp < P; ++pp) {
                            const uint32_t u = w0[pp].x & 0xffffu;
                            if (jrow[pp] < Rt && (u & 1u) != thi) {
                                const Vec<T, V> a = ldv<T, V>(slot + (int64_t)(w0[pp].y & 0xffffu) * K + col);
#pragma unroll
                                for (int v = 0; v < V; ++v) nb[pp][v] += a.v[v];
                            }
                        }
                        give();
                    }
                }
                for (int h = 0; h < nh && ok; ++h) {
                    if ((ok = take(slot))) {
#pragma unroll
                        for (int pp = 0; pp < P; ++pp)
                            if (jrow[pp] < Rt) {
                                const Vec<T, V> a = ldv<T, V>(slot + (int64_t)jrow[pp] * K + col);
#pragma unroll
                                for (int v = 0; v < V; ++v) nb[pp][v] += a.v[v];
                            }
                        give();
                    }
                }
                if (ok) {
                    T acc[P][V];
#pragma unroll
                    for (int pp = 0; pp < P; ++pp)
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[pp][v] = fma_rn((T)0.5, nb[pp][v], dx[pp][v]);
                    if (MODE != kPcgQ) {
                        const T zero[V] = {};
#pragma unroll
                        for (int pp = 0; pp < P; ++pp)
                            if (jrow[pp] < Rt)
                                finish_row<T, V, MODE>(acc[pp], 0, off + jrow[pp], Y, K, R, dinv, col, zero, part);
                    } else {
                        // r (and w, p) of the tile's rows: items of their own, in that order
                        const T *sr = nullptr, *sw = nullptr, *sp = nullptr;
                        ok = take(sr);
                        if (ok && fused_w) {
                            RingPos q = pos;
                            q.next((uint32_t)nbuf);
                            ok = take_at(q, sw);
                            q.next((uint32_t)nbuf);
                            if (ok) ok = take_at(q, sp);
                        }
                        if (ok) {
                            T alpha[V];
#pragma unroll
                            for (int v = 0; v < V; ++v) alpha[v] = s_alpha[col + v];
#pragma unroll
                            for (int pp = 0; pp < P; ++pp) {
                                if (jrow[pp] >= Rt) continue;
                                const int64_t o = (int64_t)jrow[pp] * K + col;
                                const int64_t g = (int64_t)(off + jrow[pp]) * K + col;
                                Vec<T, V> rr = ldv<T, V>(sr + o);
                                const T dd = di[pp];
#pragma unroll
                                for (int v = 0; v < V; ++v) {
                                    rr.v[v] -= alpha[v] * acc[pp][v];
                                    part[v] += rr.v[v] * (dd * rr.v[v]);
                                }
                                stv<T, V>(R + g, rr);
                                if (fused_w) {
                                    Vec<T, V> wv = ldv<T, V>(sw + o);
                                    const Vec<T, V> pv = ldv<T, V>(sp + o);
#pragma unroll
                                    for (int v = 0; v < V; ++v) wv.v[v] += alpha[v] * pv.v[v];
                                    stv<T, V>((T *)ps.w + g, wv);
                                }
                            }
                            give();
                            if (fused_w) {
                                give();
                                give();
                            }
                        }
                    }
                }
            }
            if (!ok) {
                // the ring stopped: this warp's rows of this and every later tile are NaN
                Vec<T, V> nanv;
#pragma unroll
                for (int v = 0; v < V; ++v) nanv.v[v] = (T)NAN;
                T *dst = (MODE == kPcgQ) ? R : Y;
#pragma unroll
                for (int pp = 0; pp < P; ++pp)
                    if (jrow[pp] < Rt) stv<T, V>(dst + (int64_t)(off + jrow[pp]) * K + col, nanv);
#pragma unroll
                for (int v = 0; v < V; ++v) part[v] = (T)NAN;
            }
        }
    }
    if (MODE == kPlain) return;
    pcg_block_finish<T, V, G, MODE>(red, part, K, ps, rd);
}

// ---------------------------------------------------------------------------------
// Slab product: every term of a tile's product reaches shared memory as one contiguous
// block by a bulk asynchronous copy -- the tile itself, the tile's low-pattern records,
// the joining-bond partner rows, the wrap partner tile, one block per antiparallel high
// bond, and in the q-launch the tile's rows of r -- through a ring of kSlabSlots slots of
// 32 KB.  One producer warp per block computes each tile's values (tile_meta_warp) once,
// records them beside the tile's first slot, and issues the copies; eight consumer warps
// add the blocks up.  Each consumer thread owns one 16-byte column chunk of up to
// kSlabPasses rows of the tile (G = row bytes / 16 lanes per row), so every shared-memory
// read of a row is G x 16 contiguous bytes: no bank conflicts.  A whole ring of data is in
// flight per SM without holding registers, which is what the L2 needs to deliver rows at
// its gather bandwidth.  The sums are formed in the order of the other work orders (low
// bonds, joining, wrap, high bonds): bitwise equal to them at the same tile width.  Every
// wait is bounded; a timeout stops the producer, drains its copies, and writes NaN to the
// block's remaining output rows (and its PCG partials).  The q-launch variant leaves
// w += alpha p to the direction update.

constexpr int kSlabConsumers = 8;
constexpr int kSlabThreads = 32 * (kSlabConsumers + 1);
constexpr int kSlabPasses = 8;
constexpr int kSlabSlotBytes = 32768;
#ifndef MBL_SLAB_SLOTS
#define MBL_SLAB_SLOTS 6
#endif
constexpr int kSlabSlots = MBL_SLAB_SLOTS;

template <typename T, int K>
struct SlabLayout {
    static constexpr int RB = K * (int)sizeof(T);   // row bytes
    static constexpr int V = 16 / (int)sizeof(T);   // one 16-byte vector per lane
    static constexpr int G = RB / 16;               // lanes per row
    static constexpr int RPW = G > 0 ? 32 / G : 1;  // rows per warp and pass
    static constexpr int RPP = kSlabConsumers * RPW;
    static constexpr int CAP = kSlabPasses * RPP;   // rows of the largest tile: CAP * RB = 32 KB
    static constexpr bool ok = RB >= 32 && RB <= 256 && (RB % 16) == 0 && (32 % (RB / 16)) == 0;
};

// The values of one tile the consumers need, written by the producer with the copy of
// the tile's own rows (published by that copy's mbarrier).
template <typename T>
struct SlabTile {
    uint32_t off, offper;
    int nh;
    T ct;
};

template <typename T, int K, int MODE>
__global__ void __launch_bounds__(kSlabThreads, 1)
    k_apply_slab(ChainParams cp, int B, const T *__restrict__ X, T *__restrict__ Y, T *__restrict__ R,
                 const T *__restrict__ dinv, PcgScalars ps, Reduce rd)
{
    using SL = SlabLayout<T, K>;
    constexpr int V = SL::V, G = SL::G, RPW = SL::RPW, RPP = SL::RPP, P = kSlabPasses;
    constexpr int NS = kSlabSlots;
    static_assert(SL::ok, "slab rows: 32 to 256 bytes");
    extern __shared__ __align__(128) unsigned char slab_raw[];
    __shared__ uint32_t sbin[kBinomDim * kBinomDim];
    __shared__ T tab[1024];
    __shared__ T red[kSlabConsumers + 1][64];
    __shared__ uint32_t spref[kLowMaxB + 2];
    __shared__ T s_alpha[64];
    __shared__ TileMeta<T> s_pmeta;         // the producer's scratch
    __shared__ SlabTile<T> s_tile[NS];      // per slot of a tile's own rows
    __shared__ __align__(8) uint64_t s_full[NS], s_empty[NS];
    __shared__ int s_fail;
    load_binom(sbin);
    build_field_tables<T>(tab, cp);
    if (MODE == kPcgQ && threadIdx.x < K) s_alpha[threadIdx.x] = (T)ps.alpha[threadIdx.x];
    if (threadIdx.x == 0) {
        for (int q = 0; q < NS; ++q) {
            mbar_init(&s_full[q], 1);
            mbar_init(&s_empty[q], kSlabConsumers);
        }
        s_fail = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int q = 0; q <= B + 1 && q <= kLowMaxB + 1; ++q) {
            spref[q] = acc;
            acc += binom(sbin, B, q);
        }
    }
    __syncthreads();

    const int L = cp.L, m = cp.n_up, H = L - B;
    const uint32_t ntile = 1u << H;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int *fail = &s_fail;
    const LowRec *__restrict__ tbl = g_lowtab + lowtab_base(B);
    T part[V];
#pragma unroll
    for (int v = 0; v < V; ++v) part[v] = (T)0;

    if (warp == kSlabConsumers) {
        // producer
        RingPos pos{0u, 0u};
        uint32_t k = 0;
        bool ok = true;
        for (uint32_t t = blockIdx.x; t < ntile && ok; t += gridDim.x) {
            const int p = m - __popc(t);
            if (p < 0 || p > B) continue;  // warp-uniform
            __syncwarp();
            tile_meta_warp<T>(sbin, tab, cp, B, t, p, s_pmeta);
            __syncwarp();
            if (lane == 0) {
                const uint32_t Rt = binom(sbin, B, p), c0 = binom(sbin, B - 1, p);
                const uint32_t sup = p >= 1 ? binom(sbin, B - 1, p - 1) : 0u;
                const uint32_t t0 = t & 1u;
                const uint32_t jcnt = t0 ? c0 : Rt - c0;
                const int64_t jsrc = t0 ? (int64_t)s_pmeta.off - (int64_t)c0 : (int64_t)s_pmeta.off + c0 + sup;
                auto issue = [&](const void *src, uint32_t bytes, bool own) {
                    if (!ok) return;
                    const uint32_t q = pos.s;
                    // the slot's previous use (one lap ago) must have been released
                    if (k >= (uint32_t)NS && !ring_wait(&s_empty[q], pos.ph ^ 1u, fail)) {
                        ok = false;
                        return;
                    }
                    if (own) s_tile[q] = SlabTile<T>{s_pmeta.off, s_pmeta.offper, s_pmeta.nh, s_pmeta.ct};
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(&s_full[q], bytes);
                    bulk_copy_g2s(slab_raw + (size_t)q * kSlabSlotBytes, src, bytes, &s_full[q]);
                    ++k;
                    pos.next((uint32_t)NS);
                };
                issue(X + (int64_t)s_pmeta.off * K, Rt * (uint32_t)SL::RB, true);
                issue(tbl + spref[p], Rt * (uint32_t)sizeof(LowRec), false);
                if (jcnt) issue(X + jsrc * K, jcnt * (uint32_t)SL::RB, false);
                if (cp.periodic && s_pmeta.offper != kNoRow) {
                    const int p2 = m - __popc(t ^ (1u << (H - 1)));
                    issue(X + (int64_t)s_pmeta.offper * K, binom(sbin, B, p2) * (uint32_t)SL::RB, false);
                }
                for (int h = 0; h < s_pmeta.nh; ++h)
                    issue(X + ((int64_t)s_pmeta.off + (int32_t)s_pmeta.shift[h]) * K, Rt * (uint32_t)SL::RB, false);
                if (MODE == kPcgQ) issue(R + (int64_t)s_pmeta.off * K, Rt * (uint32_t)SL::RB, false);
            }
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        }
        if (!ok && lane == 0) {
            // leave no copy in flight: wait (bounded) for the last ring of issued copies
            const uint32_t k0 = k > (uint32_t)NS ? k - (uint32_t)NS : 0u;
            for (uint32_t kk = k0; kk < k; ++kk)
                mbar_wait_bounded(&s_full[kk % (uint32_t)NS], (kk / (uint32_t)NS) & 1u);
        }
    } else {
        // consumers: thread (warp w, row group rw, chunk c) owns rows i * RPP + w * RPW + rw
        const int rw = lane / G, col = (lane % G) * V;
        const T hdelta = cp_half_delta<T>(cp);
        RingPos pos{0u, 0u};
        bool ok = true;
        for (uint32_t t = blockIdx.x; t < ntile; t += gridDim.x) {
            const int p = m - __popc(t);
            if (p < 0 || p > B) continue;  // warp-uniform
            const uint32_t Rt = binom(sbin, B, p), c0 = binom(sbin, B - 1, p);
            const uint32_t t0 = t & 1u, thi = (t >> (H - 1)) & 1u;
            const uint32_t jbase = t0 ? 0u : c0, jcnt = t0 ? c0 : Rt - c0;
            const uint32_t jw0 = (uint32_t)(warp * RPW);
            auto take = [&](const unsigned char *&slot) -> bool {
                slot = slab_raw + (size_t)pos.s * kSlabSlotBytes;
                return __all_sync(0xffffffffu, ring_wait(&s_full[pos.s], pos.ph, fail)) != 0;
            };
            auto give = [&]() {
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_empty[pos.s]);
                pos.next((uint32_t)NS);
            };
            uint32_t off = 0;
            if (ok) {
                const unsigned char *so = nullptr, *sr = nullptr, *sl = nullptr;
                const uint32_t own_slot = pos.s;
                ok = take(so);
                if (ok) {
                    pos.next((uint32_t)NS);
                    ok = take(sr);
                }
                if (ok) {
                    const SlabTile<T> st = s_tile[own_slot];
                    off = st.off;
                    const bool has_wrap = cp.periodic && st.offper != kNoRow;
                    const T *__restrict__ own = reinterpret_cast<const T *>(so);
                    const LowRec *__restrict__ rec = reinterpret_cast<const LowRec *>(sr);
                    T nb[P][V], dx[P][V];
                    uint32_t jper[P];
                    uint32_t wrapbits = 0;
#pragma unroll
                    for (int i = 0; i < P; ++i) {
                        jper[i] = 0;
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            nb[i][v] = (T)0;
                            dx[i][v] = (T)0;
                        }
                        if (i * RPP + jw0 >= Rt) continue;  // warp-uniform
                        const uint32_t j = i * RPP + jw0 + rw;
                        const bool valid = j < Rt;
                        const uint32_t jc = valid ? j : Rt - 1u;
                        const uint4 w0 = reinterpret_cast<const uint4 *>(rec + jc)[0];
                        const uint4 w1 = reinterpret_cast<const uint4 *>(rec + jc)[1];
                        const uint32_t u = w0.x & 0xffffu, cnt = (w0.x >> 16) & 0xffu, alow = w0.x >> 24;
                        const bool join = j - jbase < jcnt;
                        const bool wrap = has_wrap && (u & 1u) != thi;
                        jper[i] = w0.y & 0xffffu;
                        if (valid && wrap) wrapbits |= 1u << i;
                        // in-tile neighbours, to the largest count of the warp's rows
                        const uint32_t nbw[6] = {w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
                        const int cmax = (int)__reduce_max_sync(0xffffffffu, valid ? cnt : 0u);
#pragma unroll
                        for (int q0 = 0; q0 < 12; q0 += 4) {
                            if (q0 >= cmax) break;
                            Vec<T, V> a[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int q = q0 + e;
                                const int qq = q < 12 ? q : 11;
                                const uint32_t jn = (nbw[qq >> 1] >> (16 * (qq & 1))) & 0xffffu;
                                a[e] = ldv<T, V>(own + (int64_t)jn * K + col);
                            }
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (q0 + e < (int)cnt) vadd<T, V>(nb[i], a[e]);
                        }
                        const Vec<T, V> x = ldv<T, V>(own + (int64_t)jc * K + col);
                        const T d = (st.ct + (tab[u & 255u] + tab[256 + (u >> 8)])) -
                                    mul_rn(hdelta, (T)(alow + (join ? 1u : 0u) + (wrap ? 1u : 0u)));
                        if constexpr (sizeof(T) == 4 && V % 2 == 0) {
#pragma unroll
                            for (int v = 0; v < V; v += 2) {
                                const float2 r2 = __fmul2_rn(make_float2(d, d), make_float2(x.v[v], x.v[v + 1]));
                                dx[i][v] = r2.x;
                                dx[i][v + 1] = r2.y;
                            }
                        } else {
#pragma unroll
                            for (int v = 0; v < V; ++v) dx[i][v] = mul_rn(d, x.v[v]);
                        }
                    }
                    // own rows and records are no longer needed
                    {
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&s_empty[own_slot]);
                    }
                    give();
                    if (jcnt && ok) {
                        ok = take(sl);
                        if (ok) {
                            const T *__restrict__ sj = reinterpret_cast<const T *>(sl);
#pragma unroll
                            for (int i = 0; i < P; ++i) {
                                const uint32_t j = i * RPP + jw0 + rw;
                                if (i * RPP + jw0 < Rt && j < Rt && j - jbase < jcnt)
                                    vadd<T, V>(nb[i], ldv<T, V>(sj + (int64_t)(j - jbase) * K + col));
                            }
                            give();
                        }
                    }
                    if (has_wrap && ok) {
                        ok = take(sl);
                        if (ok) {
                            const T *__restrict__ sw = reinterpret_cast<const T *>(sl);
#pragma unroll
                            for (int i = 0; i < P; ++i)
                                if ((wrapbits >> i) & 1u) vadd<T, V>(nb[i], ldv<T, V>(sw + (int64_t)jper[i] * K + col));
                            give();
                        }
                    }
                    for (int h = 0; h < st.nh && ok; ++h) {
                        ok = take(sl);
                        if (ok) {
                            const T *__restrict__ sh = reinterpret_cast<const T *>(sl);
#pragma unroll
                            for (int i = 0; i < P; ++i) {
                                if (i * RPP + jw0 >= Rt) continue;
                                const uint32_t j = i * RPP + jw0 + rw;
                                const uint32_t jc = j < Rt ? j : Rt - 1u;
                                vadd<T, V>(nb[i], ldv<T, V>(sh + (int64_t)jc * K + col));
                            }
                            give();
                        }
                    }
                    const T *__restrict__ srr = nullptr;
                    if (MODE == kPcgQ && ok) {
                        ok = take(sl);
                        srr = reinterpret_cast<const T *>(sl);
                    }
                    if (ok) {
                        T alpha[V];
#pragma unroll
                        for (int v = 0; v < V; ++v) alpha[v] = (MODE == kPcgQ) ? s_alpha[col + v] : (T)0;
#pragma unroll
                        for (int i = 0; i < P; ++i) {
                            const uint32_t j = i * RPP + jw0 + rw;
                            if (i * RPP + jw0 >= Rt || j >= Rt) continue;
                            T acc[V];
                            if constexpr (sizeof(T) == 4 && V % 2 == 0) {
#pragma unroll
                                for (int v = 0; v < V; v += 2) {
                                    const float2 r2 = __ffma2_rn(make_float2(0.5f, 0.5f),
                                                                 make_float2(nb[i][v], nb[i][v + 1]),
                                                                 make_float2(dx[i][v], dx[i][v + 1]));
                                    acc[v] = r2.x;
                                    acc[v + 1] = r2.y;
                                }
                            } else {
#pragma unroll
                                for (int v = 0; v < V; ++v) acc[v] = fma_rn((T)0.5, nb[i][v], dx[i][v]);
                            }
                            const int64_t g = (int64_t)(off + j) * K + col;
                            Vec<T, V> y;
                            if (MODE == kPcgQ) {
                                y = ldv<T, V>(srr + (int64_t)j * K + col);
                                const T dq = dinv[off + j];
#pragma unroll
                                for (int v = 0; v < V; ++v) {
                                    y.v[v] -= alpha[v] * acc[v];
                                    part[v] += y.v[v] * (dq * y.v[v]);
                                }
                                stv<T, V>(R + g, y);
                            } else {
#pragma unroll
                                for (int v = 0; v < V; ++v) y.v[v] = acc[v];
                                if (MODE == kPlain) {
                                    stv_stream<T, V>(Y + g, y);
                                } else {
                                    stv<T, V>(Y + g, y);
#pragma unroll
                                    for (int v = 0; v < V; ++v) part[v] += acc[v] * acc[v];
                                }
                            }
                        }
                        if (MODE == kPcgQ) give();
                    }
                }
            }
            if (!ok) {
                // the ring stopped: this thread's rows of this and every later tile are NaN
                // (the tile's first row comes from the tile index, not from the ring)
                const uint32_t offt = cns_rank(sbin, (t << B) | ((1u << p) - 1u));
                Vec<T, V> nanv;
#pragma unroll
                for (int v = 0; v < V; ++v) nanv.v[v] = (T)NAN;
                T *dst = (MODE == kPcgQ) ? R : Y;
                for (uint32_t j = (uint32_t)(jw0 + rw); j < Rt; j += RPP)
                    stv<T, V>(dst + (int64_t)(offt + j) * K + col, nanv);
#pragma unroll
                for (int v = 0; v < V; ++v) part[v] = (T)NAN;
            }
        }
    }
    if (MODE == kPlain) return;
    pcg_block_finish<T, V, G, MODE, kSlabThreads>(red, part, K, ps, rd);
}

// Host side of the low-pattern table: built once per tile width and copied to the
// device table before the first tiled product of that width on the current device.
static std::mutex g_lowtab_mutex;
static bool g_lowtab_ready[64][kLowMaxB + 1] = {};

uint32_t host_binom(int n, int k);

static int host_colex_rank(uint32_t u)
{
    int r = 0, j = 0;
    for (int pos = 0; pos < 32; ++pos)
        if ((u >> pos) & 1u) {
            ++j;
            r += (int)host_binom(pos, j);
        }
    return r;
}

int ensure_lowtab(int B);

// Every tile width a product of this chain length may use, uploaded before a solve
// captures its iteration into a CUDA graph (the upload is a synchronous copy, which a
// capturing thread must not issue).
int ensure_lowtabs_for(int L)
{
    for (int B = 2; B <= kLowMaxB && B <= L - 2; ++B) {
        const int rc = ensure_lowtab(B);
        if (rc != MBL_OK) return rc;
    }
    return MBL_OK;
}

int ensure_lowtab(int B)
{
    if (B < 2 || B > kLowMaxB) return MBL_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return MBL_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_lowtab_mutex);
    if (g_lowtab_ready[dev][B]) return MBL_OK;
    std::vector<LowRec> recs((size_t)1 << B);
    size_t idx = 0;
    for (int p = 0; p <= B; ++p) {
        // words of popcount p in ascending order: their position is their colex rank
        for (uint32_t u = 0; u < (1u << B); ++u) {
            if (__builtin_popcount(u) != p) continue;
            LowRec rec{};
            rec.u = (uint16_t)u;
            int cnt = 0;
            for (int i = 0; i + 1 < B; ++i) {
                const uint32_t bi = (u >> i) & 1u, bj = (u >> (i + 1)) & 1u;
                if (bi == bj) continue;
                rec.nb[cnt++] = (uint16_t)host_colex_rank(u ^ (3u << i));
            }
            rec.cnt = (uint8_t)cnt;
            rec.alow = (uint8_t)cnt;
            rec.jper = (uint16_t)host_colex_rank(u ^ 1u);
            recs[idx++] = rec;
        }
    }
    if (cudaMemcpyToSymbol(g_lowtab, recs.data(), recs.size() * sizeof(LowRec),
                           (size_t)lowtab_base(B) * sizeof(LowRec)) != cudaSuccess)
        return MBL_ERR_CUDA;
    g_lowtab_ready[dev][B] = true;
    return MBL_OK;
}

// Runtime block width (any 1 <= k <= 256, any alignment): one warp per row, lanes
// stride the columns.  Plain product only.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_apply_generic(ChainParams cp, const T *__restrict__ X,
                                                            int64_t ldx, T *__restrict__ Y, int64_t ldy,
                                                            uint32_t n, int k)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ApplySmem<T> &sm = *reinterpret_cast<ApplySmem<T> *>(smem_raw);
    load_binom(sm.binom);
    build_field_tables<T>(sm.tab, cp);
    __syncthreads();
    const T dconst = (T)cp.diag_const, hdelta = (T)cp.half_delta, half = (T)0.5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nbatch = (n + 31u) / 32u;
    for (uint32_t b = blockIdx.x * kWarps + warp; b < nbatch; b += gridDim.x * kWarps) {
        const uint32_t base = b * 32u;
        {
            const uint32_t r = base + lane;
            int f = -1;
            T d = (T)0;
            if (r < n) {
                uint32_t s = state_of(sm.binom, cp, r);
                d = diag_shifted<T>(sm.tab, dconst, hdelta, cp, s);
                f = row_neighbours<T>(sm.binom, cp, r, s, sm.nb[warp][lane]);
            }
            sm.dsig[warp][lane] = d;
            sm.cnt[warp][lane] = f;
        }
        __syncwarp();
        for (int ri = 0; ri < 32; ++ri) {
            const int f = sm.cnt[warp][ri];
            if (f < 0) break;
            const uint32_t r = base + ri;
            const T d = sm.dsig[warp][ri];
            for (int c = lane; c < k; c += 32) {
                T acc = d * X[(int64_t)r * ldx + c];
                for (int u = 0; u < f; ++u) acc += half * X[(int64_t)sm.nb[warp][ri][u] * ldx + c];
                Y[(int64_t)r * ldy + c] = acc;
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------------
// Elementwise PCG kernels.

// dinv[r] = 1 / ((d(s) - sigma)^2 + f(s)/4): inverse diagonal of A = (H - sigma)^2.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_fold_dinv(ChainParams cp, uint32_t n, T *__restrict__ dinv)
{
    __shared__ uint32_t sb[kBinomDim * kBinomDim];
    __shared__ double tab[1024];
    load_binom(sb);
    build_field_tables<double>(tab, cp);
    __syncthreads();
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        uint32_t s = state_of(sb, cp, r);
        double d = diag_shifted<double>(tab, cp.diag_const, cp.half_delta, cp, s);
        int f = __popc((s ^ (s >> 1)) & cp.open_mask);
        if (cp.periodic) f += (int)(((s >> (cp.L - 1)) ^ s) & 1u);
        dinv[r] = (T)(1.0 / (d * d + 0.25 * (double)f));
    }
}

// Gershgorin bound max_s |d(s)| + f(s)/2 of ||H||: per-block maxima, last block folds.
__global__ void __launch_bounds__(kThreads) k_gershgorin(ChainParams cp, uint32_t n, Reduce rd, double *out)
{
    __shared__ uint32_t sb[kBinomDim * kBinomDim];
    __shared__ double tab[1024];
    __shared__ double s_red[kThreads];
    __shared__ unsigned s_last;
    load_binom(sb);
    build_field_tables<double>(tab, cp);
    __syncthreads();
    double m = 0.0;
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        uint32_t s = state_of(sb, cp, r);
        double d = diag_shifted<double>(tab, cp.diag_const, cp.half_delta, cp, s);  // sigma = 0 here
        int f = __popc((s ^ (s >> 1)) & cp.open_mask);
        if (cp.periodic) f += (int)(((s >> (cp.L - 1)) ^ s) & 1u);
        m = fmax(m, fabs(d) + 0.5 * (double)f);
    }
    s_red[threadIdx.x] = m;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s_red[threadIdx.x] = fmax(s_red[threadIdx.x], s_red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) rd.partials[blockIdx.x] = s_red[0];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(rd.counter, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x == 0) {
        double g = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) g = fmax(g, rd.partials[b]);
        *out = g;
        *rd.counter = 0u;
    }
}

// PCG start: r = b_j / ||b_j|| (b = FP64 residual block, norms given), p = dinv r,
// w = 0; finish rz = r.(dinv r), rz0 = rz, active = rz > 0.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_pcg_init(const double *__restrict__ B, int64_t ldb,
                                                       const double *__restrict__ bnorm, uint32_t n, int k,
                                                       const T *__restrict__ dinv, T *__restrict__ r,
                                                       T *__restrict__ p, T *__restrict__ w, PcgScalars ps,
                                                       Reduce rd)
{
    // thread layout: column c = threadIdx.x % k (k divides 256 when k is a power of two;
    // otherwise threads with c >= ... still map columns in a round-robin way)
    __shared__ double s_part[kThreads];
    __shared__ unsigned s_last;
    const int per = kThreads / k;  // rows per block-iteration
    const int c = threadIdx.x % k, ro = threadIdx.x / k;
    double acc = 0.0;
    if (ro < per) {
        const double inv = bnorm[c] > 0.0 ? 1.0 / bnorm[c] : 0.0;
        for (uint32_t row = blockIdx.x * per + ro; row < n; row += gridDim.x * per) {
            T rv = (T)(B[(int64_t)row * ldb + c] * inv);
            T zv = dinv[row] * rv;
            r[(int64_t)row * k + c] = rv;
            p[(int64_t)row * k + c] = zv;
            w[(int64_t)row * k + c] = (T)0;
            acc += (double)(rv * zv);
        }
    }
    s_part[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < k) {
        double t = 0.0;
        for (int q = 0; q < per; ++q) t += s_part[q * k + threadIdx.x];
        rd.partials[(int64_t)blockIdx.x * k + threadIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(rd.counter, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    __shared__ double s_tot[64];
    finish_column_sums(rd, k, s_tot);
    if (threadIdx.x < k) {
        double rz = s_tot[threadIdx.x];
        ps.rz[threadIdx.x] = rz;
        ps.rz0[threadIdx.x] = rz;
        ps.alpha[threadIdx.x] = 0.0;
        ps.beta[threadIdx.x] = 0.0;
        ps.active[threadIdx.x] = (rz > 0.0 && isfinite(rz)) ? 1 : 0;
    }
}

// PCG direction update: w += alpha p_old; p = dinv r + beta p_old (per column scalars).
// Each thread takes kUpdRows rows of one block slice and requests all their loads before
// any arithmetic, so that several rows per thread are in flight.
constexpr int kUpdRows = 4;
template <typename T, int K, bool WDONE>
__global__ void __launch_bounds__(kThreads) k_pcg_update(uint32_t n, const T *__restrict__ dinv,
                                                         const T *__restrict__ r, T *__restrict__ p,
                                                         T *__restrict__ w, PcgScalars ps)
{
    using Lay = RowLayout<T, K>;
    constexpr int V = Lay::V, G = Lay::G;
    const int col = (threadIdx.x % G) * V;
    T a[V], bt[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        a[v] = (T)ps.alpha[col + v];
        bt[v] = (T)ps.beta[col + v];
    }
    const uint32_t rows_per_block = kThreads / G;
    const uint64_t stride = (uint64_t)gridDim.x * rows_per_block * kUpdRows;
    for (uint64_t base = (uint64_t)blockIdx.x * rows_per_block * kUpdRows + threadIdx.x / G; base < n;
         base += stride) {
        Vec<T, V> rv[kUpdRows], pv[kUpdRows], wv[kUpdRows];
        T di[kUpdRows];
#pragma unroll
        for (int q = 0; q < kUpdRows; ++q) {
            const uint64_t row = base + (uint64_t)q * rows_per_block;
            const int64_t o = (int64_t)(row < n ? row : n - 1) * K + col;  // a valid row; stored only if < n
            rv[q] = ldv<T, V>(r + o);
            pv[q] = ldv<T, V>(p + o);
            if (!WDONE) wv[q] = ldv<T, V>(w + o);
            di[q] = dinv[row < n ? row : n - 1];
        }
#pragma unroll
        for (int q = 0; q < kUpdRows; ++q) {
            const uint64_t row = base + (uint64_t)q * rows_per_block;
            if (row >= n) continue;
            const int64_t o = (int64_t)row * K + col;
            if (!WDONE) {  // else the q-launch has done w += alpha p
#pragma unroll
                for (int v = 0; v < V; ++v) wv[q].v[v] += a[v] * pv[q].v[v];
                stv<T, V>(w + o, wv[q]);
            }
            Vec<T, V> pn;
#pragma unroll
            for (int v = 0; v < V; ++v) pn.v[v] = di[q] * rv[q].v[v] + bt[v] * pv[q].v[v];
            stv<T, V>(p + o, pn);
        }
    }
}

// ---------------------------------------------------------------------------------
// Batched PCG step (Sec. 3.1: realizations are independent): one launch covers the PCG
// phase of many problems ("lanes"), each with its own chain, sector size, tile width,
// vectors and per-column scalars, read from a table in device memory.  A lane's work
// items are those of the persistent tiled product (a chunk of rows of one tile); the
// items of all lanes form rounds of kWarps items, lane after lane, and each block takes a
// contiguous run of rounds, so a block meets few lanes and rebuilds its shared tables
// (chain constants, field tables) only when the lane changes.  Each round's column
// partials (t.t or r.M^-1 r, compensated FP32 pairs in FP32) go to the lane's partials
// by round; the block that completes a lane's last round sums them in round order and
// finishes alpha or beta exactly as the single-problem launches do, so the results do not
// depend on which block ran which round.  The row pass is the shared tile_row_pass.


// Last lane whose first round (or row) is <= x: lanes are ordered by both.
__device__ __forceinline__ int lane_of(const PcgLane *__restrict__ lanes, int nlanes, uint32_t x, bool by_row)
{
    int lo = 0, hi = nlanes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const uint32_t v = by_row ? __ldg(&lanes[mid].row0) : __ldg(&lanes[mid].round0);
        if (v <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename T, int K, int MODE, int LB>
__global__ void __launch_bounds__(kThreads, MBL_TILED_MIN_BLOCKS)
    k_pcg_batch(const PcgLane *__restrict__ lanes, int nlanes, uint32_t total_rounds)
{
    using Lay = WideRowLayout<T, K, LB>;
    constexpr int V = Lay::V, G = Lay::G, RPW = 32 / G, CH = Lay::CH;
    constexpr int NBr = 128 / (V * (int)sizeof(T));
    constexpr int NB = NBr < 2 ? 2 : (NBr > 8 ? 8 : NBr);
    __shared__ uint32_t sbin[kBinomDim * kBinomDim];
    __shared__ T tab[1024];
    __shared__ T red[kWarps][64];
    __shared__ uint32_t spref[kLowMaxB + 2];
    __shared__ T s_alpha[64];
    __shared__ TileMeta<T> s_meta[kWarps];
    __shared__ ChainParams s_cp;
    __shared__ int s_lane;
    __shared__ unsigned s_last;
    load_binom(sbin);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane / G;
    const int col = (lane % G) * V;
    const uint32_t r_begin = (uint32_t)(((uint64_t)total_rounds * blockIdx.x) / gridDim.x);
    const uint32_t r_end = (uint32_t)(((uint64_t)total_rounds * (blockIdx.x + 1)) / gridDim.x);
    int cur = -1;
    for (uint32_t round = r_begin; round < r_end; ++round) {
        if (threadIdx.x == 0) s_lane = lane_of(lanes, nlanes, round, false);
        __syncthreads();
        const int li = s_lane;
        const PcgLane &Ln = lanes[li];
        if (li != cur) {
            // the lane's chain constants, field tables, tile-row prefix and alpha
            const int *src = reinterpret_cast<const int *>(&Ln.cp);
            int *dst = reinterpret_cast<int *>(&s_cp);
            for (int i = threadIdx.x; i < (int)(sizeof(ChainParams) / sizeof(int)); i += kThreads) dst[i] = src[i];
            __syncthreads();
            build_field_tables<T>(tab, s_cp);
            if (MODE == kPcgQ && threadIdx.x < K) s_alpha[threadIdx.x] = (T)Ln.alpha[threadIdx.x];
            if (threadIdx.x == 0) {
                const int B = Ln.B;
                uint32_t acc = 0;
                for (int q = 0; q <= B + 1 && q <= kLowMaxB + 1; ++q) {
                    spref[q] = acc;
                    acc += binom(sbin, B, q);
                }
            }
            __syncthreads();
            cur = li;
        }
        const ChainParams &cp = s_cp;
        const int B = Ln.B;
        const int L = cp.L, m = cp.n_up, H = L - B;
        const uint32_t nchunk = (binom(sbin, B, B / 2) + CH - 1) / CH;
        const T hdelta = cp_half_delta<T>(cp);
        T *__restrict__ X = (T *)(MODE == kPcgT ? Ln.p : Ln.t);
        T *__restrict__ Y = (T *)(MODE == kPcgT ? Ln.t : nullptr);
        T *__restrict__ R = (T *)(MODE == kPcgQ ? Ln.r : nullptr);
        const T *__restrict__ dinv = (const T *)Ln.dinv;
        T part[V];
#pragma unroll
        for (int v = 0; v < V; ++v) part[v] = (T)0;
        const uint32_t item = (round - Ln.round0) * kWarps + warp;
        if (item < Ln.items) {
            const uint32_t t = item / nchunk, c = item % nchunk;
            const int p = m - __popc(t);
            const uint32_t Rt = (p >= 0 && p <= B) ? binom(sbin, B, p) : 0u;
            const uint32_t j_begin = c * CH;
            if (j_begin < Rt) {  // warp-uniform
                const uint32_t j_end = min(Rt, j_begin + CH);
                TileMeta<T> &tm = s_meta[warp];
                __syncwarp();
                tile_meta_warp<T>(sbin, tab, cp, B, t, p, tm);
                __syncwarp();
                const uint32_t t0 = t & 1u, thi = (t >> (H - 1)) & 1u;
                const uint32_t sup = p >= 1 ? binom(sbin, B - 1, p - 1) : 0u;
                const uint32_t sdn = binom(sbin, B - 1, p);
                const LowRec *__restrict__ rp = g_lowtab + lowtab_base(B) + spref[p];
                const T *__restrict__ Xt = X + (int64_t)tm.off * K;
                for (uint32_t j0 = j_begin; j0 < j_end; j0 += RPW) {
                    const uint32_t j = j0 + grp;
                    tile_row_pass<T, V, NB, MODE>(cp, B, X, K, Xt, K, rp, min(j, j_end - 1u), j < j_end, tm, tab,
                                                  hdelta, t0, thi, sup, sdn, col, Y, K, R, dinv, s_alpha, part,
                                                  nullptr, nullptr);
                }
            }
        }
        // this round's column partials -> the lane's partial slot of the round
#pragma unroll
        for (int v = 0; v < V; ++v)
            for (int off = G; off < 32; off <<= 1) part[v] += __shfl_xor_sync(0xffffffffu, part[v], off);
        if (lane < G) {
#pragma unroll
            for (int v = 0; v < V; ++v) red[warp][lane * V + v] = part[v];
        }
        __syncthreads();
        const uint32_t slot = round - Ln.round0;
        if (threadIdx.x < K) {
            if constexpr (sizeof(T) == 4) {
                float sum = 0.0f, cmp = 0.0f;
                for (int w = 0; w < kWarps; ++w) {
                    float hi, e;
                    two_sum(sum, red[w][threadIdx.x], hi, e);
                    sum = hi;
                    cmp += e;
                }
                reinterpret_cast<float2 *>(Ln.partials)[(int64_t)slot * K + threadIdx.x] = make_float2(sum, cmp);
            } else {
                double acc = 0.0;
                for (int w = 0; w < kWarps; ++w) acc += (double)red[w][threadIdx.x];
                Ln.partials[(int64_t)slot * K + threadIdx.x] = acc;
            }
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = (atomicAdd(Ln.counter, 1u) == Ln.nrounds - 1) ? 1u : 0u;
        __syncthreads();
        if (s_last) {
            // this block finished the lane's last round: sum the rounds in order
            __threadfence();
            if (threadIdx.x < K) {
                double tot;
                if constexpr (sizeof(T) == 4) {
                    const float2 *pp = reinterpret_cast<const float2 *>(Ln.partials);
                    float S = 0.0f, C = 0.0f;
                    for (uint32_t q = 0; q < Ln.nrounds; ++q) {
                        const float2 v2 = pp[(int64_t)q * K + threadIdx.x];
                        float hi, e;
                        two_sum(S, v2.x, hi, e);
                        S = hi;
                        C += e + v2.y;
                    }
                    tot = (double)S + (double)C;
                } else {
                    double S = 0.0;
                    for (uint32_t q = 0; q < Ln.nrounds; ++q) S += Ln.partials[(int64_t)q * K + threadIdx.x];
                    tot = S;
                }
                const int cc = threadIdx.x;
                if (MODE == kPcgT) {
                    const bool ok = Ln.active[cc] && tot > 0.0 && isfinite(tot);
                    Ln.alpha[cc] = ok ? Ln.rz[cc] / tot : 0.0;
                } else {
                    int act = Ln.active[cc];
                    if (!isfinite(tot)) act = 0;
                    if (Ln.tol2 > 0.0 && tot <= Ln.tol2 * Ln.rz0[cc]) act = 0;
                    Ln.beta[cc] = (act && Ln.rz[cc] > 0.0) ? tot / Ln.rz[cc] : 0.0;
                    if (!act) Ln.alpha[cc] = 0.0;
                    Ln.active[cc] = act;
                    Ln.rz[cc] = tot;
                }
            }
            if (threadIdx.x == 0) *Ln.counter = 0u;
        }
    }
}

// Batched direction update: w += alpha p, p = M^-1 r + beta p for every lane's rows (the
// lanes' rows concatenated; each thread takes kUpdRows rows, loads first).
template <typename T, int K>
__global__ void __launch_bounds__(kThreads) k_pcg_batch_update(const PcgLane *__restrict__ lanes, int nlanes,
                                                               uint32_t total_rows)
{
    using Lay = RowLayout<T, K>;
    constexpr int V = Lay::V, G = Lay::G;
    const int col = (threadIdx.x % G) * V;
    const uint32_t rows_per_block = kThreads / G;
    const uint64_t stride = (uint64_t)gridDim.x * rows_per_block * kUpdRows;
    for (uint64_t base = (uint64_t)blockIdx.x * rows_per_block * kUpdRows + threadIdx.x / G; base < total_rows;
         base += stride) {
        Vec<T, V> rv[kUpdRows], pv[kUpdRows], wv[kUpdRows];
        T di[kUpdRows];
        int li[kUpdRows];
        int64_t o[kUpdRows];
#pragma unroll
        for (int q = 0; q < kUpdRows; ++q) {
            uint64_t row = base + (uint64_t)q * rows_per_block;
            if (row >= total_rows) row = total_rows - 1;  // a valid row; stored only if in range
            li[q] = lane_of(lanes, nlanes, (uint32_t)row, true);
            const PcgLane &Ln = lanes[li[q]];
            const uint32_t lr = (uint32_t)row - Ln.row0;
            o[q] = (int64_t)lr * K + col;
            rv[q] = ldv<T, V>((const T *)Ln.r + o[q]);
            pv[q] = ldv<T, V>((const T *)Ln.p + o[q]);
            wv[q] = ldv<T, V>((const T *)Ln.w + o[q]);
            di[q] = ((const T *)Ln.dinv)[lr];
        }
#pragma unroll
        for (int q = 0; q < kUpdRows; ++q) {
            if (base + (uint64_t)q * rows_per_block >= total_rows) continue;
            const PcgLane &Ln = lanes[li[q]];
            Vec<T, V> pn;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const T a = (T)Ln.alpha[col + v], bt = (T)Ln.beta[col + v];
                wv[q].v[v] += a * pv[q].v[v];
                pn.v[v] = di[q] * rv[q].v[v] + bt * pv[q].v[v];
            }
            stv<T, V>((T *)Ln.w + o[q], wv[q]);
            stv<T, V>((T *)Ln.p + o[q], pn);
        }
    }
}

// Generic-k version of the PCG product kernels (one warp per row, lanes stride the
// columns, k <= 64).
template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_apply_pcg_generic(ChainParams cp, const T *__restrict__ X,
                                                                T *__restrict__ Y, uint32_t n, int k,
                                                                T *__restrict__ R, const T *__restrict__ dinv,
                                                                PcgScalars ps, Reduce rd)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ApplySmem<T> &sm = *reinterpret_cast<ApplySmem<T> *>(smem_raw);
    load_binom(sm.binom);
    build_field_tables<T>(sm.tab, cp);
    __syncthreads();
    const T dconst = (T)cp.diag_const, hdelta = (T)cp.half_delta, half = (T)0.5;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T part[2] = {(T)0, (T)0};
    const uint32_t nbatch = (n + 31u) / 32u;
    for (uint32_t b = blockIdx.x * kWarps + warp; b < nbatch; b += gridDim.x * kWarps) {
        const uint32_t base = b * 32u;
        {
            const uint32_t r = base + lane;
            int f = -1;
            T d = (T)0;
            if (r < n) {
                uint32_t s = state_of(sm.binom, cp, r);
                d = diag_shifted<T>(sm.tab, dconst, hdelta, cp, s);
                f = row_neighbours<T>(sm.binom, cp, r, s, sm.nb[warp][lane]);
            }
            sm.dsig[warp][lane] = d;
            sm.cnt[warp][lane] = f;
        }
        __syncwarp();
        for (int ri = 0; ri < 32; ++ri) {
            const int f = sm.cnt[warp][ri];
            if (f < 0) break;
            const uint32_t r = base + ri;
            const T d = sm.dsig[warp][ri];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int c = lane + 32 * h;
                if (c >= k) break;
                T acc = d * X[(int64_t)r * k + c];
                for (int u = 0; u < f; ++u) acc += half * X[(int64_t)sm.nb[warp][ri][u] * k + c];
                if (MODE == kPcgT) {
                    Y[(int64_t)r * k + c] = acc;
                    part[h] += acc * acc;
                } else {
                    T rv = R[(int64_t)r * k + c] - (T)ps.alpha[c] * acc;
                    R[(int64_t)r * k + c] = rv;
                    part[h] += rv * (dinv[r] * rv);
                }
            }
        }
        __syncwarp();
    }
    // block reduction: columns c = lane + 32h
    if (lane < 32) {
#pragma unroll
        for (int h = 0; h < 2; ++h) sm.red[warp][lane + 32 * h] = part[h];
    }
    __syncthreads();
    if (threadIdx.x < k) {
        double acc = 0.0;
        for (int w = 0; w < kWarps; ++w) acc += (double)sm.red[w][threadIdx.x];
        rd.partials[(int64_t)blockIdx.x * k + threadIdx.x] = acc;
    }
    __threadfence();
    __shared__ unsigned s_last;
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(rd.counter, 1u) == gridDim.x - 1) ? 1u : 0u;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    __shared__ double s_tot[64];
    finish_column_sums(rd, k, s_tot);
    if (threadIdx.x < k) {
        const int c = threadIdx.x;
        if (MODE == kPcgT) {
            double tt = s_tot[c];
            bool ok = ps.active[c] && tt > 0.0 && isfinite(tt);
            ps.alpha[c] = ok ? ps.rz[c] / tt : 0.0;
        } else {
            double rzn = s_tot[c];
            int act = ps.active[c];
            if (!isfinite(rzn)) act = 0;
            if (ps.tol2 > 0.0 && rzn <= ps.tol2 * ps.rz0[c]) act = 0;
            ps.beta[c] = (act && ps.rz[c] > 0.0) ? rzn / ps.rz[c] : 0.0;
            if (!act) ps.alpha[c] = 0.0;
            ps.active[c] = act;
            ps.rz[c] = rzn;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_pcg_update_generic(uint32_t n, int k, const T *__restrict__ dinv,
                                                                 const T *__restrict__ r, T *__restrict__ p,
                                                                 T *__restrict__ w, PcgScalars ps)
{
    const int64_t total = (int64_t)n * k;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e % k);
        const uint32_t row = (uint32_t)(e / k);
        T pv = p[e];
        w[e] += (T)ps.alpha[c] * pv;
        p[e] = dinv[row] * r[e] + (T)ps.beta[c] * pv;
    }
}

// ---------------------------------------------------------------------------------
// Host-side dispatch.

static std::atomic<int> g_num_sms{0};

int num_sms()
{
    if (g_num_sms.load() == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
        g_num_sms.store(v);
    }
    return g_num_sms.load();
}

int make_chain_params(const mbl_chain *chain, double sigma, ChainParams *cp)
{
    if (!chain || !chain->h_host) return MBL_ERR_ARG;
    const int L = chain->L;
    if (L < 2 || L > kMaxL || chain->n_up < 0 || chain->n_up > L) return MBL_ERR_ARG;
    if (!std::isfinite(chain->delta) || !std::isfinite(sigma)) return MBL_ERR_ARG;
    ChainParams p{};
    p.L = L;
    p.n_up = chain->n_up;
    p.periodic = (chain->periodic && L > 2) ? 1 : 0;
    p.nbonds = (L - 1) + p.periodic;
    p.open_mask = (L - 1 >= 32) ? 0xffffffffu : ((1u << (L - 1)) - 1u);
    double hsum = 0.0;
    for (int i = 0; i < L; ++i) {
        double hi = chain->h_host[i];
        if (!std::isfinite(hi)) return MBL_ERR_ARG;
        p.h[i] = hi;
        hsum += hi;
    }
    p.half_delta = 0.5 * chain->delta;
    p.diag_const = 0.25 * chain->delta * (double)p.nbonds - 0.5 * hsum - sigma;
    for (int i = 0; i < L; ++i) {
        p.h_hi[i] = (float)p.h[i];
        p.h_lo[i] = (float)(p.h[i] - (double)p.h_hi[i]);
    }
    p.half_delta_f = (float)p.half_delta;
    p.diag_const_f = (float)p.diag_const;
    *cp = p;
    return MBL_OK;
}

template <typename T>
static size_t apply_smem_bytes()
{
    return sizeof(ApplySmem<T>);
}

template <typename T, int K, int MODE>
static cudaError_t launch_apply_k(const ChainParams &cp, const T *X, int64_t ldx, T *Y, int64_t ldy, uint32_t n,
                                  T *R, const T *dinv, const PcgScalars &ps, const Reduce &rd, int grid,
                                  cudaStream_t st)
{
    auto kern = k_apply<T, K, MODE>;
    const size_t sm = apply_smem_bytes<T>();
    static const bool attr_set_once = [&]() {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        return true;
    }();
    (void)attr_set_once;
    note_launch();
    kern<<<grid, kThreads, sm, st>>>(cp, X, ldx, Y, ldy, n, R, dinv, ps, rd);
    return cudaGetLastError();
}

// ---- tiled product dispatch ----------------------------------------------------

// Tile width override per (block width, element size): 0 = heuristic, -1 = untiled,
// >= 2 = that many low bits.  Set by the autotuner.
static int g_tile_bits[2][8] = {};
static int g_lane_bytes[2][8] = {};  // 0: default (32), else 16, 32 or 64
static int g_schedule[2][8] = {};    // 0: by size, 1: persistent, 2: ordered, 3: staged

static int kslot(int K)
{
    switch (K) {
    case 1: return 0;
    case 2: return 1;
    case 4: return 2;
    case 8: return 3;
    case 16: return 4;
    case 32: return 5;
    case 64: return 6;
    default: return 7;
    }
}

uint32_t host_binom(int n, int k)
{
    if (k < 0 || k > n) return 0;
    uint64_t c = 1;
    for (int i = 1; i <= k; ++i) c = c * (uint64_t)(n - k + i) / (uint64_t)i;
    return (uint32_t)c;
}

// Tile width heuristic: the widest table-backed tiles (B = 13, at most L - 2 so that two
// high bits remain); measured fastest or within a few per cent of it for L = 20..26,
// k = 8..64 (wider tiles leave more bonds inside the tile).
static int heuristic_tile_bits(int L, int K, size_t es)
{
    (void)K;
    (void)es;
    int B = kLowMaxB;
    if (B > L - 2) B = L - 2;
    return B >= 2 ? B : -1;
}

int tile_bits_for(int L, int K, size_t es)
{
    if (L < 4) return -1;
    const int o = g_tile_bits[es == 8 ? 1 : 0][kslot(K)];
    if (o == -1) return -1;
    int B = (o >= 2) ? o : heuristic_tile_bits(L, K, es);
    if (B > kLowMaxB) B = kLowMaxB;
    if (B > L - 2) B = L - 2;
    return B >= 2 ? B : -1;
}

void set_tile_bits(int K, size_t es, int bits) { g_tile_bits[es == 8 ? 1 : 0][kslot(K)] = bits; }
void set_lane_bytes(int K, size_t es, int bytes) { g_lane_bytes[es == 8 ? 1 : 0][kslot(K)] = bytes; }
void set_schedule(int K, size_t es, int mode) { g_schedule[es == 8 ? 1 : 0][kslot(K)] = mode; }

// Per-(element size, block width, L) choices written by the autotuner; 0 = not tuned.
// An explicit tuning switch (g_schedule, g_lane_bytes) takes precedence; during a
// tuning run the candidate under test is forced on the tuning thread.
struct ProductTune {
    int schedule, lane;
};
static ProductTune g_tuned[2][8][kMaxL + 1] = {};
static std::mutex g_tune_mutex;
static thread_local int t_force_schedule = 0, t_force_lane = 0;

// Work order of a plain tiled product.  Persistent: a grid of a few blocks per SM, each
// warp striding over the (tile, chunk) items.  Ordered: one item per warp and as many
// blocks as needed, so the hardware hands out blocks in index order and the tiles in
// flight stay a narrow, advancing window; with the grid-stride loop, warps that meet
// many empty chunks run ahead and the window widens beyond L2.  Every block of the
// ordered grid repeats the shared-memory setup, so it only pays for wide rows: measured
// on GB300, ordered wins for rows of >= 256 bytes once the block vector is >= 1 GiB
// (FP32), or >= 128 MiB in FP64 (ALU-bound there), and loses elsewhere.
// The staged schedule (whole tiles in shared memory) is the default for 128-byte rows
// once the block vector outgrows 16 MB (measured: 2-6 % faster there, slower for
// narrower and wider rows); anything else defaults to persistent.
static int size_schedule(int L, int n_up, int K, size_t es)
{
    const double bytes = (double)host_binom(L, n_up) * K * (double)es;
    if (K * (int)es >= 256 && bytes >= (es == 8 ? 128.0 * (1 << 20) : 1024.0 * (1 << 20))) return 2;
    if (K * (int)es == 128 && bytes >= 16.0 * (1 << 20)) return 3;
    return 1;
}

static int schedule_for(int L, int n_up, int K, size_t es)
{
    if (t_force_schedule) return t_force_schedule;
    const int o = g_schedule[es == 8 ? 1 : 0][kslot(K)];
    if (o) return o;
    const int a = (L >= 0 && L <= kMaxL) ? g_tuned[es == 8 ? 1 : 0][kslot(K)][L].schedule : 0;
    if (a) return a;
    return size_schedule(L, n_up, K, es);
}
static bool ordered_schedule(int L, int n_up, int K, size_t es) { return schedule_for(L, n_up, K, es) == 2; }

// 32-byte lanes by default; 64-byte lanes for FP64 rows of >= 128 bytes (measured 13 %
// faster: the FP64 products are ALU-bound and wider lanes repeat less index work).
static int size_lane_bytes(int K, size_t es) { return (es == 8 && K * (int)es >= 128) ? 64 : 32; }

static int lane_bytes_for(int L, int K, size_t es)
{
    if (t_force_lane) return t_force_lane;
    const int v = g_lane_bytes[es == 8 ? 1 : 0][kslot(K)];
    if (v == 16 || v == 32 || v == 64) return v;
    const int a = (L >= 0 && L <= kMaxL) ? g_tuned[es == 8 ? 1 : 0][kslot(K)][L].lane : 0;
    if (a) return a;
    return size_lane_bytes(K, es);
}

template <typename T, int K, int MODE, int LB>
static cudaError_t launch_tiled_lb(const ChainParams &cp, int B, const T *X, int64_t ldx, T *Y, int64_t ldy, T *R,
                                   const T *dinv, const PcgScalars &ps, const Reduce &rd, cudaStream_t st)
{
    if (ensure_lowtab(B) != MBL_OK) return cudaErrorUnknown;
    auto kern = k_apply_tiled<T, K, MODE, LB>;
    static const int per_sm = [&]() {
        int v = 0;
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 25);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, kThreads, 0) != cudaSuccess || v < 1) v = 1;
        return v;
    }();
    const uint32_t rmax = host_binom(B, B / 2);
    constexpr int CH = WideRowLayout<T, K, LB>::CH;
    const int64_t items = ((int64_t)1 << (cp.L - B)) * (int64_t)((rmax + CH - 1) / CH);
    int64_t grid = (int64_t)num_sms() * per_sm;
    if (grid > (int64_t)num_sms() * 8) grid = (int64_t)num_sms() * 8;  // partials capacity
    const int64_t need = (items + kWarps - 1) / kWarps;
    // the ordered schedule (one item per warp) only for the plain product: the PCG
    // epilogues keep one partial per block in a buffer sized for the persistent grid
    if (MODE == kPlain && ordered_schedule(cp.L, cp.n_up, K, sizeof(T))) grid = need;
    note_launch();
    if (grid > need) grid = need;
    kern<<<(int)grid, kThreads, 0, st>>>(cp, B, X, ldx, Y, ldy, R, dinv, ps, rd);
    return cudaGetLastError();
}

// Tile width of the staged kernel: the widest table-backed B (<= L - 2) whose largest
// tile, C(B, B/2) rows, fits in the shared-memory stage.
static int staged_bits(int L, int K, size_t es)
{
    int B = kLowMaxB < L - 2 ? kLowMaxB : L - 2;
    while (B >= 2 && (size_t)host_binom(B, B / 2) * K * es > (size_t)kStageBytes) --B;
    return B;
}

static bool staged_schedule(int L, int n_up, int K, size_t es) { return schedule_for(L, n_up, K, es) == 3; }

template <typename T, int K, int MODE, int LB>
static cudaError_t launch_staged_lb(const ChainParams &cp, int Bs, const T *X, T *Y, T *R, const T *dinv,
                                    const PcgScalars &ps, const Reduce &rd, cudaStream_t st)
{
    if (ensure_lowtab(Bs) != MBL_OK) return cudaErrorUnknown;
    auto kern = k_apply_staged<T, K, MODE, LB>;
    static const int per_sm = [&]() {
        int v = 0;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kStageBytes);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, kThreads, kStageBytes) != cudaSuccess || v < 1)
            v = 1;
        return v;
    }();
    const size_t dyn = (size_t)host_binom(Bs, Bs / 2) * K * sizeof(T);
    const int64_t ntile = (int64_t)1 << (cp.L - Bs);
    int64_t grid = (int64_t)num_sms() * per_sm;
    if (grid > (int64_t)num_sms() * 8) grid = (int64_t)num_sms() * 8;  // partials capacity
    if (grid > ntile) grid = ntile;
    note_launch();
    kern<<<(int)grid, kThreads, dyn, st>>>(cp, Bs, X, Y, R, dinv, ps, rd);
    return cudaGetLastError();
}

static bool streamed_schedule(int L, int n_up, int K, size_t es) { return schedule_for(L, n_up, K, es) == 4; }

// Dynamic shared memory a streamed block can have next to the kernel's static arrays.
template <typename T, int K, int MODE>
static size_t stream_ring_capacity()
{
    static const size_t cap = []() {
        auto kern = k_apply_streamed<T, K, MODE>;
        cudaFuncAttributes fa{};
        int dev = 0, optin = 0, per_sm = 0, reserved = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, kern) != cudaSuccess)
            return (size_t)0;
        // kStreamBlocks blocks share the SM's shared memory
        size_t block = (size_t)per_sm / kStreamBlocks;
        block = block > (size_t)reserved ? block - (size_t)reserved : 0;
        if (block > (size_t)optin) block = (size_t)optin;
        const size_t avail = block > fa.sharedSizeBytes ? block - fa.sharedSizeBytes : 0;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)avail) != cudaSuccess)
            return (size_t)0;
        return avail;
    }();
    return cap;
}

// Tile width of the streamed kernel: the widest table-backed B (<= L - 2) whose largest
// tile the consumer warps cover and whose ring still holds MBL_STREAM_MIN_SLOTS tiles.
static int stream_bits_for(int L, int K, size_t es, size_t ring_bytes, int cap_rows)
{
    int B = kLowMaxB < L - 2 ? kLowMaxB : L - 2;
    for (; B >= 2; --B) {
        const size_t rows = host_binom(B, B / 2);
        if (rows > (size_t)cap_rows) continue;
        if (ring_bytes / (rows * K * es) >= (size_t)MBL_STREAM_MIN_SLOTS) return B;
    }
    return -1;
}

template <typename T, int K>
static int stream_bits(int L)
{
    using SL = StreamLayout<T, K>;
    if constexpr (!SL::ok) {
        return -1;
    } else {
        return stream_bits_for(L, K, sizeof(T), stream_ring_capacity<T, K, kPlain>(), SL::CAP);
    }
}

template <typename T, int K, int MODE>
static cudaError_t launch_streamed(const ChainParams &cp, int Bs, const T *X, T *Y, T *R, const T *dinv,
                                   const PcgScalars &ps, const Reduce &rd, cudaStream_t st)
{
    if (ensure_lowtab(Bs) != MBL_OK) return cudaErrorUnknown;
    const size_t avail = stream_ring_capacity<T, K, MODE>();
    const size_t slot = (size_t)host_binom(Bs, Bs / 2) * K * sizeof(T);
    int nbuf = (int)(avail / slot);
    if (nbuf > kMaxSlots) nbuf = kMaxSlots;
    if (nbuf < 4) return cudaErrorInvalidConfiguration;
    const int64_t ntile = (int64_t)1 << (cp.L - Bs);
    int64_t grid = (int64_t)num_sms() * kStreamBlocks;
    if (grid > ntile) grid = ntile;
    note_launch();
    k_apply_streamed<T, K, MODE><<<(int)grid, kThreads, (size_t)nbuf * slot, st>>>(cp, Bs, nbuf, X, Y, R, dinv, ps,
                                                                                   rd);
    return cudaGetLastError();
}

static bool slab_schedule(int L, int n_up, int K, size_t es) { return schedule_for(L, n_up, K, es) == 5; }

// Tile width of the slab kernel: the widest table-backed B (<= L - 2) whose largest tile
// fits one 32 KB ring slot (the consumers cover exactly that many rows).
static int slab_bits(int L, int K, size_t es)
{
    const size_t rb = (size_t)K * es;
    if (rb < 32 || rb > 256 || rb % 16 != 0) return -1;
    int B = kLowMaxB < L - 2 ? kLowMaxB : L - 2;
    while (B >= 2 && (size_t)host_binom(B, B / 2) * rb > (size_t)kSlabSlotBytes) --B;
    return B >= 2 ? B : -1;
}

template <typename T, int K, int MODE>
static cudaError_t launch_slab(const ChainParams &cp, int Bs, const T *X, T *Y, T *R, const T *dinv,
                               const PcgScalars &ps, const Reduce &rd, cudaStream_t st)
{
    if (ensure_lowtab(Bs) != MBL_OK) return cudaErrorUnknown;
    auto kern = k_apply_slab<T, K, MODE>;
    constexpr int dyn = kSlabSlots * kSlabSlotBytes;
    static const cudaError_t attr = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (attr != cudaSuccess) return attr;
    const int64_t ntile = (int64_t)1 << (cp.L - Bs);
    int64_t grid = num_sms();
    if (grid > ntile) grid = ntile;
    note_launch();
    kern<<<(int)grid, kSlabThreads, dyn, st>>>(cp, Bs, X, Y, R, dinv, ps, rd);
    return cudaGetLastError();
}

template <typename T, int K, int MODE>
static cudaError_t launch_tiled(const ChainParams &cp, int B, const T *X, int64_t ldx, T *Y, int64_t ldy, T *R,
                                const T *dinv, const PcgScalars &ps, const Reduce &rd, cudaStream_t st)
{
    if constexpr (SlabLayout<T, K>::ok) {
        // slab: contiguous rows (ld = K), 16-byte aligned bases for the bulk copies; the
        // q-launch variant leaves w to the direction update
        auto al = [](const void *q) { return q == nullptr || (uintptr_t)q % 16 == 0; };
        if (slab_schedule(cp.L, cp.n_up, K, sizeof(T)) && ldx == K && (Y == nullptr || ldy == K) && al(X) &&
            al(Y) && al(R) && (MODE != kPcgQ || ps.w == nullptr)) {
            const int Bs = slab_bits(cp.L, K, sizeof(T));
            if (Bs >= 2) return launch_slab<T, K, MODE>(cp, Bs, X, Y, R, dinv, ps, rd, st);
        }
    }
    if constexpr (StreamLayout<T, K>::ok) {
        // streamed: contiguous rows (ld = K) and 16-byte aligned bases for every streamed block
        auto al = [](const void *q) { return q == nullptr || (uintptr_t)q % 16 == 0; };
        if (streamed_schedule(cp.L, cp.n_up, K, sizeof(T)) && ldx == K && (Y == nullptr || ldy == K) && al(X) &&
            al(Y) && al(R) && al(ps.w) && al(ps.p)) {
            const int Bs = stream_bits<T, K>(cp.L);
            if (Bs >= 2) return launch_streamed<T, K, MODE>(cp, Bs, X, Y, R, dinv, ps, rd, st);
        }
    }
    if constexpr ((K * sizeof(T)) % 16 == 0) {
        // staged: contiguous rows (ld = K) and 16-byte aligned bases for the bulk copies
        const bool aligned = ((uintptr_t)X % 16 == 0) && (Y == nullptr || (uintptr_t)Y % 16 == 0) &&
                             (R == nullptr || (uintptr_t)R % 16 == 0);
        if (staged_schedule(cp.L, cp.n_up, K, sizeof(T)) && ldx == K && (Y == nullptr || ldy == K) && aligned) {
            const int Bs = staged_bits(cp.L, K, sizeof(T));
            if (Bs >= 2) {
                const int lbs = lane_bytes_for(cp.L, K, sizeof(T));
                if (lbs == 16) return launch_staged_lb<T, K, MODE, 16>(cp, Bs, X, Y, R, dinv, ps, rd, st);
                if (lbs == 64) return launch_staged_lb<T, K, MODE, 64>(cp, Bs, X, Y, R, dinv, ps, rd, st);
                return launch_staged_lb<T, K, MODE, 32>(cp, Bs, X, Y, R, dinv, ps, rd, st);
            }
        }
    }
    const int lb = lane_bytes_for(cp.L, K, sizeof(T));
    if (lb == 16) return launch_tiled_lb<T, K, MODE, 16>(cp, B, X, ldx, Y, ldy, R, dinv, ps, rd, st);
    if (lb == 64) return launch_tiled_lb<T, K, MODE, 64>(cp, B, X, ldx, Y, ldy, R, dinv, ps, rd, st);
    return launch_tiled_lb<T, K, MODE, 32>(cp, B, X, ldx, Y, ldy, R, dinv, ps, rd, st);
}

static int apply_grid(uint32_t n, int cap_per_sm)
{
    int64_t need = ((int64_t)n + 32 * kWarps - 1) / (32 * kWarps);
    int64_t cap = (int64_t)num_sms() * cap_per_sm;
    if (need < 1) need = 1;
    return (int)(need < cap ? need : cap);
}

template <typename T>
static bool vec_ok_wide(const void *p, int64_t ld, int K, int lb)
{
    const int bytes = K * (int)sizeof(T);
    const int align = bytes >= lb ? lb : bytes;  // one vector per lane: min(row, lane) bytes
    return ((uintptr_t)p % align == 0) && ((ld * (int64_t)sizeof(T)) % align == 0);
}

template <typename T>
static bool vec_ok(const void *p, int64_t ld, int K)
{
    const int bytes = K * (int)sizeof(T);
    const int align = bytes >= 16 ? 16 : bytes;
    return ((uintptr_t)p % align == 0) && ((ld * (int64_t)sizeof(T)) % align == 0);
}

template <typename T>
static int dispatch_plain(const ChainParams &cp, const T *X, int64_t ldx, T *Y, int64_t ldy, uint32_t n, int k,
                          cudaStream_t st)
{
    PcgScalars ps{};
    Reduce rd{};
    const int grid = apply_grid(n, 8);
    cudaError_t e = cudaSuccess;
    bool done = true;
    const int B = tile_bits_for(cp.L, k, sizeof(T));
    const int lb = lane_bytes_for(cp.L, k, sizeof(T));
    if (B >= 2 && vec_ok_wide<T>(X, ldx, k, lb) && vec_ok_wide<T>(Y, ldy, k, lb)) {
        switch (k) {
        case 1: e = launch_tiled<T, 1, kPlain>(cp, B, X, ldx, Y, ldy, nullptr, nullptr, ps, rd, st); break;
        case 2: e = launch_tiled<T, 2, kPlain>(cp, B, X, ldx, Y, ldy, nullptr, nullptr, ps, rd, st); break;
        case 4: e = launch_tiled<T, 4, kPlain>(cp, B, X, ldx, Y, ldy, nullptr, nullptr, ps, rd, st); break;
        case 8: e = launch_tiled<T, 8, kPlain>(cp, B, X, ldx, Y, ldy, nullptr, nullptr, ps, rd, st); break;
        case 16: e = launch_tiled<T, 16, kPlain>(cp, B, X, ldx, Y, ldy, nullptr, nullptr, ps, rd, st); break;
        case 32: e = launch_tiled<T, 32, kPlain>(cp, B, X, ldx, Y, ldy, nullptr, nullptr, ps, rd, st); break;
        case 64: e = launch_tiled<T, 64, kPlain>(cp, B, X, ldx, Y, ldy, nullptr, nullptr, ps, rd, st); break;
        default: done = false;
        }
    } else if (vec_ok<T>(X, ldx, k) && vec_ok<T>(Y, ldy, k)) {
        switch (k) {
        case 1: e = launch_apply_k<T, 1, kPlain>(cp, X, ldx, Y, ldy, n, nullptr, nullptr, ps, rd, grid, st); break;
        case 2: e = launch_apply_k<T, 2, kPlain>(cp, X, ldx, Y, ldy, n, nullptr, nullptr, ps, rd, grid, st); break;
        case 4: e = launch_apply_k<T, 4, kPlain>(cp, X, ldx, Y, ldy, n, nullptr, nullptr, ps, rd, grid, st); break;
        case 8: e = launch_apply_k<T, 8, kPlain>(cp, X, ldx, Y, ldy, n, nullptr, nullptr, ps, rd, grid, st); break;
        case 16: e = launch_apply_k<T, 16, kPlain>(cp, X, ldx, Y, ldy, n, nullptr, nullptr, ps, rd, grid, st); break;
        case 32: e = launch_apply_k<T, 32, kPlain>(cp, X, ldx, Y, ldy, n, nullptr, nullptr, ps, rd, grid, st); break;
        case 64: e = launch_apply_k<T, 64, kPlain>(cp, X, ldx, Y, ldy, n, nullptr, nullptr, ps, rd, grid, st); break;
        default: done = false;
        }
    } else {
        done = false;
    }
    if (!done) {
        const size_t sm = apply_smem_bytes<T>();
        static const bool attr_set_once = [&]() {
            cudaFuncSetAttribute(k_apply_generic<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            return true;
        }();
        (void)attr_set_once;
        note_launch();
        k_apply_generic<T><<<grid, kThreads, sm, st>>>(cp, X, ldx, Y, ldy, n, k);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

int apply_device(const ChainParams &cp, int dtype, const void *X, int64_t ldx, void *Y, int64_t ldy, uint32_t n,
                 int k, cudaStream_t st)
{
    if (dtype == MBL_F32)
        return dispatch_plain<float>(cp, (const float *)X, ldx, (float *)Y, ldy, n, k, st);
    return dispatch_plain<double>(cp, (const double *)X, ldx, (double *)Y, ldy, n, k, st);
}

template <typename T>
int pcg_fold_dinv(const ChainParams &cp, uint32_t n, T *dinv, cudaStream_t st)
{
    int grid = (int)(((int64_t)n + kThreads - 1) / kThreads);
    note_launch();
    if (grid > num_sms() * 8) grid = num_sms() * 8;
    k_fold_dinv<T><<<grid, kThreads, 0, st>>>(cp, n, dinv);
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}
template int pcg_fold_dinv<float>(const ChainParams &, uint32_t, float *, cudaStream_t);
template int pcg_fold_dinv<double>(const ChainParams &, uint32_t, double *, cudaStream_t);

int gershgorin_bound(const ChainParams &cp, uint32_t n, double *partials, unsigned *counter, double *out,
                     cudaStream_t st)
{
    int grid = (int)(((int64_t)n + kThreads - 1) / kThreads);
    if (grid > num_sms() * 4) grid = num_sms() * 4;
    Reduce rd{partials, counter};
    note_launch();
    k_gershgorin<<<grid, kThreads, 0, st>>>(cp, n, rd, out);
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

int pcg_grid(uint32_t n) { return apply_grid(n, 4); }
size_t pcg_partial_doubles() { return (size_t)num_sms() * 8 * 64 + 64; }

template <typename T>
int pcg_start(const double *B, int64_t ldb, const double *bnorm, uint32_t n, int k, const T *dinv, T *r, T *p,
              T *w, const PcgDev &pd, cudaStream_t st)
{
    PcgScalars ps{pd.rz, pd.rz0, pd.alpha, pd.beta, pd.active, pd.tol2};
    Reduce rd{pd.partials, pd.counter};
    int grid = pcg_grid(n);
    note_launch();
    k_pcg_init<T><<<grid, kThreads, 0, st>>>(B, ldb, bnorm, n, k, dinv, r, p, w, ps, rd);
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}
template int pcg_start<float>(const double *, int64_t, const double *, uint32_t, int, const float *, float *,
                              float *, float *, const PcgDev &, cudaStream_t);
template int pcg_start<double>(const double *, int64_t, const double *, uint32_t, int, const double *, double *,
                               double *, double *, const PcgDev &, cudaStream_t);

// ---- batched PCG step: host side ------------------------------------------------

// Work items and rounds of one lane (the persistent tiled product's items: a chunk of
// WideRowLayout::CH rows of one tile, all 2^(L-B) tiles).
template <typename T, int K>
static void lane_items(int L, int B, uint32_t *items, uint32_t *nrounds)
{
    constexpr int CH = WideRowLayout<T, K, 32>::CH;
    const uint32_t nchunk = (host_binom(B, B / 2) + CH - 1) / CH;
    *items = (uint32_t)(((uint64_t)1 << (L - B)) * nchunk);
    *nrounds = (*items + kWarps - 1) / kWarps;
}

int pcg_lane_fill(PcgLane *Ln, const ChainParams &cp, uint32_t n, int k, int f32, const void *dinv, void *r,
                  void *p, void *t, void *w, const PcgDev &pd, uint32_t *round0, uint32_t *row0)
{
    const size_t es = f32 ? 4 : 8;
    const int B = tile_bits_for(cp.L, k, es);
    if (B < 2) return MBL_ERR_ARG;
    if (ensure_lowtab(B) != MBL_OK) return MBL_ERR_CUDA;
    uint32_t items = 0, nrounds = 0;
    switch (k) {
    case 8: f32 ? lane_items<float, 8>(cp.L, B, &items, &nrounds) : lane_items<double, 8>(cp.L, B, &items, &nrounds); break;
    case 16: f32 ? lane_items<float, 16>(cp.L, B, &items, &nrounds) : lane_items<double, 16>(cp.L, B, &items, &nrounds); break;
    case 32: f32 ? lane_items<float, 32>(cp.L, B, &items, &nrounds) : lane_items<double, 32>(cp.L, B, &items, &nrounds); break;
    case 64: f32 ? lane_items<float, 64>(cp.L, B, &items, &nrounds) : lane_items<double, 64>(cp.L, B, &items, &nrounds); break;
    default: return MBL_ERR_ARG;
    }
    // the lane's round partials live in its PCG partials buffer
    if ((size_t)nrounds * k > pcg_partial_doubles()) return MBL_ERR_ARG;
    *Ln = PcgLane{cp, dinv, r, p, t, w, pd.rz, pd.rz0, pd.alpha, pd.beta, pd.active, pd.tol2, pd.partials,
                  pd.counter, n, B, items, *round0, nrounds, *row0};
    *round0 += nrounds;
    *row0 += n;
    return MBL_OK;
}

template <typename T, int K>
static cudaError_t pcg_batch_step_k(const PcgLane *lanes, int nlanes, uint32_t rounds, uint32_t rows, cudaStream_t st)
{
    static const int per_sm = [&]() {
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_pcg_batch<T, K, kPcgT, 32>, kThreads, 0) != cudaSuccess ||
            v < 1)
            v = 1;
        return v;
    }();
    int64_t grid = (int64_t)num_sms() * per_sm;
    if (grid > rounds) grid = rounds;
    note_launch();
    k_pcg_batch<T, K, kPcgT, 32><<<(int)grid, kThreads, 0, st>>>(lanes, nlanes, rounds);
    note_launch();
    k_pcg_batch<T, K, kPcgQ, 32><<<(int)grid, kThreads, 0, st>>>(lanes, nlanes, rounds);
    int ugrid = (int)(((int64_t)rows * RowLayout<T, K>::G + kThreads * kUpdRows - 1) / (kThreads * kUpdRows));
    if (ugrid > num_sms() * 8) ugrid = num_sms() * 8;
    if (ugrid < 1) ugrid = 1;
    note_launch();
    k_pcg_batch_update<T, K><<<ugrid, kThreads, 0, st>>>(lanes, nlanes, rows);
    return cudaGetLastError();
}

int pcg_batch_step(int f32, const PcgLane *lanes_dev, int nlanes, int k, uint32_t rounds, uint32_t rows,
                   cudaStream_t st)
{
    if (nlanes < 1 || rounds < 1 || rows < 1) return MBL_ERR_ARG;
    cudaError_t e;
    switch (k) {
    case 8: e = f32 ? pcg_batch_step_k<float, 8>(lanes_dev, nlanes, rounds, rows, st)
                    : pcg_batch_step_k<double, 8>(lanes_dev, nlanes, rounds, rows, st); break;
    case 16: e = f32 ? pcg_batch_step_k<float, 16>(lanes_dev, nlanes, rounds, rows, st)
                     : pcg_batch_step_k<double, 16>(lanes_dev, nlanes, rounds, rows, st); break;
    case 32: e = f32 ? pcg_batch_step_k<float, 32>(lanes_dev, nlanes, rounds, rows, st)
                     : pcg_batch_step_k<double, 32>(lanes_dev, nlanes, rounds, rows, st); break;
    case 64: e = f32 ? pcg_batch_step_k<float, 64>(lanes_dev, nlanes, rounds, rows, st)
                     : pcg_batch_step_k<double, 64>(lanes_dev, nlanes, rounds, rows, st); break;
    default: return MBL_ERR_ARG;
    }
    return e == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

template <typename T, int K>
static cudaError_t pcg_step_k(const ChainParams &cp, uint32_t n, const T *dinv, T *r, T *p, T *t, T *w,
                              const PcgScalars &ps, const Reduce &rd, int grid, cudaStream_t st)
{
    cudaError_t e;
    const int B = tile_bits_for(cp.L, K, sizeof(T));
    bool wdone = false;
    if (B >= 2) {
        e = launch_tiled<T, K, kPcgT>(cp, B, p, K, t, K, nullptr, dinv, ps, rd, st);
        if (e != cudaSuccess) return e;
        PcgScalars psq = ps;
        if (!MBL_PCG_W_IN_UPDATE) {  // the q-launch also updates w (alpha is known by then)
            psq.w = w;
            psq.p = p;
            wdone = true;
        }
        e = launch_tiled<T, K, kPcgQ>(cp, B, t, K, nullptr, K, r, dinv, psq, rd, st);
    } else {
        e = launch_apply_k<T, K, kPcgT>(cp, p, K, t, K, n, nullptr, dinv, ps, rd, grid, st);
        if (e != cudaSuccess) return e;
        e = launch_apply_k<T, K, kPcgQ>(cp, t, K, nullptr, K, n, r, dinv, ps, rd, grid, st);
    }
    if (e != cudaSuccess) return e;
    int ugrid = (int)(((int64_t)n * RowLayout<T, K>::G + kThreads * kUpdRows - 1) / (kThreads * kUpdRows));
    note_launch();
    if (ugrid > num_sms() * 8) ugrid = num_sms() * 8;
    if (wdone) k_pcg_update<T, K, true><<<ugrid, kThreads, 0, st>>>(n, dinv, r, p, w, ps);
    else k_pcg_update<T, K, false><<<ugrid, kThreads, 0, st>>>(n, dinv, r, p, w, ps);
    return cudaGetLastError();
}

// One PCG iteration on A = (H - sigma)^2: t = (H - sigma)p, alpha; r -= alpha (H - sigma)t,
// beta; w += alpha p, p = M^-1 r + beta p.  Three launches, no host synchronisation.
template <typename T>
int pcg_step(const ChainParams &cp, uint32_t n, int k, const T *dinv, T *r, T *p, T *t, T *w, const PcgDev &pd,
             cudaStream_t st)
{
    PcgScalars ps{pd.rz, pd.rz0, pd.alpha, pd.beta, pd.active, pd.tol2};
    Reduce rd{pd.partials, pd.counter};
    const int grid = pcg_grid(n);
    cudaError_t e = cudaSuccess;
    switch (k) {
    case 8: e = pcg_step_k<T, 8>(cp, n, dinv, r, p, t, w, ps, rd, grid, st); break;
    case 16: e = pcg_step_k<T, 16>(cp, n, dinv, r, p, t, w, ps, rd, grid, st); break;
    case 32: e = pcg_step_k<T, 32>(cp, n, dinv, r, p, t, w, ps, rd, grid, st); break;
    case 64: e = pcg_step_k<T, 64>(cp, n, dinv, r, p, t, w, ps, rd, grid, st); break;
    default: {
        const size_t sm = apply_smem_bytes<T>();
        static const bool attr_set_once = [&]() {
            cudaFuncSetAttribute(k_apply_pcg_generic<T, kPcgT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            cudaFuncSetAttribute(k_apply_pcg_generic<T, kPcgQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            return true;
        }();
        (void)attr_set_once;
        note_launch();
        k_apply_pcg_generic<T, kPcgT><<<grid, kThreads, sm, st>>>(cp, p, t, n, k, nullptr, dinv, ps, rd);
        note_launch();
        k_apply_pcg_generic<T, kPcgQ><<<grid, kThreads, sm, st>>>(cp, t, nullptr, n, k, r, dinv, ps, rd);
        int ugrid = num_sms() * 8;
        note_launch();
        k_pcg_update_generic<T><<<ugrid, kThreads, 0, st>>>(n, k, dinv, r, p, w, ps);
        e = cudaGetLastError();
    }
    }
    return e == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}
template int pcg_step<float>(const ChainParams &, uint32_t, int, const float *, float *, float *, float *, float *,
                             const PcgDev &, cudaStream_t);
template int pcg_step<double>(const ChainParams &, uint32_t, int, const double *, double *, double *, double *,
                              double *, const PcgDev &, cudaStream_t);

}  // namespace mbl

// ---------------------------------------------------------------------------------
// C ABI: the product.

extern "C" int mbl_set_product_tile_bits(int k, int dtype, int bits)
{
    if (k < 1 || k > 256 || (dtype != MBL_F32 && dtype != MBL_F64) || bits < -1 || bits > 16 || bits == 1)
        return MBL_ERR_ARG;
    mbl::set_tile_bits(k, dtype == MBL_F32 ? 4 : 8, bits);
    return MBL_OK;
}

// Streamed tile width for a runtime block width (-1: no streamed kernel for it).
static int stream_bits_k(int L, int k, size_t es)
{
    using namespace mbl;
    if (es == 4) {
        switch (k) {
        case 8: return stream_bits<float, 8>(L);
        case 16: return stream_bits<float, 16>(L);
        case 32: return stream_bits<float, 32>(L);
        case 64: return stream_bits<float, 64>(L);
        default: return -1;
        }
    }
    switch (k) {
    case 4: return stream_bits<double, 4>(L);
    case 8: return stream_bits<double, 8>(L);
    case 16: return stream_bits<double, 16>(L);
    case 32: return stream_bits<double, 32>(L);
    case 64: return stream_bits<double, 64>(L);
    default: return -1;
    }
}

extern "C" int mbl_product_tile_width(int L, int dtype, int k, int schedule)
{
    using namespace mbl;
    if ((dtype != MBL_F32 && dtype != MBL_F64) || k < 1 || k > 256 || L < 4 || L > kMaxL || schedule < 1 ||
        schedule > 5)
        return MBL_ERR_ARG;
    const size_t es = dtype == MBL_F32 ? 4 : 8;
    const bool tiled_k = (k == 1 || k == 2 || k == 4 || k == 8 || k == 16 || k == 32 || k == 64);
    const int B = tiled_k ? tile_bits_for(L, k, es) : -1;
    if (B < 2) return 0;
    int w = B;
    if (schedule == 3) w = (k * (int)es) % 16 == 0 ? staged_bits(L, k, es) : -1;
    if (schedule == 4) w = stream_bits_k(L, k, es);
    if (schedule == 5) w = (k == 2 || k == 4 || k == 8 || k == 16 || k == 32 || k == 64) ? slab_bits(L, k, es) : -1;
    return w >= 2 ? w : 0;
}

extern "C" int mbl_set_product_schedule(int k, int dtype, int schedule)
{
    if (k < 1 || k > 256 || (dtype != MBL_F32 && dtype != MBL_F64) || schedule < 0 || schedule > 5)
        return MBL_ERR_ARG;
    mbl::set_schedule(k, dtype == MBL_F32 ? 4 : 8, schedule);
    return MBL_OK;
}

extern "C" int mbl_set_product_lane_bytes(int k, int dtype, int bytes)
{
    if (k < 1 || k > 256 || (dtype != MBL_F32 && dtype != MBL_F64) || (bytes != 0 && bytes != 16 && bytes != 32 && bytes != 64))
        return MBL_ERR_ARG;
    mbl::set_lane_bytes(k, dtype == MBL_F32 ? 4 : 8, bytes);
    return MBL_OK;
}

extern "C" int mbl_autotune_product(const mbl_chain *chain, int dtype, const void *X_dev, void *Y_dev, int64_t n,
                                    int k, int reps, mbl_product_choice *choice, mbl_stream_t stream)
{
    using namespace mbl;
    ChainParams cp;
    int rc = make_chain_params(chain, 0.0, &cp);
    if (rc != MBL_OK) return rc;
    if (dtype != MBL_F32 && dtype != MBL_F64) return MBL_ERR_ARG;
    if (k < 1 || k > 256 || reps < 1 || reps > 1000) return MBL_ERR_ARG;
    if (n != mbl_basis_size(chain->L, chain->n_up) || n == 0 || !X_dev || !Y_dev) return MBL_ERR_ARG;
    const size_t es = dtype == MBL_F32 ? 4 : 8;
    const char *xb = (const char *)X_dev, *yb = (const char *)Y_dev;
    if (xb < yb + n * k * (int64_t)es && yb < xb + n * k * (int64_t)es) return MBL_ERR_ARG;
    if (choice) *choice = mbl_product_choice{0, 0, 0, 0.0};
    const bool tiled_k = (k == 1 || k == 2 || k == 4 || k == 8 || k == 16 || k == 32 || k == 64);
    if (!tiled_k || tile_bits_for(cp.L, k, es) < 2) return MBL_OK;  // one kernel only: nothing to choose
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return MBL_ERR_CUDA;
    }
    const int rows = (int)(k * es);
    float best = -1.0f, def_ms = -1.0f;
    int best_s = 1, best_l = 32;
    // the size-based default, kept unless a candidate beats it by more than timing noise
    const int def_s = size_schedule(cp.L, cp.n_up, k, es), def_l = rows >= 64 ? size_lane_bytes(k, es) : 32;
    rc = MBL_OK;
    const int sbits = stream_bits_k(cp.L, k, es);
    const int slbits = slab_bits(cp.L, k, es);
    for (int sch = 1; sch <= 5 && rc == MBL_OK; ++sch) {
        if (sch == 3 && (rows % 16 != 0 || staged_bits(cp.L, k, es) < 2)) continue;
        if (sch == 4 && sbits < 2) continue;
        if (sch == 5 && slbits < 2) continue;
        for (int lane = 32; lane <= 64 && rc == MBL_OK; lane *= 2) {
            if (lane == 64 && rows < 64) continue;  // narrower rows: one lane holds the row either way
            if (lane == 64 && (sch == 4 || sch == 5)) continue;  // one lane width there
            t_force_schedule = sch;
            t_force_lane = lane;
            float ms = 0.0f;
            rc = apply_device(cp, dtype, X_dev, k, Y_dev, k, (uint32_t)n, k, st);  // warm-up
            if (rc == MBL_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = MBL_ERR_CUDA;
            for (int r = 0; r < reps && rc == MBL_OK; ++r)
                rc = apply_device(cp, dtype, X_dev, k, Y_dev, k, (uint32_t)n, k, st);
            if (rc == MBL_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                 cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                rc = MBL_ERR_CUDA;
            t_force_schedule = 0;
            t_force_lane = 0;
            if (rc == MBL_OK && (best < 0.0f || ms < best)) {
                best = ms;
                best_s = sch;
                best_l = lane;
            }
            if (rc == MBL_OK && sch == def_s && lane == def_l) def_ms = ms;
        }
    }
    if (rc == MBL_OK && def_ms > 0.0f && best > 0.98f * def_ms) {
        best = def_ms;
        best_s = def_s;
        best_l = def_l;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != MBL_OK) return rc;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tuned[es == 8 ? 1 : 0][kslot(k)][cp.L] = ProductTune{best_s, best_l};
    }
    if (choice)
        *choice = mbl_product_choice{best_s, best_l,
                                     best_s == 3   ? staged_bits(cp.L, k, es)
                                     : best_s == 4 ? sbits
                                     : best_s == 5 ? slbits
                                                   : tile_bits_for(cp.L, k, es),
                                     1000.0 * (double)best / reps};
    return MBL_OK;
}

extern "C" int mbl_hamiltonian_apply(const mbl_chain *chain, double sigma, int dtype, const void *X_dev,
                                     int64_t ldx, void *Y_dev, int64_t ldy, int64_t n, int k, mbl_stream_t stream)
{
    using namespace mbl;
    ChainParams cp;
    int rc = make_chain_params(chain, sigma, &cp);
    if (rc != MBL_OK) return rc;
    if (dtype != MBL_F32 && dtype != MBL_F64) return MBL_ERR_ARG;
    if (k < 1 || k > 256 || ldx < k || ldy < k) return MBL_ERR_ARG;
    if (n != mbl_basis_size(chain->L, chain->n_up)) return MBL_ERR_ARG;
    if (n == 0) return MBL_OK;
    if (!X_dev || !Y_dev) return MBL_ERR_ARG;
    const size_t es = dtype == MBL_F32 ? 4 : 8;
    // X and Y must not overlap (the gather reads X rows that other groups write in Y)
    const char *xb = (const char *)X_dev, *yb = (const char *)Y_dev;
    const char *xe = xb + ((n - 1) * ldx + k) * (int64_t)es, *ye = yb + ((n - 1) * ldy + k) * (int64_t)es;
    if (xb < ye && yb < xe) return MBL_ERR_ARG;
    return apply_device(cp, dtype, X_dev, ldx, Y_dev, ldy, (uint32_t)n, k, (cudaStream_t)stream);
}
