// mbl_device.cuh -- device-side building blocks shared by the sm_103a kernels:
// binomial table, combinatorial-number-system rank/unrank of S^z-sector states,
// and the per-chain constants of the diagonal.  (Sec. 2.1: sector basis and the
// matrix elements of Eq. (model).)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mbl.h"

namespace mbl {

constexpr int kMaxL = 32;
constexpr int kBinomDim = kMaxL + 1;  // C(i, j) for 0 <= i, j <= 32

struct BinomTable {
    uint32_t v[kBinomDim * kBinomDim];
};

constexpr BinomTable make_binom_table()
{
    BinomTable t{};
    for (int i = 0; i < kBinomDim; ++i)
        for (int j = 0; j < kBinomDim; ++j) {
            uint32_t c = 0;
            if (j == 0) c = 1;
            else if (i > 0) c = t.v[(i - 1) * kBinomDim + (j - 1)] + t.v[(i - 1) * kBinomDim + j];
            t.v[i * kBinomDim + j] = c;
        }
    return t;
}

// C(32, 16) = 601,080,390 < 2^32, so every entry fits in uint32.  One copy per
// translation unit (no relocatable device code needed), in global memory: blocks copy it
// into shared memory with consecutive threads reading consecutive words (from L2 after
// the first launch).  From constant memory that copy cost ~3 us per product launch at
// L = 20: the constant cache serves the 32 different addresses of a warp one at a time.
static __device__ const BinomTable g_binom = make_binom_table();

// Copy the binomial table into shared memory (call with all threads, then sync).
__device__ __forceinline__ void load_binom(uint32_t *sb)
{
    for (int i = threadIdx.x; i < kBinomDim * kBinomDim; i += blockDim.x) sb[i] = __ldg(&g_binom.v[i]);
}

__device__ __forceinline__ uint32_t binom(const uint32_t *sb, int i, int j)
{
    return sb[i * kBinomDim + j];
}

// rank(s) = sum_{j=1..m} C(p_j, j), p_1 < ... < p_m the set bits of s.
__device__ __forceinline__ uint32_t cns_rank(const uint32_t *sb, uint32_t s)
{
    uint32_t r = 0;
    int j = 0;
    while (s) {
        int p = __ffs(s) - 1;
        s &= s - 1;
        ++j;
        r += binom(sb, p, j);
    }
    return r;
}

// Inverse of cns_rank on the sector (L sites, m up spins), 0 <= r < C(L, m):
// choose the highest up spin first, the largest p with C(p, j) <= r.
__device__ __forceinline__ uint32_t cns_unrank(const uint32_t *sb, int L, int m, uint32_t r)
{
    uint32_t s = 0;
    int p = L - 1;
    for (int j = m; j >= 1; --j) {
        while (binom(sb, p, j) > r) --p;
        s |= 1u << p;
        r -= binom(sb, p, j);
        --p;
    }
    return s;
}

// Next word with the same popcount in ascending order (Gosper's hack): add the
// lowest set bit, then refill the cleared low run at the bottom.  s must not be the
// last word of the sector.
__device__ __forceinline__ uint32_t next_same_popcount(uint32_t s)
{
    uint32_t c = s & (0u - s);
    uint32_t r = s + c;
    return (((r ^ s) >> 2) >> (__ffs(s) - 1)) | r;
}

// Per-chain constants needed by every product kernel.  Passed by value as a kernel
// argument, so no device allocation is needed for h.
struct ChainParams {
    int L;
    int n_up;
    int periodic;      // 1 when the wrap bond (L-1, 0) exists (periodic and L > 2)
    int nbonds;        // |B|
    uint32_t open_mask;  // bits i = 0..L-2: bond (i, i+1)
    double half_delta;   // delta / 2: each antiparallel bond lowers d by delta/2
    double diag_const;   // delta |B| / 4 - sum_i h_i / 2 - sigma
    double h[kMaxL];     // fields
    const uint32_t *states;  // optional sector basis (n words); nullptr: unrank on the fly
    // FP32 copies for the FP32 kernels, split on the host so no kernel needs the FP64
    // pipe (about 1/64 of the FP32 rate on GB300): h = h_hi + h_lo exactly to 48 bits
    float h_hi[kMaxL], h_lo[kMaxL];
    float half_delta_f, diag_const_f;  // rounded once
};

// One problem (lane) of a batched PCG launch: its chain, vectors, per-column scalars and
// its place in the launch's rounds and concatenated rows (filled by pcg_lane_fill).
struct PcgLane {
    ChainParams cp;
    const void *dinv;
    void *r, *p, *t, *w;
    double *rz, *rz0, *alpha, *beta;
    int *active;
    double tol2;
    double *partials;   // >= nrounds * 64 doubles
    unsigned *counter;  // zero between launches (the finishing block resets it)
    uint32_t n;
    int B;              // tile width
    uint32_t items;     // work items of the lane
    uint32_t round0;    // first round of the lane
    uint32_t nrounds;   // ceil(items / kWarps)
    uint32_t row0;      // first row of the lane in the concatenated rows (update launch)
};

// The chain constants in the kernel's own type.
template <typename T>
__device__ __forceinline__ T cp_diag_const(const ChainParams &cp);
template <>
__device__ __forceinline__ float cp_diag_const<float>(const ChainParams &cp) { return cp.diag_const_f; }
template <>
__device__ __forceinline__ double cp_diag_const<double>(const ChainParams &cp) { return cp.diag_const; }
template <typename T>
__device__ __forceinline__ T cp_half_delta(const ChainParams &cp);
template <>
__device__ __forceinline__ float cp_half_delta<float>(const ChainParams &cp) { return cp.half_delta_f; }
template <>
__device__ __forceinline__ double cp_half_delta<double>(const ChainParams &cp) { return cp.half_delta; }

// Error-free sum of two FP32 numbers: s + e == a + b exactly (Knuth's TwoSum, TAOCP
// vol. 2, 4.2.2); six additions, no products, so nothing can be contracted.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Sector word of row r: from the basis table when one is given, else by unranking.
__device__ __forceinline__ uint32_t state_of(const uint32_t *sb, const ChainParams &cp, uint32_t r)
{
    return cp.states ? __ldg(cp.states + r) : cns_unrank(sb, cp.L, cp.n_up, r);
}

// Field part of the diagonal from 4 byte tables: sum over up spins of h_i.
// tab[b * 256 + v] = sum_{bit t of v} h[8b + t].
template <typename T>
__device__ __forceinline__ T field_sum(const T *tab, uint32_t s)
{
    return (tab[s & 255u] + tab[256 + ((s >> 8) & 255u)]) +
           (tab[512 + ((s >> 16) & 255u)] + tab[768 + (s >> 24)]);
}

// Build the byte tables in shared memory: entries summed in FP64, rounded once to T.
template <typename T>
__device__ __forceinline__ void build_field_tables(T *tab, const ChainParams &cp)
{
    for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
        int b = e >> 8;
        uint32_t v = (uint32_t)(e & 255);
        double acc = 0.0;
        for (int t = 0; t < 8; ++t) {
            int site = 8 * b + t;
            if (((v >> t) & 1u) && site < cp.L) acc += cp.h[site];
        }
        tab[e] = (T)acc;
    }
}

// FP32 tables without FP64 arithmetic: each entry is a compensated sum of the (h_hi,
// h_lo) pairs, rounded once at the end (equal to the rounded FP64 sum to within one
// unit in the last place).
template <>
__device__ __forceinline__ void build_field_tables<float>(float *tab, const ChainParams &cp)
{
    for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
        const int b = e >> 8;
        const uint32_t v = (uint32_t)(e & 255);
        float s = 0.0f, c = 0.0f;
        for (int t = 0; t < 8; ++t) {
            const int site = 8 * b + t;
            if (((v >> t) & 1u) && site < cp.L) {
                float hi, err;
                two_sum(s, cp.h_hi[site], hi, err);
                s = hi;
                c += err + cp.h_lo[site];
            }
        }
        tab[e] = s + c;
    }
}

// d(s) - sigma.  z_i z_j = +1 for parallel, -1 for antiparallel spins; with a the
// number of antiparallel bonds, sum_bonds delta/4 z_i z_j = delta|B|/4 - (delta/2) a.
// sum_i h_i/2 z_i = sum_{up} h_i - sum_i h_i / 2.
template <typename T>
__device__ __forceinline__ T diag_shifted(const T *tab, T dconst, T hdelta, const ChainParams &cp,
                                          uint32_t s)
{
    uint32_t anti = (s ^ (s >> 1)) & cp.open_mask;
    int a = __popc(anti);
    if (cp.periodic) a += (int)(((s >> (cp.L - 1)) ^ s) & 1u);
    return (dconst + field_sum(tab, s)) - hdelta * (T)a;
}

}  // namespace mbl
