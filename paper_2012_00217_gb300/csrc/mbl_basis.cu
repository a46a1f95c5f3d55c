// mbl_basis.cu -- S^z-sector basis (Sec. 2.1: block-diagonalisation by total S^z,
// sector dimension C(L, n_up), Table 1).  States are listed in ascending integer
// order; position <-> word by the combinatorial number system, so no lookup table of
// 2^L entries is ever needed.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mbl_device.cuh"
#include "mbl_internal.h"

namespace mbl {

// states[r] = cns_unrank(r) for a contiguous run of rows per thread: one unrank, then
// Gosper successors (cheaper than an unrank per row).
__global__ void __launch_bounds__(256) k_basis_build(int L, int m, uint32_t n, uint32_t run, uint32_t *states)
{
    __shared__ uint32_t sb[kBinomDim * kBinomDim];
    load_binom(sb);
    __syncthreads();
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t r0 = t * run;
    if (r0 >= n) return;
    uint32_t s = cns_unrank(sb, L, m, (uint32_t)r0);
    const uint64_t r1 = (r0 + run < n) ? r0 + run : n;
    for (uint64_t r = r0; r < r1; ++r) {
        states[r] = s;
        if (r + 1 < r1) s = next_same_popcount(s);
    }
}

__global__ void __launch_bounds__(256) k_basis_rank(int L, int m, const uint32_t *__restrict__ words,
                                                    int64_t *__restrict__ ranks, int64_t cnt)
{
    __shared__ uint32_t sb[kBinomDim * kBinomDim];
    load_binom(sb);
    __syncthreads();
    const uint32_t hi = (L >= 32) ? 0u : ~((1u << L) - 1u);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += (int64_t)gridDim.x * blockDim.x) {
        uint32_t s = words[q];
        ranks[q] = ((s & hi) || __popc(s) != m) ? -1 : (int64_t)cns_rank(sb, s);
    }
}

}  // namespace mbl

extern "C" int64_t mbl_basis_size(int L, int n_up)
{
    if (L < 1 || L > mbl::kMaxL || n_up < 0 || n_up > L) return -1;
    constexpr mbl::BinomTable t = mbl::make_binom_table();
    return (int64_t)t.v[L * mbl::kBinomDim + n_up];
}

extern "C" int mbl_basis_build(int L, int n_up, uint32_t *states_dev, int64_t n, mbl_stream_t stream)
{
    if (mbl_basis_size(L, n_up) < 0 || n != mbl_basis_size(L, n_up)) return MBL_ERR_ARG;
    if (n == 0) return MBL_OK;
    if (!states_dev) return MBL_ERR_ARG;
    const uint32_t run = 16;
    const int64_t threads = (n + run - 1) / run;
    const int grid = (int)((threads + 255) / 256);
    mbl::note_launch();
    mbl::k_basis_build<<<grid, 256, 0, (cudaStream_t)stream>>>(L, n_up, (uint32_t)n, run, states_dev);
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

extern "C" int mbl_basis_rank(int L, int n_up, const uint32_t *words_dev, int64_t *ranks_dev, int64_t cnt,
                              mbl_stream_t stream)
{
    if (mbl_basis_size(L, n_up) < 0 || cnt < 0) return MBL_ERR_ARG;
    if (cnt == 0) return MBL_OK;
    if (!words_dev || !ranks_dev) return MBL_ERR_ARG;
    int64_t blocks = (cnt + 255) / 256;
    const int64_t cap = (int64_t)mbl::num_sms() * 16;
    mbl::note_launch();
    mbl::k_basis_rank<<<(int)(blocks < cap ? blocks : cap), 256, 0, (cudaStream_t)stream>>>(L, n_up, words_dev,
                                                                                          ranks_dev, cnt);
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

extern "C" const char *mbl_status_string(int status)
{
    switch (status) {
    case MBL_OK: return "ok";
    case MBL_ERR_ARG: return "invalid argument";
    case MBL_ERR_WORKSPACE: return "workspace too small";
    case MBL_ERR_CUDA: return "CUDA error";
    case MBL_ERR_NOT_CONVERGED: return "not converged within max_iter";
    case MBL_ERR_BREAKDOWN: return "orthonormalisation breakdown";
    case MBL_ERR_NUMERIC: return "NaN or Inf encountered";
    default: return "unknown status";
    }
}
