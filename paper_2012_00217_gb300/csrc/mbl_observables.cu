// mbl_observables.cu -- localization indicators of converged eigenpairs (Sec. 2.2): the
// ABI entries of the adjacent gap ratio (kernel below) and of the half-chain entanglement
// entropy (kernels in mbl_small.cu, next to the Jacobi eigensolver they use).
//
// Adjacent gap ratio: one block per disorder realization.  The block loads the
// realization's m levels into shared memory (padded to a power of two with +inf),
// sorts them with a bitonic network, forms r_j = min(d_{j-1}, d_j) / max(d_{j-1}, d_j)
// from the gaps d_j = E_{j+1} - E_j of every interior level (a level whose two gaps are
// both zero has no ratio), and reduces the ratios and their count in a fixed order, so
// results are bitwise reproducible.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "mbl.h"
#include "mbl_internal.h"

namespace mbl {
namespace {

constexpr int kGapThreads = 256;
constexpr int kGapMaxLevels = 4096;

__global__ void __launch_bounds__(kGapThreads)
    k_gap_ratio(int m, int P, const double *__restrict__ E, int64_t ld, double *__restrict__ r_mean,
                int *__restrict__ count)
{
    extern __shared__ double s_lv[];  // P levels
    __shared__ double s_sum[kGapThreads];
    __shared__ int s_cnt[kGapThreads];
    __shared__ int s_bad;
    const int tid = threadIdx.x;
    const double *e = E + (int64_t)blockIdx.x * ld;
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int j = tid; j < P; j += kGapThreads) {
        double v = INFINITY;
        if (j < m) {
            v = e[j];
            if (!isfinite(v)) s_bad = 1;
        }
        s_lv[j] = v;
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) {
            r_mean[blockIdx.x] = NAN;
            count[blockIdx.x] = 0;
        }
        return;
    }
    // bitonic sort, ascending
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < P; i += kGapThreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const double a = s_lv[i], b = s_lv[ixj];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        s_lv[i] = b;
                        s_lv[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    double acc = 0.0;
    int c = 0;
    for (int j = 1 + tid; j <= m - 2; j += kGapThreads) {
        const double d0 = s_lv[j] - s_lv[j - 1], d1 = s_lv[j + 1] - s_lv[j];
        const double hi = fmax(d0, d1), lo = fmin(d0, d1);
        if (hi > 0.0) {
            acc += lo / hi;
            ++c;
        }
    }
    s_sum[tid] = acc;
    s_cnt[tid] = c;
    __syncthreads();
    for (int h = kGapThreads / 2; h > 0; h >>= 1) {
        if (tid < h) {
            s_sum[tid] += s_sum[tid + h];
            s_cnt[tid] += s_cnt[tid + h];
        }
        __syncthreads();
    }
    if (tid == 0) {
        r_mean[blockIdx.x] = s_cnt[0] > 0 ? s_sum[0] / (double)s_cnt[0] : NAN;
        count[blockIdx.x] = s_cnt[0];
    }
}

}  // namespace
}  // namespace mbl

extern "C" int mbl_gap_ratio(int nprob, int m, const double *evals_dev, int64_t ld, double *r_mean_dev,
                             int *count_dev, mbl_stream_t stream)
{
    using namespace mbl;
    if (nprob < 0 || m < 1 || m > kGapMaxLevels || ld < m) return MBL_ERR_ARG;
    if (nprob == 0) return MBL_OK;
    if (!evals_dev || !r_mean_dev || !count_dev) return MBL_ERR_ARG;
    int P = 2;
    while (P < m) P <<= 1;
    note_launch();
    k_gap_ratio<<<nprob, kGapThreads, (size_t)P * sizeof(double), (cudaStream_t)stream>>>(m, P, evals_dev, ld,
                                                                                           r_mean_dev, count_dev);
    return cudaGetLastError() == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

// Largest Gram side the entanglement kernels accept (a one-block Jacobi per block).
static constexpr int64_t kEntMaxSide = 512;

static int ent_check(const mbl_chain *chain, int l_a, int nvec, mbl::EntanglementPlan *pl)
{
    if (!chain || nvec < 0) return MBL_ERR_ARG;
    const int L = chain->L, m = chain->n_up;
    if (L < 2 || L > 32 || m < 0 || m > L || l_a < 1 || l_a > L - 1) return MBL_ERR_ARG;
    *pl = mbl::entanglement_plan(L, m, l_a);
    if (pl->dmax > kEntMaxSide) return MBL_ERR_ARG;
    return MBL_OK;
}

extern "C" int mbl_entanglement_workspace_size(const mbl_chain *chain, int l_a, int nvec, size_t *bytes)
{
    mbl::EntanglementPlan pl;
    const int rc = ent_check(chain, l_a, nvec, &pl);
    if (rc != MBL_OK) return rc;
    if (!bytes) return MBL_ERR_ARG;
    *bytes = mbl::entanglement_work_bytes(pl, nvec);
    return MBL_OK;
}

extern "C" int mbl_entanglement_entropy(const mbl_chain *chain, int l_a, int nvec, const double *V_dev,
                                        int64_t ldv, double *S_dev, void *workspace_dev, size_t workspace_bytes,
                                        mbl_stream_t stream)
{
    mbl::EntanglementPlan pl;
    const int rc = ent_check(chain, l_a, nvec, &pl);
    if (rc != MBL_OK) return rc;
    if (ldv < nvec) return MBL_ERR_ARG;
    if (nvec == 0) return MBL_OK;
    if (!V_dev || !S_dev || !workspace_dev) return MBL_ERR_ARG;
    if (workspace_bytes < mbl::entanglement_work_bytes(pl, nvec)) return MBL_ERR_WORKSPACE;
    return mbl::entanglement_launch(chain->L, chain->n_up, l_a, nvec, V_dev, ldv, S_dev, workspace_dev,
                                    workspace_bytes, (cudaStream_t)stream);
}
