// mbl_lanczos.cu -- spectrum bounds E_min, E_max of the sector Hamiltonian (placing sigma
// at the middle of the spectrum and scaling the tolerance, Sec. 6.2) by an FP64 Lanczos
// recurrence on H:
//   w = H v_j,  alpha_j = v_j^T w,  w -= alpha_j v_j + beta_{j-1} v_{j-1},
//   beta_j = ||w||,  v_{j+1} = w / beta_j,
// one block product of width 1 and three small streaming kernels per step.  Both ends come
// from the same tridiagonal T_m = tridiag(beta, alpha, beta): its extreme eigenvalues by
// Sturm bisection, and the residual of each extreme Ritz pair as beta_m |y_m| (y the
// eigenvector of T_m, by inverse iteration).  No reorthogonalisation: the extreme Ritz
// values converge to the extreme eigenvalues whatever copies the loss of orthogonality
// adds inside the spectrum.  The dot products are deterministic (block partials, then a
// fixed-order sum in the last block).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mbl_dense.h"
#include "mbl_device.cuh"
#include "mbl_internal.h"

namespace mbl {

namespace {

constexpr int kLzThreads = 256;
constexpr int kLzMaxSteps = 4096;
constexpr int kLzCheckEvery = 20;

struct LzDev {
    double *v[3];        // the three Lanczos vectors (roles rotate)
    double *alpha, *beta;  // kLzMaxSteps each
    double *part;        // grid partials
    unsigned *counter;   // zero; the last block resets it
};

// Sum of the block partials in a fixed order, in the last block to finish; true there.
__device__ __forceinline__ bool lz_last_block(double v, double *part, unsigned *counter, double *s_sum)
{
    __shared__ double s_red[kLzThreads / 32];
    __shared__ unsigned s_last;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < kLzThreads / 32; ++w) b += s_red[w];
        part[blockIdx.x] = b;
        __threadfence();
        s_last = (atomicAdd(counter, 1u) == gridDim.x - 1) ? 1u : 0u;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) t += part[b];
        *s_sum = t;
        *counter = 0u;
    }
    __syncthreads();
    return true;
}

// alpha_j = v . w
__global__ void __launch_bounds__(kLzThreads) k_lz_alpha(const double *__restrict__ v, const double *__restrict__ w,
                                                         int64_t n, double *alpha_j, double *part, unsigned *counter)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += v[i] * w[i];
    __shared__ double s_sum;
    if (lz_last_block(acc, part, counter, &s_sum) && threadIdx.x == 0) *alpha_j = s_sum;
}

// w -= alpha_j v + beta_{j-1} v_prev;  beta_j = ||w||
__global__ void __launch_bounds__(kLzThreads) k_lz_update(const double *__restrict__ v, const double *__restrict__ vp,
                                                          double *__restrict__ w, int64_t n, const double *alpha_j,
                                                          const double *beta_prev, double *beta_j, double *part,
                                                          unsigned *counter)
{
    const double a = *alpha_j, b = beta_prev ? *beta_prev : 0.0;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = w[i] - a * v[i] - b * vp[i];
        w[i] = x;
        acc += x * x;
    }
    __shared__ double s_sum;
    if (lz_last_block(acc, part, counter, &s_sum) && threadIdx.x == 0) *beta_j = sqrt(s_sum);
}

// x *= 1 / s (s > 0), or x = 0 when s is 0 (an invariant subspace: the recurrence ends)
__global__ void __launch_bounds__(kLzThreads) k_lz_scale(double *__restrict__ x, int64_t n, const double *s)
{
    const double d = *s;
    const double f = d > 0.0 ? 1.0 / d : 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] *= f;
}

// x = column c of X (ld), and its squared norm
__global__ void __launch_bounds__(kLzThreads) k_lz_start(const double *__restrict__ X, int64_t ld,
                                                         double *__restrict__ x, int64_t n, double *nrm2,
                                                         double *part, unsigned *counter)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double t = X[i * ld];
        x[i] = t;
        acc += t * t;
    }
    __shared__ double s_sum;
    if (lz_last_block(acc, part, counter, &s_sum) && threadIdx.x == 0) *nrm2 = sqrt(s_sum);
}

// ---- host: the tridiagonal T_m -------------------------------------------------------

// Number of eigenvalues of T_m below x (Sturm sequence of the LDL^T pivots).
int sturm_below(const std::vector<double> &a, const std::vector<double> &b, int m, double x)
{
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < m; ++i) {
        const double off = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
        d = (a[i] - x) - (i > 0 ? off / d : 0.0);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++cnt;
    }
    return cnt;
}

// The idx-th smallest eigenvalue of T_m (0-based) by bisection on [lo, hi].
double tri_eig(const std::vector<double> &a, const std::vector<double> &b, int m, int idx, double lo, double hi)
{
    for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_below(a, b, m, mid) > idx) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// |last component| of the normalised eigenvector of T_m for its extreme eigenvalue theta
// (lowest: the smallest; else the largest), by two steps of inverse iteration on
// M = s (T - theta I) + delta I, s = +1 for the lowest end and -1 for the highest: M is
// symmetric positive definite (its eigenvalues are >= delta), so the LDL^T (Thomas) solve
// needs no pivoting, and 1 / delta amplifies the wanted eigenvector.
double tri_last_component(const std::vector<double> &a, const std::vector<double> &b, int m, double theta,
                          bool lowest)
{
    if (m == 1) return 1.0;
    double scale = std::fabs(theta);
    for (int i = 0; i < m; ++i) scale = std::max(scale, std::fabs(a[i]) + std::fabs(b[i]));
    const double delta = 1e-10 * std::max(scale, 1e-300);
    const double sg = lowest ? 1.0 : -1.0;
    std::vector<double> dd(m), ll(m, 0.0), y(m, 1.0 / std::sqrt((double)m)), w(m);
    dd[0] = sg * (a[0] - theta) + delta;
    if (!(dd[0] > 1e-300)) dd[0] = 1e-300;  // rounding at the very edge of definiteness
    for (int i = 1; i < m; ++i) {
        const double off = sg * b[i - 1];
        ll[i] = off / dd[i - 1];
        dd[i] = sg * (a[i] - theta) + delta - ll[i] * off;
        if (!(dd[i] > 1e-300)) dd[i] = 1e-300;
    }
    for (int pass = 0; pass < 2; ++pass) {
        w[0] = y[0];
        for (int i = 1; i < m; ++i) w[i] = y[i] - ll[i] * w[i - 1];
        for (int i = 0; i < m; ++i) w[i] /= dd[i];
        for (int i = m - 2; i >= 0; --i) w[i] -= ll[i + 1] * w[i + 1];
        double nrm = 0.0;
        for (int i = 0; i < m; ++i) nrm += w[i] * w[i];
        nrm = std::sqrt(nrm);
        if (!(nrm > 0.0) || !std::isfinite(nrm)) return 1.0;
        for (int i = 0; i < m; ++i) y[i] = w[i] / nrm;
    }
    return std::fabs(y[m - 1]);
}

}  // namespace

size_t lanczos_workspace_bytes(int64_t n)
{
    const size_t vec = ((size_t)n * sizeof(double) + 255) & ~(size_t)255;
    return 3 * vec + 2 * (size_t)kLzMaxSteps * sizeof(double) + (size_t)(4 * num_sms() + 64) * sizeof(double) + 512;
}

int lanczos_bounds(const ChainParams &cp, int64_t n, const double *X0, int64_t ldx0, double tol, int max_iter,
                   void *ws, size_t ws_bytes, double *emin, double *emax, int *iters, cudaStream_t st)
{
    if (ws_bytes < lanczos_workspace_bytes(n)) return MBL_ERR_WORKSPACE;
    if (max_iter > kLzMaxSteps) max_iter = kLzMaxSteps;
    char *p = (char *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
    const size_t vec = ((size_t)n * sizeof(double) + 255) & ~(size_t)255;
    LzDev d;
    for (int i = 0; i < 3; ++i) {
        d.v[i] = (double *)p;
        p += vec;
    }
    d.alpha = (double *)p;
    p += (size_t)kLzMaxSteps * sizeof(double);
    d.beta = (double *)p;
    p += (size_t)kLzMaxSteps * sizeof(double);
    const int grid = std::max(1, std::min(2 * num_sms(), (int)((n + kLzThreads - 1) / kLzThreads)));
    d.part = (double *)p;
    p += (size_t)(4 * num_sms() + 8) * sizeof(double);
    d.counter = (unsigned *)p;
    double *nrm0 = (double *)(p + 64);
    if (cudaMemsetAsync(d.counter, 0, sizeof(unsigned), st) != cudaSuccess ||
        cudaMemsetAsync(d.v[0], 0, (size_t)n * sizeof(double), st) != cudaSuccess)
        return MBL_ERR_CUDA;
    // v_0 = X0[:, 0] / ||X0[:, 0]||;  v_prev = 0
    note_launch();
    k_lz_start<<<grid, kLzThreads, 0, st>>>(X0, ldx0, d.v[1], n, nrm0, d.part, d.counter);
    note_launch();
    k_lz_scale<<<grid, kLzThreads, 0, st>>>(d.v[1], n, nrm0);
    if (cudaGetLastError() != cudaSuccess) return MBL_ERR_CUDA;

    std::vector<double> a, b;
    int ip = 0, iv = 1, iw = 2;  // roles: v_prev, v, w
    int m = 0;
    double lo = 0.0, hi = 0.0;
    bool done = false, ok = false;
    for (int j = 0; j < max_iter && !done; ++j) {
        const int rc = apply_device(cp, MBL_F64, d.v[iv], 1, d.v[iw], 1, (uint32_t)n, 1, st);
        if (rc != MBL_OK) return rc;
        note_launch();
        k_lz_alpha<<<grid, kLzThreads, 0, st>>>(d.v[iv], d.v[iw], n, d.alpha + j, d.part, d.counter);
        note_launch();
        k_lz_update<<<grid, kLzThreads, 0, st>>>(d.v[iv], d.v[ip], d.v[iw], n, d.alpha + j,
                                                  j > 0 ? d.beta + j - 1 : nullptr, d.beta + j, d.part, d.counter);
        note_launch();
        k_lz_scale<<<grid, kLzThreads, 0, st>>>(d.v[iw], n, d.beta + j);
        if (cudaGetLastError() != cudaSuccess) return MBL_ERR_CUDA;
        const int t = ip;
        ip = iv;
        iv = iw;
        iw = t;
        m = j + 1;
        if (m % kLzCheckEvery != 0 && m != max_iter) continue;
        a.resize(m);
        b.resize(m);
        if (cudaMemcpyAsync(a.data(), d.alpha, m * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(b.data(), d.beta, m * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return MBL_ERR_CUDA;
        for (int i = 0; i < m; ++i)
            if (!std::isfinite(a[i]) || !std::isfinite(b[i])) return MBL_ERR_NUMERIC;
        // Gershgorin interval of T_m, then both ends by bisection
        double glo = a[0], ghi = a[0];
        for (int i = 0; i < m; ++i) {
            const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
            glo = std::min(glo, a[i] - r);
            ghi = std::max(ghi, a[i] + r);
        }
        lo = tri_eig(a, b, m, 0, glo, ghi);
        hi = tri_eig(a, b, m, m - 1, glo, ghi);
        const double bm = b[m - 1];
        const double rlo = std::fabs(bm) * tri_last_component(a, b, m, lo, true);
        const double rhi = std::fabs(bm) * tri_last_component(a, b, m, hi, false);
        ok = (rlo <= tol * std::fabs(lo) && rhi <= tol * std::fabs(hi)) || bm == 0.0;
        done = ok;
    }
    if (m == 0) return MBL_ERR_ARG;
    *emin = lo;
    *emax = hi;
    if (iters) *iters = m;
    return ok ? MBL_OK : MBL_ERR_NOT_CONVERGED;
}

}  // namespace mbl
