// mbl_lobpcg.cu -- folded-spectrum LOBPCG with a Jacobi-PCG preconditioner (Sec. 3.2,
// Sec. 6.2), and the ABI entries of the spectrum bounds used to place sigma (the Lanczos
// recurrence itself is in mbl_lanczos.cu).
//
// One iteration (every product of H runs in the gather kernels of mbl_apply.cu; every
// reduction is deterministic):
//   1. H Rayleigh-Ritz on span(X): M = X^T (H - sigma)X, eig M = V mu V^T,
//      E = (H - sigma)X - X M, residual_j = ||E v_j||; accept the nev values nearest 0.
//   2. R = AX - X (X^T A X)              (A = (H - sigma)^2)
//   3. W = PCG_m(R / ||R||) column-wise, Jacobi M = diag(A)      [FP32 in mixed mode]
//   4. W <- W - X (X^T W), twice;  AW = A W
//   5. P <- P - X (X^T P), twice;  AP = A P     (from the second iteration on)
//   6. SVQB on S = [X W P] and Rayleigh-Ritz with A; keep the k smallest
//   7. X <- S C_X, P <- [W P] C_[W,P] (unit columns), X <- Cholesky-QR(X)
//   8. T = (H - sigma)X, AX = (H - sigma)T
// Steps 2..8 plus step 1 of the next iteration are enqueued without host
// synchronisation and can be captured once as a CUDA graph and replayed; the host
// reads a few status words per iteration.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <mutex>
#include <thread>
#include <vector>

#include "mbl_dense.h"
#include "mbl_device.cuh"
#include "mbl_internal.h"

namespace mbl {

static std::atomic<int64_t> g_kernel_launches{0};
static thread_local bool t_capturing = false;

void note_launch(int64_t count)
{
    if (!t_capturing) g_kernel_launches.fetch_add(count, std::memory_order_relaxed);
}

void set_capturing(bool on) { t_capturing = on; }

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Carver {
    size_t off = 0;
    char *base = nullptr;
    template <typename T>
    T *take(size_t count)
    {
        size_t o = off;
        off = align_up(off + count * sizeof(T));
        return base ? reinterpret_cast<T *>(base + o) : nullptr;
    }
};

// Device buffers of one solve (the workspace carve-up).
struct Buffers {
    double *S, *AS, *T, *Tmp, *Xn;
    void *pr, *pp, *pt, *pw, *dinv;  // PCG vectors (float or double)
    double *G1, *G2, *G3, *Gk;       // Grams: (3k)^2 x 2, k^2 x 2
    double *part;                    // Gram / column partials
    double *mu, *V, *Rinv, *coef, *theta, *Csel, *res_all, *res_sel, *rn, *eigw;
    double *pcg_s;                   // rz, rz0, alpha, beta (4 x 64)
    int *pcg_active;
    double *pcg_part;
    unsigned *counter;
    int *iflags;                     // [0] chol flag, [1..2] rr info, [4..5] hrr status, [8..] sel
    double *dstat;                   // [0] max rel resid, [1] gershgorin
    uint32_t *states;                // sector basis, n words
};

// Largest scratch any reduction of the iteration needs: Grams of widths k, 2k, 3k and
// the column norms.
size_t part_doubles(int64_t n, int k)
{
    size_t m = colnorm_partial_doubles(k);
    for (int w = 1; w <= 3; ++w) {
        size_t a = gram_partial_doubles(n, w * k, w * k);
        if (a > m) m = a;
    }
    return m;
}

Buffers carve(char *base, int64_t n, int k, int pcg_f32, size_t *bytes)
{
    Carver c;
    c.base = base;
    Buffers b{};
    const size_t nk = (size_t)n * k;
    const size_t es = pcg_f32 ? 4 : 8;
    b.S = c.take<double>(3 * nk);
    b.AS = c.take<double>(3 * nk);
    b.T = c.take<double>(nk);
    b.Tmp = c.take<double>(nk);
    b.Xn = c.take<double>(nk);
    b.pr = c.take<char>(nk * es);
    b.pp = c.take<char>(nk * es);
    b.pt = c.take<char>(nk * es);
    b.pw = c.take<char>(nk * es);
    b.dinv = c.take<char>((size_t)n * es);
    const size_t w2 = (size_t)9 * k * k;
    b.G1 = c.take<double>(w2);
    b.G2 = c.take<double>(w2);
    b.G3 = c.take<double>(w2);
    b.Gk = c.take<double>((size_t)k * k);
    b.part = c.take<double>(part_doubles(n, k));
    b.mu = c.take<double>(3 * k);
    b.V = c.take<double>((size_t)k * k);
    b.Rinv = c.take<double>((size_t)k * k);
    b.coef = c.take<double>(w2);
    b.theta = c.take<double>(3 * k);
    b.Csel = c.take<double>((size_t)k * k);
    b.res_all = c.take<double>(k);
    b.res_sel = c.take<double>(k);
    b.rn = c.take<double>(k);
    size_t ew = small_rr_work_doubles(3 * k);
    size_t ew2 = small_eig_work_doubles(3 * k);
    b.eigw = c.take<double>(ew > ew2 ? ew : ew2);
    b.pcg_s = c.take<double>(4 * 64);
    b.pcg_active = c.take<int>(64);
    b.pcg_part = c.take<double>(pcg_partial_doubles());
    b.counter = c.take<unsigned>(4);
    b.iflags = c.take<int>(16 + 64);
    b.dstat = c.take<double>(8);
    b.states = c.take<uint32_t>((size_t)n);
    *bytes = c.off;
    return b;
}

int check_opts(const mbl_chain *chain, const mbl_lobpcg_opts *o, int64_t *n_out)
{
    if (!chain || !o) return MBL_ERR_ARG;
    int64_t n = mbl_basis_size(chain->L, chain->n_up);
    if (n <= 0 || chain->L < 2) return MBL_ERR_ARG;
    if (o->k < 1 || o->k > 64 || o->nev < 1 || o->nev > o->k) return MBL_ERR_ARG;
    if ((int64_t)3 * o->k > n) return MBL_ERR_ARG;
    if (o->max_iter < 0 || o->pcg_iters < 0) return MBL_ERR_ARG;
    if (!(o->tol > 0.0) || !(o->pcg_tol >= 0.0)) return MBL_ERR_ARG;
    if (o->mode != MBL_MODE_FP64 && o->mode != MBL_MODE_MIXED) return MBL_ERR_ARG;
    *n_out = n;
    return MBL_OK;
}

#define MBL_TRY(expr)                   \
    do {                                \
        int rc__ = (expr);              \
        if (rc__ != MBL_OK) return rc__; \
    } while (0)

// The solver state for one call.
struct Solver {
    ChainParams cp;
    int64_t n;
    int k, nev, m;
    int mixed;
    int gmix;     // Rayleigh-Ritz Grams and eigensolves in FP32 (mixed mode until a stall)
    int largest;  // bounds mode, -H: keep the largest Ritz values
    int folded;   // 1: A = (H - sigma)^2 with PCG; 0: A = H - sigma, no preconditioner
    double tol_abs, norm_h, pcg_tol;
    Buffers b;
    cudaStream_t st;
    int64_t matvecs = 0;
    // optional phase timing: events recorded at the phase boundaries of each iteration
    bool timing = false;
    cudaEvent_t ev[10] = {};
    double tphase[10] = {};
    void mark(int i)
    {
        if (timing) cudaEventRecord(ev[i], st);
    }
    void accumulate(int first, int last, int slot0)  // tphase[slot0 + j] += ev[first+j] -> ev[first+j+1]
    {
        if (!timing) return;
        for (int i = first; i < last; ++i) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess) tphase[slot0 + i - first] += 1e-3 * ms;
        }
    }

    double *X() { return b.S; }
    double *W() { return b.S + k; }
    double *P() { return b.S + 2 * k; }
    double *AX() { return b.AS; }
    double *AW() { return b.AS + k; }
    double *AP() { return b.AS + 2 * k; }
    int64_t ld3() const { return 3 * (int64_t)k; }

    int apply64(const double *Xp, int64_t ldx, double *Yp, int64_t ldy)
    {
        matvecs += k;
        return apply_device(cp, MBL_F64, Xp, ldx, Yp, ldy, (uint32_t)n, k, st);
    }
    // Y = A X: two products through Tmp when folded
    int applyA(const double *Xp, int64_t ldx, double *Yp, int64_t ldy)
    {
        if (!folded) return apply64(Xp, ldx, Yp, ldy);
        MBL_TRY(apply64(Xp, ldx, b.Tmp, k));
        return apply64(b.Tmp, k, Yp, ldy);
    }
    // X <- X - X_ref (X_ref^T X), twice (block classical Gram-Schmidt against X)
    // B -= X (X^T B), twice.  B is a search direction (W from the preconditioner, or P):
    // the Rayleigh-Ritz that follows resolves it only to FP32 in mixed mode, so the
    // projection runs in FP32 there (X itself and every residual stay FP64).
    int ortho_against_x(double *Bp)
    {
        for (int pass = 0; pass < 2; ++pass) {
            MBL_TRY(gram(X(), ld3(), k, Bp, ld3(), k, n, b.Gk, k, 0, gmix, b.part, st));
            MBL_TRY(update(X(), ld3(), k, b.Gk, k, k, Bp, ld3(), Bp, ld3(), n, -1.0, 1.0, gmix, st));
        }
        return MBL_OK;
    }
    // X <- Cholesky-QR(src) into the X slice; flag -> iflags[0]
    int cholqr_into_x(const double *src, int64_t lds)
    {
        MBL_TRY(gram(src, lds, k, src, lds, k, n, b.Gk, k, 1, 0, b.part, st));
        MBL_TRY(small_chol_inv(k, b.Gk, k, b.Rinv, b.eigw, b.iflags + 0, st));
        return update(src, lds, k, b.Rinv, k, k, nullptr, 0, X(), ld3(), n, 1.0, 0.0, 0, st);
    }
    int refresh_tx()  // T = (H - sigma)X, AX = (H - sigma)T   (or AX = T when unfolded)
    {
        MBL_TRY(apply64(X(), ld3(), b.T, k));
        if (folded) return apply64(b.T, k, AX(), ld3());
        return copy_block(b.T, k, AX(), ld3(), k, n, st);
    }
    // Step 1: H Rayleigh-Ritz on span(X) and the convergence status (folded mode).
    int enqueue_hrr()
    {
        MBL_TRY(gram(X(), ld3(), k, b.T, k, k, n, b.Gk, k, 1, 0, b.part, st));
        MBL_TRY(small_eig(k, b.Gk, k, b.mu, b.V, b.eigw, st));
        MBL_TRY(update(X(), ld3(), k, b.Gk, k, k, b.T, k, b.Tmp, k, n, -1.0, 1.0, 0, st));
        // E^T E in FP64 in both modes: a converged pair's residual is read off this Gram
        // next to the guard columns' much larger ones, and FP32 rounding of the latter
        // (sqrt(u32) times their norm) would hide residuals below ~1e-7 of them
        MBL_TRY(gram(b.Tmp, k, k, b.Tmp, k, k, n, b.G3, k, 1, 0, b.part, st));
        return hrr_select(k, nev, b.mu, b.V, b.G3, tol_abs, norm_h, b.res_all, b.iflags + 8, b.res_sel,
                          b.iflags + 4, b.dstat, st);
    }
    // Bounds mode status: theta_0 and ||R_0|| from AX = H X (sign handled by 'largest').
    int enqueue_bounds_status()
    {
        MBL_TRY(gram(X(), ld3(), k, AX(), ld3(), k, n, b.Gk, k, 1, 0, b.part, st));
        MBL_TRY(update(X(), ld3(), k, b.Gk, k, k, AX(), ld3(), b.Tmp, k, n, -1.0, 1.0, 0, st));
        MBL_TRY(colnorms(b.Tmp, k, k, n, b.rn, 1, b.part, st));
        return MBL_OK;
    }
    PcgDev pcg_dev() const
    {
        return PcgDev{b.pcg_s, b.pcg_s + 64, b.pcg_s + 128, b.pcg_s + 192, b.pcg_active, pcg_tol * pcg_tol,
                      b.pcg_part, b.counter};
    }
    // Step 2 and the start of step 3: the residual of the current block and, folded, the
    // PCG start from its normalised columns.
    int enqueue_pre_pcg()
    {
        mark(0);
        MBL_TRY(gram(X(), ld3(), k, AX(), ld3(), k, n, b.Gk, k, 1, gmix, b.part, st));
        MBL_TRY(update(X(), ld3(), k, b.Gk, k, k, AX(), ld3(), b.Tmp, k, n, -1.0, 1.0, 0, st));
        mark(1);
        if (!folded) return MBL_OK;
        MBL_TRY(colnorms(b.Tmp, k, k, n, b.rn, 1, b.part, st));
        const PcgDev pd = pcg_dev();
        if (mixed)
            return pcg_start<float>(b.Tmp, k, b.rn, (uint32_t)n, k, (const float *)b.dinv, (float *)b.pr,
                                    (float *)b.pp, (float *)b.pw, pd, st);
        return pcg_start<double>(b.Tmp, k, b.rn, (uint32_t)n, k, (const double *)b.dinv, (double *)b.pr,
                                 (double *)b.pp, (double *)b.pw, pd, st);
    }
    // Step 3: the m PCG steps of this problem alone.
    int enqueue_pcg_steps()
    {
        const PcgDev pd = pcg_dev();
        for (int it = 0; it < m; ++it) {
            if (mixed)
                MBL_TRY(pcg_step<float>(cp, (uint32_t)n, k, (const float *)b.dinv, (float *)b.pr, (float *)b.pp,
                                        (float *)b.pt, (float *)b.pw, pd, st));
            else
                MBL_TRY(pcg_step<double>(cp, (uint32_t)n, k, (const double *)b.dinv, (double *)b.pr,
                                         (double *)b.pp, (double *)b.pt, (double *)b.pw, pd, st));
        }
        return MBL_OK;
    }
    // Steps 4..8 (+ the status of the next iteration), after the preconditioner.
    int enqueue_post_pcg(bool have_p)
    {
        if (folded) {
            matvecs += (int64_t)2 * m * k;
            MBL_TRY(widen(mixed, b.pw, k, W(), ld3(), k, n, st));
        } else {
            MBL_TRY(copy_block(b.Tmp, k, W(), ld3(), k, n, st));
        }
        mark(2);
        // 4. W against X, then A W
        MBL_TRY(ortho_against_x(W()));
        MBL_TRY(applyA(W(), ld3(), AW(), ld3()));
        // 5. P against X, then A P
        if (have_p) {
            MBL_TRY(ortho_against_x(P()));
            MBL_TRY(applyA(P(), ld3(), AP(), ld3()));
        }
        mark(3);
        // 6. SVQB + Rayleigh-Ritz with A
        const int w = have_p ? 3 * k : 2 * k;
        MBL_TRY(gram(b.S, ld3(), w, b.S, ld3(), w, n, b.G1, w, 1, gmix, b.part, st));
        MBL_TRY(gram(b.S, ld3(), w, b.AS, ld3(), w, n, b.G2, w, 1, gmix, b.part, st));
        mark(4);
        MBL_TRY(small_svqb_rr(w, k, largest, gmix, b.G1, b.G2, svqb_tau(), b.coef, b.theta, b.eigw, b.iflags + 1, st));
        mark(5);
        // 7. updates.  The new direction P = [W P] C_WP first (FP32 in mixed mode, like W and
        // P themselves), then X_new = S C = X C_X + P: the [W P] product is formed once, and
        // the FP64 update of X only spans X's own k columns
        MBL_TRY(update(W(), ld3(), w - k, b.coef + (int64_t)k * k, k, k, nullptr, 0, P(), ld3(), n, 1.0, 0.0, gmix,
                       st));
        MBL_TRY(update(X(), ld3(), k, b.coef, k, k, P(), ld3(), b.Xn, k, n, 1.0, 1.0, 0, st));
        MBL_TRY(colnorms(P(), ld3(), k, n, b.rn, 1, b.part, st));
        MBL_TRY(scale_cols_inv(P(), ld3(), k, n, b.rn, st));
        MBL_TRY(cholqr_into_x(b.Xn, k));
        mark(6);
        // 8. products for the new block, and the status of the next iteration
        MBL_TRY(refresh_tx());
        mark(7);
        MBL_TRY(folded ? enqueue_hrr() : enqueue_bounds_status());
        mark(8);
        return MBL_OK;
    }
    // Steps 2..8 (+ the status of the next iteration).
    int enqueue_body(bool have_p)
    {
        MBL_TRY(enqueue_pre_pcg());
        if (folded) MBL_TRY(enqueue_pcg_steps());
        return enqueue_post_pcg(have_p);
    }
    // Directions below the resolution of the Gram matrix are dropped: its entries carry
    // FP32 rounding in mixed mode.
    double svqb_tau() const { return gmix ? 1e-7 : 1e-14; }
};

// The rotation of the start block onto A's Ritz vectors (X, T, AX <- . C).
int initial_rr(Solver &s)
{
    MBL_TRY(gram(s.X(), s.ld3(), s.k, s.AX(), s.ld3(), s.k, s.n, s.b.Gk, s.k, 1, 0, s.b.part, s.st));
    MBL_TRY(small_eig(s.k, s.b.Gk, s.k, s.b.mu, s.b.V, s.b.eigw, s.st));
    if (s.largest) {
        // reverse column order so that column 0 is the largest Ritz value
        // (done by a tiny gather with reversed indices)
        int sel_rev[64];
        for (int j = 0; j < s.k; ++j) sel_rev[j] = s.k - 1 - j;
        MBL_TRY(cudaMemcpyAsync(s.b.iflags + 8, sel_rev, sizeof(int) * s.k, cudaMemcpyHostToDevice, s.st) ==
                        cudaSuccess
                    ? MBL_OK
                    : MBL_ERR_CUDA);
        MBL_TRY(gather_cols(s.k, s.k, s.b.V, s.b.iflags + 8, s.b.Csel, s.st));
        // keep the host array alive until the copy is done
        if (cudaStreamSynchronize(s.st) != cudaSuccess) return MBL_ERR_CUDA;
    } else {
        MBL_TRY(copy_block(s.b.V, s.k, s.b.Csel, s.k, s.k, s.k, s.st));
    }
    MBL_TRY(update(s.X(), s.ld3(), s.k, s.b.Csel, s.k, s.k, nullptr, 0, s.b.Xn, s.k, s.n, 1.0, 0.0, 0, s.st));
    MBL_TRY(copy_block(s.b.Xn, s.k, s.X(), s.ld3(), s.k, s.n, s.st));
    return s.refresh_tx();
}

struct HostStatus {
    int iflags[16];
    double dstat[8];
};

int read_status(Solver &s, HostStatus *h)
{
    if (cudaMemcpyAsync(h->iflags, s.b.iflags, sizeof(h->iflags), cudaMemcpyDeviceToHost, s.st) != cudaSuccess)
        return MBL_ERR_CUDA;
    if (cudaMemcpyAsync(h->dstat, s.b.dstat, sizeof(h->dstat), cudaMemcpyDeviceToHost, s.st) != cudaSuccess)
        return MBL_ERR_CUDA;
    if (cudaStreamSynchronize(s.st) != cudaSuccess) return MBL_ERR_CUDA;
    return MBL_OK;
}

// Capture body(have_p) once into an executable graph.
struct GraphCache {
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    int64_t kernels[2] = {0, 0};  // kernel nodes per graph
    cudaStream_t cap = nullptr;
    // drop the captured bodies (after a change of the body's precision)
    void reset()
    {
        for (int i = 0; i < 2; ++i) {
            if (exec[i]) cudaGraphExecDestroy(exec[i]);
            exec[i] = nullptr;
            kernels[i] = 0;
        }
    }
    ~GraphCache()
    {
        reset();
        if (cap) cudaStreamDestroy(cap);
    }
};

int run_body(Solver &s, bool have_p, bool use_graph, GraphCache &gc)
{
    if (!use_graph) return s.enqueue_body(have_p);
    const int slot = have_p ? 1 : 0;
    if (!gc.exec[slot]) {
        if (!gc.cap && cudaStreamCreateWithFlags(&gc.cap, cudaStreamNonBlocking) != cudaSuccess) return MBL_ERR_CUDA;
        cudaStream_t user = s.st;
        s.st = gc.cap;
        int64_t mv = s.matvecs;
        if (cudaStreamBeginCapture(gc.cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            s.st = user;
            return MBL_ERR_CUDA;
        }
        set_capturing(true);
        int rc = s.enqueue_body(have_p);
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(gc.cap, &g);
        set_capturing(false);
        s.st = user;
        s.matvecs = mv;  // counted again at each replay below
        if (rc != MBL_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ce != cudaSuccess || !g) return MBL_ERR_CUDA;
        size_t nn = 0;
        if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
            std::vector<cudaGraphNode_t> nodes(nn);
            if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
                for (size_t i = 0; i < nn; ++i) {
                    cudaGraphNodeType ty;
                    if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel)
                        ++gc.kernels[slot];
                }
        }
        ce = cudaGraphInstantiate(&gc.exec[slot], g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) return MBL_ERR_CUDA;
    }
    // matvec accounting of one body
    s.matvecs += (int64_t)(s.folded ? 2 * s.m * s.k + 2 * s.k + (have_p ? 2 * s.k : 0) + 2 * s.k
                                    : s.k + (have_p ? s.k : 0) + s.k);
    if (cudaGraphLaunch(gc.exec[slot], s.st) != cudaSuccess) return MBL_ERR_CUDA;
    note_launch(gc.kernels[slot]);
    return MBL_OK;
}

// Everything before the first iteration, enqueued on st: the workspace carve-up, the
// sector basis, the norm of the tolerance (a Gershgorin bound, read back with a host
// synchronisation, when opts->norm_h <= 0), the preconditioner diagonal, and the start
// block orthonormalised and rotated onto A's Ritz vectors with its first H Rayleigh-Ritz
// status.
int solver_setup(Solver &s, const mbl_chain *chain, double sigma, const mbl_lobpcg_opts *opts, int64_t n,
                 const double *X0_dev, void *workspace_dev, size_t workspace_bytes, cudaStream_t st)
{
    const mbl_stream_t stream = (mbl_stream_t)st;
    int rc = make_chain_params(chain, sigma, &s.cp);
    if (rc != MBL_OK) return rc;
    size_t need = 0;
    const int mixed = opts->mode == MBL_MODE_MIXED;
    s.b = carve((char *)workspace_dev, n, opts->k, mixed, &need);
    if (workspace_bytes < need) return MBL_ERR_WORKSPACE;
    s.n = n;
    s.k = opts->k;
    s.nev = opts->nev;
    s.m = opts->pcg_iters;
    s.mixed = mixed;
    s.gmix = mixed;
    s.largest = 0;
    s.folded = 1;
    s.pcg_tol = opts->pcg_tol;
    s.st = st;
    s.matvecs = 0;
    const int k = s.k;
    if (cudaMemsetAsync(s.b.counter, 0, 4 * sizeof(unsigned), s.st) != cudaSuccess ||
        cudaMemsetAsync(s.b.iflags, 0, (16 + 64) * sizeof(int), s.st) != cudaSuccess)
        return MBL_ERR_CUDA;
    s.timing = opts->timing != 0;
    if (s.timing) {
        for (auto &e : s.ev)
            if (cudaEventCreate(&e) != cudaSuccess) return MBL_ERR_CUDA;
        s.mark(9);
    }
    // sector basis, read by every product kernel of the solve
    MBL_TRY(ensure_lowtabs_for(chain->L));  // before any graph capture
    MBL_TRY(mbl_basis_build(chain->L, chain->n_up, s.b.states, n, stream));
    s.cp.states = s.b.states;
    // norm used to scale the tolerance
    double norm_h = opts->norm_h;
    if (!(norm_h > 0.0)) {
        ChainParams c0;
        make_chain_params(chain, 0.0, &c0);
        MBL_TRY(gershgorin_bound(c0, (uint32_t)n, s.b.part, s.b.counter, s.b.dstat + 1, s.st));
        if (cudaMemcpyAsync(&norm_h, s.b.dstat + 1, sizeof(double), cudaMemcpyDeviceToHost, s.st) != cudaSuccess ||
            cudaStreamSynchronize(s.st) != cudaSuccess)
            return MBL_ERR_CUDA;
    }
    s.norm_h = norm_h;
    s.tol_abs = opts->tol * norm_h;

    // Jacobi preconditioner diagonal
    if (mixed)
        MBL_TRY(pcg_fold_dinv<float>(s.cp, (uint32_t)n, (float *)s.b.dinv, s.st));
    else
        MBL_TRY(pcg_fold_dinv<double>(s.cp, (uint32_t)n, (double *)s.b.dinv, s.st));

    // start block: orthonormalise, products, rotate onto A's Ritz vectors
    MBL_TRY(s.cholqr_into_x(X0_dev, k));
    MBL_TRY(s.refresh_tx());
    MBL_TRY(initial_rr(s));
    MBL_TRY(s.enqueue_hrr());
    if (s.timing) cudaEventRecord(s.ev[0], s.st);
    return MBL_OK;
}

}  // namespace

}  // namespace mbl

using namespace mbl;

extern "C" int mbl_lobpcg_workspace_size(const mbl_chain *chain, const mbl_lobpcg_opts *opts, size_t *bytes)
{
    int64_t n;
    if (!bytes) return MBL_ERR_ARG;
    int rc = check_opts(chain, opts, &n);
    if (rc != MBL_OK) return rc;
    carve(nullptr, n, opts->k, opts->mode == MBL_MODE_MIXED, bytes);
    return MBL_OK;
}

extern "C" int mbl_lobpcg_solve(const mbl_chain *chain, double sigma, const mbl_lobpcg_opts *opts,
                                const double *X0_dev, void *workspace_dev, size_t workspace_bytes,
                                double *evals_host, double *evecs_dev, double *resid_host, mbl_lobpcg_stats *stats,
                                mbl_stream_t stream)
{
    auto t0 = std::chrono::steady_clock::now();
    int64_t n;
    int rc = check_opts(chain, opts, &n);
    if (rc != MBL_OK) return rc;
    if (!X0_dev || !workspace_dev) return MBL_ERR_ARG;
    if ((uintptr_t)workspace_dev % kAlign) return MBL_ERR_ARG;
    Solver s;
    rc = solver_setup(s, chain, sigma, opts, n, X0_dev, workspace_dev, workspace_bytes, (cudaStream_t)stream);
    if (rc != MBL_OK) {
        if (s.timing)
            for (auto &e : s.ev)
                if (e) cudaEventDestroy(e);
        return rc;
    }
    const int k = s.k;
    const double norm_h = s.norm_h;

    HostStatus hs;
    GraphCache gc;
    int it = 0;
    bool have_p = false;
    int status = MBL_OK;
    const bool graphs = opts->use_graph != 0 && !s.timing;
    // Mixed mode keeps its Rayleigh-Ritz in FP32 while the residual keeps falling; once the
    // largest wanted residual has not dropped by 10 % for kStallIters iterations, the FP32
    // Grams of the folded operator are taken to limit it (their rounding, ~1e-7 ||A||,
    // swamps the small gaps of A near sigma) and the remaining iterations run them in FP64.
    constexpr int kStallIters = 20;
    double r_mark = 0.0;
    int it_mark = 0;
    for (;;) {
        MBL_TRY(read_status(s, &hs));
        if (s.gmix) {
            const double r = hs.dstat[0];
            if (it == 0 || r < 0.9 * r_mark) {
                r_mark = r;
                it_mark = it;
            } else if (it - it_mark >= kStallIters) {
                s.gmix = 0;
                gc.reset();
            }
        }
        if (s.timing) {
            if (it == 0) {
                float ms = 0.f;
                if (cudaEventElapsedTime(&ms, s.ev[9], s.ev[0]) == cudaSuccess) s.tphase[9] += 1e-3 * ms;
            } else {
                s.accumulate(0, 8, 0);
            }
        }
        if (hs.iflags[5] || hs.iflags[2]) {
            status = MBL_ERR_NUMERIC;
            break;
        }
        if (hs.iflags[0]) {
            status = MBL_ERR_BREAKDOWN;
            break;
        }
        if (hs.iflags[4]) break;
        if (it >= opts->max_iter) {
            status = MBL_ERR_NOT_CONVERGED;
            break;
        }
        MBL_TRY(run_body(s, have_p, graphs, gc));
        have_p = true;
        ++it;
    }
    // final extraction: evecs = X V[:, sel]
    MBL_TRY(gather_cols(k, s.nev, s.b.V, s.b.iflags + 8, s.b.Csel, s.st));
    if (evecs_dev)
        MBL_TRY(update(s.X(), s.ld3(), k, s.b.Csel, s.nev, s.nev, nullptr, 0, evecs_dev, s.nev, n, 1.0, 0.0, 0, s.st));
    double mu_h[64], res_h[64];
    int sel_h[64];
    if (cudaMemcpyAsync(mu_h, s.b.mu, sizeof(double) * k, cudaMemcpyDeviceToHost, s.st) != cudaSuccess ||
        cudaMemcpyAsync(sel_h, s.b.iflags + 8, sizeof(int) * s.nev, cudaMemcpyDeviceToHost, s.st) != cudaSuccess ||
        cudaMemcpyAsync(res_h, s.b.res_sel, sizeof(double) * s.nev, cudaMemcpyDeviceToHost, s.st) != cudaSuccess ||
        cudaStreamSynchronize(s.st) != cudaSuccess)
        return MBL_ERR_CUDA;
    double mx = 0.0;
    for (int j = 0; j < s.nev; ++j) {
        if (evals_host) evals_host[j] = sigma + mu_h[sel_h[j]];
        if (resid_host) resid_host[j] = res_h[j];
        mx = fmax(mx, res_h[j] / norm_h);
    }
    if (stats) {
        stats->iters = it;
        stats->converged = (status == MBL_OK) ? 1 : 0;
        stats->matvecs = s.matvecs;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        stats->max_rel_resid = mx;
        stats->norm_h = norm_h;
        stats->t_setup = s.tphase[9];
        stats->t_resid = s.tphase[0];
        stats->t_pcg = s.tphase[1];
        stats->t_wp = s.tphase[2];
        stats->t_gram = s.tphase[3];
        stats->t_small = s.tphase[4];
        stats->t_update = s.tphase[5];
        stats->t_refresh = s.tphase[6];
        stats->t_hrr = s.tphase[7];
    }
    if (s.timing)
        for (auto &e : s.ev) cudaEventDestroy(e);
    return status;
}

// ------------------------------------------------------------------------------------
// Spectrum bounds.

extern "C" int mbl_bounds_workspace_size(const mbl_chain *chain, int k, size_t *bytes)
{
    if (!chain || !bytes || k < 2 || k > 16) return MBL_ERR_ARG;
    int64_t n = mbl_basis_size(chain->L, chain->n_up);
    if (n <= 0 || (int64_t)3 * k > n) return MBL_ERR_ARG;
    *bytes = lanczos_workspace_bytes(n);
    return MBL_OK;
}

extern "C" int mbl_spectrum_bounds(const mbl_chain *chain, int k, double tol, int max_iter, const double *X0_dev,
                                   void *workspace_dev, size_t workspace_bytes, double *emin_host, double *emax_host,
                                   int *iters_host, mbl_stream_t stream)
{
    size_t need = 0;
    int rc = mbl_bounds_workspace_size(chain, k, &need);
    if (rc != MBL_OK) return rc;
    if (!X0_dev || !workspace_dev || !(tol > 0.0) || max_iter < 1) return MBL_ERR_ARG;
    if (workspace_bytes < need) return MBL_ERR_WORKSPACE;
    ChainParams cp;
    rc = make_chain_params(chain, 0.0, &cp);
    if (rc != MBL_OK) return rc;
    MBL_TRY(ensure_lowtabs_for(chain->L));
    if (iters_host) *iters_host = 0;
    double lo = 0.0, hi = 0.0;
    const int64_t n = mbl_basis_size(chain->L, chain->n_up);
    rc = lanczos_bounds(cp, n, X0_dev, k, tol, max_iter, workspace_dev, workspace_bytes, &lo, &hi, iters_host,
                        (cudaStream_t)stream);
    if (rc != MBL_OK && rc != MBL_ERR_NOT_CONVERGED) return rc;
    if (emin_host) *emin_host = lo;
    if (emax_host) *emax_host = hi;
    return rc;
}

// ------------------------------------------------------------------------------------
// Solve without any allocation: the workspace is a fixed array in device memory that
// exists from module load to process exit on every device that loads this library.

namespace {

constexpr size_t kNoAllocBytes = (size_t)MBL_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Host code must not use g_noalloc_scratch as an address: its name only stands for the
// device symbol.  The device address is looked up once per device (with that device
// current) and cached.
constexpr int kMaxDevices = 64;
void *g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mutex;

int noalloc_scratch(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MBL_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return MBL_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MBL_ERR_CUDA;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return MBL_OK;
}

}  // namespace

extern "C" int mbl_lobpcg_solve_noalloc(const mbl_chain *chain, double sigma, const mbl_lobpcg_opts *opts,
                                        const double *X0_dev, double *evals_host, double *evecs_dev,
                                        double *resid_host, mbl_lobpcg_stats *stats, mbl_stream_t stream)
{
    size_t need = 0;
    int rc = mbl_lobpcg_workspace_size(chain, opts, &need);
    if (rc != MBL_OK) return rc;
    if (need > kNoAllocBytes) return MBL_ERR_WORKSPACE;
    // the array looked up below is the current device's: the stream must run there
    int cur = 0, sdev = 0;
    if (cudaGetDevice(&cur) != cudaSuccess || cudaStreamGetDevice((cudaStream_t)stream, &sdev) != cudaSuccess)
        return MBL_ERR_CUDA;
    if (sdev != cur) return MBL_ERR_ARG;
    void *ws = nullptr;
    rc = noalloc_scratch(&ws);
    if (rc != MBL_OK) return rc;
    // graph instantiation and timing events would allocate: both are switched off
    mbl_lobpcg_opts o = *opts;
    o.use_graph = 0;
    o.timing = 0;
    return mbl_lobpcg_solve(chain, sigma, &o, X0_dev, ws, kNoAllocBytes, evals_host, evecs_dev, resid_host, stats,
                            stream);
}

// ------------------------------------------------------------------------------------
// Batched solve: many disorder realisations (any mix of L) advanced in lock step.  The
// workspace holds nlanes slots; each lane solves one problem at a time, and every round
// advances every lane by one LOBPCG iteration on the caller's stream: the steps before
// and after the preconditioner are enqueued lane by lane, and the m PCG steps of all
// lanes run as three launches per step over a table of the lanes (pcg_batch_step).  A
// lane whose problem has converged (or reached max_iter) writes its results and takes
// the next problem.  The host synchronises once per round and reads each lane's status
// words.  When no shifts are given, each problem's spectrum bounds are found first by
// nlanes host threads, one stream and one slot each.

namespace {

constexpr int kBatchBoundsK = 4;
constexpr double kBatchBoundsTol = 1e-7;

size_t batch_slot_bytes(int nprob, const mbl_chain *chains, const mbl_lobpcg_opts *opts, int *rc)
{
    size_t slot = 0;
    *rc = MBL_OK;
    for (int i = 0; i < nprob; ++i) {
        size_t a = 0, b = 0;
        int r = mbl_lobpcg_workspace_size(&chains[i], opts, &a);
        if (r != MBL_OK) {
            *rc = r;
            return 0;
        }
        if (mbl_bounds_workspace_size(&chains[i], kBatchBoundsK, &b) != MBL_OK) b = 0;
        slot = std::max(slot, std::max(a, b));
    }
    return align_up(slot);
}

size_t batch_table_bytes(int nlanes) { return align_up((size_t)nlanes * sizeof(PcgLane)); }

// sigma_i and ||H||_i of every problem from its own Lanczos bounds, nth host threads.
int batch_bounds(int nprob, const mbl_chain *chains, const double *X0_dev, const std::vector<int64_t> &off_x,
                 int k, void *workspace_dev, size_t slot, int nth, cudaStream_t after, double norm_given,
                 std::vector<double> &sig, std::vector<double> &nh)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MBL_ERR_CUDA;
    cudaEvent_t start_ev;
    if (cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming) != cudaSuccess) return MBL_ERR_CUDA;
    if (cudaEventRecord(start_ev, after) != cudaSuccess) {
        cudaEventDestroy(start_ev);
        return MBL_ERR_CUDA;
    }
    std::atomic<int> next{0};
    std::atomic<int> first_error{MBL_OK};
    auto worker = [&](int wid) {
        if (cudaSetDevice(dev) != cudaSuccess) {
            first_error.store(MBL_ERR_CUDA);
            return;
        }
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            first_error.store(MBL_ERR_CUDA);
            return;
        }
        cudaStreamWaitEvent(st, start_ev, 0);
        void *ws = (char *)workspace_dev + slot * (size_t)wid;
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= nprob || first_error.load() != MBL_OK) break;
            const mbl_chain &ch = chains[i];
            double lo = 0.0, hi = 0.0;
            int it = 0;
            ChainParams cpb;
            int r1 = make_chain_params(&ch, 0.0, &cpb);
            if (r1 == MBL_OK) r1 = ensure_lowtabs_for(ch.L);
            if (r1 == MBL_OK)
                r1 = lanczos_bounds(cpb, mbl_basis_size(ch.L, ch.n_up), X0_dev + off_x[i], k, kBatchBoundsTol, 1000,
                                    ws, slot, &lo, &hi, &it, st);
            if (r1 != MBL_OK && r1 != MBL_ERR_NOT_CONVERGED) {
                int expect = MBL_OK;
                first_error.compare_exchange_strong(expect, r1);
                break;
            }
            sig[i] = 0.5 * (lo + hi);
            nh[i] = norm_given > 0.0 ? norm_given : std::max(std::fabs(lo), std::fabs(hi));
        }
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    };
    std::vector<std::thread> pool;
    for (int w = 0; w < nth; ++w) pool.emplace_back(worker, w);
    for (auto &t : pool) t.join();
    cudaEventDestroy(start_ev);
    return first_error.load();
}

constexpr int kBatchSubStreams = 16;

// The streams (and their join events) of a batched solve, released on scope exit.
struct SubStreams {
    cudaStream_t cap = nullptr;  // for capturing the lanes' graphs
    cudaStream_t st[kBatchSubStreams] = {};
    cudaEvent_t ev[kBatchSubStreams] = {};
    cudaEvent_t ev_main = nullptr;
    int count = 0;
    int create(int n)
    {
        if (cudaEventCreateWithFlags(&ev_main, cudaEventDisableTiming) != cudaSuccess ||
            cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
            return MBL_ERR_CUDA;
        for (; count < n; ++count)
            if (cudaStreamCreateWithFlags(&st[count], cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&ev[count], cudaEventDisableTiming) != cudaSuccess)
                return MBL_ERR_CUDA;
        return MBL_OK;
    }
    ~SubStreams()
    {
        for (int j = 0; j < kBatchSubStreams; ++j) {
            if (st[j]) {
                cudaStreamSynchronize(st[j]);
                cudaStreamDestroy(st[j]);
            }
            if (ev[j]) cudaEventDestroy(ev[j]);
        }
        if (ev_main) cudaEventDestroy(ev_main);
        if (cap) cudaStreamDestroy(cap);
    }
};

// The captured steps of one lane's problem: before the preconditioner, and after it
// without / with the previous direction P (about 40 small kernels each, launched as one
// graph per round), with the products each counts.
struct LaneGraphs {
    cudaGraphExec_t pre = nullptr, post[2] = {nullptr, nullptr};
    int64_t kernels_pre = 0, kernels_post[2] = {0, 0};
    int64_t matvecs_post[2] = {0, 0};
    void reset()
    {
        if (pre) cudaGraphExecDestroy(pre);
        for (auto &g : post)
            if (g) cudaGraphExecDestroy(g);
        pre = post[0] = post[1] = nullptr;
        kernels_pre = kernels_post[0] = kernels_post[1] = 0;
        matvecs_post[0] = matvecs_post[1] = 0;
    }
};

// Capture what enqueue() puts on s.st into an executable graph (s.st is swapped for the
// capture stream meanwhile); *kernels = its kernel nodes.
template <typename F>
int capture_graph(Solver &s, cudaStream_t cap, F enqueue, cudaGraphExec_t *exec, int64_t *kernels)
{
    cudaStream_t user = s.st;
    s.st = cap;
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        s.st = user;
        return MBL_ERR_CUDA;
    }
    set_capturing(true);
    const int rc = enqueue();
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cap, &g);
    set_capturing(false);
    s.st = user;
    if (rc != MBL_OK || ce != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        return rc != MBL_OK ? rc : MBL_ERR_CUDA;
    }
    size_t nn = 0;
    *kernels = 0;
    if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
        std::vector<cudaGraphNode_t> nodes(nn);
        if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
            for (size_t i = 0; i < nn; ++i) {
                cudaGraphNodeType ty;
                if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++*kernels;
            }
    }
    const cudaError_t ie = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    return ie == cudaSuccess ? MBL_OK : MBL_ERR_CUDA;
}

// One lane of the lock-step batch.
struct Lane {
    LaneGraphs graphs;
    ~Lane() { graphs.reset(); }
    Solver s;
    int prob = -1;  // problem in the lane, -1: idle
    int it = 0;
    bool have_p = false;
    bool body = false;  // advances this round
    double r_mark = 0.0;
    int it_mark = 0;
    std::chrono::steady_clock::time_point t0;
};

}  // namespace

extern "C" int mbl_batched_workspace_size(int nprob, const mbl_chain *chains, const mbl_lobpcg_opts *opts,
                                          int nstreams, size_t *bytes)
{
    if (nprob < 1 || !chains || !opts || !bytes || nstreams < 1 || nstreams > 64) return MBL_ERR_ARG;
    int rc;
    const size_t slot = batch_slot_bytes(nprob, chains, opts, &rc);
    if (rc != MBL_OK) return rc;
    const int ns = std::min(nstreams, nprob);
    *bytes = slot * (size_t)ns + batch_table_bytes(ns);
    return MBL_OK;
}

extern "C" int mbl_lobpcg_solve_batched(int nprob, const mbl_chain *chains, const double *sigmas,
                                        const mbl_lobpcg_opts *opts, const double *X0_dev, int nstreams,
                                        void *workspace_dev, size_t workspace_bytes, double *evals_host,
                                        double *evecs_dev, double *resid_host, mbl_lobpcg_stats *stats,
                                        mbl_stream_t stream)
{
    if (nprob < 1 || !chains || !opts || !X0_dev || !workspace_dev || nstreams < 1 || nstreams > 64)
        return MBL_ERR_ARG;
    if ((uintptr_t)workspace_dev % kAlign) return MBL_ERR_ARG;
    int rc;
    const size_t slot = batch_slot_bytes(nprob, chains, opts, &rc);
    if (rc != MBL_OK) return rc;
    const int ns = std::min(nstreams, nprob);
    if (workspace_bytes < slot * (size_t)ns + batch_table_bytes(ns)) return MBL_ERR_WORKSPACE;
    if (opts->use_graph == 0 && opts->timing) return MBL_ERR_ARG;
    // packed offsets of each problem's start block and eigenvectors
    std::vector<int64_t> off_x(nprob + 1, 0), off_v(nprob + 1, 0);
    for (int i = 0; i < nprob; ++i) {
        const int64_t n = mbl_basis_size(chains[i].L, chains[i].n_up);
        if (n <= 0 || (sigmas == nullptr && chains[i].L < 2)) return MBL_ERR_ARG;
        off_x[i + 1] = off_x[i] + n * opts->k;
        off_v[i + 1] = off_v[i] + n * opts->nev;
    }
    const cudaStream_t st = (cudaStream_t)stream;
    // shifts and tolerance norms
    std::vector<double> sig(nprob), nh(nprob, opts->norm_h);
    if (sigmas) {
        for (int i = 0; i < nprob; ++i) sig[i] = sigmas[i];
    } else {
        MBL_TRY(batch_bounds(nprob, chains, X0_dev, off_x, opts->k, workspace_dev, slot, ns, st, opts->norm_h, sig, nh));
    }
    PcgLane *table_dev = reinterpret_cast<PcgLane *>((char *)workspace_dev + slot * (size_t)ns);
    std::vector<PcgLane> table((size_t)ns);
    std::vector<Lane> lanes((size_t)ns);
    // the lanes' own steps run on nsub streams (lane l on stream l mod nsub), so that the
    // small kernels of different lanes overlap on the GPU; events join them to `st` around
    // the batched PCG launches and at the end of each round
    const int nsub = std::min(ns, kBatchSubStreams);
    SubStreams sub;
    MBL_TRY(sub.create(nsub));
    auto fork = [&]() -> int {  // the sub-streams wait for the work queued on st
        if (cudaEventRecord(sub.ev_main, st) != cudaSuccess) return MBL_ERR_CUDA;
        for (int j = 0; j < nsub; ++j)
            if (cudaStreamWaitEvent(sub.st[j], sub.ev_main, 0) != cudaSuccess) return MBL_ERR_CUDA;
        return MBL_OK;
    };
    auto join = [&]() -> int {  // st waits for the work queued on the sub-streams
        for (int j = 0; j < nsub; ++j)
            if (cudaEventRecord(sub.ev[j], sub.st[j]) != cudaSuccess || cudaStreamWaitEvent(st, sub.ev[j], 0) != cudaSuccess)
                return MBL_ERR_CUDA;
        return MBL_OK;
    };
    const int mixed = opts->mode == MBL_MODE_MIXED;
    const int k = opts->k, nev = opts->nev;
    const bool graphs = opts->use_graph != 0;
    constexpr int kStallIters = 20;  // as in mbl_lobpcg_solve
    int next = 0, not_converged = 0;

    // put problem next (if any) into lane l: its setup is enqueued now, its first status
    // is read in the next round
    auto assign = [&](int l) -> int {
        Lane &ln = lanes[(size_t)l];
        ln.prob = -1;
        if (next >= nprob) return MBL_OK;
        const int i = next++;
        mbl_lobpcg_opts o = *opts;
        o.norm_h = nh[(size_t)i];
        o.timing = 0;
        ln.graphs.reset();
        ln.s = Solver{};
        ln.t0 = std::chrono::steady_clock::now();
        MBL_TRY(solver_setup(ln.s, &chains[i], sig[(size_t)i], &o, mbl_basis_size(chains[i].L, chains[i].n_up),
                             X0_dev + off_x[i], (char *)workspace_dev + slot * (size_t)l, slot, sub.st[l % nsub]));
        ln.prob = i;
        ln.it = 0;
        ln.have_p = false;
        ln.r_mark = 0.0;
        ln.it_mark = 0;
        return MBL_OK;
    };
    // results of lane l's problem (its status words say it is done); evecs by a kernel
    auto finish = [&](int l, int status) -> int {
        Lane &ln = lanes[(size_t)l];
        Solver &s = ln.s;
        const int i = ln.prob;
        MBL_TRY(gather_cols(k, nev, s.b.V, s.b.iflags + 8, s.b.Csel, s.st));
        if (evecs_dev)
            MBL_TRY(update(s.X(), s.ld3(), k, s.b.Csel, nev, nev, nullptr, 0, evecs_dev + off_v[i], nev, s.n, 1.0, 0.0,
                           0, s.st));
        double mu_h[64], res_h[64];
        int sel_h[64];
        if (cudaMemcpy(mu_h, s.b.mu, sizeof(double) * k, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(sel_h, s.b.iflags + 8, sizeof(int) * nev, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(res_h, s.b.res_sel, sizeof(double) * nev, cudaMemcpyDeviceToHost) != cudaSuccess)
            return MBL_ERR_CUDA;
        double mx = 0.0;
        for (int j = 0; j < nev; ++j) {
            if (evals_host) evals_host[(size_t)i * nev + j] = sig[(size_t)i] + mu_h[sel_h[j]];
            if (resid_host) resid_host[(size_t)i * nev + j] = res_h[j];
            mx = std::fmax(mx, res_h[j] / s.norm_h);
        }
        if (stats) {
            mbl_lobpcg_stats sv{};
            sv.iters = ln.it;
            sv.converged = status == MBL_OK ? 1 : 0;
            sv.matvecs = s.matvecs;
            sv.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - ln.t0).count();
            sv.max_rel_resid = mx;
            sv.norm_h = s.norm_h;
            stats[i] = sv;
        }
        if (status == MBL_ERR_NOT_CONVERGED) ++not_converged;
        return MBL_OK;
    };

    MBL_TRY(fork());
    for (int l = 0; l < ns; ++l) MBL_TRY(assign(l));
    MBL_TRY(join());
    for (;;) {
        if (cudaStreamSynchronize(st) != cudaSuccess) return MBL_ERR_CUDA;
        MBL_TRY(fork());
        int busy = 0;
        for (int l = 0; l < ns; ++l) {
            Lane &ln = lanes[(size_t)l];
            ln.body = false;
            if (ln.prob < 0) continue;
            Solver &s = ln.s;
            HostStatus hs;
            if (cudaMemcpy(hs.iflags, s.b.iflags, sizeof(hs.iflags), cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(hs.dstat, s.b.dstat, sizeof(hs.dstat), cudaMemcpyDeviceToHost) != cudaSuccess)
                return MBL_ERR_CUDA;
            if (s.gmix) {  // the stall rule of mbl_lobpcg_solve
                const double r = hs.dstat[0];
                if (ln.it == 0 || r < 0.9 * ln.r_mark) {
                    ln.r_mark = r;
                    ln.it_mark = ln.it;
                } else if (ln.it - ln.it_mark >= kStallIters) {
                    s.gmix = 0;
                    ln.graphs.reset();
                }
            }
            if (hs.iflags[5] || hs.iflags[2]) return MBL_ERR_NUMERIC;
            if (hs.iflags[0]) return MBL_ERR_BREAKDOWN;
            const bool done = hs.iflags[4] != 0;
            if (done || ln.it >= opts->max_iter) {
                MBL_TRY(finish(l, done ? MBL_OK : MBL_ERR_NOT_CONVERGED));
                MBL_TRY(assign(l));
                if (ln.prob >= 0) ++busy;  // its first status comes next round
                continue;
            }
            ln.body = true;
            ++busy;
        }
        if (busy == 0) {
            MBL_TRY(join());
            break;
        }
        // one LOBPCG iteration of every advancing lane
        int nb = 0;
        for (int l = 0; l < ns; ++l) {
            Lane &ln = lanes[(size_t)l];
            if (!ln.body) continue;
            ++nb;
            if (!graphs) {
                MBL_TRY(ln.s.enqueue_pre_pcg());
                continue;
            }
            if (!ln.graphs.pre)
                MBL_TRY(capture_graph(ln.s, sub.cap, [&]() { return ln.s.enqueue_pre_pcg(); }, &ln.graphs.pre,
                                      &ln.graphs.kernels_pre));
            if (cudaGraphLaunch(ln.graphs.pre, ln.s.st) != cudaSuccess) return MBL_ERR_CUDA;
            note_launch(ln.graphs.kernels_pre);
        }
        MBL_TRY(join());
        if (nb > 0 && opts->pcg_iters > 0) {
            // the lanes' table for the batched PCG launches; widths or tile settings without a
            // tiled kernel (pcg_lane_fill refuses them) run each lane's own PCG launches
            uint32_t round0 = 0, row0 = 0;
            int nt = 0, fill = MBL_OK;
            for (int l = 0; l < ns && fill == MBL_OK; ++l) {
                Lane &ln = lanes[(size_t)l];
                if (!ln.body) continue;
                Solver &s = ln.s;
                fill = pcg_lane_fill(&table[(size_t)nt++], s.cp, (uint32_t)s.n, k, mixed, s.b.dinv, s.b.pr, s.b.pp,
                                     s.b.pt, s.b.pw, s.pcg_dev(), &round0, &row0);
            }
            if (fill == MBL_ERR_ARG) {
                MBL_TRY(fork());
                for (int l = 0; l < ns; ++l)
                    if (lanes[(size_t)l].body) MBL_TRY(lanes[(size_t)l].s.enqueue_pcg_steps());
                MBL_TRY(join());
            } else {
                MBL_TRY(fill);
                if (cudaMemcpyAsync(table_dev, table.data(), sizeof(PcgLane) * (size_t)nt, cudaMemcpyHostToDevice,
                                    st) != cudaSuccess)
                    return MBL_ERR_CUDA;
                for (int step = 0; step < opts->pcg_iters; ++step)
                    MBL_TRY(pcg_batch_step(mixed, table_dev, nt, k, round0, row0, st));
            }
        }
        MBL_TRY(fork());
        for (int l = 0; l < ns; ++l) {
            Lane &ln = lanes[(size_t)l];
            if (!ln.body) continue;
            if (!graphs) {
                MBL_TRY(ln.s.enqueue_post_pcg(ln.have_p));
            } else {
                const int g = ln.have_p ? 1 : 0;
                if (!ln.graphs.post[g]) {
                    const int64_t mv = ln.s.matvecs;
                    MBL_TRY(capture_graph(ln.s, sub.cap, [&]() { return ln.s.enqueue_post_pcg(ln.have_p); },
                                          &ln.graphs.post[g], &ln.graphs.kernels_post[g]));
                    ln.graphs.matvecs_post[g] = ln.s.matvecs - mv;
                    ln.s.matvecs = mv;
                }
                if (cudaGraphLaunch(ln.graphs.post[g], ln.s.st) != cudaSuccess) return MBL_ERR_CUDA;
                note_launch(ln.graphs.kernels_post[g]);
                ln.s.matvecs += ln.graphs.matvecs_post[g];
            }
            ln.have_p = true;
            ++ln.it;
        }
        MBL_TRY(join());
    }
    return not_converged ? MBL_ERR_NOT_CONVERGED : MBL_OK;
}

extern "C" int64_t mbl_kernel_launch_count(void) { return g_kernel_launches.load(std::memory_order_relaxed); }

extern "C" int mbl_set_gram_engine(int engine)
{
    if (engine < 0 || engine > 2) return MBL_ERR_ARG;
    mbl::set_gram_engine(engine);
    return MBL_OK;
}

extern "C" int mbl_gram_workspace_size(int64_t n, int p, int q, size_t *bytes)
{
    if (!bytes || n < 1 || n > ((int64_t)1 << 31) || p < 1 || q < 1 || p > 256 || q > 256) return MBL_ERR_ARG;
    *bytes = mbl::gram_partial_doubles(n, p, q) * sizeof(double) + 256;
    return MBL_OK;
}

extern "C" int mbl_gram(const double *A_dev, int64_t lda, int p, const double *B_dev, int64_t ldb, int q, int64_t n,
                        double *C_dev, int64_t ldc, int precision, int engine, void *workspace_dev,
                        size_t workspace_bytes, mbl_stream_t stream)
{
    size_t need = 0;
    if (mbl_gram_workspace_size(n, p, q, &need) != MBL_OK) return MBL_ERR_ARG;
    if (!A_dev || !B_dev || !C_dev || !workspace_dev || lda < p || ldb < q || ldc < q) return MBL_ERR_ARG;
    if ((precision != MBL_F32 && precision != MBL_F64) || engine < 0 || engine > 2) return MBL_ERR_ARG;
    if (precision == MBL_F64 && engine == 2) return MBL_ERR_ARG;  // the tensor-core path is FP32-accurate
    if (workspace_bytes < need) return MBL_ERR_WORKSPACE;
    double *part = (double *)(((uintptr_t)workspace_dev + 255) & ~(uintptr_t)255);
    const int f32 = precision == MBL_F32;
    mbl::set_gram_engine_local(f32 ? engine : 1);
    const int rc = mbl::gram(A_dev, lda, p, B_dev, ldb, q, n, C_dev, ldc, 0, f32, part, (cudaStream_t)stream);
    mbl::set_gram_engine_local(0);
    return rc;
}

extern "C" int mbl_update(const double *A_dev, int64_t lda, int p, const double *M_dev, int64_t ldm, int q,
                          const double *C_dev, int64_t ldc, double *D_dev, int64_t ldd, int64_t n, double alpha,
                          double beta, int precision, int engine, mbl_stream_t stream)
{
    if (!A_dev || !M_dev || !D_dev || n < 0 || n > ((int64_t)1 << 31) || p < 1 || q < 1 || p > 192 || q > 64)
        return MBL_ERR_ARG;
    if (lda < p || ldm < q || ldd < q || (C_dev && ldc < q) || (!C_dev && beta != 0.0)) return MBL_ERR_ARG;
    if (!std::isfinite(alpha) || !std::isfinite(beta)) return MBL_ERR_ARG;
    if ((precision != MBL_F32 && precision != MBL_F64) || engine < 0 || engine > 2) return MBL_ERR_ARG;
    if (precision == MBL_F64 && engine == 2) return MBL_ERR_ARG;  // the tensor-core path is FP32-accurate
    const int f32 = precision == MBL_F32;
    mbl::set_gram_engine_local(f32 ? engine : 1);
    const int rc = mbl::update(A_dev, lda, p, M_dev, ldm, q, C_dev, C_dev ? ldc : 0, D_dev, ldd, n, alpha, beta, f32,
                               (cudaStream_t)stream);
    mbl::set_gram_engine_local(0);
    return rc;
}
