/*
 * mbl.h -- C ABI of the GB300 (sm_103a) library for the matrix-free MBL eigensolver:
 * interior eigenpairs of the disordered Heisenberg chain restricted to one S^z sector.
 *
 * Model (Sec. 2.1, Eq. (model) and Eq. (Hmatrix)), with an anisotropy delta on the
 * Z_iZ_j part (delta = 1 is the paper's isotropic model):
 *     H = sum_bonds [ (X_iX_j + Y_iY_j)/4 + delta Z_iZ_j/4 ] + sum_i h_i Z_i/2
 * Bonds are (i, i+1), i = 0..L-2, plus (L-1, 0) on a periodic chain with L > 2.
 * Basis: the L-bit words s with popcount n_up (bit i = site i, 1 = spin up), in
 * ascending integer order; the sector dimension is n = C(L, n_up) (Sec. 2.1, Table 1).
 * Matrix elements: diagonal d(s) = sum_bonds delta/4 z_i z_j + sum_i h_i/2 z_i
 * (z = +1 up, -1 down); off-diagonal 1/2 between s and s with the two differing
 * spins of one bond exchanged.
 *
 * Conventions shared by every entry point:
 *   - All functions return an int status (MBL_OK = 0, negative on error) and never
 *     throw.  Arguments are validated before any launch; on MBL_ERR_ARG nothing is
 *     enqueued.
 *   - "_dev" pointers are device pointers owned by the caller; "_host" pointers are
 *     host memory owned by the caller.  The library allocates no device memory: the
 *     solvers take a caller-owned workspace sized by the matching *_workspace_size.
 *   - Work is enqueued on the caller's stream (mbl_stream_t is cudaStream_t; NULL is
 *     the legacy default stream).  Entry points that return host results (the
 *     solvers) synchronise that stream before returning; the others do not.
 *   - Blocks of vectors are row-major n x k with a leading dimension ld >= k
 *     (element (r, c) at ptr[r * ld + c]).
 */
#ifndef MBL_H
#define MBL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *mbl_stream_t; /* identical to cudaStream_t */

/* status codes */
#define MBL_OK 0
#define MBL_ERR_ARG -1            /* invalid argument; nothing was launched */
#define MBL_ERR_WORKSPACE -2      /* workspace smaller than *_workspace_size reported */
#define MBL_ERR_CUDA -3           /* a CUDA runtime call or launch failed */
#define MBL_ERR_NOT_CONVERGED -4  /* max_iter reached; outputs hold the best estimates */
#define MBL_ERR_BREAKDOWN -5      /* orthonormalisation lost rank beyond recovery */
#define MBL_ERR_NUMERIC -6        /* NaN or Inf met in a residual or Gram matrix */

#define MBL_F32 0
#define MBL_F64 1

#define MBL_MODE_FP64 0  /* every step in FP64 */
#define MBL_MODE_MIXED 1 /* FP32 preconditioner and FP32 Gram matrices; FP64 products
                            of H for X, W, P, FP64 Rayleigh-Ritz with H, orthonormalisation
                            of X and residual norms (Sec. 6.2: PCG in single, LOBPCG in
                            double).  If the largest wanted residual has not fallen by 10 %
                            in 20 iterations, the Rayleigh-Ritz Grams of the fold switch to
                            FP64 for the rest of the solve. */

/* Human-readable text for a status code (static storage). */
const char *mbl_status_string(int status);

/* Number of GPU kernels this library has launched in the calling process since it was
 * loaded, over all threads and devices: each direct launch counts one, each replay of a
 * captured CUDA graph counts its kernel nodes.  Monotone; for instrumentation (the
 * difference of two readings is the launches in between).  Never fails. */
int64_t mbl_kernel_launch_count(void);

/* One disorder realisation of the chain.  h_host: L FP64 fields (host memory, read
 * during the call only).  Requirements: 2 <= L <= 32, 0 <= n_up <= L, finite h and
 * delta. */
typedef struct {
    int L;
    int n_up;
    int periodic; /* 0 = open chain (the paper's choice), 1 = periodic */
    double delta;
    const double *h_host;
} mbl_chain;

/* ---- basis (Sec. 2.1 sector block-diagonalisation; Table 1) ---------------------- */

/* n = C(L, n_up), or -1 when 1 <= L <= 32 and 0 <= n_up <= L do not hold. */
int64_t mbl_basis_size(int L, int n_up);

/* states_dev[r] = the r-th L-bit word with popcount n_up in ascending order, for
 * r = 0..n-1 (combinatorial-number-system unranking).  n must equal
 * mbl_basis_size(L, n_up).  states_dev: n uint32 words. */
int mbl_basis_build(int L, int n_up, uint32_t *states_dev, int64_t n, mbl_stream_t stream);

/* ranks_dev[q] = position of words_dev[q] in that list (sum over up spins of
 * C(position, index)), or -1 when the word is not in the sector (wrong popcount or
 * bits at or above L).  cnt words in, cnt int64 out. */
int mbl_basis_rank(int L, int n_up, const uint32_t *words_dev, int64_t *ranks_dev, int64_t cnt,
                   mbl_stream_t stream);

/* ---- Hamiltonian product (Sec. 4.1, the MATVEC) ---------------------------------- */

/* Y = (H - sigma I) X on the sector, X and Y row-major n x k blocks (n = C(L, n_up))
 * with leading dimensions ldx, ldy >= k, element type dtype (MBL_F32 or MBL_F64,
 * accumulation in the same type).  Gather form: every output row is written once by
 * one thread group, no atomics, so results are bitwise reproducible.  X and Y must
 * not overlap.  Requires 1 <= k <= 256. */
int mbl_hamiltonian_apply(const mbl_chain *chain, double sigma, int dtype, const void *X_dev,
                          int64_t ldx, void *Y_dev, int64_t ldy, int64_t n, int k,
                          mbl_stream_t stream);

/* Tuning: the product kernels split a state into B low bits and L - B high bits; all
 * states with the same high bits form one tile of consecutive rows, in-tile neighbours
 * come from a per-B table of low patterns, and high-bond neighbours are whole tiles at
 * the same in-tile offsets.  This sets B for products of block width k and type dtype
 * in this process: 0 = built-in heuristic (default), -1 = untiled kernel, 2..16 = that
 * B (capped at 13 and at L - 2).  Results differ only in the order of floating-point
 * additions.  Returns MBL_ERR_ARG for k outside 1..256, an unknown dtype or bits
 * outside {-1, 0, 2..16}.  Not thread-safe against concurrent products. */
int mbl_set_product_tile_bits(int k, int dtype, int bits);

/* Tuning: bytes of each row that one lane moves per neighbour in the tiled product
 * (16, 32 or 64; 0 = default 32) for block width k and type dtype.  Returns MBL_ERR_ARG
 * for any other value, k outside 1..256 or an unknown dtype. */
int mbl_set_product_lane_bytes(int k, int dtype, int bytes);

/* Tuning: work order of the tiled product for block width k and type dtype.
 * 0 = by size (default, unless mbl_autotune_product chose for this L: ordered for plain
 * products with rows of k * element size >= 256 bytes once C(L, n_up) * k * element size
 * reaches 1 GiB in FP32 or 128 MiB in FP64, staged for 128-byte rows from 16 MB, else
 * persistent), 1 = persistent (a few blocks per SM striding over the tiles), 2 = ordered
 * (plain products only: one chunk of rows per warp; the hardware dispatches blocks in
 * index order, so the tiles being read advance as a narrow window that stays in L2),
 * 3 = staged (each block copies whole tiles of at most 48 KB into shared memory with bulk
 * asynchronous copies and reads the in-tile neighbours there), 4 = streamed (two blocks
 * per SM; a producer warp copies every row block a tile's product reads -- joining-bond
 * partners, wrap partner tile, the tile, one block per antiparallel high bond, and for the
 * PCG launches the rows of r, w, p -- into a ring of shared-memory slots with bulk
 * asynchronous copies, and the other warps add them up; rows of 32 to 512 bytes), 5 = slab
 * (one block of 288 threads per SM; a producer warp copies every term of a tile's product
 * -- the tile, its low-pattern records, joining-bond partners, wrap partner tile, one
 * block per antiparallel high bond, and for the q-launch of the PCG the rows of r -- into
 * a ring of six 32 KB shared-memory slots; each consumer thread owns one 16-byte column
 * chunk of up to 8 rows of the tile; rows of 32 to 256 bytes).  3, 4 and 5 need ld = k and
 * 16-byte aligned buffers (else persistent).  Results are bitwise identical under every
 * order for the same tile width (mbl_product_tile_width).  Returns MBL_ERR_ARG for
 * schedule outside 0..5, k outside 1..256 or an unknown dtype. */
int mbl_set_product_schedule(int k, int dtype, int schedule);

/* Tile width B (>= 2) that work order `schedule` (1..5, as above) uses for a chain of
 * length L, block width k and type dtype under the current switches, or 0 when that
 * order has no tiled kernel for this shape (3 and 4 then fall back to persistent, 1 and
 * 2 to the untiled kernel).  Schedule 4 reads the device's shared-memory limit (a CUDA
 * device must be current); 1..3 and 5 are host-only.  Returns MBL_ERR_ARG for an unknown
 * dtype, k outside 1..256, L outside 4..32 or schedule outside 1..5. */
int mbl_product_tile_width(int L, int dtype, int k, int schedule);

/* Autotuner of the product (the tile widths and work orders above): times the plain
 * product of this chain, block width k, type dtype, under every candidate -- schedule
 * persistent / ordered / staged / streamed / slab (where its conditions hold) times 32- or
 * 64-byte lanes (64 only for rows of >= 64 bytes; streamed and slab have one lane width) -- on the
 * caller's buffers X_dev, Y_dev (n x k, ld = k, n = C(L, n_up); X is read, Y
 * overwritten; they must not overlap): one warm-up and `reps` timed launches each
 * (1 <= reps <= 1000), CUDA events on `stream`.  The fastest is kept -- the size-based
 * default of mbl_set_product_schedule unless another candidate is more than 2 % faster
 * -- for all later products with this L, k and dtype in this process (the explicit
 * switches above still take precedence) and reported in *choice (optional): schedule
 * 1..5, lane bytes, tile bits and the mean microseconds per product.  Widths k without a
 * tiled kernel leave nothing to choose: MBL_OK with *choice zeroed.
 * Host-synchronous (waits for its timing launches). */
typedef struct {
    int schedule;
    int lane_bytes;
    int tile_bits;
    double microseconds;
} mbl_product_choice;
int mbl_autotune_product(const mbl_chain *chain, int dtype, const void *X_dev, void *Y_dev, int64_t n, int k,
                         int reps, mbl_product_choice *choice, mbl_stream_t stream);

/* Tuning: engine of the FP32 Gram matrices of mixed mode (S^T S, S^T A S, X^T A X; the
 * tall-skinny contraction of the Rayleigh-Ritz step, Sec. 3.2) and of its FP32 block
 * updates (the projections of W and P against X and the new direction P): 0 = default
 * (tensor cores for Grams whose sides are both >= 64 and for updates of at least 16,384
 * rows, CUDA cores otherwise), 1 = CUDA cores
 * (FP32 FMA), 2 = tensor cores whenever the shape fits (tcgen05.mma kind::tf32 with FP32
 * accumulators in tensor memory; each FP32 operand split into two TF32 parts, three
 * products, error of the order of FP32 rounding; Grams up to 256 x 256, updates with
 * p <= 192, q <= 64).  Applies to later solves in this process.  Returns MBL_ERR_ARG for
 * any other value. */
int mbl_set_gram_engine(int engine);

/* The tall-skinny Gram of the Rayleigh-Ritz step (Sec. 3.2), on its own: C = A^T B for
 * FP64 device blocks A (n x p, row-major, lda >= p) and B (n x q, ldb >= q), 1 <= p, q
 * <= 256, into C (p x q, row-major, ldc >= q, FP64 device memory).  precision MBL_F64:
 * FP64 arithmetic (CUDA cores); MBL_F32: inputs rounded to FP32, products accumulated in
 * FP32 per slab of rows, slabs summed in FP64 in a fixed order, on the engine given
 * (0: the process-wide choice of mbl_set_gram_engine, 1: CUDA cores, 2: tensor cores --
 * A and B read by TMA, tcgen05.mma kind::tf32 with each operand split into two TF32 parts,
 * the accumulators drained every 256 rows into float-float slab sums; it needs A and B
 * 16-byte aligned with even leading dimensions and otherwise runs on the CUDA cores; 2 with
 * MBL_F64 is MBL_ERR_ARG).  Workspace: mbl_gram_workspace_size bytes of device memory.
 * Deterministic for a given engine. */
int mbl_gram_workspace_size(int64_t n, int p, int q, size_t *bytes);
int mbl_gram(const double *A_dev, int64_t lda, int p, const double *B_dev, int64_t ldb, int q, int64_t n,
             double *C_dev, int64_t ldc, int precision, int engine, void *workspace_dev, size_t workspace_bytes,
             mbl_stream_t stream);

/* The block update of the LOBPCG step (Sec. 3.2: X <- S C, P <- [W P] C and the
 * projections B - X (X^T B)) on its own: D = beta C + alpha A M for FP64 device blocks
 * A (n x p, row-major, lda >= p), M (p x q, ldm >= q), C and D (n x q, ldc, ldd >= q; C may
 * be D, or NULL when beta = 0), 1 <= p <= 192, 1 <= q <= 64.  precision MBL_F64: FP64
 * arithmetic (CUDA cores); MBL_F32: inputs rounded to FP32 and FP32 arithmetic, so
 * |D - exact| is of the order of 2^-21 (|alpha| |A| |M| + |beta C|) elementwise, on the
 * engine given (0: the process-wide choice of mbl_set_gram_engine, 1: CUDA cores, which add
 * beta C in FP64, 2: tensor cores -- A, C and D moved by TMA, tcgen05.mma kind::tf32 over
 * 128-row tiles with the accumulator in tensor memory, each FP32 operand split into two
 * TF32 parts, three products; it needs A, D (and C when beta != 0) 16-byte aligned with even
 * leading dimensions and otherwise runs on the CUDA cores; 2 with MBL_F64 is MBL_ERR_ARG).
 * Allocates nothing; deterministic for a given engine; runs on `stream`. */
int mbl_update(const double *A_dev, int64_t lda, int p, const double *M_dev, int64_t ldm, int q,
               const double *C_dev, int64_t ldc, double *D_dev, int64_t ldd, int64_t n, double alpha,
               double beta, int precision, int engine, mbl_stream_t stream);

/* ---- folded-spectrum LOBPCG (Sec. 3.2, Sec. 6.2) ---------------------------------- */

typedef struct {
    int nev;        /* wanted eigenpairs nearest sigma, 1 <= nev <= k */
    int k;          /* block width, nev <= k <= 64, 3k <= n */
    int max_iter;   /* LOBPCG iterations before MBL_ERR_NOT_CONVERGED */
    int pcg_iters;  /* Jacobi-PCG steps per LOBPCG iteration (the preconditioner) */
    double tol;     /* accept when ||H y - lambda y||_2 <= tol * norm_h for all nev pairs */
    double pcg_tol; /* 0: always pcg_iters steps; > 0: freeze a column once
                       r^T M^-1 r <= pcg_tol^2 times its initial value */
    double norm_h;  /* scale of the tolerance; <= 0: a Gershgorin bound max_s |d(s)| + f(s)/2 */
    int mode;       /* MBL_MODE_FP64 or MBL_MODE_MIXED */
    int use_graph;  /* 1: capture the body of an iteration once as a CUDA graph and replay it */
    int timing;     /* 1: record CUDA events between the phases of every iteration and report
                       the per-phase device time in mbl_lobpcg_stats (disables use_graph) */
} mbl_lobpcg_opts;

typedef struct {
    int iters;            /* LOBPCG iterations taken */
    int converged;        /* 1 when every wanted pair met the tolerance */
    int64_t matvecs;      /* single-column applications of H (a block of k counts k) */
    double seconds;       /* wall time of the call */
    double max_rel_resid; /* max over the returned pairs of ||Hy - lambda y|| / norm_h */
    double norm_h;        /* the norm the tolerance was scaled by */
    /* device seconds per phase when opts->timing = 1 (else 0): setup (preconditioner
       diagonal, start block), residual block R, Jacobi-PCG sweeps, orthogonalisation of
       W and P with their products, Gram matrices of S, small dense steps (SVQB,
       Rayleigh-Ritz), block updates with Cholesky-QR, products of the new block, and the
       H Rayleigh-Ritz convergence test */
    double t_setup, t_resid, t_pcg, t_wp, t_gram, t_small, t_update, t_refresh, t_hrr;
} mbl_lobpcg_stats;

/* Bytes of device workspace mbl_lobpcg_solve needs for this chain and options. */
int mbl_lobpcg_workspace_size(const mbl_chain *chain, const mbl_lobpcg_opts *opts,
                              size_t *bytes);

/* The opts->nev eigenpairs of H nearest sigma, by LOBPCG on A = (H - sigma I)^2 with a
 * column-wise Jacobi-PCG preconditioner (M = diag(A) = (d - sigma)^2 + f/4).  Every
 * iteration a Rayleigh-Ritz with H on span(X) gives the Ritz pairs whose residuals
 * decide convergence; the same step is the final extraction.
 *   X0_dev:    n x k FP64 starting block, row-major, ld = k (read only).
 *   workspace: >= mbl_lobpcg_workspace_size bytes of device memory, 256-byte aligned.
 *   evals_host: nev FP64, ascending.  evecs_dev: n x nev FP64, row-major, ld = nev,
 *   unit columns.  resid_host: nev FP64 absolute residual norms ||Hy - lambda y||_2
 *   (each may be NULL).  stats: may be NULL.
 * Returns MBL_OK, or MBL_ERR_NOT_CONVERGED with the current estimates written. */
int mbl_lobpcg_solve(const mbl_chain *chain, double sigma, const mbl_lobpcg_opts *opts,
                     const double *X0_dev, void *workspace_dev, size_t workspace_bytes,
                     double *evals_host, double *evecs_dev, double *resid_host,
                     mbl_lobpcg_stats *stats, mbl_stream_t stream);

/* Same solve for callers that cannot allocate device memory when they need a solve:
 * plug-ins whose host application's own allocator owns the whole device memory pool,
 * and real-time callers whose memory budget is fixed up front.  The paper has no
 * counterpart; this entry point only changes where the workspace lives.
 * The workspace is one fixed device array of MBL_NOALLOC_SCRATCH_BYTES (16 MiB) inside
 * the library, present on every GPU that loads the library until the process exits;
 * problems whose mbl_lobpcg_workspace_size exceeds it are rejected with
 * MBL_ERR_WORKSPACE before anything is launched (16 MiB covers, for instance, L = 12 with
 * k <= 64, L = 14 with k <= 32 and L = 16 with k = 8).  The call allocates nothing: no
 * cudaMalloc or cudaFree, no graph instantiation (opts->use_graph is ignored) and no
 * timing events (opts->timing is ignored).
 * Set-up: the first call on a device looks up the array's device address with that
 * device current; with lazy module loading the module (and its 16 MiB) is loaded at the
 * library's first use on that device, so make one call of this library on each device
 * (this one, or any other) before the caller's memory budget is fixed.
 * The stream must belong to the current device (else MBL_ERR_ARG).  Like
 * mbl_lobpcg_solve, the call synchronises the stream at set-up and once per iteration
 * and writes host results, so it cannot be issued on a stream that is being captured
 * into a CUDA graph.
 * Every call shares the one array and leaves its contents behind; the solver clears
 * what must start at zero.  Calls whose work overlaps on the GPU (other streams, other
 * host threads) race on the array: serialise them.
 * Arguments and results are those of mbl_lobpcg_solve. */
#define MBL_NOALLOC_SCRATCH_BYTES (16u << 20)
int mbl_lobpcg_solve_noalloc(const mbl_chain *chain, double sigma, const mbl_lobpcg_opts *opts,
                             const double *X0_dev, double *evals_host, double *evecs_dev,
                             double *resid_host, mbl_lobpcg_stats *stats, mbl_stream_t stream);

/* Batched disorder averaging (Sec. 3.1: realisations and disorder strengths are
 * independent levels of concurrency): nprob problems, any mix of L and fields, solved
 * with the same opts.  The workspace holds nstreams lanes; each lane solves one problem at
 * a time, and all lanes advance in lock step on `stream`, one LOBPCG iteration per round:
 * the steps before and after the preconditioner are enqueued lane by lane, and each of the
 * pcg_iters PCG steps of all advancing lanes runs as three launches over a table of the
 * lanes (so a round issues about 40 launches per lane plus 3 per PCG step, not 3 per PCG
 * step per lane).  When a lane's problem converges (or reaches max_iter) its results are
 * written and it takes the next problem.  The host synchronises `stream` once per round
 * to read the lanes' status words.  With opts->use_graph, each lane's steps before and
 * after the preconditioner are captured once per problem as two small CUDA graphs and
 * replayed every round; opts->timing is ignored (use_graph = 0 with timing = 1 is
 * MBL_ERR_ARG).  Every problem's results equal the single-problem solve's to within
 * rounding (the PCG of a lane runs the same arithmetic in a batched launch; widths k other
 * than 8, 16, 32, 64 run each lane's own PCG launches and then equal them exactly).
 *   sigmas:   nprob shifts, or NULL: sigma_i = (E_min + E_max)/2 of problem i from
 *             the Lanczos bounds of mbl_spectrum_bounds (tolerance 1e-7, at most 1000
 *             steps, started from column 0 of its X0 block), found before the solves by
 *             nstreams host threads with a stream and a lane's slot each (started after
 *             the work already queued on `stream`); then, if opts->norm_h <= 0,
 *             ||H|| = max |E|.
 *   X0_dev:   the problems' n_i x k FP64 start blocks packed one after another.
 *   workspace: mbl_batched_workspace_size bytes (nstreams slots of the largest problem and
 *             the lanes' table).
 *   evals_host, resid_host: nprob x nev (problem-major); evecs_dev: the n_i x nev blocks
 *   packed one after another, or NULL; stats: nprob entries or NULL (per-phase times 0).
 * Returns MBL_OK, MBL_ERR_NOT_CONVERGED when some problem did not converge (all outputs
 * written), or the first error met (remaining problems are skipped). */
int mbl_batched_workspace_size(int nprob, const mbl_chain *chains, const mbl_lobpcg_opts *opts,
                               int nstreams, size_t *bytes);
int mbl_lobpcg_solve_batched(int nprob, const mbl_chain *chains, const double *sigmas,
                             const mbl_lobpcg_opts *opts, const double *X0_dev, int nstreams,
                             void *workspace_dev, size_t workspace_bytes, double *evals_host,
                             double *evecs_dev, double *resid_host, mbl_lobpcg_stats *stats,
                             mbl_stream_t stream);

/* Spectrum bounds E_min, E_max of the sector Hamiltonian (used to place sigma at the
 * middle of the spectrum and to scale tolerances): one FP64 Lanczos recurrence on H
 * started from column 0 of X0_dev (n x k FP64, ld = k; the other columns are not read;
 * 2 <= k <= 16 and 3k <= n are checked), without reorthogonalisation.  Every 20 steps the
 * extreme eigenvalues theta of the tridiagonal T_m are found by Sturm bisection and each
 * end's residual ||H y - theta y|| = beta_m |last component of T_m's eigenvector| by
 * inverse iteration; the call stops when both are <= tol |theta| (or the recurrence
 * meets an invariant subspace), or after max_iter steps (at most 4096; then
 * MBL_ERR_NOT_CONVERGED with the current estimates).  *iters_host: the Lanczos steps.
 * Host-synchronous every 20 steps.  Workspace: mbl_bounds_workspace_size bytes. */
int mbl_bounds_workspace_size(const mbl_chain *chain, int k, size_t *bytes);
int mbl_spectrum_bounds(const mbl_chain *chain, int k, double tol, int max_iter,
                        const double *X0_dev, void *workspace_dev, size_t workspace_bytes,
                        double *emin_host, double *emax_host, int *iters_host,
                        mbl_stream_t stream);

/* ---- localization indicators (Sec. 2.2) ------------------------------------------- */

/* Adjacent gap ratio of converged eigenvalues (Sec. 2.2, in the form of the work it cites):
 * for each of nprob disorder realizations, its m levels evals_dev[i * ld + 0 .. m-1] (FP64
 * device memory, any order) are sorted; with the gaps d_j = E_{j+1} - E_j, every interior
 * level j = 1 .. m-2 gives r_j = min(d_{j-1}, d_j) / max(d_{j-1}, d_j), and a level whose
 * two gaps are both zero is skipped.  Writes r_mean_dev[i] (FP64 device memory) = the mean
 * of realization i's ratios, and count_dev[i] (int32 device memory) = their number; NaN
 * and 0 when it has none (m < 3) or when one of its levels is not finite.  The mean over
 * several realizations is sum(r_mean * count) / sum(count) (skip count 0).  One block per
 * realization on `stream`; fixed-order sums, bitwise reproducible.  Returns MBL_ERR_ARG
 * (nothing launched) for nprob < 0, m outside 1..4096, ld < m or a null pointer with
 * nprob > 0; nprob = 0 is a no-op. */
int mbl_gap_ratio(int nprob, int m, const double *evals_dev, int64_t ld, double *r_mean_dev,
                  int *count_dev, mbl_stream_t stream);

/* Half-chain entanglement entropy of sector vectors (Sec. 2.2): the chain is cut after
 * its first l_a sites (1 <= l_a <= L - 1) and S = -sum lambda ln lambda over the
 * eigenvalues lambda of the reduced density matrix of sites 0 .. l_a-1, for each of the
 * nvec columns of V_dev (n x nvec, row-major, ld ldv >= nvec, FP64 device memory,
 * n = C(L, n_up) rows in the basis order of mbl_basis_build; a column need not be
 * normalised: lambda is taken relative to its squared norm).  The reduced density matrix
 * is the direct sum over p (up spins on the left) of M_p M_p^T, M_p holding the column's
 * entries with p up spins on the left (rows: left patterns, columns: right patterns); its
 * eigenvalues come from the smaller Gram of each M_p by FP64 Jacobi.  Writes S_dev[nvec]
 * (FP64 device memory; NaN for a zero column).  chain->h, delta and periodic are not used.
 * Limit: every Gram side min(C(l_a, p), C(L - l_a, n_up - p)) <= 512 (the half cut up to
 * L = 22), else MBL_ERR_ARG.  Workspace: mbl_entanglement_workspace_size bytes of device
 * memory (about 1 MB per column and p at L = 20, l_a = 10).  Deterministic (fixed-order
 * sums).  Runs on `stream`; nvec = 0 is a no-op. */
int mbl_entanglement_workspace_size(const mbl_chain *chain, int l_a, int nvec, size_t *bytes);
int mbl_entanglement_entropy(const mbl_chain *chain, int l_a, int nvec, const double *V_dev, int64_t ldv,
                             double *S_dev, void *workspace_dev, size_t workspace_bytes,
                             mbl_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* MBL_H */
