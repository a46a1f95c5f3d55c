// mbl_internal.h -- host-side interfaces between the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "mbl.h"

namespace mbl {

struct ChainParams;

// Device-resident per-column PCG state plus the block-partials scratch used by the
// deterministic reductions (partials: >= grid * 64 doubles; counter: one zeroed word).
struct PcgDev {
    double *rz, *rz0, *alpha, *beta;
    int *active;
    double tol2;
    double *partials;
    unsigned *counter;
};

// Count of the kernels this library has launched in the process.  Every launch site
// calls note_launch(); a launch made while this thread captures a CUDA graph is not
// counted there but once per replay of the graph (note_launch(kernel nodes)).
void note_launch(int64_t count = 1);
void set_capturing(bool on);

int num_sms();
// Spectrum bounds by FP64 Lanczos on H (mbl_lanczos.cu); X0: start vector in column 0 (ld).
size_t lanczos_workspace_bytes(int64_t n);
int lanczos_bounds(const ChainParams &cp, int64_t n, const double *X0, int64_t ldx0, double tol, int max_iter,
                   void *ws, size_t ws_bytes, double *emin, double *emax, int *iters, cudaStream_t st);
// Upload the low-pattern tables of every tile width usable at chain length L.
int ensure_lowtabs_for(int L);
int make_chain_params(const mbl_chain *chain, double sigma, ChainParams *cp);
int apply_device(const ChainParams &cp, int dtype, const void *X, int64_t ldx, void *Y, int64_t ldy, uint32_t n,
                 int k, cudaStream_t st);
int gershgorin_bound(const ChainParams &cp, uint32_t n, double *partials, unsigned *counter, double *out,
                     cudaStream_t st);
int pcg_grid(uint32_t n);
size_t pcg_partial_doubles();
// Tile width (low bits per tile) used by the product kernels for block width K and
// element size es; -1 = untiled kernel.  set_tile_bits: 0 heuristic, -1 untiled, >= 2 fixed.
int tile_bits_for(int L, int K, size_t es);
void set_tile_bits(int K, size_t es, int bits);
void set_lane_bytes(int K, size_t es, int bytes);
void set_schedule(int K, size_t es, int mode);
template <typename T>
int pcg_fold_dinv(const ChainParams &cp, uint32_t n, T *dinv, cudaStream_t st);
template <typename T>
int pcg_start(const double *B, int64_t ldb, const double *bnorm, uint32_t n, int k, const T *dinv, T *r, T *p,
              T *w, const PcgDev &pd, cudaStream_t st);
template <typename T>
int pcg_step(const ChainParams &cp, uint32_t n, int k, const T *dinv, T *r, T *p, T *t, T *w, const PcgDev &pd,
             cudaStream_t st);
// Batched PCG step over nlanes problems (lanes_dev: a device copy of PcgLane entries filled
// by pcg_lane_fill, in round order); every lane has block width k, FP32 (f32) or FP64
// vectors.  Three launches for all lanes.
struct PcgLane;
int pcg_lane_fill(PcgLane *lane, const ChainParams &cp, uint32_t n, int k, int f32, const void *dinv, void *r,
                  void *p, void *t, void *w, const PcgDev &pd, uint32_t *round0, uint32_t *row0);
int pcg_batch_step(int f32, const PcgLane *lanes_dev, int nlanes, int k, uint32_t rounds, uint32_t rows,
                   cudaStream_t st);

uint32_t host_binom(int n, int k);

// Half-chain entanglement entropy (mbl_small.cu): per cut, the largest Gram side dmax,
// the largest right-pattern count tmax, the largest block R x T (mmax), and the
// workspace doubles of one (vector, p) block.
struct EntanglementPlan {
    int64_t dmax, tmax, mmax, block_doubles;
    int blocks_per_vector;
};
EntanglementPlan entanglement_plan(int L, int n_up, int la);
size_t entanglement_work_bytes(const EntanglementPlan &pl, int nvec);
int entanglement_launch(int L, int n_up, int la, int nvec, const double *V, int64_t ldv, double *S, void *work,
                        size_t work_bytes, cudaStream_t st);

}  // namespace mbl
