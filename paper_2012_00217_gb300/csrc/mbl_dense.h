// mbl_dense.h -- dense kernels of the LOBPCG iteration (host launchers).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "mbl_internal.h"

namespace mbl {

// C (p x q, ldc) = A^T B over n rows; FP64 storage, FP32 or FP64 arithmetic; sym: store
// (C + C^T)/2.  part: gram_partial_doubles(n, p, q) doubles of scratch.
int gram(const double *A, int64_t lda, int p, const double *B, int64_t ldb, int q, int64_t n, double *C,
         int64_t ldc, int sym, int compute_f32, double *part, cudaStream_t st);
size_t gram_partial_doubles(int64_t n, int p, int q);
// Engine of the FP32 Grams and block updates: 0 = default, 1 = CUDA cores, 2 = tensor
// cores (tcgen05).
void set_gram_engine(int engine);
void set_gram_engine_local(int engine);  // this thread's next Grams (0: use the switch)
// Tensor-core slab partials (mbl_gram_tc.cu): part[slab][i][j] for nslab slabs; the blocks
// are read by TMA, so they must be 16-byte aligned with even leading dimensions.
bool gram_tc_supported(int p, int q);
bool gram_tc_eligible(const double *A, int64_t lda, int p, const double *B, int64_t ldb, int q);
int gram_tc_slabs(int64_t n, int p);
int gram_tc_partial(const double *A, int64_t lda, int p, const double *B, int64_t ldb, int q, int64_t n, int nslab,
                    double *part, cudaStream_t st);
// Tensor-core block update D = beta C + alpha A M with FP32 accuracy (mbl_gram_tc.cu):
// p <= 192, q <= 64, A, D (and C when beta != 0) 16-byte aligned with even leading
// dimensions (they are read and written by TMA).
bool update_tc_supported(const double *A, int64_t lda, int p, int q, const double *C, int64_t ldc, const double *D,
                         int64_t ldd, double beta);
int update_tc(const double *A, int64_t lda, int p, const double *M, int64_t ldm, int q, const double *C, int64_t ldc,
              double *D, int64_t ldd, int64_t n, double alpha, double beta, cudaStream_t st);

// D = beta C + alpha A M  (A: n x p, M: p x q, C, D: n x q); D may alias C.
int update(const double *A, int64_t lda, int p, const double *M, int64_t ldm, int q, const double *C, int64_t ldc,
           double *D, int64_t ldd, int64_t n, double alpha, double beta, int compute_f32, cudaStream_t st);

int colnorms(const double *A, int64_t lda, int k, int64_t n, double *out, int take_sqrt, double *part,
             cudaStream_t st);
size_t colnorm_partial_doubles(int k);
int widen(int src_f32, const void *src, int64_t lds, double *dst, int64_t ldd, int k, int64_t n, cudaStream_t st);
int scale_cols_inv(double *A, int64_t lda, int k, int64_t n, const double *norms, cudaStream_t st);
int copy_block(const double *S, int64_t lds, double *D, int64_t ldd, int k, int64_t n, cudaStream_t st);

int small_eig(int n, const double *G, int64_t ldg, double *w, double *Z, double *work, cudaStream_t st);
size_t small_eig_work_doubles(int n);
int small_chol_inv(int n, const double *G, int64_t ldg, double *Rinv, double *work, int *flag, cudaStream_t st);
int small_svqb_rr(int w, int k, int largest, int mixed, const double *GS, const double *GA, double tau,
                  double *coef, double *theta, double *work, int *info, cudaStream_t st);
size_t small_rr_work_doubles(int w);
int hrr_select(int k, int nev, const double *mu, const double *V, const double *EtE, double tol_abs, double norm_h,
               double *res_all, int *sel, double *res_sel, int *st, double *dst, cudaStream_t s);
int gather_cols(int k, int nev, const double *V, const int *sel, double *Csel, cudaStream_t st);

}  // namespace mbl
