// Internal declarations shared by the CUDA translation units of the CUP library.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "modp.cuh"

#define CUP_BMAX 64        // most rows a leaf slab may hold
#define CUP_WNMAX 128      // widest pivot-search window of a leaf
#define CUP_NSLOT (CUP_WNMAX + 2)
#define CUP_QT 64          // column positions per CTA in the leaf finish kernel

// What the leaf pivot kernel hands to the leaf finish kernel (device memory).
// Positions are relative to the slab's first active column col0.
struct SlabScratch {
    int r_s;                 // pivots found
    int i_stop;              // rows resolved (the rest need the node update first)
    int wne;                 // window width used
    int ext_pos;             // position >= wne that received window column 0, or -1
    int ext_slot;            // slot of ext_pos in Dorig
    int n_slot;
    int prof[CUP_BMAX];      // slab-relative row of pivot t
    int win_col[CUP_WNMAX];  // original position held by window position q
    int win_slot[CUP_WNMAX]; // Dorig slot of window position q, or -1 if not displaced
    uint32_t Cn[CUP_BMAX][CUP_BMAX];     // C[i][t] for slab rows i < i_stop, t < r_s
    uint32_t Minv[CUP_BMAX][CUP_BMAX];   // U rows = Minv * (pivot rows of the original slab)
    uint32_t Dorig[CUP_NSLOT][CUP_BMAX]; // original pivot-row values of displaced positions
};

// Kernel launchers (cup_kernels.cu). All are asynchronous on `st`.
cudaError_t launch_slab_pivots(const uint32_t *A, int64_t lda, int64_t a, int brows, int64_t col0,
                               int64_t w, int wn, ModP M, SlabScratch *S, int64_t *ipiv,
                               int64_t *prof, cudaStream_t st);
cudaError_t launch_slab_finish(uint32_t *A, int64_t lda, int64_t a, int64_t col0, int64_t w,
                               ModP M, const SlabScratch *S, cudaStream_t st);
cudaError_t launch_swaplist(const int64_t *ipiv, int64_t k0, int64_t k1, int2 *pairs, int *count,
                            cudaStream_t st);
cudaError_t launch_laswp(uint32_t *A, int64_t lda, int64_t row0, int64_t nrows, const int2 *pairs,
                         const int *count, cudaStream_t st);
cudaError_t launch_trsm_ruu_leaf(const uint32_t *U, int64_t ldu, uint32_t *B, int64_t ldb,
                                 int64_t m, int n, ModP M, cudaStream_t st);
cudaError_t launch_gemm_sub_cc(const uint32_t *A, int64_t lda, const uint32_t *B, int64_t ldb,
                               uint32_t *C, int64_t ldc, int64_t Mr, int64_t N, int64_t K, ModP M,
                               cudaStream_t st);
cudaError_t launch_det_reduce(const uint32_t *A, int64_t lda, int64_t n, const int64_t *ipiv, ModP M,
                              uint32_t *out, cudaStream_t st);

// Tensor-core Schur update (cup_tc.cu).
int tc_limbs(uint32_t p);
size_t tc_workspace_bytes(uint32_t p, int64_t M, int64_t N, int64_t K);
cudaError_t launch_gemm_sub_tc(const uint32_t *A, int64_t lda, const uint32_t *B, int64_t ldb, uint32_t *C,
                               int64_t ldc, int64_t M, int64_t N, int64_t K, ModP Mp, void *ws, int *err,
                               cudaStream_t st, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr);
