// Internal (non-ABI) entry points shared between the library's translation units.
#pragma once

#include "common.cuh"

namespace wp {

enum LiftOpId { LIFT_FWD = 0, LIFT_INV = 1, LIFT_ADJ = 2, LIFT_IADJ = 3 };

// Fused L-level lifting of a (p, plane) tensor; see lift.cu.  `interleaved`:
// the wavelet-domain side uses the group-interleaved slice order (local index
// t of tube group g at slice g * 2^L + t) instead of the Mallat order; only
// for L <= kMaxInterleavedLevels (WP_ERR_UNSUPPORTED beyond).
constexpr int kMaxInterleavedLevels = 5;
int lift_dispatch(int op, const float* in, float* out, int64_t plane, int64_t p, int L,
                  cudaStream_t st, bool interleaved = false);

// Plain FP32 SIMT batched GEMM; see gemm_simt.cu.
int sgemm_batched(const float* A, const float* B, float* C, int M, int N, int K, bool transA,
                  bool transB, int batch, cudaStream_t st);

// Tensor-core face-products (BF16, BF16x3, FP8) of FP32 wavelet-domain
// operands; see gemm_tc.cu.  Workspace holds the converted operands.
size_t tc_facewise_workspace(int64_t M, int64_t N, int64_t K, int64_t p, int prec);
int tc_facewise(const float* A, const float* B, float* C, int64_t M, int64_t N, int64_t K,
                int64_t p, bool transA, bool transB, int prec, void* ws, size_t ws_bytes,
                cudaStream_t st);
// Fused tensor-core w-product (lift + split producers, inverse-lift epilogue);
// WP_ERR_UNSUPPORTED outside its domain (no transposes, 1 <= L <= 5).
int tc_wprod_fused(const float* A, const float* B, float* C, int64_t n1, int64_t n2, int64_t n4,
                   int64_t p, int L, int prec, void* ws, size_t ws_bytes, cudaStream_t st);

}  // namespace wp

namespace wp {

// Batched one-sided Jacobi SVD (jacobi.cu): leading r singular triplets of
// slices [slice0, slice0 + nslices) of X (p, n1, n2).  vec_out (p, max(n1,n2), r)
// receives unit left vectors when n1 >= n2, unit right vectors otherwise;
// sig_out (p, r) the singular values in descending order.
int jacobi_svd(const float* X, int n1, int n2, int slice0, int nslices, int r, float* vec_out, float* sig_out,
               cudaStream_t st);
bool jacobi_supported(int n1, int n2);
// Device address of the Jacobi sweep counters ([0] total slice-sweeps, [1] max).
unsigned long long* jacobi_stats_ptr();
// Sweep limit passed to every Jacobi launch (default kJacobiMaxSweeps; set by
// wp_set_jacobi_max_sweeps).
constexpr int kJacobiMaxSweeps = 40;
int jacobi_max_sweeps();

}  // namespace wp
