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
// True when wp_wprod (no transposes) has several tensor-core kernels to
// choose from for these arguments: the fused inverse-lift epilogue kernel,
// the persistent GEMM into C_hat plus a separate inverse lift, and (where
// wprod_lift_ok also holds) the lifted-operand kernel.
bool wprod_tunable(int64_t n1, int64_t n2, int64_t n4, int64_t p, int L, int prec);
// True when the third kernel, which lifts the spatial operands in its
// producer warps (L <= 3, n2 and n4 multiples of 4, 16-byte aligned A, B, C),
// takes these arguments.
bool wprod_lift_ok(const float* A, const float* B, const float* C, int64_t n1, int64_t n2, int64_t n4, int64_t p,
                   int L, int prec);
constexpr int kVariantFused = 1, kVariantPersistent = 2, kVariantLifted = 3;
// The tuned variant for this shape (tune.cu); 0 if none.
int wprod_plan_lookup(int64_t n1, int64_t n2, int64_t n4, int64_t p, int L, int prec);

}  // namespace wp

namespace wp {

// Batched one-sided Jacobi SVD (jacobi.cu): leading r singular triplets of
// slices [slice0, slice0 + nslices) of X (p, n1, n2).  vec_out (p, max(n1,n2), r)
// receives unit left vectors when n1 >= n2, unit right vectors otherwise;
// sig_out (p, r) the singular values in descending order.
// Slices too large for a thread-block cluster's shared memory run on the
// global-memory kernel (jacobi_global.cu), which needs `work` of
// jacobi_work_bytes(n1, n2, nslices) bytes (0 for every other shape).
int jacobi_svd(const float* X, int n1, int n2, int slice0, int nslices, int r, float* vec_out, float* sig_out,
               cudaStream_t st, void* work = nullptr, size_t work_bytes = 0);
bool jacobi_supported(int n1, int n2);
size_t jacobi_work_bytes(int n1, int n2, int nslices);
// global-memory kernel (jacobi_global.cu)
size_t jacobi_global_work_bytes(int n1, int n2, int nslices);
bool jacobi_global_supported(int n1, int n2);
struct JacobiArgs;
int jacobi_global_launch(const JacobiArgs& a, int nslices, void* work, size_t work_bytes, cudaStream_t st);
// Householder QR preconditioner of the Jacobi SVD (qr.cu): R^T (row-major)
// of the working matrix of each of slices [0, nslices) of X (p, n1, n2).
bool qr_supported(int m_len, int n_vec);
// Register-resident cluster QR (qr_cols.cu) of working matrices of at most
// 256 x 256: writes R^T row-major (nslices, n, n) to R like qr_r.
bool qr_cols_fits(int m_len, int n_vec);
int qr_cols_launch(const float* X, int n1, int n2, int nslices, float* R, cudaStream_t st);
size_t qr_work_bytes(int m_len, int n_vec, int nslices);
int qr_r(const float* X, int n1, int n2, int nslices, void* work, size_t work_bytes, float** Rt_out,
         cudaStream_t st);
// True when w-svd / wpinv precondition the Jacobi SVD of (n1, n2) slices by
// a QR (setting of wp_set_jacobi_precondition, and the slice shape: at
// least 32 columns, at most 1024 rows, within the register kernel's reach).
bool jacobi_preconditioned(int n1, int n2);
// Device address of the Jacobi sweep counters ([0] total slice-sweeps, [1] max).
unsigned long long* jacobi_stats_ptr();
// Sweep limit passed to every Jacobi launch (default kJacobiMaxSweeps; set by
// wp_set_jacobi_max_sweeps).
constexpr int kJacobiMaxSweeps = 40;
int jacobi_max_sweeps();

}  // namespace wp
