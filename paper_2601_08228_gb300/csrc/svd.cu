// w-svd, sp-w-svd (Algorithm 2, Thm 2.5, Sec. IV-B) and the Moore-Penrose
// inverse (Def. 2.6, Thm 2.6) built on the batched Jacobi SVD.
//
// w-svd:   A_hat = W(A); per slice the leading r triplets (jacobi.cu);
//          C_hat_k = U_r U_r^T A_hat_k  (= U_r Sigma_r V_r^T) when n1 >= n2,
//          C_hat_k = A_hat_k V_r V_r^T  otherwise;  C_r = W^{-1}(C_hat).
//          The other factor comes from the same small product:
//          V_r = (U_r^T A_hat_k)^T Sigma_r^{-1}, or U_r = A_hat_k V_r Sigma_r^{-1}.
// sp-w-svd: the same on the s_L and d_L slices only (Mallat rows [0, 2m));
//          every finer detail slice of C_hat is zero.
// wpinv:   full Jacobi SVD per slice; with the singular values above
//          rtol * sigma_max kept (w_i = 1 / sigma_i^2, else 0)
//          n1 >= n2:  X_hat_k = (A_k^T U) diag(w) U^T   (V = A^T U Sigma^-1)
//          n1 <  n2:  X_hat_k = V diag(w) (A_k V)^T      (U = A V Sigma^-1)
//          then optional refinement X <- X + X (I - A X) with the residual
//          in compensated (twice working precision) arithmetic, and
//          X = W^{-1}(X_hat).

#include "common.cuh"
#include "internal.cuh"

namespace wp {

// ---- small element-wise kernels ------------------------------------------------------

// Factor outputs of w-svd: U (p, n1, r), S (p, r), V (p, n2, r) from the
// Jacobi vectors `vec`, the product T and the singular values; slices
// [nsl, p) are zero (sp-w-svd).
__global__ void __launch_bounds__(256) wsvd_factors_kernel(const float* __restrict__ vec, const float* __restrict__ T,
                                                           const float* __restrict__ sig, int trans, int n1, int n2,
                                                           int r, int nsl, int p, float* __restrict__ U,
                                                           float* __restrict__ S, float* __restrict__ V) {
  const int64_t nu = int64_t(p) * n1 * r, nv = int64_t(p) * n2 * r, ns = int64_t(p) * r;
  const int64_t total = nu + nv + ns;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    if (i < nu) {
      const int64_t s = i / (int64_t(n1) * r);
      const int rem = int(i - s * n1 * r), row = rem / r, k = rem % r;
      float v = 0.f;
      if (s < nsl) {
        if (!trans) v = vec[i];
        else {
          const float sg = sig[s * r + k];
          v = sg > 0.f ? T[(s * n1 + row) * r + k] / sg : 0.f;   // T = A V (n1 x r)
        }
      }
      U[i] = v;
    } else if (i < nu + nv) {
      const int64_t j = i - nu;
      const int64_t s = j / (int64_t(n2) * r);
      const int rem = int(j - s * n2 * r), col = rem / r, k = rem % r;
      float v = 0.f;
      if (s < nsl) {
        if (trans) v = vec[j];
        else {
          const float sg = sig[s * r + k];
          v = sg > 0.f ? T[(s * r + k) * n2 + col] / sg : 0.f;   // T = U^T A (r x n2)
        }
      }
      V[j] = v;
    } else {
      const int64_t j = i - nu - nv;
      S[j] = (j / r < nsl) ? sig[j] : 0.f;
    }
  }
}

// T[:, k] *= w_k with w_k = 1/sigma_k^2 if sigma_k > rtol * sigma_0, else 0
// (T is (batch, rows, n) with n = number of singular values per slice).
__global__ void __launch_bounds__(256) pinv_scale_kernel(float* __restrict__ T, const float* __restrict__ sig, int rows,
                                                         int n, int batch, float rtol) {
  const int64_t total = int64_t(batch) * rows * n;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t s = i / (int64_t(rows) * n);
    const int k = int(i % n);
    const float smax = sig[s * n];
    const float sk = sig[s * n + k];
    const float w = (smax > 0.f && sk > rtol * smax) ? 1.f / (sk * sk) : 0.f;
    T[i] *= w;
  }
}

// R = I - A X per slice (A: m x n, X: n x m), each entry a compensated dot
// product: the algorithm Dot2 of Ogita, Rump and Oishi ("Accurate sum and
// dot product", SIAM J. Sci. Comput. 26, 2005), as accurate as if computed
// in twice the working precision and then rounded.  Every product a x is
// split exactly into p + e with one FMA (e = fma(a, x, -p)), the p are
// added with TwoSum (s + t = hi + p exactly), and the rounding errors e and
// t are summed plainly into `lo`.  With X close to the pseudo-inverse,
// A X is I + E with E of order kappa * eps, so R needs the extra precision;
// GB300 runs FP32 arithmetic at many times its FP64 rate.  The diagonal
// 1 - hi is exact (Sterbenz: hi is within a factor 2 of 1), so R rounds once.
// Every thread takes RB consecutive rows of one column of R, so each loaded
// element of X serves RB dot products (the rows of A are broadcast loads
// shared by the warp's lanes).
constexpr int RES_RB = 8;

__global__ void __launch_bounds__(256) residual_dot2_kernel(const float* __restrict__ A, const float* __restrict__ X,
                                                            float* __restrict__ R, int m, int n, int batch) {
  const int mb = (m + RES_RB - 1) / RES_RB;
  const int64_t total = int64_t(batch) * mb * m;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t s = i / (int64_t(mb) * m);
    const int rem = int(i - s * mb * m), rb = rem / m, col = rem % m;
    const int row0 = rb * RES_RB;
    const float* a = A + (s * m + row0) * n;
    const float* x = X + s * int64_t(n) * m + col;
    float hi[RES_RB], lo[RES_RB];
#pragma unroll
    for (int q = 0; q < RES_RB; ++q) hi[q] = lo[q] = 0.f;
    for (int l = 0; l < n; ++l) {
      const float xv = __ldg(x + int64_t(l) * m);
#pragma unroll
      for (int q = 0; q < RES_RB; ++q) {
        if (row0 + q < m) {
          const float av = __ldg(a + int64_t(q) * n + l);
          // _rn intrinsics: never contracted into FMAs, so every step rounds as written
          const float pr = __fmul_rn(av, xv);
          const float pe = fmaf(av, xv, -pr);          // av * xv = pr + pe exactly
          const float sm = __fadd_rn(hi[q], pr);       // TwoSum(hi, pr) = sm + se exactly
          const float bb = __fsub_rn(sm, hi[q]);
          const float se = __fadd_rn(__fsub_rn(hi[q], __fsub_rn(sm, bb)), __fsub_rn(pr, bb));
          hi[q] = sm;
          lo[q] = __fadd_rn(lo[q], __fadd_rn(pe, se));
        }
      }
    }
#pragma unroll
    for (int q = 0; q < RES_RB; ++q) {
      const int row = row0 + q;
      if (row < m) {
        const float d = (row == col) ? 1.f - hi[q] : -hi[q];
        R[(s * m + row) * int64_t(m) + col] = d - lo[q];
      }
    }
  }
}

__global__ void __launch_bounds__(256) axpy_kernel(float* __restrict__ y, const float* __restrict__ x, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] += x[i];
}

static unsigned grid_for(int64_t total) {
  const int64_t cap = int64_t(sm_count()) * 8;
  return unsigned(std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, cap)));
}

// ---- w-svd ------------------------------------------------------------------------

// Work of the QR preconditioner (0 when the shape is not preconditioned).
static size_t precond_bytes(int64_t n1, int64_t n2, int64_t p) {
  if (!jacobi_preconditioned(int(n1), int(n2))) return 0;
  return qr_work_bytes(int(std::max(n1, n2)), int(std::min(n1, n2)), int(p));
}

// Facewise Jacobi SVD of slices [0, nsl) of Ah, preconditioned by a QR where
// jacobi_preconditioned() says so.  *right = true when the vectors written
// to vec are right singular vectors (n2 x r per slice), false for left ones
// (n1 x r): the plain Jacobi yields the long side's vectors, the
// preconditioned one (Jacobi on R^T) the short side's.
static int facewise_svd(const float* Ah, int64_t n1, int64_t n2, int nsl, int r, float* vec, float* sig, void* qwork,
                        size_t qbytes, void* jwork, size_t jbytes, bool* right, cudaStream_t st) {
  const int N1 = int(n1), N2 = int(n2);
  if (qbytes > 0) {
    float* Rt = nullptr;
    WP_TRY(qr_r(Ah, N1, N2, nsl, qwork, qbytes, &Rt, st));
    const int nv = std::min(N1, N2);
    WP_TRY(jacobi_svd(Rt, nv, nv, 0, nsl, r, vec, sig, st));
    *right = n1 >= n2;
    return WP_OK;
  }
  WP_TRY(jacobi_svd(Ah, N1, N2, 0, nsl, r, vec, sig, st, jwork, jbytes));
  *right = n1 < n2;
  return WP_OK;
}

static void wsvd_layout(int64_t n1, int64_t n2, int64_t p, int r, Sizer& s) {
  const int64_t mx = std::max(n1, n2);
  s.take<float>(size_t(p) * n1 * n2);   // A_hat
  s.take<float>(size_t(p) * mx * r);    // Jacobi vectors
  s.take<float>(size_t(p) * r);         // singular values
  s.take<float>(size_t(p) * mx * r);    // T
  s.take<float>(size_t(p) * n1 * n2);   // C_hat
  s.take<float>(size_t(p) * n1 * r);    // spatial-domain factor staging: U
  s.take<float>(size_t(p) * r);         //                              S
  s.take<float>(size_t(p) * n2 * r);    //                              V
  s.take<char>(jacobi_work_bytes(int(n1), int(n2), int(p)));   // large slices: Jacobi work buffer
  s.take<char>(precond_bytes(n1, n2, p));                        // QR preconditioner
}

static int check_wsvd(int64_t n1, int64_t n2, int64_t p, int L, int r) {
  if (n1 < 1 || n2 < 1 || p < 1) return WP_ERR_SHAPE;
  if (n1 > 4096 || n2 > 4096 || p > INT32_MAX) return WP_ERR_SHAPE;
  WP_TRY(check_levels(p, L));
  if (r < 1 || r > std::min(n1, n2)) return WP_ERR_RANK;
  if (!jacobi_supported(int(n1), int(n2))) return WP_ERR_UNSUPPORTED;
  return WP_OK;
}

}  // namespace wp

using namespace wp;

extern "C" int wp_wsvd_workspace(int64_t n1, int64_t n2, int64_t p, int L, int r, size_t* bytes) {
  if (!bytes) return WP_ERR_NULL;
  WP_TRY(check_wsvd(n1, n2, p, L, r));
  Sizer s;
  wsvd_layout(n1, n2, p, r, s);
  *bytes = s.bytes();
  return WP_OK;
}

extern "C" int wp_wsvd(const float* A, float* C_r, float* U, float* S, float* V, int64_t n1, int64_t n2, int64_t p,
                       int L, int r, int sparse, int factors_in_wavelet_domain, void* ws, size_t ws_bytes,
                       void* stream) {
  WP_TRY(check_wsvd(n1, n2, p, L, r));
  if (!A || !C_r) return WP_ERR_NULL;
  const bool want_f = (U || S || V);
  if (want_f && !(U && S && V)) return WP_ERR_NULL;
  if (!aligned16(A) || !aligned16(C_r) || (want_f && (!aligned16(U) || !aligned16(S) || !aligned16(V))))
    return WP_ERR_ALIGN;
  const size_t ca = size_t(p) * n1 * n2 * 4;
  if (overlaps(A, ca, C_r, ca)) return WP_ERR_ALIAS;
  if (want_f && (overlaps(A, ca, U, size_t(p) * n1 * r * 4) || overlaps(A, ca, V, size_t(p) * n2 * r * 4) ||
                 overlaps(A, ca, S, size_t(p) * r * 4)))
    return WP_ERR_ALIAS;
  Sizer need;
  wsvd_layout(n1, n2, p, r, need);
  if (!ws || ws_bytes < need.bytes()) return WP_ERR_WORKSPACE;
  Carver cv(ws, ws_bytes);
  const int64_t mx = std::max(n1, n2);
  float* Ah = cv.take<float>(size_t(p) * n1 * n2);
  float* vec = cv.take<float>(size_t(p) * mx * r);
  float* sig = cv.take<float>(size_t(p) * r);
  float* T = cv.take<float>(size_t(p) * mx * r);
  float* Ch = cv.take<float>(size_t(p) * n1 * n2);
  float* Uw = cv.take<float>(size_t(p) * n1 * r);
  float* Sw = cv.take<float>(size_t(p) * r);
  float* Vw = cv.take<float>(size_t(p) * n2 * r);
  const size_t jw = jacobi_work_bytes(int(n1), int(n2), int(p));
  void* jwork = jw ? cv.take<char>(jw) : nullptr;
  const size_t qb = precond_bytes(n1, n2, p);
  void* qwork = qb ? cv.take<char>(qb) : nullptr;
  if (!cv.ok) return WP_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  const int N1 = int(n1), N2 = int(n2);
  const int64_t m = p >> L;
  const int nsl = int(sparse ? std::min<int64_t>(2 * m, p) : p);

  WP_TRY(lift_dispatch(LIFT_FWD, A, Ah, n1 * n2, p, L, st));
  bool trans = false;   // the Jacobi vectors are right singular vectors
  WP_TRY(facewise_svd(Ah, n1, n2, nsl, r, vec, sig, qwork, qb, jwork, jw, &trans, st));
  if (!trans) {
    // T = U_r^T A_hat (r x n2), C_hat = U_r T
    WP_TRY(sgemm_batched(vec, Ah, T, r, N2, N1, true, false, nsl, st));
    WP_TRY(sgemm_batched(vec, T, Ch, N1, N2, r, false, false, nsl, st));
  } else {
    // T = A_hat V_r (n1 x r), C_hat = T V_r^T
    WP_TRY(sgemm_batched(Ah, vec, T, N1, r, N2, false, false, nsl, st));
    WP_TRY(sgemm_batched(T, vec, Ch, N1, N2, r, false, true, nsl, st));
  }
  if (nsl < p)
    WP_CUDA_TRY(cudaMemsetAsync(Ch + int64_t(nsl) * n1 * n2, 0, size_t(p - nsl) * n1 * n2 * sizeof(float), st));
  WP_TRY(lift_dispatch(LIFT_INV, Ch, C_r, n1 * n2, p, L, st));
  if (want_f) {
    const bool wav = factors_in_wavelet_domain != 0;
    float* Uo = wav ? U : Uw;
    float* So = wav ? S : Sw;
    float* Vo = wav ? V : Vw;
    const int64_t total = p * (n1 + n2 + 1) * r;
    {
      WP_PROFILE("wsvd_factors", st);
      wsvd_factors_kernel<<<grid_for(total), 256, 0, st>>>(vec, T, sig, trans ? 1 : 0, N1, N2, r, nsl, int(p), Uo,
                                                           So, Vo);
      WP_TRY(launch_status());
    }
    if (!wav) {
      WP_TRY(lift_dispatch(LIFT_INV, Uw, U, n1 * r, p, L, st));
      WP_TRY(lift_dispatch(LIFT_INV, Sw, S, r, p, L, st));
      WP_TRY(lift_dispatch(LIFT_INV, Vw, V, n2 * r, p, L, st));
    }
  }
  return WP_OK;
}

// ---- Moore-Penrose inverse -------------------------------------------------------------

static void wpinv_layout(int64_t m, int64_t n, int64_t p, Sizer& s) {
  const int64_t mx = std::max(m, n), mn = std::min(m, n);
  s.take<float>(size_t(p) * m * n);     // A_hat
  s.take<float>(size_t(p) * mx * mn);   // Jacobi vectors (all)
  s.take<float>(size_t(p) * mn);        // singular values
  s.take<float>(size_t(p) * mx * mx);   // T
  s.take<float>(size_t(p) * n * m);     // X_hat
  s.take<float>(size_t(p) * m * m);     // residual R
  s.take<float>(size_t(p) * n * m);     // X R
  s.take<char>(jacobi_work_bytes(int(m), int(n), int(p)));   // large slices: Jacobi work buffer
}

extern "C" int wp_wpinv_workspace(int64_t m, int64_t n, int64_t p, int L, size_t* bytes) {
  if (!bytes) return WP_ERR_NULL;
  if (m < 1 || n < 1 || p < 1 || m > 4096 || n > 4096) return WP_ERR_SHAPE;
  WP_TRY(check_levels(p, L));
  if (!jacobi_supported(int(m), int(n))) return WP_ERR_UNSUPPORTED;
  Sizer s;
  wpinv_layout(m, n, p, s);
  *bytes = s.bytes();
  return WP_OK;
}

extern "C" int wp_wpinv(const float* A, float* X, int64_t m, int64_t n, int64_t p, int L, double rtol,
                        int refine_iters, void* ws, size_t ws_bytes, void* stream) {
  if (m < 1 || n < 1 || p < 1 || m > 4096 || n > 4096) return WP_ERR_SHAPE;
  WP_TRY(check_levels(p, L));
  if (!A || !X) return WP_ERR_NULL;
  if (!aligned16(A) || !aligned16(X)) return WP_ERR_ALIGN;
  if (refine_iters < 0 || refine_iters > 100) return WP_ERR_SHAPE;
  if (!jacobi_supported(int(m), int(n))) return WP_ERR_UNSUPPORTED;
  const size_t bytes = size_t(p) * m * n * 4;
  if (overlaps(A, bytes, X, bytes)) return WP_ERR_ALIAS;
  Sizer need;
  wpinv_layout(m, n, p, need);
  if (!ws || ws_bytes < need.bytes()) return WP_ERR_WORKSPACE;
  Carver cv(ws, ws_bytes);
  const int64_t mx = std::max(m, n), mn = std::min(m, n);
  float* Ah = cv.take<float>(size_t(p) * m * n);
  float* vec = cv.take<float>(size_t(p) * mx * mn);
  float* sig = cv.take<float>(size_t(p) * mn);
  float* T = cv.take<float>(size_t(p) * mx * mx);
  float* Xh = cv.take<float>(size_t(p) * n * m);
  float* R = cv.take<float>(size_t(p) * m * m);
  float* XR = cv.take<float>(size_t(p) * n * m);
  const size_t jw = jacobi_work_bytes(int(m), int(n), int(p));
  void* jwork = jw ? cv.take<char>(jw) : nullptr;
  if (!cv.ok) return WP_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  const int M = int(m), N = int(n), P = int(p), K = int(mn);
  const float tol = rtol < 0 ? float(mx) * 1.1920929e-7f : float(rtol);

  WP_TRY(lift_dispatch(LIFT_FWD, A, Ah, m * n, p, L, st));
  // the plain Jacobi: the pseudo-inverse needs every singular value down to
  // the cut-off, and R^T's columns (R's rows, graded like the singular
  // values) fall below the Jacobi's numerically-zero threshold there
  bool right = false;
  WP_TRY(facewise_svd(Ah, m, n, P, K, vec, sig, nullptr, 0, jwork, jw, &right, st));
  if (!right) {
    // U = vec (m x K); T = A^T U (n x K); T *= w; X_hat = T U^T (n x m)
    WP_TRY(sgemm_batched(Ah, vec, T, N, K, M, true, false, P, st));
    {
      WP_PROFILE("pinv_scale", st);
      pinv_scale_kernel<<<grid_for(p * n * K), 256, 0, st>>>(T, sig, N, K, P, tol);
      WP_TRY(launch_status());
    }
    WP_TRY(sgemm_batched(T, vec, Xh, N, M, K, false, true, P, st));
  } else {
    // V = vec (n x K); T = A V (m x K); T *= w; X_hat = V T^T (n x m)
    WP_TRY(sgemm_batched(Ah, vec, T, M, K, N, false, false, P, st));
    {
      WP_PROFILE("pinv_scale", st);
      pinv_scale_kernel<<<grid_for(p * m * K), 256, 0, st>>>(T, sig, M, K, P, tol);
      WP_TRY(launch_status());
    }
    WP_TRY(sgemm_batched(vec, T, Xh, N, M, K, false, true, P, st));
  }
  for (int it = 0; it < refine_iters; ++it) {
    {
      WP_PROFILE("pinv_residual", st);
      residual_dot2_kernel<<<grid_for(p * ((m + RES_RB - 1) / RES_RB) * m), 256, 0, st>>>(Ah, Xh, R, M, N, P);
      WP_TRY(launch_status());
    }
    WP_TRY(sgemm_batched(Xh, R, XR, N, M, M, false, false, P, st));
    {
      WP_PROFILE("pinv_update", st);
      axpy_kernel<<<grid_for(p * n * m), 256, 0, st>>>(Xh, XR, p * n * m);
      WP_TRY(launch_status());
    }
  }
  return lift_dispatch(LIFT_INV, Xh, X, n * m, p, L, st);
}
