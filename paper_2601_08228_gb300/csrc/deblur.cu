// One gradient step of w-product deblurring, the deblurring application of
// Sec. IV-C in its one-sided least-squares form:
//
//   f(X) = ||K *w X - Y||_F^2 + lam ||X||_F^2
//   grad f(X) = 2 K^T *w (K *w X - Y) + 2 lam X,     X <- X - eta grad f(X)
//
// The K^T *w R term is the backward pass of the w-product with respect to its
// second operand (adjoint route: W^T (K_hat^T Delta W^{-T} R)), so the step is
//   C = K *w X;  R = C - Y (and f(X) accumulated);  dX = backward_B(K, X, R);
//   X <- X - eta (2 dX + 2 lam X).
// Every launch is stream-ordered with no host synchronisation and no
// allocation, so a loop of steps can be captured in a CUDA graph.

#include "common.cuh"
#include "internal.cuh"

namespace wp {

// R = C - Y; with LOSS also loss += sum(R^2) + lam * sum(X^2).  Each thread
// sums its terms in FP32 with Kahan compensation and the threads' sums are
// combined in FP64: GB300's FP64 pipe is a small fraction of its FP32 rate,
// and FP64 arithmetic per element made this pass four times slower than
// its memory traffic.  Relative error of the loss: a few FP32 roundings.
template <bool LOSS>
__global__ void __launch_bounds__(256) residual_loss_kernel(const float* __restrict__ C, const float* __restrict__ Y,
                                                            const float* __restrict__ X, float* __restrict__ R,
                                                            int64_t n, float lam, double* loss) {
  float sum = 0.f, comp = 0.f;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float r = C[i] - Y[i];
    R[i] = r;
    if constexpr (LOSS) {
      const float x = X[i];
      const float term = fmaf(lam * x, x, r * r);
      const float yk = term - comp;
      const float t = sum + yk;
      comp = (t - sum) - yk;
      sum = t;
    }
  }
  if constexpr (LOSS) {
    double acc = double(sum) - double(comp);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double wsum[8];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < int(blockDim.x >> 5); ++w) t += wsum[w];
      atomicAdd(loss, t);
    }
  }
}

// X <- X - eta (2 dX + 2 lam X)
__global__ void __launch_bounds__(256) gd_update_kernel(float* __restrict__ X, const float* __restrict__ dX, int64_t n,
                                                        float lam, float eta) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float x = X[i];
    X[i] = x - eta * (2.f * dX[i] + 2.f * lam * x);
  }
}

static unsigned grid_elems(int64_t n) {
  return unsigned(std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, int64_t(sm_count()) * 8)));
}

static void deblur_layout(int64_t n1, int64_t n2, int64_t p, int L, int prec, Sizer& s, size_t* prod_ws,
                          size_t* bwd_ws) {
  wp_wprod_workspace(n1, n1, n2, p, L, prec, prod_ws);
  wp_wprod_backward_workspace(n1, n1, n2, p, L, prec, bwd_ws);
  s.take<float>(size_t(p) * n1 * n2);      // C = K *w X, then dX
  s.take<float>(size_t(p) * n1 * n2);      // R
  s.take<char>(std::max(*prod_ws, *bwd_ws));
}

}  // namespace wp

using namespace wp;

extern "C" int wp_deblur_workspace(int64_t n1, int64_t n2, int64_t p, int L, int prec, size_t* bytes) {
  if (!bytes) return WP_ERR_NULL;
  if (n1 < 1 || n2 < 1 || p < 1) return WP_ERR_SHAPE;
  WP_TRY(check_levels(p, L));
  if (prec < WP_PREC_FP32 || prec > WP_PREC_FP8) return WP_ERR_PREC;
  Sizer s;
  size_t a = 0, b = 0;
  deblur_layout(n1, n2, p, L, prec, s, &a, &b);
  *bytes = s.bytes();
  return WP_OK;
}

extern "C" int wp_deblur_step(const float* K, const float* Y, float* X, int64_t n1, int64_t n2, int64_t p, int L,
                              float lam, float eta, int prec, double* loss, void* ws, size_t ws_bytes,
                              void* stream) {
  if (n1 < 1 || n2 < 1 || p < 1) return WP_ERR_SHAPE;
  WP_TRY(check_levels(p, L));
  if (!K || !Y || !X) return WP_ERR_NULL;
  if (prec < WP_PREC_FP32 || prec > WP_PREC_FP8) return WP_ERR_PREC;
  if (!aligned16(K) || !aligned16(Y) || !aligned16(X)) return WP_ERR_ALIGN;
  const size_t bx = size_t(p) * n1 * n2 * 4, bk = size_t(p) * n1 * n1 * 4;
  if (overlaps(X, bx, K, bk) || overlaps(X, bx, Y, bx)) return WP_ERR_ALIAS;
  Sizer need;
  size_t prod_ws = 0, bwd_ws = 0;
  deblur_layout(n1, n2, p, L, prec, need, &prod_ws, &bwd_ws);
  if (!ws || ws_bytes < need.bytes()) return WP_ERR_WORKSPACE;
  Carver cv(ws, ws_bytes);
  float* C = cv.take<float>(size_t(p) * n1 * n2);
  float* R = cv.take<float>(size_t(p) * n1 * n2);
  void* inner = cv.take<char>(std::max(prod_ws, bwd_ws));
  if (!cv.ok) return WP_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  const int64_t n = p * n1 * n2;
  WP_TRY(wp_wprod(K, X, C, n1, n1, n2, p, L, 0, 0, prec, inner, prod_ws, stream));
  {
    WP_PROFILE("deblur_residual", st);
    if (loss) residual_loss_kernel<true><<<grid_elems(n), 256, 0, st>>>(C, Y, X, R, n, lam, loss);
    else residual_loss_kernel<false><<<grid_elems(n), 256, 0, st>>>(C, Y, X, R, n, lam, nullptr);
    WP_TRY(launch_status());
  }
  // dX = K^T *w R by the adjoint backward of the w-product (second operand)
  WP_TRY(wp_wprod_backward(K, X, R, nullptr, C, n1, n1, n2, p, L, prec, inner, bwd_ws, stream));
  WP_PROFILE("deblur_update", st);
  gd_update_kernel<<<grid_elems(n), 256, 0, st>>>(X, C, n, lam, eta);
  return launch_status();
}

// ---- two-sided pseudo-inverse deblurring (Sec. IV-C) ----------------------------------
//
// X = A_V^dagger *w B *w (A_H^T)^dagger: two w-pseudo-inverses (wp_wpinv) and
// two w-products.  (A_H^T)^dagger = (A_H^dagger)^T (facewise, and the
// transform commutes with the slice transpose, Thm 2.1), so the second
// product takes P_H = A_H^dagger with transB.

static int deblur_pinv_layout(int64_t n1, int64_t n2, int64_t p, int L, int prec, Sizer& s, size_t* inner) {
  size_t a = 0, b = 0, c = 0, d = 0;
  WP_TRY(wp_wpinv_workspace(n1, n1, p, L, &a));
  WP_TRY(wp_wpinv_workspace(n2, n2, p, L, &b));
  WP_TRY(wp_wprod_workspace(n1, n1, n2, p, L, prec, &c));   // P_V *w B
  WP_TRY(wp_wprod_workspace(n1, n2, n2, p, L, prec, &d));   // T *w P_H^T
  *inner = std::max(std::max(a, b), std::max(c, d));
  s.take<float>(size_t(p) * n1 * n1);   // P_V
  s.take<float>(size_t(p) * n2 * n2);   // P_H
  s.take<float>(size_t(p) * n1 * n2);   // T = P_V *w B
  s.take<char>(*inner);
  return WP_OK;
}

extern "C" int wp_deblur_pinv_workspace(int64_t n1, int64_t n2, int64_t p, int L, int prec, size_t* bytes) {
  if (!bytes) return WP_ERR_NULL;
  if (n1 < 1 || n2 < 1 || p < 1) return WP_ERR_SHAPE;
  WP_TRY(check_levels(p, L));
  if (prec < WP_PREC_FP32 || prec > WP_PREC_FP8) return WP_ERR_PREC;
  Sizer s;
  size_t inner = 0;
  WP_TRY(deblur_pinv_layout(n1, n2, p, L, prec, s, &inner));
  *bytes = s.bytes();
  return WP_OK;
}

extern "C" int wp_deblur_pinv(const float* AV, const float* AH, const float* B, float* X, int64_t n1, int64_t n2,
                              int64_t p, int L, double rtol, int refine_iters, int prec, void* ws, size_t ws_bytes,
                              void* stream) {
  if (n1 < 1 || n2 < 1 || p < 1) return WP_ERR_SHAPE;
  WP_TRY(check_levels(p, L));
  if (!AV || !AH || !B || !X) return WP_ERR_NULL;
  if (prec < WP_PREC_FP32 || prec > WP_PREC_FP8) return WP_ERR_PREC;
  if (!aligned16(AV) || !aligned16(AH) || !aligned16(B) || !aligned16(X)) return WP_ERR_ALIGN;
  const size_t bx = size_t(p) * n1 * n2 * 4;
  if (overlaps(X, bx, AV, size_t(p) * n1 * n1 * 4) || overlaps(X, bx, AH, size_t(p) * n2 * n2 * 4) ||
      overlaps(X, bx, B, bx))
    return WP_ERR_ALIAS;
  Sizer need;
  size_t inner_bytes = 0;
  WP_TRY(deblur_pinv_layout(n1, n2, p, L, prec, need, &inner_bytes));
  if (!ws || ws_bytes < need.bytes()) return WP_ERR_WORKSPACE;
  Carver cv(ws, ws_bytes);
  float* PV = cv.take<float>(size_t(p) * n1 * n1);
  float* PH = cv.take<float>(size_t(p) * n2 * n2);
  float* T = cv.take<float>(size_t(p) * n1 * n2);
  void* inner = cv.take<char>(inner_bytes);
  if (!cv.ok) return WP_ERR_WORKSPACE;
  WP_TRY(wp_wpinv(AV, PV, n1, n1, p, L, rtol, refine_iters, inner, inner_bytes, stream));
  WP_TRY(wp_wpinv(AH, PH, n2, n2, p, L, rtol, refine_iters, inner, inner_bytes, stream));
  WP_TRY(wp_wprod(PV, B, T, n1, n1, n2, p, L, 0, 0, prec, inner, inner_bytes, stream));
  return wp_wprod(T, PH, X, n1, n2, n2, p, L, 0, 1, prec, inner, inner_bytes, stream);
}
