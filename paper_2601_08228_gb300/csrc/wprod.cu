// The w-product (Def. 2.1, Algorithm 1), its face-product and its backward.
//
//   C = W^{-1}( W(op A) Delta W(op B) )
//
// Forward: lift A and B (one fused pass each), face-product of the p
// wavelet-domain slices, inverse-lift C.  For the tensor-core precisions
// without transposes the transform is folded into the operand preparation
// and the GEMM epilogue instead (tc_wprod_fused in gemm_tc.cu).  The transform acts tube by tube,
// so a transposed operand is lifted in its stored layout and the transpose is
// applied by the GEMM (Thm 2.1: W(A^T) = W(A)^T).
//
// Backward (adjoint route; the transform is not orthogonal, Remark 2.1):
//   G_hat = W^{-T} G,  dA = W^T (G_hat Delta B_hat^T),  dB = W^T (A_hat^T Delta G_hat)
// A_hat and B_hat are recomputed from A and B, not stored by the forward.

#include "common.cuh"
#include "internal.cuh"

namespace wp {

static bool valid_prec(int prec) { return prec >= WP_PREC_FP32 && prec <= WP_PREC_FP8; }

static size_t facewise_ws(int64_t n1, int64_t n2, int64_t n4, int64_t p, int prec) {
  return prec == WP_PREC_FP32 ? 0 : tc_facewise_workspace(n1, n4, n2, p, prec);
}

static int facewise_run(const float* Ah, const float* Bh, float* Ch, int64_t n1, int64_t n2,
                        int64_t n4, int64_t p, bool tA, bool tB, int prec, void* ws,
                        size_t ws_bytes, cudaStream_t st) {
  if (prec == WP_PREC_FP32) {
    if (n1 > INT32_MAX || n2 > INT32_MAX || n4 > INT32_MAX || p > INT32_MAX) return WP_ERR_SHAPE;
    return sgemm_batched(Ah, Bh, Ch, int(n1), int(n4), int(n2), tA, tB, int(p), st);
  }
  return tc_facewise(Ah, Bh, Ch, n1, n4, n2, p, tA, tB, prec, ws, ws_bytes, st);
}

static int check_prod_args(const float* A, const float* B, const float* C, int64_t n1,
                           int64_t n2, int64_t n4, int64_t p, int prec) {
  if (n1 < 1 || n2 < 1 || n4 < 1 || p < 1) return WP_ERR_SHAPE;
  if (!A || !B || !C) return WP_ERR_NULL;
  if (n1 > (1 << 24) || n2 > (1 << 24) || n4 > (1 << 24)) return WP_ERR_SHAPE;
  if (!valid_prec(prec)) return WP_ERR_PREC;
  if (!aligned16(A) || !aligned16(B) || !aligned16(C)) return WP_ERR_ALIGN;
  const size_t ca = size_t(p) * n1 * n2 * 4, cb = size_t(p) * n2 * n4 * 4, cc = size_t(p) * n1 * n4 * 4;
  if (overlaps(C, cc, A, ca) || overlaps(C, cc, B, cb)) return WP_ERR_ALIAS;
  return WP_OK;
}

}  // namespace wp

using namespace wp;

extern "C" int wp_facewise_workspace(int64_t n1, int64_t n2, int64_t n4, int64_t p, int prec,
                                     size_t* bytes) {
  if (!bytes) return WP_ERR_NULL;
  if (n1 < 1 || n2 < 1 || n4 < 1 || p < 1) return WP_ERR_SHAPE;
  if (!valid_prec(prec)) return WP_ERR_PREC;
  *bytes = facewise_ws(n1, n2, n4, p, prec);
  return WP_OK;
}

extern "C" int wp_facewise(const float* Ah, const float* Bh, float* Ch, int64_t n1, int64_t n2,
                           int64_t n4, int64_t p, int transA, int transB, int prec, void* ws,
                           size_t ws_bytes, void* stream) {
  WP_TRY(check_prod_args(Ah, Bh, Ch, n1, n2, n4, p, prec));
  const size_t need = facewise_ws(n1, n2, n4, p, prec);
  if (need > 0 && (ws == nullptr || ws_bytes < need)) return WP_ERR_WORKSPACE;
  return facewise_run(Ah, Bh, Ch, n1, n2, n4, p, transA != 0, transB != 0, prec, ws, ws_bytes,
                      as_stream(stream));
}

static void wprod_layout(int64_t n1, int64_t n2, int64_t n4, int64_t p, int prec, Sizer& s) {
  s.take<float>(size_t(p) * n1 * n2);   // A_hat
  s.take<float>(size_t(p) * n2 * n4);   // B_hat
  s.take<float>(size_t(p) * n1 * n4);   // C_hat
  s.take<char>(facewise_ws(n1, n2, n4, p, prec));
}

extern "C" int wp_wprod_workspace(int64_t n1, int64_t n2, int64_t n4, int64_t p, int L, int prec,
                                  size_t* bytes) {
  if (!bytes) return WP_ERR_NULL;
  if (n1 < 1 || n2 < 1 || n4 < 1 || p < 1) return WP_ERR_SHAPE;
  WP_TRY(check_levels(p, L));
  if (!valid_prec(prec)) return WP_ERR_PREC;
  Sizer s;
  wprod_layout(n1, n2, n4, p, prec, s);
  *bytes = s.bytes();
  return WP_OK;
}

extern "C" int wp_wprod(const float* A, const float* B, float* C, int64_t n1, int64_t n2,
                        int64_t n4, int64_t p, int L, int transA, int transB, int prec, void* ws,
                        size_t ws_bytes, void* stream) {
  WP_TRY(check_prod_args(A, B, C, n1, n2, n4, p, prec));
  WP_TRY(check_levels(p, L));
  Sizer need;
  wprod_layout(n1, n2, n4, p, prec, need);
  if (ws == nullptr || ws_bytes < need.bytes()) return WP_ERR_WORKSPACE;
  if (!transA && !transB && prec != WP_PREC_FP32) {
    const int st_fused = tc_wprod_fused(A, B, C, n1, n2, n4, p, L, prec, ws, ws_bytes, as_stream(stream));
    if (st_fused != WP_ERR_UNSUPPORTED) return st_fused;
  }
  Carver cv(ws, ws_bytes);
  float* Ah = cv.take<float>(size_t(p) * n1 * n2);
  float* Bh = cv.take<float>(size_t(p) * n2 * n4);
  float* Ch = cv.take<float>(size_t(p) * n1 * n4);
  const size_t fws = facewise_ws(n1, n2, n4, p, prec);
  void* fw = fws ? cv.take<char>(fws) : nullptr;
  if (!cv.ok) return WP_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  // A_hat, B_hat and C_hat never leave this call: group-interleaved order
  const bool il = L <= kMaxInterleavedLevels;
  WP_TRY(lift_dispatch(LIFT_FWD, A, Ah, n1 * n2, p, L, st, il));
  WP_TRY(lift_dispatch(LIFT_FWD, B, Bh, n2 * n4, p, L, st, il));
  WP_TRY(facewise_run(Ah, Bh, Ch, n1, n2, n4, p, transA != 0, transB != 0, prec, fw, fws, st));
  return lift_dispatch(LIFT_INV, Ch, C, n1 * n4, p, L, st, il);
}

static void backward_layout(int64_t n1, int64_t n2, int64_t n4, int64_t p, int prec, Sizer& s) {
  s.take<float>(size_t(p) * n1 * n2);   // A_hat
  s.take<float>(size_t(p) * n2 * n4);   // B_hat
  s.take<float>(size_t(p) * n1 * n4);   // G_hat
  s.take<float>(size_t(p) * std::max(n1 * n2, n2 * n4));   // dA_hat / dB_hat
  s.take<char>(std::max(facewise_ws(n1, n4, n2, p, prec), facewise_ws(n2, n1, n4, p, prec)));
}

extern "C" int wp_wprod_backward_workspace(int64_t n1, int64_t n2, int64_t n4, int64_t p, int L,
                                           int prec, size_t* bytes) {
  if (!bytes) return WP_ERR_NULL;
  if (n1 < 1 || n2 < 1 || n4 < 1 || p < 1) return WP_ERR_SHAPE;
  WP_TRY(check_levels(p, L));
  if (!valid_prec(prec)) return WP_ERR_PREC;
  Sizer s;
  backward_layout(n1, n2, n4, p, prec, s);
  *bytes = s.bytes();
  return WP_OK;
}

extern "C" int wp_wprod_backward(const float* A, const float* B, const float* G, float* dA,
                                 float* dB, int64_t n1, int64_t n2, int64_t n4, int64_t p, int L,
                                 int prec, void* ws, size_t ws_bytes, void* stream) {
  if (!A || !B || !G) return WP_ERR_NULL;
  if (n1 < 1 || n2 < 1 || n4 < 1 || p < 1) return WP_ERR_SHAPE;
  WP_TRY(check_levels(p, L));
  if (!valid_prec(prec)) return WP_ERR_PREC;
  if (!aligned16(A) || !aligned16(B) || !aligned16(G)) return WP_ERR_ALIGN;
  if ((dA && !aligned16(dA)) || (dB && !aligned16(dB))) return WP_ERR_ALIGN;
  const size_t ca = size_t(p) * n1 * n2 * 4, cb = size_t(p) * n2 * n4 * 4, cg = size_t(p) * n1 * n4 * 4;
  for (const float* out : {static_cast<const float*>(dA), static_cast<const float*>(dB)}) {
    if (!out) continue;
    const size_t co = (out == dA) ? ca : cb;
    if (overlaps(out, co, A, ca) || overlaps(out, co, B, cb) || overlaps(out, co, G, cg))
      return WP_ERR_ALIAS;
  }
  if (dA && dB && overlaps(dA, ca, dB, cb)) return WP_ERR_ALIAS;
  Sizer need;
  backward_layout(n1, n2, n4, p, prec, need);
  if (ws == nullptr || ws_bytes < need.bytes()) return WP_ERR_WORKSPACE;
  Carver cv(ws, ws_bytes);
  float* Ah = cv.take<float>(size_t(p) * n1 * n2);
  float* Bh = cv.take<float>(size_t(p) * n2 * n4);
  float* Gh = cv.take<float>(size_t(p) * n1 * n4);
  float* dXh = cv.take<float>(size_t(p) * std::max(n1 * n2, n2 * n4));
  const size_t fws = std::max(facewise_ws(n1, n4, n2, p, prec), facewise_ws(n2, n1, n4, p, prec));
  void* fw = fws ? cv.take<char>(fws) : nullptr;
  if (!cv.ok) return WP_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  // the wavelet-domain intermediates never leave this call: group-interleaved order
  const bool il = L <= kMaxInterleavedLevels;
  WP_TRY(lift_dispatch(LIFT_IADJ, G, Gh, n1 * n4, p, L, st, il));
  if (dA) {
    // dA_hat_k = G_hat_k B_hat_k^T: (n1 x n4) (n4 x n2)
    WP_TRY(lift_dispatch(LIFT_FWD, B, Bh, n2 * n4, p, L, st, il));
    WP_TRY(facewise_run(Gh, Bh, dXh, n1, n4, n2, p, false, true, prec, fw, fws, st));
    WP_TRY(lift_dispatch(LIFT_ADJ, dXh, dA, n1 * n2, p, L, st, il));
  }
  if (dB) {
    // dB_hat_k = A_hat_k^T G_hat_k: (n2 x n1) (n1 x n4)
    WP_TRY(lift_dispatch(LIFT_FWD, A, Ah, n1 * n2, p, L, st, il));
    WP_TRY(facewise_run(Ah, Gh, dXh, n2, n1, n4, p, true, false, prec, fw, fws, st));
    WP_TRY(lift_dispatch(LIFT_ADJ, dXh, dB, n2 * n4, p, L, st, il));
  }
  return WP_OK;
}
