// Lifting with general per-level predict / update operators (Sec. II-A,
// Eq. 2-3 with arbitrary P_j and U_j; Example 2.1; Remark 3.1), its inverse
// and both adjoints, and the w-product and backward built on them.
//
// Level j splits its input f (length n) into odd[k] = f[2k] and
// even[k] = f[2k + 1] (Algorithm 1's 1-based odd / even positions) and
//   forward   d = odd - P(even),   s = even + U(d)
//   inverse   even = s - U(d),     odd = d + P(even)
//   W^T       b = g_d + U^T g_s,   g_even = g_s - P^T b,  g_odd = b
//   W^{-T}    a = even + P^T odd,  g_d = odd - U^T a,     g_s = a
// with stencil operators (Op y)[k] = sum_t c_t y[refl(k + off + t)] under
// half-sample symmetric extension (refl(-1 - i) = i, refl(N + i) = N - 1 - i)
// and their exact transposes, evaluated as gathers: (Op^T y)[i] sums
// c_t y[k] over the k with refl(k + off + t) = i, which (the stencil reaching
// less than N) are k = i - off - t, -1 - i - off - t and 2N - 1 - i - off - t
// whenever they lie in [0, N).  With P = I and U = I / 2 this is the
// lazy-Haar transform of lift.cu.
//
// The operators couple neighbouring tube positions across the 2^L-slice
// groups of the Haar transform, so the transform is no longer local to a
// group: a CTA owns 32 whole mode-3 tubes (all p slices of 32 consecutive
// plane elements), held in shared memory as [p][32] tiles (the 32 tubes of
// a slice on 32 consecutive banks).  Four threads share a tube -- one in
// each of the CTA's four warps -- and split every pass of every level over
// k, with a CTA barrier between passes.  A spatial input tile arrives by
// p bulk copies of one 128-byte slice row each (cp.async.bulk, one
// mbarrier, bounded wait); Mallat-ordered inputs are read level by level.
// Each tube element is read from HBM once and written once (stores
// coalesced across the 32 tubes).

#include "common.cuh"
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace wp {

struct GOp {
  int off, len;
  float c[4];
};
struct GLevels {
  GOp P[WP_MAX_LEVELS], U[WP_MAX_LEVELS];
};

constexpr int kGTile = 32;           // tubes (plane elements) per CTA
constexpr int kGParts = 4;           // threads per tube
constexpr int kGThreads = kGTile * kGParts;

__device__ __forceinline__ int refl(int i, int n) {
  // half-sample symmetric extension; stencils reach less than n (host check)
  if (i < 0) i = -1 - i;
  if (i >= n) i = 2 * n - 1 - i;
  return i;
}

// (Op y)[k], k < n; y[i] at y0[i * ys]
__device__ __forceinline__ float op_at(const GOp& op, const float* y0, int ys, int k, int n) {
  float acc = 0.f;
  for (int t = 0; t < op.len; ++t) acc = fmaf(op.c[t], y0[refl(k + op.off + t, n) * ys], acc);
  return acc;
}

// (Op^T y)[i], i < n: the three preimages of i under k -> refl(k + off + t)
__device__ __forceinline__ float opT_at(const GOp& op, const float* y0, int ys, int i, int n) {
  float acc = 0.f;
  for (int t = 0; t < op.len; ++t) {
    const int k0 = i - op.off - t, k1 = -1 - i - op.off - t, k2 = 2 * n - 1 - i - op.off - t;
    if (k0 >= 0 && k0 < n) acc = fmaf(op.c[t], y0[k0 * ys], acc);
    if (k1 >= 0 && k1 < n) acc = fmaf(op.c[t], y0[k1 * ys], acc);
    if (k2 >= 0 && k2 < n) acc = fmaf(op.c[t], y0[k2 * ys], acc);
  }
  return acc;
}

__device__ __forceinline__ void bulk_row(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   ptx::smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(ptx::smem_u32(bar))
               : "memory");
}

// OP: 0 forward, 1 inverse, 2 W^T, 3 W^{-T}.  bulk: the spatial input (OP 0,
// 3) arrives by bulk copies (plane % 4 == 0, 16-byte aligned input).
template <int OP>
__global__ void __launch_bounds__(kGThreads) glift_kernel(const float* __restrict__ in, float* __restrict__ out,
                                                          int64_t plane, int p, int L, GLevels lv, int bulk,
                                                          int* status) {
  extern __shared__ __align__(128) float sm[];      // two buffers [p][kGTile]
  __shared__ __align__(8) uint64_t bar;
  constexpr int S = kGTile;                           // stride between tube positions in a buffer
  const int t = int(threadIdx.x) % kGTile, part = int(threadIdx.x) / kGTile;
  const int64_t e0 = int64_t(blockIdx.x) * kGTile, e = e0 + t;
  const bool act = e < plane;
  float* cur = sm + t;
  float* nxt = sm + size_t(p) * kGTile + t;
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (OP == 0 || OP == 3) {
    // spatial tube in, coefficients out: finest level first
    if (bulk) {
      const int width = int(plane - e0 < kGTile ? plane - e0 : int64_t(kGTile));
      __shared__ int s_ok;
      if (threadIdx.x == 0) {
        ptx::mbar_init(&bar, 1);
        ptx::fence_mbar_init();
        ptx::mbar_arrive_expect_tx(&bar, uint32_t(p) * uint32_t(width) * 4u);
        for (int k = 0; k < p; ++k) bulk_row(sm + k * S, in + k * plane + e0, uint32_t(width) * 4u, &bar);
        // one bounded wait for the CTA; on expiry (status word set) wait once
        // more, bounded, for the copies still in flight, and give up
        s_ok = ptx::mbar_wait(&bar, 0, status) ? 1 : 0;
        if (!s_ok) ptx::mbar_wait(&bar, 0, nullptr, 100000000ull);
      }
      __syncthreads();
      if (!s_ok) return;
      ptx::mbar_try_wait(&bar, 0);   // completed phase: orders the copied data before this thread's reads
    } else if (act) {
      for (int k = part; k < p; k += kGParts) cur[k * S] = __ldg(in + k * plane + e);
    }
    __syncthreads();
    for (int j = 1; j <= L; ++j) {
      const int h = p >> j;
      const GOp& P = lv.P[j - 1];
      const GOp& U = lv.U[j - 1];
      if (OP == 0) {
        // d -> nxt[h..2h) and out, then s -> nxt[0..h)
        if (act)
          for (int k = part; k < h; k += kGParts) {
            const float d = cur[(2 * k) * S] - op_at(P, cur + S, 2 * S, k, h);
            nxt[(h + k) * S] = d;
            out[int64_t(h + k) * plane + e] = d;
          }
        __syncthreads();
        if (act)
          for (int k = part; k < h; k += kGParts) nxt[k * S] = cur[(2 * k + 1) * S] + op_at(U, nxt + h * S, S, k, h);
      } else {
        // a = even + P^T odd -> nxt[0..h), then g_d = odd - U^T a -> nxt[h..2h) and out
        if (act)
          for (int k = part; k < h; k += kGParts) nxt[k * S] = cur[(2 * k + 1) * S] + opT_at(P, cur, 2 * S, k, h);
        __syncthreads();
        if (act)
          for (int k = part; k < h; k += kGParts) {
            const float gd = cur[(2 * k) * S] - opT_at(U, nxt, S, k, h);
            nxt[(h + k) * S] = gd;
            out[int64_t(h + k) * plane + e] = gd;
          }
      }
      __syncthreads();
      float* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
    if (act)
      for (int k = part; k < (p >> L); k += kGParts) out[k * plane + e] = cur[k * S];
  } else {
    // coefficients in, spatial tube out: coarsest level first
    if (act)
      for (int k = part; k < (p >> L); k += kGParts) cur[k * S] = __ldg(in + k * plane + e);
    for (int j = L; j >= 1; --j) {
      const int h = p >> j;
      const GOp& P = lv.P[j - 1];
      const GOp& U = lv.U[j - 1];
      if (act)
        for (int k = part; k < h; k += kGParts) nxt[(h + k) * S] = __ldg(in + int64_t(h + k) * plane + e);
      __syncthreads();
      if (OP == 1) {
        // even = s - U(d) -> nxt[0..h); then f[2k+1] = even, f[2k] = d + P(even) -> cur[0..2h)
        if (act)
          for (int k = part; k < h; k += kGParts) nxt[k * S] = cur[k * S] - op_at(U, nxt + h * S, S, k, h);
        __syncthreads();
        if (act)
          for (int k = part; k < h; k += kGParts) {
            cur[(2 * k + 1) * S] = nxt[k * S];
            cur[(2 * k) * S] = nxt[(h + k) * S] + op_at(P, nxt, S, k, h);
          }
      } else {
        // b = g_d + U^T g_s -> nxt[h..2h) (in place: each k reads its own g_d);
        // g_even = g_s - P^T b -> nxt[0..h); then interleave into cur[0..2h)
        if (act)
          for (int k = part; k < h; k += kGParts) nxt[(h + k) * S] += opT_at(U, cur, S, k, h);
        __syncthreads();
        if (act)
          for (int k = part; k < h; k += kGParts) nxt[k * S] = cur[k * S] - opT_at(P, nxt + h * S, S, k, h);
        __syncthreads();
        if (act)
          for (int k = part; k < h; k += kGParts) {
            cur[(2 * k + 1) * S] = nxt[k * S];
            cur[(2 * k) * S] = nxt[(h + k) * S];
          }
      }
      __syncthreads();
    }
    if (act)
      for (int k = part; k < p; k += kGParts) out[k * plane + e] = cur[k * S];
  }
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---- host side ----------------------------------------------------------------------

constexpr int kGMaxP = 800;         // two [p][32] FP32 buffers in 200 KB of shared memory

static int to_levels(const wp_lift_ops* ops, int64_t p, int L, GLevels* lv) {
  if (L < 0 || L > WP_MAX_LEVELS) return WP_ERR_LEVELS;
  if (L > 0 && !ops) return WP_ERR_NULL;
  *lv = GLevels{};
  for (int j = 1; j <= L; ++j) {
    const int64_t h = p >> j;
    const wp_lift_ops& o = ops[j - 1];
    const int32_t offs[2] = {o.predict_offset, o.update_offset};
    const int32_t lens[2] = {o.predict_taps, o.update_taps};
    for (int q = 0; q < 2; ++q) {
      if (lens[q] < 0 || lens[q] > 4) return WP_ERR_SHAPE;
      if (lens[q] > 0) {
        const int64_t reach = std::max<int64_t>(std::abs(int64_t(offs[q])), std::abs(int64_t(offs[q]) + lens[q] - 1));
        if (reach >= h) return WP_ERR_SHAPE;
      }
    }
    GOp P{o.predict_offset, o.predict_taps, {0.f, 0.f, 0.f, 0.f}};
    GOp U{o.update_offset, o.update_taps, {0.f, 0.f, 0.f, 0.f}};
    for (int t = 0; t < 4; ++t) {
      P.c[t] = o.predict[t];
      U.c[t] = o.update[t];
    }
    lv->P[j - 1] = P;
    lv->U[j - 1] = U;
  }
  return WP_OK;
}

template <int OP>
static int launch_glift(const float* in, float* out, int64_t plane, int64_t p, int L, const GLevels& lv,
                        cudaStream_t st) {
  const size_t smem = size_t(2) * p * kGTile * sizeof(float);
  const int bulk = (OP == 0 || OP == 3) && plane % 4 == 0 && aligned16(in);
  static bool attr = false;
  if (!attr) {
    WP_CUDA_TRY(cudaFuncSetAttribute(glift_kernel<OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(size_t(2) * kGMaxP * kGTile * sizeof(float))));
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned((plane + kGTile - 1) / kGTile), 1, 1);
  cfg.blockDim = dim3(kGThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attrs[1];
  attrs[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attrs[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attrs;
  cfg.numAttrs = 1;
  static const char* const names[4] = {"glift_forward", "glift_inverse", "glift_adjoint", "glift_inverse_adjoint"};
  WP_PROFILE(names[OP], st);
  WP_CUDA_TRY(cudaLaunchKernelEx(&cfg, glift_kernel<OP>, in, out, plane, int(p), L, lv, bulk, device_status_ptr()));
  return launch_status();
}

static int glift_dispatch(int op, const float* in, float* out, int64_t plane, int64_t p, int L, const GLevels& lv,
                          cudaStream_t st) {
  if (plane > int64_t(INT32_MAX) * kGTile) return WP_ERR_SHAPE;
  switch (op) {
    case 0: return launch_glift<0>(in, out, plane, p, L, lv, st);
    case 1: return launch_glift<1>(in, out, plane, p, L, lv, st);
    case 2: return launch_glift<2>(in, out, plane, p, L, lv, st);
    default: return launch_glift<3>(in, out, plane, p, L, lv, st);
  }
}

static int check_glift(int64_t p, int L, const wp_lift_ops* ops, GLevels* lv) {
  WP_TRY(check_levels(p, L));
  if (p > kGMaxP) return WP_ERR_UNSUPPORTED;
  return to_levels(ops, p, L, lv);
}

}  // namespace wp

using namespace wp;

extern "C" int wp_glift(const float* x, float* y, int64_t n1, int64_t n2, int64_t p, int L, const wp_lift_ops* ops,
                        int op, void* stream) {
  if (n1 < 1 || n2 < 1 || p < 1) return WP_ERR_SHAPE;
  if (!x || !y) return WP_ERR_NULL;
  if (op < 0 || op > 3) return WP_ERR_SHAPE;
  GLevels lv;
  WP_TRY(check_glift(p, L, ops, &lv));
  const size_t bytes = size_t(n1) * n2 * p * sizeof(float);
  if (overlaps(x, bytes, y, bytes)) return WP_ERR_ALIAS;
  if (!aligned16(x) || !aligned16(y)) return WP_ERR_ALIGN;
  return glift_dispatch(op, x, y, n1 * n2, p, L, lv, as_stream(stream));
}

static int facewise_any(const float* Ah, const float* Bh, float* Ch, int64_t n1, int64_t n2, int64_t n4, int64_t p,
                        bool tA, bool tB, int prec, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (prec == WP_PREC_FP32) {
    if (n1 > INT32_MAX || n2 > INT32_MAX || n4 > INT32_MAX || p > INT32_MAX) return WP_ERR_SHAPE;
    return sgemm_batched(Ah, Bh, Ch, int(n1), int(n4), int(n2), tA, tB, int(p), st);
  }
  return tc_facewise(Ah, Bh, Ch, n1, n4, n2, p, tA, tB, prec, ws, ws_bytes, st);
}

static size_t facewise_bytes(int64_t M, int64_t N, int64_t K, int64_t p, int prec) {
  return prec == WP_PREC_FP32 ? 0 : tc_facewise_workspace(M, N, K, p, prec);
}

static void gwprod_layout(int64_t n1, int64_t n2, int64_t n4, int64_t p, int prec, Sizer& s) {
  s.take<float>(size_t(p) * n1 * n2);
  s.take<float>(size_t(p) * n2 * n4);
  s.take<float>(size_t(p) * n1 * n4);
  s.take<char>(facewise_bytes(n1, n4, n2, p, prec));
}

extern "C" int wp_gwprod_workspace(int64_t n1, int64_t n2, int64_t n4, int64_t p, int L, int prec, size_t* bytes) {
  if (!bytes) return WP_ERR_NULL;
  if (n1 < 1 || n2 < 1 || n4 < 1 || p < 1) return WP_ERR_SHAPE;
  WP_TRY(check_levels(p, L));
  if (prec < WP_PREC_FP32 || prec > WP_PREC_FP8) return WP_ERR_PREC;
  Sizer s;
  gwprod_layout(n1, n2, n4, p, prec, s);
  *bytes = s.bytes();
  return WP_OK;
}

extern "C" int wp_gwprod(const float* A, const float* B, float* C, int64_t n1, int64_t n2, int64_t n4, int64_t p,
                         int L, const wp_lift_ops* ops, int prec, void* ws, size_t ws_bytes, void* stream) {
  if (n1 < 1 || n2 < 1 || n4 < 1 || p < 1) return WP_ERR_SHAPE;
  if (!A || !B || !C) return WP_ERR_NULL;
  if (prec < WP_PREC_FP32 || prec > WP_PREC_FP8) return WP_ERR_PREC;
  GLevels lv;
  WP_TRY(check_glift(p, L, ops, &lv));
  if (!aligned16(A) || !aligned16(B) || !aligned16(C)) return WP_ERR_ALIGN;
  const size_t ca = size_t(p) * n1 * n2 * 4, cb = size_t(p) * n2 * n4 * 4, cc = size_t(p) * n1 * n4 * 4;
  if (overlaps(C, cc, A, ca) || overlaps(C, cc, B, cb)) return WP_ERR_ALIAS;
  Sizer need;
  gwprod_layout(n1, n2, n4, p, prec, need);
  if (!ws || ws_bytes < need.bytes()) return WP_ERR_WORKSPACE;
  Carver cv(ws, ws_bytes);
  float* Ah = cv.take<float>(size_t(p) * n1 * n2);
  float* Bh = cv.take<float>(size_t(p) * n2 * n4);
  float* Ch = cv.take<float>(size_t(p) * n1 * n4);
  const size_t fb = facewise_bytes(n1, n4, n2, p, prec);
  void* fw = fb ? cv.take<char>(fb) : nullptr;
  if (!cv.ok) return WP_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  WP_TRY(glift_dispatch(0, A, Ah, n1 * n2, p, L, lv, st));
  WP_TRY(glift_dispatch(0, B, Bh, n2 * n4, p, L, lv, st));
  WP_TRY(facewise_any(Ah, Bh, Ch, n1, n2, n4, p, false, false, prec, fw, fb, st));
  return glift_dispatch(1, Ch, C, n1 * n4, p, L, lv, st);
}

static void gbackward_layout(int64_t n1, int64_t n2, int64_t n4, int64_t p, int prec, Sizer& s) {
  s.take<float>(size_t(p) * n1 * n2);
  s.take<float>(size_t(p) * n2 * n4);
  s.take<float>(size_t(p) * n1 * n4);
  s.take<float>(size_t(p) * std::max(n1 * n2, n2 * n4));
  s.take<char>(std::max(facewise_bytes(n1, n2, n4, p, prec), facewise_bytes(n2, n4, n1, p, prec)));
}

extern "C" int wp_gwprod_backward_workspace(int64_t n1, int64_t n2, int64_t n4, int64_t p, int L, int prec,
                                            size_t* bytes) {
  if (!bytes) return WP_ERR_NULL;
  if (n1 < 1 || n2 < 1 || n4 < 1 || p < 1) return WP_ERR_SHAPE;
  WP_TRY(check_levels(p, L));
  if (prec < WP_PREC_FP32 || prec > WP_PREC_FP8) return WP_ERR_PREC;
  Sizer s;
  gbackward_layout(n1, n2, n4, p, prec, s);
  *bytes = s.bytes();
  return WP_OK;
}

extern "C" int wp_gwprod_backward(const float* A, const float* B, const float* G, float* dA, float* dB, int64_t n1,
                                  int64_t n2, int64_t n4, int64_t p, int L, const wp_lift_ops* ops, int prec, void* ws,
                                  size_t ws_bytes, void* stream) {
  if (n1 < 1 || n2 < 1 || n4 < 1 || p < 1) return WP_ERR_SHAPE;
  if (!A || !B || !G) return WP_ERR_NULL;
  if (prec < WP_PREC_FP32 || prec > WP_PREC_FP8) return WP_ERR_PREC;
  GLevels lv;
  WP_TRY(check_glift(p, L, ops, &lv));
  if (!aligned16(A) || !aligned16(B) || !aligned16(G)) return WP_ERR_ALIGN;
  if ((dA && !aligned16(dA)) || (dB && !aligned16(dB))) return WP_ERR_ALIGN;
  const size_t ca = size_t(p) * n1 * n2 * 4, cb = size_t(p) * n2 * n4 * 4, cg = size_t(p) * n1 * n4 * 4;
  for (const float* o : {static_cast<const float*>(dA), static_cast<const float*>(dB)}) {
    if (!o) continue;
    const size_t co = (o == dA) ? ca : cb;
    if (overlaps(o, co, A, ca) || overlaps(o, co, B, cb) || overlaps(o, co, G, cg)) return WP_ERR_ALIAS;
  }
  if (dA && dB && overlaps(dA, ca, dB, cb)) return WP_ERR_ALIAS;
  Sizer need;
  gbackward_layout(n1, n2, n4, p, prec, need);
  if (!ws || ws_bytes < need.bytes()) return WP_ERR_WORKSPACE;
  Carver cv(ws, ws_bytes);
  float* Ah = cv.take<float>(size_t(p) * n1 * n2);
  float* Bh = cv.take<float>(size_t(p) * n2 * n4);
  float* Gh = cv.take<float>(size_t(p) * n1 * n4);
  float* dXh = cv.take<float>(size_t(p) * std::max(n1 * n2, n2 * n4));
  const size_t fb = std::max(facewise_bytes(n1, n2, n4, p, prec), facewise_bytes(n2, n4, n1, p, prec));
  void* fw = fb ? cv.take<char>(fb) : nullptr;
  if (!cv.ok) return WP_ERR_WORKSPACE;
  cudaStream_t st = as_stream(stream);
  // adjoint route: G_hat = W^{-T} G, dA = W^T (G_hat Delta B_hat^T), dB = W^T (A_hat^T Delta G_hat)
  WP_TRY(glift_dispatch(3, G, Gh, n1 * n4, p, L, lv, st));
  if (dA) {
    WP_TRY(glift_dispatch(0, B, Bh, n2 * n4, p, L, lv, st));
    WP_TRY(facewise_any(Gh, Bh, dXh, n1, n4, n2, p, false, true, prec, fw, fb, st));
    WP_TRY(glift_dispatch(2, dXh, dA, n1 * n2, p, L, lv, st));
  }
  if (dB) {
    WP_TRY(glift_dispatch(0, A, Ah, n1 * n2, p, L, lv, st));
    WP_TRY(facewise_any(Ah, Gh, dXh, n2, n1, n4, p, true, false, prec, fw, fb, st));
    WP_TRY(glift_dispatch(2, dXh, dB, n2 * n4, p, L, lv, st));
  }
  return WP_OK;
}
