// Lifting transforms along mode 3 (Sec. II-A, Eq. 1-3, Algorithm 1): forward,
// inverse and the two adjoints, all L levels fused into one pass over HBM.
//
// Data layout: slice-major (p, n1, n2) float32; the n1*n2 "plane" of a slice is
// contiguous, so the mode-3 tube of element e is {x[k*plane + e]}.  A thread
// owns VEC adjacent plane elements (one 128-bit access when VEC = 4) of one
// tube group of G = 2^L slices: it issues G coalesced loads, lifts in
// registers, and issues G coalesced stores to the Mallat positions.  Every
// element is read once and written once -- the algorithmic minimum of
// 2 * 4 * p * n1 * n2 bytes per call.
//
// For L > 5 the group no longer fits in registers; a shared-memory variant
// stages a (G x E)-element tile and lifts level by level.
//
// Wavelet-side slice order.  The exported transforms use the Mallat order of
// Eq. (1).  Buffers that stay inside one library call (the w-product's
// W(A), W(B), C_hat and the backward's cotangents) may instead use the
// group-interleaved order, local index t of group g at slice g * 2^L + t:
// a pass over it reads and writes G consecutive slices per group.  Reading
// the Mallat positions of a group (slices g, m + g, 2m + 2g, ...) streams at
// about half the copy rate on GB300 at L = 4 (measured: 3.5 vs 6.6 TB/s for
// the same bytes), so the internal round trips avoid it.

#include <algorithm>

#include "common.cuh"
#include "internal.cuh"
#include "lift_math.cuh"

namespace wp {

enum LiftOp { OP_FWD = LIFT_FWD, OP_INV = LIFT_INV, OP_ADJ = LIFT_ADJ, OP_IADJ = LIFT_IADJ };

static const char* const kLiftNames[4] = {"lift_forward", "lift_inverse", "lift_adjoint",
                                          "lift_inverse_adjoint"};

// Ops that read spatial groups and write Mallat positions.
__host__ __device__ constexpr bool reads_spatial(int op) { return op == OP_FWD || op == OP_IADJ; }

template <int L, int OP>
__device__ __forceinline__ void group_op(const float* in, float* out) {
  if constexpr (OP == OP_FWD) lift_group<L>(in, out);
  else if constexpr (OP == OP_INV) ilift_group<L>(in, out);
  else if constexpr (OP == OP_ADJ) lift_adjoint_group<L>(in, out);
  else ilift_adjoint_group<L>(in, out);
}

template <int VEC> struct VecT;
template <> struct VecT<1> { using T = float; };
template <> struct VecT<2> { using T = float2; };
template <> struct VecT<4> { using T = float4; };

template <int VEC>
__device__ __forceinline__ void load_vec(const float* p, float* v) {
  if constexpr (VEC == 4) {
    float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else if constexpr (VEC == 2) {
    float2 t = __ldg(reinterpret_cast<const float2*>(p));
    v[0] = t.x; v[1] = t.y;
  } else {
    v[0] = __ldg(p);
  }
}

template <int VEC>
__device__ __forceinline__ void store_vec(float* p, const float* v) {
  if constexpr (VEC == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (VEC == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else {
    *p = v[0];
  }
}

// Register kernel: grid-stride over items = (group g, vector index e).
// Launched with programmatic serialisation: it may start while the previous
// kernel of the stream finishes and waits for that kernel's completion before
// reading; it lets its own successor start early the same way.
//
// GF (group-fastest): CTA-sized chunks are ordered with the tube group
// fastest, so the CTAs in flight cover every group at nearby plane offsets
// instead of every offset of two or three groups.  Used for the ops that
// gather a group from its Mallat positions at L >= 4, where it streams
// faster (measured at 256 slices of 1024 x 512: 4.4 against 3.5 TB/s at
// L = 4, 2.8 against 2.2 TB/s at L = 5).
// S2: the coarse pass of a split inverse / adjoint (see launch_split): local
// index t of group g is written to output slice 4 (g G + t) + 3 instead of
// g G + t.
template <int L, int VEC, int OP, bool IL, bool GF, bool S2 = false>
__global__ void __launch_bounds__(256) lift_reg_kernel(const float* __restrict__ in,
                                                       float* __restrict__ out, int64_t plane,
                                                       int64_t p, int64_t nvec, int64_t total) {
  constexpr int G = 1 << L;
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int64_t m = p >> L;
  const int64_t nchunk = (nvec + blockDim.x - 1) / blockDim.x;
  const int64_t nwork = GF ? m * nchunk : total;
  const int64_t first = GF ? int64_t(blockIdx.x) : int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int64_t stride = GF ? int64_t(gridDim.x) : int64_t(gridDim.x) * blockDim.x;
  for (int64_t w = first; w < nwork; w += stride) {
    int64_t g, iv;
    if constexpr (GF) {
      g = w % m;
      iv = (w / m) * blockDim.x + threadIdx.x;
      if (iv >= nvec) continue;
    } else {
      g = w / nvec;
      iv = w - g * nvec;
    }
    const int64_t e = iv * VEC;
    float v[G][VEC];
#pragma unroll
    for (int t = 0; t < G; ++t) {
      const int64_t slice = (reads_spatial(OP) || IL) ? g * G + t : mallat_slice<L>(t, g, p);
      load_vec<VEC>(in + slice * plane + e, v[t]);
    }
    float w2[G][VEC];
#pragma unroll
    for (int c = 0; c < VEC; ++c) {
      float x[G], y[G];
#pragma unroll
      for (int t = 0; t < G; ++t) x[t] = v[t][c];
      group_op<L, OP>(x, y);
#pragma unroll
      for (int t = 0; t < G; ++t) w2[t][c] = y[t];
    }
#pragma unroll
    for (int t = 0; t < G; ++t) {
      int64_t slice = (reads_spatial(OP) && !IL) ? mallat_slice<L>(t, g, p) : g * G + t;
      if constexpr (S2) slice = 4 * slice + 3;
      store_vec<VEC>(out + slice * plane + e, w2[t]);
    }
  }
}

// Fine pass of a split inverse / adjoint: the last two levels (L = 2 groups
// of four slices k) with the smooth coefficient s_2[k] taken from slice
// 4k + 3 of x, where the coarse pass left it; d_2 and d_1 from their Mallat
// positions in y (p/4 + k, p/2 + 2k, p/2 + 2k + 1).  Every thread reads its
// element of slice 4k + 3 before it writes slices 4k .. 4k + 3 of the same
// element, so reusing x needs no synchronisation (x is not __restrict__).
template <int VEC, int OP>
__global__ void __launch_bounds__(256) lift_tail_kernel(const float* __restrict__ y, float* x, int64_t plane,
                                                        int64_t p, int64_t nvec, int64_t total) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  for (int64_t w = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; w < total; w += int64_t(gridDim.x) * blockDim.x) {
    const int64_t k = w / nvec;
    const int64_t e = (w - k * nvec) * VEC;
    float v[4][VEC];
    {
      const float* src = x + (4 * k + 3) * plane + e;   // written by the coarse pass: read through L2
      if constexpr (VEC == 4) {
        const float4 q = __ldcg(reinterpret_cast<const float4*>(src));
        v[0][0] = q.x; v[0][1] = q.y; v[0][2] = q.z; v[0][3] = q.w;
      } else if constexpr (VEC == 2) {
        const float2 q = __ldcg(reinterpret_cast<const float2*>(src));
        v[0][0] = q.x; v[0][1] = q.y;
      } else {
        v[0][0] = __ldcg(src);
      }
    }
    load_vec<VEC>(y + ((p >> 2) + k) * plane + e, v[1]);
    load_vec<VEC>(y + ((p >> 1) + 2 * k) * plane + e, v[2]);
    load_vec<VEC>(y + ((p >> 1) + 2 * k + 1) * plane + e, v[3]);
    float o[4][VEC];
#pragma unroll
    for (int c = 0; c < VEC; ++c) {
      float a[4], b[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) a[t] = v[t][c];
      group_op<2, OP>(a, b);
#pragma unroll
      for (int t = 0; t < 4; ++t) o[t][c] = b[t];
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) store_vec<VEC>(x + (4 * k + t) * plane + e, o[t]);
  }
}

// Shared-memory kernel for large groups (L > 5): one CTA per (group, E-element
// chunk).  Three G x E buffers: X keeps the gathered group, S0 / S1 ping-pong
// the smooth part level by level, so no level ever reads what it writes; one
// barrier per level.
__device__ __forceinline__ int64_t mallat_slice_rt(int t, int64_t g, int64_t p, int L) {
  if (t == 0) return g;
  const int hb = 31 - __clz(t);
  return (p >> (L - hb)) + g * (int64_t(1) << hb) + (t - (1 << hb));
}

template <int OP, int E>
__global__ void __launch_bounds__(256) lift_smem_kernel(const float* __restrict__ in,
                                                        float* __restrict__ out, int64_t plane,
                                                        int64_t p, int L, int64_t nchunk) {
  extern __shared__ float smem[];
  const int G = 1 << L;
  float* X = smem;                 // [G][E] gathered input, local order
  float* S[2] = {smem + G * E, smem + 2 * G * E};
  const int64_t g = blockIdx.y;
  for (int64_t chunk = blockIdx.x; chunk < nchunk; chunk += gridDim.x) {
    const int64_t e0 = chunk * E;
    const int width = (plane - e0 < E) ? int(plane - e0) : E;
    for (int idx = threadIdx.x; idx < G * E; idx += blockDim.x) {
      const int t = idx / E, c = idx % E;
      const int64_t slice = reads_spatial(OP) ? g * G + t : mallat_slice_rt(t, g, p, L);
      X[idx] = (c < width) ? in[slice * plane + e0 + c] : 0.f;
    }
    __syncthreads();
    if (reads_spatial(OP)) {
      // finest level first; level j turns cur = G >> (j-1) smooth rows into
      // half = cur / 2 smooth rows (next buffer) and half detail rows (global)
      const float* src = X;
      for (int j = 1; j <= L; ++j) {
        const int half = G >> j;
        float* dst = S[j & 1];
        for (int idx = threadIdx.x; idx < half * E; idx += blockDim.x) {
          const int k = idx / E, c = idx % E;
          const float a = src[(2 * k) * E + c], b = src[(2 * k + 1) * E + c];
          float sv, dv;
          if (OP == OP_FWD) { dv = a - b; sv = fmaf(0.5f, dv, b); }
          else { dv = 0.5f * (a - b); sv = a + b; }
          dst[k * E + c] = sv;
          if (c < width) out[((p >> j) + g * half + k) * plane + e0 + c] = dv;
        }
        __syncthreads();
        src = dst;
      }
      if (threadIdx.x < width) out[g * plane + e0 + threadIdx.x] = src[threadIdx.x];
    } else {
      // coarsest level first; level j expands s_j (src rows [0, half)) with
      // d_j (X rows [half, 2 half)) into 2 half smooth rows of the next buffer
      const float* src = X;
      for (int j = L; j >= 1; --j) {
        const int half = G >> j;
        float* dst = S[j & 1];
        for (int idx = threadIdx.x; idx < half * E; idx += blockDim.x) {
          const int k = idx / E, c = idx % E;
          const float s = src[k * E + c], d = X[(half + k) * E + c];
          float av, bv;
          if (OP == OP_INV) { bv = fmaf(-0.5f, d, s); av = d + bv; }
          else { av = fmaf(0.5f, s, d); bv = fmaf(0.5f, s, -d); }
          dst[(2 * k) * E + c] = av;
          dst[(2 * k + 1) * E + c] = bv;
        }
        __syncthreads();
        src = dst;
      }
      for (int idx = threadIdx.x; idx < G * E; idx += blockDim.x) {
        const int t = idx / E, c = idx % E;
        if (c < width) out[(g * G + t) * plane + e0 + c] = src[idx];
      }
    }
    __syncthreads();
  }
}

template <int L, int VEC, int OP, bool IL, bool S2 = false>
static int launch_reg(const float* in, float* out, int64_t plane, int64_t p, cudaStream_t st) {
  const int64_t nvec = plane / VEC;
  const int64_t total = (p >> L) * nvec;
  const int threads = 256;
  int64_t blocks = (total + threads - 1) / threads;
  const int64_t cap = int64_t(sm_count()) * 8;   // 2048 resident threads per SM
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(blocks), 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // group-fastest chunk order for the Mallat-position gathers at L >= 4
  constexpr bool GF = !IL && !reads_spatial(OP) && L >= 4;
  WP_PROFILE(kLiftNames[OP], st);
  WP_CUDA_TRY(cudaLaunchKernelEx(&cfg, lift_reg_kernel<L, VEC, OP, IL, GF, S2>, in, out, plane, p, nvec, total));
  return launch_status();
}

// Mallat-input inverse / adjoint at L = 4, 5, split by levels.  Gathering a
// group from its L + 1 Mallat runs reads far below the copy rate at L >= 4
// (measured 4.4 / 2.8 TB/s at L = 4 / 5 against 5.5 at L = 3, 256 slices of
// 1024 x 512), so the transform runs as two passes with short gathers:
//   coarse  levels L .. 3 on the first p/4 slices of y -- the Mallat-ordered
//           (L-2)-level transform of s_2 -- writing s_2[k] to slice 4k + 3 of x;
//   fine    levels 2 and 1 (lift_tail_kernel), s_2 from x, d_2, d_1 from y.
// x (the output, distinct from y) doubles as the scratch space; the extra
// traffic is p/4 slices written and read once (2.5 p slices moved against 2 p).
template <int L, int VEC, int OP>
static int launch_split(const float* y, float* x, int64_t plane, int64_t p, cudaStream_t st) {
  static_assert(L == 4 || L == 5, "split passes for L = 4, 5");
  WP_TRY((launch_reg<L - 2, VEC, OP, false, true>(y, x, plane, p >> 2, st)));
  const int64_t nvec = plane / VEC;
  const int64_t total = (p >> 2) * nvec;
  int64_t blocks = std::min<int64_t>((total + 255) / 256, int64_t(sm_count()) * 8);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(std::max<int64_t>(blocks, 1)), 1, 1);
  cfg.blockDim = dim3(256, 1, 1);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  WP_PROFILE(kLiftNames[OP], st);
  WP_CUDA_TRY(cudaLaunchKernelEx(&cfg, lift_tail_kernel<VEC, OP>, y, x, plane, p, nvec, total));
  return launch_status();
}

template <int OP, int E>
static int launch_smem_e(const float* in, float* out, int64_t plane, int64_t p, int L,
                         cudaStream_t st) {
  const int G = 1 << L;
  const size_t smem = size_t(3) * G * E * sizeof(float);
  static bool attr_set = false;
  if (!attr_set) {
    WP_CUDA_TRY(cudaFuncSetAttribute(lift_smem_kernel<OP, E>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  const int64_t nchunk = (plane + E - 1) / E;
  const int64_t groups = p >> L;
  if (groups > 65535) return WP_ERR_SHAPE;
  int64_t bx = nchunk;
  const int64_t cap = std::max<int64_t>(1, int64_t(sm_count()) * 4 / std::max<int64_t>(1, groups));
  if (bx > cap) bx = cap;
  const dim3 grid{unsigned(bx), unsigned(groups), 1u};
  WP_PROFILE(kLiftNames[OP], st);
  lift_smem_kernel<OP, E><<<grid, 256, smem, st>>>(in, out, plane, p, L, nchunk);
  return launch_status();
}

template <int OP>
static int launch_smem(const float* in, float* out, int64_t plane, int64_t p, int L,
                       cudaStream_t st) {
  // 3 * G * E floats of shared memory: E = 32 up to G = 512 (192 KB), E = 16 beyond
  return (L <= 9) ? launch_smem_e<OP, 32>(in, out, plane, p, L, st)
                  : launch_smem_e<OP, 16>(in, out, plane, p, L, st);
}

template <int OP, bool IL>
static int dispatch(const float* in, float* out, int64_t plane, int64_t p, int L, cudaStream_t st) {
  const bool v4 = (plane % 4 == 0) && aligned16(in) && aligned16(out);
  const bool v2 = (plane % 2 == 0);
  // Mallat-input ops at L = 4, 5 with a separate output: two passes (launch_split)
  if constexpr (!IL && !reads_spatial(OP)) {
    if ((L == 4 || L == 5) && in != out) {
      if (L == 4) return v4 ? launch_split<4, 4, OP>(in, out, plane, p, st) : launch_split<4, 1, OP>(in, out, plane, p, st);
      return v4 ? launch_split<5, 4, OP>(in, out, plane, p, st) : launch_split<5, 1, OP>(in, out, plane, p, st);
    }
  }
  switch (L) {
    case 0: return v4 ? launch_reg<0, 4, OP, IL>(in, out, plane, p, st) : launch_reg<0, 1, OP, IL>(in, out, plane, p, st);
    case 1: return v4 ? launch_reg<1, 4, OP, IL>(in, out, plane, p, st) : launch_reg<1, 1, OP, IL>(in, out, plane, p, st);
    case 2: return v4 ? launch_reg<2, 4, OP, IL>(in, out, plane, p, st) : launch_reg<2, 1, OP, IL>(in, out, plane, p, st);
    case 3: return v4 ? launch_reg<3, 4, OP, IL>(in, out, plane, p, st) : launch_reg<3, 1, OP, IL>(in, out, plane, p, st);
    case 4: return v4 ? launch_reg<4, 4, OP, IL>(in, out, plane, p, st) : launch_reg<4, 1, OP, IL>(in, out, plane, p, st);
    case 5: return v2 ? launch_reg<5, 2, OP, IL>(in, out, plane, p, st) : launch_reg<5, 1, OP, IL>(in, out, plane, p, st);
    default:
      if (IL) return WP_ERR_UNSUPPORTED;
      return launch_smem<OP>(in, out, plane, p, L, st);
  }
}

template <bool IL>
static int dispatch_op(int op, const float* in, float* out, int64_t plane, int64_t p, int L, cudaStream_t st) {
  switch (op) {
    case OP_FWD: return dispatch<OP_FWD, IL>(in, out, plane, p, L, st);
    case OP_INV: return dispatch<OP_INV, IL>(in, out, plane, p, L, st);
    case OP_ADJ: return dispatch<OP_ADJ, IL>(in, out, plane, p, L, st);
    default: return dispatch<OP_IADJ, IL>(in, out, plane, p, L, st);
  }
}

int lift_dispatch(int op, const float* in, float* out, int64_t plane, int64_t p, int L, cudaStream_t st,
                  bool interleaved) {
  return interleaved ? dispatch_op<true>(op, in, out, plane, p, L, st)
                     : dispatch_op<false>(op, in, out, plane, p, L, st);
}

static int lift_entry(int op, const float* in, float* out, int64_t n1, int64_t n2, int64_t p,
                      int L, void* stream) {
  if (n1 < 1 || n2 < 1 || p < 1) return WP_ERR_SHAPE;
  if (!in || !out) return WP_ERR_NULL;
  WP_TRY(check_levels(p, L));
  if (!aligned16(in) || !aligned16(out)) return WP_ERR_ALIGN;
  const size_t bytes = size_t(n1) * size_t(n2) * size_t(p) * sizeof(float);
  if (overlaps(in, bytes, out, bytes)) return WP_ERR_ALIAS;
  return lift_dispatch(op, in, out, n1 * n2, p, L, as_stream(stream));
}

}  // namespace wp

extern "C" int wp_lift_forward(const float* x, float* y, int64_t n1, int64_t n2, int64_t p,
                               int L, void* stream) {
  return wp::lift_entry(wp::OP_FWD, x, y, n1, n2, p, L, stream);
}

extern "C" int wp_lift_inverse(const float* y, float* x, int64_t n1, int64_t n2, int64_t p,
                               int L, void* stream) {
  return wp::lift_entry(wp::OP_INV, y, x, n1, n2, p, L, stream);
}

extern "C" int wp_lift_adjoint(const float* g, float* h, int64_t n1, int64_t n2, int64_t p,
                               int L, int of_inverse, void* stream) {
  return wp::lift_entry(of_inverse ? wp::OP_IADJ : wp::OP_ADJ, g, h, n1, n2, p, L, stream);
}
