// Tensor-core face-products on tcgen05 (Def. 2.1, Algorithm 1 middle loop):
// C[b] = op(A[b]) op(B[b]) for every wavelet-domain frontal slice b, with BF16
// operands and FP32 accumulation in tensor memory.
//
// Precision modes
//   BF16    one product of the BF16-rounded operands.
//   BF16X3  split precision: every FP32 operand is written as hi + lo with
//           hi = bf16(x), lo = bf16(x - hi), so hi + lo carries ~16 bits of
//           the mantissa; the kernel accumulates hi*hi + hi*lo + lo*hi (the
//           dropped lo*lo term is ~2^-18 relative) into one FP32 accumulator.
//   FP8     E4M3 operands with one scale per wavelet-domain slice and operand:
//           s = amax(|X_k|) / 448 (448 = largest finite E4M3), q = e4m3(x / s);
//           kind::f8f6f4 MMAs accumulate q_a q_b in FP32 and the epilogue
//           multiplies by s_a[k] s_b[k].  The scales are taken on the
//           wavelet-domain slices, after the lifting has mixed the 2^L
//           spatial slices of a group.
//
// Kernels
//   tc_gemm_kernel        persistent: one CTA per SM walks every (slice, row
//                         tile, column tile) tile of 128 x BN; warp 0 lane 0
//                         issues TMA loads of the 128-byte-swizzled BF16 / E4M3
//                         tiles into a STAGES-deep ring, warp 1 owns TMEM and
//                         one lane issues tcgen05.mma (M = 128, N = BN), warps
//                         2-5 drain one of two TMEM accumulators (tcgen05.ld)
//                         and store C through swizzled shared-memory staging and
//                         TMA bulk stores while the next tile is multiplied.
//   tc_gemm_ilift_kernel  one CTA per 128 x (512 / 2^L) tile of all 2^L slices
//                         of a tube group, 2^L TMEM accumulators, inverse lift
//                         (Eq. 3) across them in the epilogue: the fused
//                         w-product for small slices.
//   tc_wprod_lift_kernel  the same tile with the forward lift (Eq. 2) and the
//                         BF16 split done by its own converter warps on the
//                         spatial FP32 operands (L <= 3): the w-product in one
//                         launch, nothing but A, B and C in HBM.
// Operands are prepared by `split` kernels that round the FP32 wavelet-domain
// slices to BF16 hi (/ lo) and, where the stored layout is not K-major,
// transpose through shared memory, or by lift-and-split kernels that also
// apply the forward transform.  Every mbarrier wait is bounded.

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "internal.cuh"
#include "lift_math.cuh"
#include "tc_ptx.cuh"

#include <cooperative_groups.h>
namespace cg = cooperative_groups;

namespace wp {

// ---- operand preparation ---------------------------------------------------------

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// in (batch, R, C) fp32 -> hi/lo (batch, R, Cp) bf16, columns [C, Cp) zero.
__global__ void __launch_bounds__(256) split_rows_kernel(const float* __restrict__ in,
                                                         __nv_bfloat16* __restrict__ hi,
                                                         __nv_bfloat16* __restrict__ lo, int64_t rows,
                                                         int C, int Cp) {
  const int64_t total = rows * Cp;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = i / Cp;
    const int c = int(i - r * Cp);
    const float x = (c < C) ? __ldg(in + r * C + c) : 0.f;
    __nv_bfloat16 h, l;
    split_bf16(x, h, l);
    hi[i] = h;
    if (lo) lo[i] = l;
  }
}

// in (batch, R, C) fp32 -> hi/lo (batch, C, Rp) bf16 (transposed), rows of
// the output padded with zeros to Rp.  32 x 32 tiles through shared memory.
__global__ void __launch_bounds__(256) split_transpose_kernel(const float* __restrict__ in,
                                                              __nv_bfloat16* __restrict__ hi,
                                                              __nv_bfloat16* __restrict__ lo, int R, int C,
                                                              int Rp, int batch) {
  __shared__ float tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int b = blockIdx.z; b < batch; b += gridDim.z) {
    const float* src = in + int64_t(b) * R * C;
    for (int i = threadIdx.y; i < 32; i += 8) {
      const int r = r0 + i, c = c0 + threadIdx.x;
      tile[i][threadIdx.x] = (r < R && c < C) ? __ldg(src + int64_t(r) * C + c) : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
      const int c = c0 + i, r = r0 + threadIdx.x;
      if (c < C && r < Rp) {
        __nv_bfloat16 h, l;
        split_bf16(tile[threadIdx.x][i], h, l);
        const int64_t o = (int64_t(b) * C + c) * Rp + r;
        hi[o] = h;
        if (lo) lo[o] = l;
      }
    }
    __syncthreads();
  }
}

// The same for C % 4 == 0 and a 16-byte aligned input: 64 x 64 tiles, four
// 16-byte loads per thread in flight, and every thread stores 8 consecutive
// K-elements of one output row as one 16-byte vector per BF16 copy (the 32
// lanes of a warp on 32 output rows: conflict-free shared-memory reads).
// Rp must be a multiple of 8.
__global__ void __launch_bounds__(256) split_transpose4_kernel(const float* __restrict__ in,
                                                               __nv_bfloat16* __restrict__ hi,
                                                               __nv_bfloat16* __restrict__ lo, int R, int C,
                                                               int Rp) {
  constexpr int T = 64, LD = T + 1;
  __shared__ float tile[T * LD];
  const int c0 = blockIdx.x * T, r0 = blockIdx.y * T;
  const int64_t b = blockIdx.z;
  const float* src = in + b * R * int64_t(C);
  const int tid = threadIdx.x;
  float4 v[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = (tid >> 4) + 16 * k, j = (tid & 15) * 4;
    const int r = r0 + i, c = c0 + j;
    v[k] = (r < R && c < C) ? __ldg(reinterpret_cast<const float4*>(src + int64_t(r) * C + c))
                            : make_float4(0.f, 0.f, 0.f, 0.f);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    float* d = tile + ((tid >> 4) + 16 * k) * LD + (tid & 15) * 4;
    d[0] = v[k].x; d[1] = v[k].y; d[2] = v[k].z; d[3] = v[k].w;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int w = tid + 256 * k;
    const int cc = w & 63, chunk = w >> 6;
    const int c = c0 + cc, rs = r0 + chunk * 8;
    if (c < C && rs < Rp) {
      __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) split_bf16(tile[(chunk * 8 + q) * LD + cc], h[q], l[q]);
      const int64_t o = (b * C + c) * int64_t(Rp) + rs;
      *reinterpret_cast<uint4*>(hi + o) = *reinterpret_cast<const uint4*>(h);
      if (lo) *reinterpret_cast<uint4*>(lo + o) = *reinterpret_cast<const uint4*>(l);
    }
  }
}

// ---- FP8 operand preparation ------------------------------------------------------------

// amax_bits[b] = max |X[b]| (as the bit pattern of a non-negative float, so
// integer atomicMax orders it); one CTA row of the grid per slice.
__global__ void __launch_bounds__(256) amax_slices_kernel(const float* __restrict__ X, int64_t per_slice,
                                                          unsigned* __restrict__ amax_bits) {
  const int64_t b = blockIdx.y;
  const float* x = X + b * per_slice;
  float m = 0.f;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < per_slice; i += int64_t(gridDim.x) * blockDim.x)
    m = fmaxf(m, fabsf(__ldg(x + i)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax_bits + b, __float_as_uint(m));
}

__device__ __forceinline__ float fp8_scale(unsigned amax_bits) {
  const float a = __uint_as_float(amax_bits);
  return a > 0.f ? a / 448.f : 1.f;
}

__device__ __forceinline__ uint8_t to_e4m3(float x) {
  return static_cast<uint8_t>(__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3));
}

// Four E4M3 codes packed little-endian (a in the lowest byte), converted in pairs.
__device__ __forceinline__ uint32_t to_e4m3x4(float a, float b, float c, float d) {
  const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
  const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
  return (lo & 0xffffu) | (hi << 16);
}

// inv[i] = 1 / s_i for the per-slice scales s_i = amax_i / 448 (1 for amax_i = 0).
__global__ void __launch_bounds__(256) fp8_inv_scales_kernel(const unsigned* __restrict__ amax_bits,
                                                             float* __restrict__ inv, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) inv[i] = 1.f / fp8_scale(amax_bits[i]);
}

// in (batch, R, C) fp32 -> q (batch, R, Cp) e4m3 with the slice's scale.
__global__ void __launch_bounds__(256) quant_rows_kernel(const float* __restrict__ in, uint8_t* __restrict__ q,
                                                         const unsigned* __restrict__ amax_bits, int64_t rows_per_slice,
                                                         int64_t total_rows, int C, int Cp) {
  const int64_t total = total_rows * Cp;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = i / Cp;
    const int c = int(i - r * Cp);
    const float inv = 1.f / fp8_scale(amax_bits[r / rows_per_slice]);
    q[i] = (c < C) ? to_e4m3(__ldg(in + r * C + c) * inv) : uint8_t(0);
  }
}

// in (batch, R, C) fp32 -> q (batch, C, Rp) e4m3 (transposed) with the slice's scale.
__global__ void __launch_bounds__(256) quant_transpose_kernel(const float* __restrict__ in, uint8_t* __restrict__ q,
                                                              const unsigned* __restrict__ amax_bits, int R, int C,
                                                              int Rp, int batch) {
  __shared__ float tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int b = blockIdx.z; b < batch; b += gridDim.z) {
    const float* src = in + int64_t(b) * R * C;
    const float inv = 1.f / fp8_scale(amax_bits[b]);
    for (int i = threadIdx.y; i < 32; i += 8) {
      const int r = r0 + i, c = c0 + threadIdx.x;
      tile[i][threadIdx.x] = (r < R && c < C) ? __ldg(src + int64_t(r) * C + c) : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
      const int c = c0 + i, r = r0 + threadIdx.x;
      if (c < C && r < Rp) q[(int64_t(b) * C + c) * Rp + r] = to_e4m3(tile[threadIdx.x][i] * inv);
    }
    __syncthreads();
  }
}

// ---- the GEMM kernel ---------------------------------------------------------------

namespace tc {

constexpr int BM = 128;
constexpr int BK = 64;          // BF16 elements per 128-byte swizzle row
constexpr int THREADS = 192;

// Persistent tcgen05 GEMM C[b] = op(A[b]) op(B[b]) over all (batch, row tile,
// column tile) tiles of 128 x BN: one CTA per SM walks the tiles with stride
// gridDim.x; the shared-memory stage ring runs on across tiles; two TMEM
// accumulators (2 BN columns) let the epilogue of one tile overlap the MMAs
// of the next.  Roles: warp 0 lane 0 issues TMA loads, warp 1 lane 0 issues
// the MMAs, warps 2..5 drain the accumulators (tcgen05.ld) and write C --
// as 32 x 32 chunks staged in shared memory with the 128-byte swizzle and
// stored by TMA (double-buffered per warp) when N % 4 == 0, else directly.
template <int BN, int NPROD, int STAGES>
struct Layout {
  static constexpr int NCOPY = (NPROD == 3) ? 2 : 1;   // BF16x3 keeps hi and lo copies
  static constexpr int A_TILE = BM * 128;               // 128-byte K rows (64 BF16 or 128 FP8)
  static constexpr int B_TILE = BN * 128;
  static constexpr int STAGE = NCOPY * (A_TILE + B_TILE);
  static constexpr int STG_OFF = STAGES * STAGE;         // epilogue staging: 4 warps x 2 x 4 KB
  static constexpr int BAR_OFF = STG_OFF + 4 * 2 * 4096;
  static constexpr int SMEM = BAR_OFF + (2 * STAGES + 5) * 8 + 16 + 1024;   // + alignment slack
  static constexpr uint32_t TMEM_COLS = (2 * BN) < 32 ? 32 : 2 * BN;
};

// NPROD: 1 = BF16, 3 = BF16x3, 8 = FP8 E4M3 (then sa_bits / sb_bits hold the
// per-slice amax of each operand and the epilogue applies s_a s_b).  BMN: B
// is MN-major (N contiguous, 64-column boxes; BF16 only).
template <int BN, int NPROD, int STAGES, bool BMN = false>
__global__ void __launch_bounds__(THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                   const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                   const __grid_constant__ CUtensorMap tmC, int tma_store, float* __restrict__ C, int M, int N,
                   int K, int batch, int* status, const unsigned* __restrict__ sa_bits,
                   const unsigned* __restrict__ sb_bits) {
  using Lay = Layout<BN, NPROD, STAGES>;
  static_assert(!BMN || (NPROD != 8 && BN % 64 == 0), "MN-major B: BF16, 64-column blocks");
  constexpr int BKE = (NPROD == 8) ? 128 : BK;          // K elements per 128-byte row
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Lay::BAR_OFF);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;     // [2] accumulator ready (MMA -> epilogue)
  uint64_t* tempty = tfull + 2;         // [2] accumulator drained (epilogue -> MMA)
  uint64_t* mma_done = tempty + 2;      // every issued MMA has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  // every CTA is resident from the start (one per SM): the next kernel of the
  // stream, if launched with programmatic serialisation, may be scheduled now
  // (it waits for this grid's completion before reading)
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int nk = (K + BKE - 1) / BKE;
  const int mt = (M + BM - 1) / BM, nt = (N + BN - 1) / BN;
  const int64_t tiles = int64_t(batch) * mt * nt;
  auto tile_of = [&](int64_t t, int& b, int& m0, int& n0) {
    b = int(t / (int64_t(mt) * nt));
    const int rem = int(t - int64_t(b) * mt * nt);
    m0 = (rem / nt) * BM;
    n0 = (rem % nt) * BN;
  };

  auto a_tile = [&](int s, int copy) { return smem + s * Lay::STAGE + copy * Lay::A_TILE; };
  auto b_tile = [&](int s, int copy) {
    return smem + s * Lay::STAGE + Lay::NCOPY * Lay::A_TILE + copy * Lay::B_TILE;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      ptx::mbar_init(&tfull[a], 1);
      ptx::mbar_init(&tempty[a], 4);
    }
    ptx::mbar_init(mma_done, 1);
    ptx::fence_mbar_init();
  }
  if (warp == 1) ptx::tmem_alloc(tmem_slot, Lay::TMEM_COLS);
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer ----
    ptx::tma_prefetch_desc(&tmAh);
    ptx::tma_prefetch_desc(&tmBh);
    // operands written by the preceding launch (programmatic serialisation)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    uint32_t it = 0;
    for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
      int b, m0, n0;
      tile_of(t, b, m0, n0);
      for (int kb = 0; kb < nk; ++kb, ++it) {
        const uint32_t s = it % STAGES;
        if (it >= uint32_t(STAGES)) ok = ptx::mbar_wait(&empty[s], ((it / STAGES) - 1) & 1, status);
        if (!ok) break;
        ptx::mbar_arrive_expect_tx(&full[s], Lay::STAGE);
        ptx::tma_load_3d(a_tile(s, 0), &tmAh, kb * BKE, m0, b, &full[s]);
        if (NPROD == 3) ptx::tma_load_3d(a_tile(s, 1), &tmAl, kb * BKE, m0, b, &full[s]);
        if constexpr (BMN) {
#pragma unroll
          for (int j = 0; j < BN / 64; ++j) {
            ptx::tma_load_3d(b_tile(s, 0) + j * 8192, &tmBh, n0 + 64 * j, kb * BK, b, &full[s]);
            if (NPROD == 3) ptx::tma_load_3d(b_tile(s, 1) + j * 8192, &tmBl, n0 + 64 * j, kb * BK, b, &full[s]);
          }
        } else {
          ptx::tma_load_3d(b_tile(s, 0), &tmBh, kb * BKE, n0, b, &full[s]);
          if (NPROD == 3) ptx::tma_load_3d(b_tile(s, 1), &tmBl, kb * BKE, n0, b, &full[s]);
        }
      }
    }
    if (!ok) {
      // drain: wait (bounded) for the loads still in flight into the ring
      for (uint32_t k = (it > uint32_t(STAGES) ? it - STAGES : 0); k < it; ++k)
        ptx::mbar_wait(&full[k % STAGES], (k / STAGES) & 1, nullptr, 100000000ull);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    constexpr uint32_t idesc = (NPROD == 8)  ? ptx::idesc_e4m3_f32(BM, BN)
                               : BMN         ? ptx::idesc_bf16_f32_bmn(BM, BN)
                                             : ptx::idesc_bf16_f32(BM, BN);
    auto bdesc = [&](int s, int copy, int kk) {
      if constexpr (BMN) return ptx::sdesc_mnmajor_sw128(b_tile(s, copy) + kk * 2048, 8192);
      else return ptx::sdesc_kmajor_sw128(b_tile(s, copy) + kk * 32);
    };
    uint32_t it = 0, ti = 0;
    for (int64_t t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++ti) {
      const uint32_t acc = ti & 1;
      // the epilogue has drained this accumulator (both start free)
      ok = ptx::mbar_wait(&tempty[acc], ((ti >> 1) & 1) ^ 1, status);
      if (!ok) break;
      ptx::tc_fence_after();
      const uint32_t d = tmem + acc * BN;
      for (int kb = 0; kb < nk; ++kb, ++it) {
        const uint32_t s = it % STAGES;
        ok = ptx::mbar_wait(&full[s], (it / STAGES) & 1, status);
        if (!ok) break;
        ptx::tc_fence_after();
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {            // 4 MMAs of 32 bytes of K per 128-byte row
          const uint64_t ah = ptx::sdesc_kmajor_sw128(a_tile(s, 0) + kk * 32);
          const uint64_t bh = bdesc(s, 0, kk);
          if (NPROD == 8) {
            ptx::mma_e4m3(d, ah, bh, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
            continue;
          }
          ptx::mma_bf16(d, ah, bh, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
          if (NPROD == 3) {
            const uint64_t al = ptx::sdesc_kmajor_sw128(a_tile(s, 1) + kk * 32);
            const uint64_t bl = bdesc(s, 1, kk);
            ptx::mma_bf16(d, ah, bl, idesc, 1u);
            ptx::mma_bf16(d, al, bh, idesc, 1u);
          }
        }
        ptx::mma_commit(&empty[s]);
      }
      if (!ok) break;
      ptx::mma_commit(&tfull[acc]);
    }
    ptx::mma_commit(mma_done);   // also on failure: tracks completion of all issued MMAs
  } else if (warp >= 2) {
    // ---- epilogue ----
    const int quad = warp & 3;                  // TMEM lanes this warp may access
    const int ew = warp - 2;                    // staging buffers of this warp
    uint32_t ti = 0, chunk = 0;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x, ++ti) {
      const uint32_t acc = ti & 1;
      if (ok) ok = ptx::mbar_wait(&tfull[acc], (ti >> 1) & 1, status);
      if (!ok) break;
      ptx::tc_fence_after();
      int b, m0, n0;
      tile_of(t, b, m0, n0);
      float scale = 1.f;
      if constexpr (NPROD == 8) scale = fp8_scale(sa_bits[b]) * fp8_scale(sb_bits[b]);
      const int row = m0 + quad * 32 + lane;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        if (n0 + c0 >= N) break;
        float v[32];
        ptx::tmem_ld_32cols(tmem + (uint32_t(quad * 32) << 16) + acc * BN + uint32_t(c0), v);
        if constexpr (NPROD == 8) {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] *= scale;
        }
        if (tma_store) {
          uint8_t* stg = smem + Lay::STG_OFF + (ew * 2 + (chunk & 1)) * 4096;
          // the store issued from this buffer two chunks ago has read it
          if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
          __syncwarp();
#pragma unroll
          for (int q = 0; q < 8; ++q)
            *reinterpret_cast<float4*>(stg + lane * 128 + ((q ^ (lane & 7)) << 4)) =
                make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
          ptx::fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) {
            ptx::tma_store_3d(&tmC, stg, n0 + c0, m0 + quad * 32, b);
            ptx::bulk_commit();
          }
          ++chunk;
        } else if (row < M) {
          float* crow = C + (int64_t(b) * M + row) * N;
          const int col = n0 + c0;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (col + j < N) crow[col + j] = v[j];
        }
      }
      // this warp's reads of the accumulator are complete
      ptx::tc_fence_before();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&tempty[acc]);
    }
    if (lane == 0) ptx::bulk_wait_all();
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    ptx::mbar_wait(mma_done, 0, nullptr, 100000000ull);   // MMAs finished before TMEM is freed
    __syncwarp();
    ptx::tmem_dealloc(tmem, Lay::TMEM_COLS);
  }
}

}  // namespace tc

// ---- fused w-product: lift + split producers, inverse-lift epilogue ------------------------
//
// For C = A *w B (no transposes, 1 <= L <= 5) the operand preparation and
// the inverse transform are folded into the neighbouring passes:
//   lift_split_rows_kernel       spatial A (p, n1, n2) -> W(A) as BF16 hi/lo,
//                                K-major (p, n1, Kp): one HBM pass
//   lift_split_transpose_kernel  spatial B (p, n2, n4) -> W(B)^T as BF16 hi/lo,
//                                K-major (p, n4, Kp), transposed through a
//                                shared-memory tile: one HBM pass
//   tc_gemm_ilift_kernel         one CTA owns a 128 x BN tile of all G = 2^L
//                                wavelet-domain slices of a tube group, with G
//                                TMEM accumulators of BN = 512 / G columns; the
//                                epilogue reads the G accumulators of a few
//                                columns at a time, applies W^{-1} across them in
//                                registers (Eq. 3) and stores spatial C.  The
//                                wavelet-domain product never reaches HBM.

// The wavelet-domain operands of these kernels, and C_hat on the three-pass
// path, stay inside one w-product call, so they use the group-interleaved
// slice order (local index t of tube group g at slice g * 2^L + t, local
// order s_L, d_L, d_{L-1}, ..., d_1 as in lift_math.cuh): every pass over
// them streams G consecutive slices per group.  The face-product does not
// depend on the slice order, and the result C is spatial.

// One operand of lift_split_rows_kernel: spatial (p, R, C) in, wavelet-domain
// BF16 hi (/ lo) (p, R, Cp) out (group-interleaved); `items` = (p / 2^L) * R * C / VEC.
struct SplitOperand {
  const float* in;
  __nv_bfloat16* hi;
  __nv_bfloat16* lo;
  int R, C, Cp;
  int64_t items;
};

template <int L, int VEC>
__device__ __forceinline__ void lift_split_item(const SplitOperand& d, int64_t p, int64_t item) {
  constexpr int G = 1 << L;
  const int64_t plane = int64_t(d.R) * d.C;
  const int64_t nvec = plane / VEC;
  const int64_t g = item / nvec;
  const int64_t e = (item - g * nvec) * VEC;
  const int r = int(e / d.C), c = int(e - int64_t(r) * d.C);
  float v[G][VEC];
#pragma unroll
  for (int t = 0; t < G; ++t) {
    const float* src = d.in + (g * G + t) * plane + e;
    if constexpr (VEC == 4) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(src));
      v[t][0] = q.x; v[t][1] = q.y; v[t][2] = q.z; v[t][3] = q.w;
    } else {
      v[t][0] = __ldg(src);
    }
  }
#pragma unroll
  for (int j = 0; j < VEC; ++j) {
    float x[G], y[G];
#pragma unroll
    for (int t = 0; t < G; ++t) x[t] = v[t][j];
    lift_group<L>(x, y);
#pragma unroll
    for (int t = 0; t < G; ++t) v[t][j] = y[t];
  }
#pragma unroll
  for (int t = 0; t < G; ++t) {
    const int64_t o = (g * G + t) * int64_t(d.R) * d.Cp + int64_t(r) * d.Cp + c;
    if constexpr (VEC == 4) {
      __nv_bfloat16 h[4], l[4];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) split_bf16(v[t][jj], h[jj], l[jj]);
      *reinterpret_cast<uint2*>(d.hi + o) = *reinterpret_cast<uint2*>(h);
      if (d.lo) *reinterpret_cast<uint2*>(d.lo + o) = *reinterpret_cast<uint2*>(l);
    } else {
      __nv_bfloat16 h, l;
      split_bf16(v[t][0], h, l);
      d.hi[o] = h;
      if (d.lo) d.lo[o] = l;
    }
  }
}

// Lift + BF16 split of one or two operands (d1.items = 0: one) in a single
// grid-stride launch.  Every CTA signals at once that the dependent launch
// (the GEMM, launched with programmatic serialisation) may start its
// prologue; the GEMM waits for this grid's completion before reading.
template <int L, int VEC>
__global__ void __launch_bounds__(256) lift_split_rows_kernel(SplitOperand d0, SplitOperand d1, int64_t p) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int64_t total = d0.items + d1.items;
  for (int64_t item = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; item < total;
       item += int64_t(gridDim.x) * blockDim.x) {
    if (item < d0.items) lift_split_item<L, VEC>(d0, p, item);
    else lift_split_item<L, VEC>(d1, p, item - d0.items);
  }
}

// Spatial B (p, R, C) -> transposed wavelet-domain BF16 hi/lo (p, C, Rp),
// group-interleaved.
// A CTA (256 threads) takes a TR x CW tile of the plane (TR = min(64, 512/G)
// input rows, CW = 2048/TR columns) of one tube group: coalesced loads into
// shared memory, the lift across the group's G slices in registers, then
// every thread writes 8 consecutive K-elements of one output row as a
// 16-byte vector per BF16 copy.
template <int L>
__global__ void __launch_bounds__(256) lift_split_transpose_kernel(const float* __restrict__ in,
                                                                   __nv_bfloat16* __restrict__ hi,
                                                                   __nv_bfloat16* __restrict__ lo, int64_t p, int R,
                                                                   int C, int Rp) {
  constexpr int G = 1 << L;
  constexpr int E = (G <= 16) ? 2048 : 1024;          // tile elements per slice (smem <= 132 KB)
  constexpr int PER = E / 256;
  constexpr int TR = (512 / G) < 64 ? (512 / G) : 64;
  constexpr int CW = E / TR;
  constexpr int LD = CW + 1;
  extern __shared__ float tile[];   // [G][TR][LD]
  const int c0 = blockIdx.x * CW, r0 = blockIdx.y * TR;
  const int64_t g = blockIdx.z;
  const int64_t plane = int64_t(R) * C;
  const int tid = threadIdx.x;
#pragma unroll 2
  for (int t = 0; t < G; ++t) {
    const float* src = in + (g * G + t) * plane;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int idx = tid + 256 * q, i = idx / CW, j = idx % CW;
      const int r = r0 + i, c = c0 + j;
      tile[(t * TR + i) * LD + j] = (r < R && c < C) ? __ldg(src + int64_t(r) * C + c) : 0.f;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int idx = tid + 256 * q, i = idx / CW, j = idx % CW;
    float x[G], y[G];
#pragma unroll
    for (int t = 0; t < G; ++t) x[t] = tile[(t * TR + i) * LD + j];
    lift_group<L>(x, y);
#pragma unroll
    for (int t = 0; t < G; ++t) tile[(t * TR + i) * LD + j] = y[t];
  }
  __syncthreads();
  const int cl = tid / (TR / 8), chunk = tid % (TR / 8);
  const int c = c0 + cl, rs = r0 + chunk * 8;
  if (tid < CW * (TR / 8) && c < C && rs < Rp) {
#pragma unroll 2
    for (int t = 0; t < G; ++t) {
      const int64_t s = g * G + t;
      __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) split_bf16(tile[(t * TR + chunk * 8 + q) * LD + cl], h[q], l[q]);
      const int64_t o = (s * C + c) * Rp + rs;
      *reinterpret_cast<uint4*>(hi + o) = *reinterpret_cast<const uint4*>(h);
      if (lo) *reinterpret_cast<uint4*>(lo + o) = *reinterpret_cast<const uint4*>(l);
    }
  }
}

// ---- FP8 w-product: lift fused into the amax and quantisation passes ------------------
//
// The per-slice scale needs the amax of each wavelet-domain slice before any
// of its elements is quantised, so the spatial operands are read twice:
//   lift_amax_kernel        lift A and B in registers, per-slice max |W(X)_k|
//                           into amax (bit patterns, atomicMax); no writes
//   fp8_inv_scales_kernel   1 / s_k for every slice, once
//   lift_quant_rows_kernel  lift again, q = e4m3(W(X)_k / s_k) in row order:
//                           A K-major (p, n1, Kp), B (p, n2, n4)
//   transpose_bytes_kernel  B's codes to K-major (p, n4, Kp)
// which moves 2 |X| + |q| (+ 2 |q_B|) bytes per operand instead of the
// 4 |X| + |q| of a lift into FP32 followed by separate amax and
// quantisation passes.  A lift-and-transpose in one pass (shared-memory tile
// of all 2^L slices) was measured slower than the row pass plus the byte
// transpose: its load, lift and store phases serialise within a CTA.

// VEC consecutive floats (16-, 8- or 4-byte aligned load).
template <int VEC>
__device__ __forceinline__ void load_floats(const float* src, float* v) {
  if constexpr (VEC == 4) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(src));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else if constexpr (VEC == 2) {
    const float2 q = __ldg(reinterpret_cast<const float2*>(src));
    v[0] = q.x; v[1] = q.y;
  } else {
    v[0] = __ldg(src);
  }
}

// One operand of the FP8 passes: spatial (p, R, C) FP32 in, E4M3 codes q
// (p, R, Cp) (rows kernel) and the per-slice amax bit patterns (p).
struct Fp8Operand {
  const float* in;
  uint8_t* q;
  unsigned* amax;
  const float* inv;     // 1 / s per slice (after the amax pass)
  int R, C, Cp;
};

// grid (x, m0 + m1): blockIdx.y < m0 takes tube group y of d0, otherwise
// group y - m0 of d1; blockIdx.x strides over the group's plane.
template <int L, int VEC>
__global__ void __launch_bounds__(256) lift_amax_kernel(Fp8Operand d0, Fp8Operand d1, int64_t p, int m0) {
  constexpr int G = 1 << L;
  const bool first = int(blockIdx.y) < m0;
  const Fp8Operand d = first ? d0 : d1;
  const int64_t g = first ? blockIdx.y : blockIdx.y - m0;
  const int64_t plane = int64_t(d.R) * d.C;
  const int64_t nvec = plane / VEC;
  float mx[G];
#pragma unroll
  for (int t = 0; t < G; ++t) mx[t] = 0.f;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < nvec; i += int64_t(gridDim.x) * blockDim.x) {
    float v[G][VEC];
#pragma unroll
    for (int t = 0; t < G; ++t) load_floats<VEC>(d.in + (g * G + t) * plane + i * VEC, v[t]);
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      float x[G], y[G];
#pragma unroll
      for (int t = 0; t < G; ++t) x[t] = v[t][j];
      lift_group<L>(x, y);
#pragma unroll
      for (int t = 0; t < G; ++t) mx[t] = fmaxf(mx[t], fabsf(y[t]));
    }
  }
  __shared__ float red[8][G];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int t = 0; t < G; ++t) {
    float m = mx[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) red[warp][t] = m;
  }
  __syncthreads();
  if (threadIdx.x < G) {
    float m = red[0][threadIdx.x];
#pragma unroll
    for (int w = 1; w < 8; ++w) m = fmaxf(m, red[w][threadIdx.x]);
    atomicMax(d.amax + g * G + threadIdx.x, __float_as_uint(m));
  }
}

// Spatial X (p, R, C) -> E4M3 codes of W(X) with the slices' scales in row
// order (p, R, Cp), for two operands in one grid-stride launch over
// (operand, tube group, VEC-vector) items.
template <int L, int VEC>
__global__ void __launch_bounds__(256) lift_quant_rows_kernel(Fp8Operand d0, Fp8Operand d1, int64_t p) {
  constexpr int G = 1 << L;
  const int64_t items0 = (p >> L) * (int64_t(d0.R) * d0.C / VEC);
  const int64_t total = items0 + (p >> L) * (int64_t(d1.R) * d1.C / VEC);
  for (int64_t it = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; it < total;
       it += int64_t(gridDim.x) * blockDim.x) {
    const bool first = it < items0;
    const Fp8Operand d = first ? d0 : d1;
    const int64_t item = first ? it : it - items0;
    const int64_t plane = int64_t(d.R) * d.C;
    const int64_t nvec = plane / VEC;
    const int64_t g = item / nvec;
    const int64_t e = (item - g * nvec) * VEC;
    const int r = int(e / d.C), c = int(e - int64_t(r) * d.C);
    float v[G][VEC];
#pragma unroll
    for (int t = 0; t < G; ++t) load_floats<VEC>(d.in + (g * G + t) * plane + e, v[t]);
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
      float x[G], y[G];
#pragma unroll
      for (int t = 0; t < G; ++t) x[t] = v[t][j];
      lift_group<L>(x, y);
#pragma unroll
      for (int t = 0; t < G; ++t) v[t][j] = y[t];
    }
#pragma unroll
    for (int t = 0; t < G; ++t) {
      const int64_t s = g * G + t;
      const float inv = __ldg(d.inv + s);
      uint8_t* o = d.q + (s * d.R + r) * int64_t(d.Cp) + c;
      if constexpr (VEC == 4) {
        *reinterpret_cast<uint32_t*>(o) = to_e4m3x4(v[t][0] * inv, v[t][1] * inv, v[t][2] * inv, v[t][3] * inv);
      } else if constexpr (VEC == 2) {
        *reinterpret_cast<uint16_t*>(o) =
            uint16_t(__nv_cvt_float2_to_fp8x2(make_float2(v[t][0] * inv, v[t][1] * inv), __NV_SATFINITE, __NV_E4M3));
      } else {
        *o = to_e4m3(v[t][0] * inv);
      }
    }
  }
}

// E4M3 codes (batch, R, C) -> (batch, C, Rp), Rp a multiple of 16: 64 x 64
// byte tiles through shared memory.  Loads take 16 bytes per thread along a
// row; every thread then gathers 16 consecutive K-bytes of one output row
// (the 32 lanes of a warp on 32 different rows, so their shared-memory
// reads hit distinct words or broadcast) and stores them as one 16-byte
// vector.  Output rows beyond R (padding up to Rp) receive zeros.
__global__ void __launch_bounds__(256) transpose_bytes_kernel(const uint8_t* __restrict__ in,
                                                              uint8_t* __restrict__ out, int R, int C, int Rp,
                                                              int vec16) {
  constexpr int T = 64, S = 80;   // tile edge, shared row stride (16-byte aligned)
  __shared__ __align__(16) uint8_t tile[T * S];
  const int c0 = blockIdx.x * T, r0 = blockIdx.y * T;
  const int64_t b = blockIdx.z;
  const int tid = threadIdx.x;
  {
    const int i = tid >> 2, j = (tid & 3) * 16;
    const int r = r0 + i, c = c0 + j;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (r < R) {
      const uint8_t* src = in + (b * R + r) * int64_t(C) + c;
      if (vec16 && c + 15 < C) {
        v = __ldg(reinterpret_cast<const uint4*>(src));
      } else {
        uint8_t t[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) t[k] = (c + k < C) ? src[k] : uint8_t(0);
        v = *reinterpret_cast<const uint4*>(t);
      }
    }
    *reinterpret_cast<uint4*>(tile + i * S + j) = v;
  }
  __syncthreads();
  const int cc = tid & 63, k = tid >> 6;
  const int c = c0 + cc, rs = r0 + k * 16;
  if (c < C && rs < Rp) {
    __align__(16) uint8_t t[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) t[q] = tile[(k * 16 + q) * S + cc];
    *reinterpret_cast<uint4*>(out + (b * C + c) * int64_t(Rp) + rs) = *reinterpret_cast<const uint4*>(t);
  }
}

namespace tc {

// Slices per store pass of the fused epilogue: the largest power of two <= G
// whose 128 x BN FP32 tiles fit in `bytes` of staging memory (0: none fit).
__host__ __device__ constexpr int fused_store_slices(int G, int BN, int bytes) {
  int s = G;
  while (s > 0 && s * 128 * BN * 4 > bytes) s >>= 1;
  return s;
}

template <int L, int NPROD, int STAGES, int TMEM = 512>
struct FusedLayout {
  static constexpr int G = 1 << L;
  static constexpr int TMEM_COLS = TMEM;
  static constexpr int BN = TMEM / G;                   // G accumulators fill the CTA's TMEM columns
  static constexpr int NCOPY = (NPROD == 1) ? 1 : 2;
  static constexpr int A_TILE = BM * BK * 2;
  static constexpr int B_TILE = BN * BK * 2;
  static constexpr int STAGE = NCOPY * (A_TILE + B_TILE);
  static constexpr int BAR_OFF = STAGES * STAGE;
  static constexpr int SMEM = BAR_OFF + (2 * STAGES + 1) * 8 + 16 + 1024;
  static constexpr int CH = 64 / G < 16 ? 64 / G : 16;  // columns per epilogue chunk (registers: G * CH = 64)
};

// Each CTA loads its own A tiles; the N tiles of one row tile re-read them
// through L2.  BMN: B is MN-major -- W(B) in its natural (K rows, N contiguous) layout,
// loaded as 64-column boxes -- instead of K-major.
template <int L, int NPROD, int STAGES, int TMEM, bool BMN>
__global__ void __launch_bounds__(THREADS, 1)
    tc_gemm_ilift_kernel(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                         const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                         const __grid_constant__ CUtensorMap tmC, int tma_store, float* __restrict__ C, int M,
                         int N, int K, int64_t p, int* status) {
  using Lay = FusedLayout<L, NPROD, STAGES, TMEM>;
  constexpr int G = Lay::G, BN = Lay::BN, CH = Lay::CH;
  // TMA-store epilogue: the output tiles of SPP slices are staged in the
  // (then idle) pipeline buffers as 32-column blocks of 128-byte rows with
  // the 128-byte swizzle, and written by one 3-D bulk store per block
  constexpr bool TMA_EPI = (BN >= 32) && (CH >= 4);
  constexpr int SPP = fused_store_slices(G, BN, STAGES * Lay::STAGE);
  static_assert(!BMN || BN % 64 == 0, "MN-major B needs 64-column blocks");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Lay::BAR_OFF);
  uint64_t* empty = full + STAGES;
  uint64_t* accum = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
  const int64_t g = blockIdx.z;
  const int nk = (K + BK - 1) / BK;
  const int iters = G * nk;

  auto a_tile = [&](int s, int copy) { return smem + s * Lay::STAGE + copy * Lay::A_TILE; };
  auto b_tile = [&](int s, int copy) {
    return smem + s * Lay::STAGE + Lay::NCOPY * Lay::A_TILE + copy * Lay::B_TILE;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(&full[s], 1);
      ptx::mbar_init(&empty[s], 1);
    }
    ptx::mbar_init(accum, 1);
    ptx::fence_mbar_init();
  }
  if (warp == 1) ptx::tmem_alloc(tmem_slot, TMEM);
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (warp == 0 && lane == 0) {
    ptx::tma_prefetch_desc(&tmAh);
    ptx::tma_prefetch_desc(&tmBh);
    // the operands are written by the preceding launch (programmatic
    // serialisation): wait for its completion before the first load
    asm volatile("griddepcontrol.wait;" ::: "memory");
    int issued = 0;
    for (int it = 0; it < iters && ok; ++it) {
      const int s = it % STAGES;
      const int t = it / nk, kb = it % nk;
      const int z = int(g * G + t);
      if (it >= STAGES) ok = ptx::mbar_wait(&empty[s], ((it / STAGES) - 1) & 1, status);
      if (!ok) break;
      ptx::mbar_arrive_expect_tx(&full[s], Lay::STAGE);
      ptx::tma_load_3d(a_tile(s, 0), &tmAh, kb * BK, m0, z, &full[s]);
      if (NPROD == 3) ptx::tma_load_3d(a_tile(s, 1), &tmAl, kb * BK, m0, z, &full[s]);
      if constexpr (BMN) {
#pragma unroll
        for (int j = 0; j < BN / 64; ++j) {
          ptx::tma_load_3d(b_tile(s, 0) + j * 8192, &tmBh, n0 + 64 * j, kb * BK, z, &full[s]);
          if (NPROD == 3) ptx::tma_load_3d(b_tile(s, 1) + j * 8192, &tmBl, n0 + 64 * j, kb * BK, z, &full[s]);
        }
      } else {
        ptx::tma_load_3d(b_tile(s, 0), &tmBh, kb * BK, n0, z, &full[s]);
        if (NPROD == 3) ptx::tma_load_3d(b_tile(s, 1), &tmBl, kb * BK, n0, z, &full[s]);
      }
      ++issued;
    }
    if (!ok) {
      for (int it = (issued > STAGES ? issued - STAGES : 0); it < issued; ++it)
        ptx::mbar_wait(&full[it % STAGES], (it / STAGES) & 1, nullptr, 100000000ull);
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = BMN ? ptx::idesc_bf16_f32_bmn(BM, BN) : ptx::idesc_bf16_f32(BM, BN);
    // B descriptor of K step kk: K-major advances 32 bytes along the row,
    // MN-major 16 rows of 128 bytes
    auto bdesc = [&](int s, int copy, int kk) {
      if constexpr (BMN) return ptx::sdesc_mnmajor_sw128(b_tile(s, copy) + kk * 2048, 8192);
      else return ptx::sdesc_kmajor_sw128(b_tile(s, copy) + kk * 32);
    };
    for (int it = 0; it < iters && ok; ++it) {
      const int s = it % STAGES;
      const int t = it / nk, kb = it % nk;
      ok = ptx::mbar_wait(&full[s], (it / STAGES) & 1, status);
      if (!ok) break;
      ptx::tc_fence_after();
      const uint32_t d = tmem + uint32_t(t * BN);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint64_t ah = ptx::sdesc_kmajor_sw128(a_tile(s, 0) + kk * 32);
        const uint64_t bh = bdesc(s, 0, kk);
        ptx::mma_bf16(d, ah, bh, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
        if (NPROD == 3) {
          const uint64_t al = ptx::sdesc_kmajor_sw128(a_tile(s, 1) + kk * 32);
          const uint64_t bl = bdesc(s, 1, kk);
          ptx::mma_bf16(d, ah, bl, idesc, 1u);
          ptx::mma_bf16(d, al, bh, idesc, 1u);
        }
      }
      ptx::mma_commit(&empty[s]);
    }
    ptx::mma_commit(accum);
  } else if (warp >= 2) {
    ok = ptx::mbar_wait(accum, 0, status);
    ptx::tc_fence_after();
    const int quad = warp & 3;
    const int r = quad * 32 + lane;   // row within the tile
    const int row = m0 + r;
    const uint32_t lane_base = tmem + (uint32_t(quad * 32) << 16);
    // columns [c0, c0 + CH) of all G accumulators, inverse-transformed across
    // the group's G slices (Eq. 3): v[t][j] = spatial slice t, column c0 + j
    auto load_chunk = [&](int c0, float (&v)[G][CH]) {
      uint32_t raw[G * CH];   // all G loads in flight, then one wait
#pragma unroll
      for (int t = 0; t < G; ++t) ptx::tmem_ld_cols_async<CH>(lane_base + uint32_t(t * BN + c0), raw + t * CH);
      ptx::tmem_wait_regs<G * CH>(raw);
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        float y[G], x[G];
#pragma unroll
        for (int t = 0; t < G; ++t) y[t] = __uint_as_float(raw[t * CH + j]);
        ilift_group<L>(y, x);
#pragma unroll
        for (int t = 0; t < G; ++t) v[t][j] = x[t];
      }
    };
    if (TMA_EPI && SPP >= 1 && tma_store) {
      if constexpr (TMA_EPI && SPP >= 1) {
        const bool leader = (warp == 2 && lane == 0);
        auto epi_sync = [] { asm volatile("bar.sync 1, 128;" ::: "memory"); };
#pragma unroll
        for (int pass = 0; pass < G / SPP; ++pass) {
          if (pass > 0) {
            // the previous pass's stores have read the staging buffers
            if (leader) ptx::bulk_wait_read_all();
            epi_sync();
          }
          if (ok) {
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += CH) {
              if (n0 + c0 >= N) break;
              float v[G][CH];
              load_chunk(c0, v);
              const int h = c0 / 32, q0 = (c0 % 32) / 4;
#pragma unroll
              for (int tt = 0; tt < SPP; ++tt) {
                uint8_t* base = smem + (h * SPP + tt) * 16384 + r * 128;
#pragma unroll
                for (int k = 0; k < CH / 4; ++k) {
                  const int t = pass * SPP + tt;
                  *reinterpret_cast<float4*>(base + (((q0 + k) ^ (r & 7)) << 4)) =
                      make_float4(v[t][4 * k], v[t][4 * k + 1], v[t][4 * k + 2], v[t][4 * k + 3]);
                }
              }
            }
          }
          ptx::fence_proxy_async_smem();
          epi_sync();
          if (leader && ok) {
#pragma unroll
            for (int h = 0; h < BN / 32; ++h)
              ptx::tma_store_3d(&tmC, smem + h * SPP * 16384, n0 + 32 * h, m0, int(g * G + pass * SPP));
            ptx::bulk_commit();
          }
        }
        if (leader) ptx::bulk_wait_all();
      }
    } else if (ok) {
      const bool vec = (N % 4) == 0;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += CH) {
        if (n0 + c0 >= N) break;
        float v[G][CH];
        load_chunk(c0, v);
        if (row < M) {
          const int col = n0 + c0;
#pragma unroll
          for (int t = 0; t < G; ++t) {
            float* dst = C + ((g * G + t) * M + row) * int64_t(N) + col;
            if (vec && col + CH <= N) {
#pragma unroll
              for (int j = 0; j < CH; j += 4 < CH ? 4 : CH) {
                if constexpr (CH >= 4)
                  *reinterpret_cast<float4*>(dst + j) = make_float4(v[t][j], v[t][j + 1], v[t][j + 2], v[t][j + 3]);
                else
                  *reinterpret_cast<float2*>(dst + j) = make_float2(v[t][j], v[t][j + 1]);
              }
            } else {
#pragma unroll
              for (int j = 0; j < CH; ++j)
                if (col + j < N) dst[j] = v[t][j];
            }
          }
        }
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    if (!ok) ptx::mbar_wait(accum, 0, nullptr, 100000000ull);
    __syncwarp();
    ptx::tmem_dealloc(tmem, TMEM);
  }
}

// ---- w-product with the forward lift in the operand producer ----------------------------
//
// tc_wprod_lift_kernel has the tile of tc_gemm_ilift_kernel (one CTA owns a
// 128 x BN tile of all G = 2^L wavelet-domain slices of a tube group, G TMEM
// accumulators of BN = 512 / G columns, the inverse lift in the epilogue) but
// reads the SPATIAL operands: for every K step of 16, converter warps load
// the FP32 tiles of the group's G slices (A: 128 rows x 16 K; B: 16 K rows x
// BN columns), apply the forward lift across the group in registers (Eq. 2),
// split each value into BF16 hi + lo and store the 2G operand tiles of the
// step into shared memory in the layouts the MMA reads: A K-major without
// swizzle (8-row x 16-byte core matrices), B MN-major with the 128-byte
// swizzle (the layout a TMA load of W(B) in its natural orientation gives).
// Neither W(A), W(B) nor the wavelet-domain product reaches HBM: A and B are
// read once from HBM (the neighbouring tiles re-read them through L2) and C
// is written once.
template <int L, int NPROD>
struct LiftLayout {
  static constexpr int G = 1 << L;
  static constexpr int BN = 512 / G;                    // G accumulators fill the 512 TMEM columns
  static constexpr int KS = 16;                         // K per stage: one MMA K step
  static constexpr int NCOPY = (NPROD == 1) ? 1 : 2;
  static constexpr int A_TILE = BM * KS * 2;            // 16 row groups x 2 core matrices of 128 B
  static constexpr int B_TILE = BN * KS * 2;            // BN / 64 blocks of 16 K rows x 128 B
  static constexpr int B_OFF = NCOPY * G * A_TILE;      // A tiles [copy][slice], then B tiles [copy][slice]
  static constexpr int STAGE = NCOPY * G * (A_TILE + B_TILE);
  static constexpr int STAGES = (196608 / STAGE) < 8 ? (196608 / STAGE) : 8;
  static constexpr int BAR_OFF = STAGES * STAGE;
  static constexpr int SMEM = BAR_OFF + (2 * STAGES + 1) * 8 + 16 + 1024;
  static constexpr int CH = 64 / G < 16 ? 64 / G : 16;  // columns per epilogue chunk
  // converter work units of one stage: A, 8 rows x 16 K; B, 2 K rows x 64
  // columns; each unit covers all G slices (4 consecutive values per lane)
  static constexpr int A_UNITS = BM / 8;
  static constexpr int B_UNITS = (KS / 2) * (BN / 64);
  static constexpr int UNITS = A_UNITS + B_UNITS;
  static constexpr int CONV = (L == 3) ? 12 : 16;       // converter warps: UNITS / CONV units each
  static constexpr int THREADS = 32 * (1 + CONV);
  static constexpr int UPW = (UNITS + CONV - 1) / CONV;
  static_assert(STAGES >= 2, "two stages at least");
  static_assert(BN % 64 == 0 && CH >= 4, "MN-major B blocks and the TMA-store epilogue");
};

// 16-byte read-only load that does not allocate in L1 and has L2 fetch the
// whole 128-byte line (the converter warps read each line in two halves, one
// K step apart, long after L1 would have evicted it).
__device__ __forceinline__ float4 ldg_stream4(const float* p) {
  float4 v;
  asm("ld.global.nc.L1::no_allocate.L2::128B.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

// Component c (a compile-time constant after unrolling) of a float4.
__device__ __forceinline__ float f4_get(const float4& v, int c) {
  return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w;
}
__device__ __forceinline__ void f4_set(float4& v, int c, float x) {
  if (c == 0) v.x = x;
  else if (c == 1) v.y = x;
  else if (c == 2) v.z = x;
  else v.w = x;
}

// hi / lo BF16 pairs of four FP32 values (hi = bf16(x), lo = bf16(x - hi)),
// packed as they are stored: value j in bits [16 (j % 2), 16 (j % 2) + 16) of word j / 2.
__device__ __forceinline__ void split4_bf16(const float (&x)[4], uint2& hi, uint2& lo) {
  const __nv_bfloat162 h0 = __floats2bfloat162_rn(x[0], x[1]);
  const __nv_bfloat162 h1 = __floats2bfloat162_rn(x[2], x[3]);
  const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
  const __nv_bfloat162 l0 = __floats2bfloat162_rn(x[0] - f0.x, x[1] - f0.y);
  const __nv_bfloat162 l1 = __floats2bfloat162_rn(x[2] - f1.x, x[3] - f1.y);
  hi = make_uint2(*reinterpret_cast<const uint32_t*>(&h0), *reinterpret_cast<const uint32_t*>(&h1));
  lo = make_uint2(*reinterpret_cast<const uint32_t*>(&l0), *reinterpret_cast<const uint32_t*>(&l1));
}

// A (p, M, K) and B (p, K, N) spatial FP32, K % 4 == 0, N % 4 == 0, 16-byte
// aligned; C (p, M, N) written through tmC (boxes of 32 columns x 128 rows x
// SPP slices).  Grid (ceil(N / BN), ceil(M / 128), p / G).
template <int L, int NPROD>
__global__ void __launch_bounds__(LiftLayout<L, NPROD>::THREADS, 1)
    tc_wprod_lift_kernel(const float* __restrict__ A, const float* __restrict__ B,
                         const __grid_constant__ CUtensorMap tmC, int M, int N, int K, int* status) {
  using Lay = LiftLayout<L, NPROD>;
  constexpr int G = Lay::G, BN = Lay::BN, CH = Lay::CH, STAGES = Lay::STAGES, CONV = Lay::CONV;
  constexpr int SPP = fused_store_slices(G, BN, STAGES * Lay::STAGE);
  static_assert(SPP >= 1, "staging room for one slice");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Lay::BAR_OFF);
  uint64_t* empty = full + STAGES;
  uint64_t* accum = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM;
  const int64_t g = blockIdx.z;
  const int nk = (K + Lay::KS - 1) / Lay::KS;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(&full[s], CONV);    // one arrival per converter warp
      ptx::mbar_init(&empty[s], 1);      // the MMA commit
    }
    ptx::mbar_init(accum, 1);
    ptx::fence_mbar_init();
  }
  if (warp == 0) ptx::tmem_alloc(tmem_slot, 512);
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0) {
      constexpr uint32_t idesc = ptx::idesc_bf16_f32_bmn(BM, BN);
      for (int it = 0; it < nk && ok; ++it) {
        const int s = it % STAGES;
        ok = ptx::mbar_wait(&full[s], (it / STAGES) & 1, status);
        if (!ok) break;
        ptx::tc_fence_after();
        const uint8_t* st = smem + s * Lay::STAGE;
#pragma unroll
        for (int t = 0; t < G; ++t) {
          const uint32_t d = tmem + uint32_t(t * BN);
          const uint64_t ah = ptx::sdesc_kmajor_noswz(st + t * Lay::A_TILE, 128, 256);
          const uint64_t bh = ptx::sdesc_mnmajor_sw128(st + Lay::B_OFF + t * Lay::B_TILE, 2048);
          ptx::mma_bf16(d, ah, bh, idesc, it > 0 ? 1u : 0u);
          if constexpr (NPROD == 3) {
            const uint64_t al = ptx::sdesc_kmajor_noswz(st + (G + t) * Lay::A_TILE, 128, 256);
            const uint64_t bl = ptx::sdesc_mnmajor_sw128(st + Lay::B_OFF + (G + t) * Lay::B_TILE, 2048);
            ptx::mma_bf16(d, ah, bl, idesc, 1u);
            ptx::mma_bf16(d, al, bh, idesc, 1u);
          }
        }
        ptx::mma_commit(&empty[s]);
      }
      ptx::mma_commit(accum);
    }
    __syncwarp();
  } else {
    const int cw = warp - 1;
    const int64_t MK = int64_t(M) * K, KN = int64_t(K) * N;
    const float* Ag = A + g * G * MK;
    const float* Bg = B + g * G * KN;
    // lane roles, fixed for the whole loop
    const int ar = (lane & 15) >> 1;                      // A: row within the 8-row group
    const int aq = ((lane >> 4) << 1) | (lane & 1);       // A: K quarter (4 values)
    const int a_soff = (lane >> 4) * 128 + ar * 16 + (lane & 1) * 8;
    const int bh = lane >> 4, bc = lane & 15;             // B: K row of the pair, 4-column group
    for (int it = 0; it < nk; ++it) {
      const int s = it % STAGES, k0 = it * Lay::KS;
      // this warp's units of the stage: loads first (no dependence on the ring)
      float4 v[Lay::UPW][G];
#pragma unroll
      for (int i = 0; i < Lay::UPW; ++i) {
        const int u = cw + i * CONV;
        bool in = false;
        const float* src = nullptr;
        int64_t sstride = 0;
        if (u < Lay::A_UNITS) {
          const int row = m0 + 8 * u + ar, kc = k0 + 4 * aq;
          in = row < M && kc < K;
          src = Ag + int64_t(row) * K + kc;
          sstride = MK;
        } else if (u < Lay::UNITS) {
          const int ub = u - Lay::A_UNITS, j = ub % (Lay::KS / 2), cb = ub / (Lay::KS / 2);
          const int krow = k0 + 2 * j + bh, col = n0 + 64 * cb + 4 * bc;
          in = krow < K && col < N;
          src = Bg + int64_t(krow) * N + col;
          sstride = KN;
        }
#pragma unroll
        for (int t = 0; t < G; ++t)
          v[i][t] = in ? ldg_stream4(src + t * sstride) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      if (it >= STAGES) ok = ptx::mbar_wait(&empty[s], ((it / STAGES) - 1) & 1, status);
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
      uint8_t* st = smem + s * Lay::STAGE;
#pragma unroll
      for (int i = 0; i < Lay::UPW; ++i) {
        const int u = cw + i * CONV;
        if (u >= Lay::UNITS) break;
        // forward lift across the group, one of the four values at a time
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float x[G], y[G];
#pragma unroll
          for (int t = 0; t < G; ++t) x[t] = f4_get(v[i][t], c);
          lift_group<L>(x, y);
#pragma unroll
          for (int t = 0; t < G; ++t) f4_set(v[i][t], c, y[t]);
        }
        int off;
        uint8_t* base;
        int tile;
        if (u < Lay::A_UNITS) {
          off = u * 256 + a_soff;
          base = st;
          tile = Lay::A_TILE;
        } else {
          const int ub = u - Lay::A_UNITS, j = ub % (Lay::KS / 2), cb = ub / (Lay::KS / 2);
          const int kr = 2 * j + bh;
          off = cb * 2048 + kr * 128 + ((((bc >> 1) ^ (kr & 7))) << 4) + (bc & 1) * 8;
          base = st + Lay::B_OFF;
          tile = Lay::B_TILE;
        }
#pragma unroll
        for (int t = 0; t < G; ++t) {
          const float x4[4] = {v[i][t].x, v[i][t].y, v[i][t].z, v[i][t].w};
          uint2 hi, lo;
          split4_bf16(x4, hi, lo);
          *reinterpret_cast<uint2*>(base + t * tile + off) = hi;
          if constexpr (NPROD == 3) *reinterpret_cast<uint2*>(base + (G + t) * tile + off) = lo;
        }
      }
      // make the stores visible to the tensor core, then one arrival per warp
      ptx::fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) ptx::mbar_arrive(&full[s]);
    }

    // epilogue: the CONV warps read the G accumulators (warp & 3 selects the
    // 32-lane quarter of TMEM), inverse-lift across them (Eq. 3), stage SPP
    // slices at a time in the idle pipeline buffers and store them with TMA
    constexpr int NGRP = CONV / 4;
    const int grp = cw / 4;
    const bool wait_ok = ptx::mbar_wait(accum, 0, status);
    ok = ok && wait_ok;
    ptx::tc_fence_after();
    const int quad = warp & 3;
    const int r = quad * 32 + lane;
    const uint32_t lane_base = tmem + (uint32_t(quad * 32) << 16);
    const bool leader = (warp == 1 && lane == 0);
    auto epi_sync = [] { asm volatile("bar.sync 1, %0;" ::"n"(Lay::CONV * 32) : "memory"); };
#pragma unroll
    for (int pass = 0; pass < G / SPP; ++pass) {
      if (pass > 0) {
        if (leader) ptx::bulk_wait_read_all();
        epi_sync();
      }
      if (ok) {
#pragma unroll 1
        for (int c0 = grp * CH; c0 < BN; c0 += NGRP * CH) {
          if (n0 + c0 >= N) break;
          uint32_t raw[G * CH];
#pragma unroll
          for (int t = 0; t < G; ++t) ptx::tmem_ld_cols_async<CH>(lane_base + uint32_t(t * BN + c0), raw + t * CH);
          ptx::tmem_wait_regs<G * CH>(raw);
          const int h = c0 / 32, q0 = (c0 % 32) / 4;
#pragma unroll
          for (int j = 0; j < CH; j += 4) {
            float xs[SPP][4];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              float y[G], x[G];
#pragma unroll
              for (int t = 0; t < G; ++t) y[t] = __uint_as_float(raw[t * CH + j + jj]);
              ilift_group<L>(y, x);
#pragma unroll
              for (int tt = 0; tt < SPP; ++tt) xs[tt][jj] = x[pass * SPP + tt];
            }
#pragma unroll
            for (int tt = 0; tt < SPP; ++tt) {
              uint8_t* rowp = smem + (h * SPP + tt) * 16384 + r * 128;
              *reinterpret_cast<float4*>(rowp + (((q0 + j / 4) ^ (r & 7)) << 4)) =
                  make_float4(xs[tt][0], xs[tt][1], xs[tt][2], xs[tt][3]);
            }
          }
        }
      }
      ptx::fence_proxy_async_smem();
      epi_sync();
      if (leader && ok) {
#pragma unroll
        for (int h = 0; h < BN / 32; ++h)
          if (n0 + 32 * h < N) ptx::tma_store_3d(&tmC, smem + h * SPP * 16384, n0 + 32 * h, m0, int(g * G + pass * SPP));
        ptx::bulk_commit();
      }
    }
    if (leader) ptx::bulk_wait_all();
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    ptx::tc_fence_after();
    if (!ok) ptx::mbar_wait(accum, 0, nullptr, 100000000ull);
    __syncwarp();
    ptx::tmem_dealloc(tmem, 512);
  }
}

}  // namespace tc

// ---- host side -------------------------------------------------------------------------

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Tensor map of a (batch, rows, Kp) operand array whose rows are K-major with
// `esize`-byte elements (2: BF16, 1: FP8 bytes); box = one 128-byte row
// segment x box_rows rows, 128B swizzle.
static int make_map(CUtensorMap* map, const void* base, int64_t K, int64_t Kp, int64_t rows, int64_t batch,
                    int box_rows, int esize = 2) {
  auto fn = encode_fn();
  if (!fn) return WP_ERR_CUDA;
  cuuint64_t dims[3] = {cuuint64_t(K), cuuint64_t(rows), cuuint64_t(batch)};
  cuuint64_t strides[2] = {cuuint64_t(Kp * esize), cuuint64_t(rows * Kp * esize)};
  cuuint32_t box[3] = {cuuint32_t(128 / esize), cuuint32_t(box_rows), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapDataType dt = (esize == 2) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
  CUresult r = fn(map, dt, 3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? WP_OK : WP_ERR_CUDA;
}

// Tensor map of an FP32 (batch, rows, cols) array, box bx x by x bz with the
// 128-byte swizzle (bx * 4 = 128 bytes), for tiled stores.
static int make_map_f32(CUtensorMap* map, const float* base, int64_t cols, int64_t rows, int64_t batch, int bx,
                        int by, int bz) {
  auto fn = encode_fn();
  if (!fn) return WP_ERR_CUDA;
  cuuint64_t dims[3] = {cuuint64_t(cols), cuuint64_t(rows), cuuint64_t(batch)};
  cuuint64_t strides[2] = {cuuint64_t(cols * 4), cuuint64_t(rows * cols * 4)};
  cuuint32_t box[3] = {cuuint32_t(bx), cuuint32_t(by), cuuint32_t(bz)};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? WP_OK : WP_ERR_CUDA;
}

static int64_t pad8(int64_t k) { return (k + 7) / 8 * 8; }
static int64_t pad16(int64_t k) { return (k + 15) / 16 * 16; }

size_t tc_facewise_workspace(int64_t M, int64_t N, int64_t K, int64_t p, int prec) {
  if (prec == WP_PREC_FP8) {
    Sizer s;
    s.take<uint8_t>(size_t(p) * M * pad16(K));
    s.take<uint8_t>(size_t(p) * N * pad16(K));
    s.take<unsigned>(2 * size_t(p));
    return s.bytes();
  }
  if (prec != WP_PREC_BF16 && prec != WP_PREC_BF16X3) return 0;
  const int64_t Kp = pad8(K);
  const int ncopy = (prec == WP_PREC_BF16X3) ? 2 : 1;
  Sizer s;
  for (int c = 0; c < ncopy; ++c) {
    s.take<__nv_bfloat16>(size_t(p) * M * Kp);
    s.take<__nv_bfloat16>(size_t(p) * N * Kp);
  }
  return s.bytes();
}

// Round an FP32 operand to BF16 hi (/ lo), K-major with row stride Kp.
// kmajor_in: the stored operand already has K as its contiguous dimension.
static int split_operand(const float* X, int64_t rows, int64_t K, int64_t Kp, int64_t p, bool kmajor_in,
                         __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t st) {
  if (kmajor_in) {
    const int64_t total = p * rows * Kp;
    int64_t blocks = std::min<int64_t>((total + 255) / 256, int64_t(sm_count()) * 8);
    WP_PROFILE("split_bf16", st);
    split_rows_kernel<<<unsigned(std::max<int64_t>(blocks, 1)), 256, 0, st>>>(X, hi, lo, p * rows, int(K), int(Kp));
    return launch_status();
  }
  // stored (p, K, rows): transpose to (p, rows, Kp)
  if (rows % 4 == 0 && aligned16(X) && Kp % 8 == 0 && p <= 65535) {
    const dim3 grid{unsigned((rows + 63) / 64), unsigned((Kp + 63) / 64), unsigned(p)};
    WP_PROFILE("split_transpose_bf16", st);
    split_transpose4_kernel<<<grid, 256, 0, st>>>(X, hi, lo, int(K), int(rows), int(Kp));
    return launch_status();
  }
  const dim3 grid{unsigned((rows + 31) / 32), unsigned((Kp + 31) / 32), unsigned(std::min<int64_t>(p, 65535))};
  WP_PROFILE("split_transpose_bf16", st);
  split_transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(X, hi, lo, int(K), int(rows), int(Kp), int(p));
  return launch_status();
}

template <int BN, int NPROD, int STAGES, bool BMN = false>
static int launch_gemm(const CUtensorMap& ah, const CUtensorMap& al, const CUtensorMap& bh, const CUtensorMap& bl,
                       float* C, int64_t M, int64_t N, int64_t K, int64_t p, cudaStream_t st, const char* name,
                       const unsigned* sa = nullptr, const unsigned* sb = nullptr) {
  using Lay = tc::Layout<BN, NPROD, STAGES>;
  auto kern = tc::tc_gemm_kernel<BN, NPROD, STAGES, BMN>;
  static bool attr = false;
  if (!attr) {
    WP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::SMEM));
    attr = true;
  }
  // C as (p, M, N) FP32, 32 x 32 boxes for the TMA-store epilogue (N % 4 == 0)
  CUtensorMap mc = ah;
  int tma_store = 0;
  if (N % 4 == 0 && aligned16(C)) {
    WP_TRY(make_map_f32(&mc, C, N, M, p, 32, 32, 1));
    tma_store = 1;
  }
  const int64_t tiles = p * ((M + tc::BM - 1) / tc::BM) * ((N + BN - 1) / BN);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(std::min<int64_t>(tiles, sm_count())), 1, 1);
  cfg.blockDim = dim3(tc::THREADS, 1, 1);
  cfg.dynamicSmemBytes = Lay::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attrs[1];
  attrs[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attrs[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attrs;
  cfg.numAttrs = 1;
  WP_PROFILE(name, st);
  WP_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, ah, al, bh, bl, mc, tma_store, C, int(M), int(N), int(K), int(p),
                                 device_status_ptr(), sa, sb));
  return launch_status();
}

// FP8: per-slice amax of both operands, E4M3 quantisation (K-major, rows
// padded to 16 bytes), E4M3 GEMM with the scales applied in the epilogue.
static int tc_facewise_fp8(const float* A, const float* B, float* C, int64_t M, int64_t N, int64_t K, int64_t p,
                           bool transA, bool transB, void* ws, size_t ws_bytes, cudaStream_t st) {
  const int64_t Kp = pad16(K);
  Carver cv(ws, ws_bytes);
  uint8_t* A8 = cv.take<uint8_t>(size_t(p) * M * Kp);
  uint8_t* B8 = cv.take<uint8_t>(size_t(p) * N * Kp);
  unsigned* amax = cv.take<unsigned>(2 * size_t(p));
  if (!cv.ok) return WP_ERR_WORKSPACE;
  WP_CUDA_TRY(cudaMemsetAsync(amax, 0, 2 * size_t(p) * sizeof(unsigned), st));
  {
    const dim3 grid{unsigned(std::max<int64_t>(1, std::min<int64_t>(64, (M * K + 255) / 256))), unsigned(p), 1u};
    WP_PROFILE("amax_fp8", st);
    amax_slices_kernel<<<grid, 256, 0, st>>>(A, M * K, amax);
    WP_TRY(launch_status());
  }
  {
    const dim3 grid{unsigned(std::max<int64_t>(1, std::min<int64_t>(64, (N * K + 255) / 256))), unsigned(p), 1u};
    WP_PROFILE("amax_fp8", st);
    amax_slices_kernel<<<grid, 256, 0, st>>>(B, N * K, amax + p);
    WP_TRY(launch_status());
  }
  auto quant = [&](const float* X, int64_t rows, bool kmajor_in, uint8_t* out, const unsigned* am) -> int {
    if (kmajor_in) {
      const int64_t total = p * rows * Kp;
      const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, int64_t(sm_count()) * 8));
      WP_PROFILE("quant_fp8", st);
      quant_rows_kernel<<<unsigned(blocks), 256, 0, st>>>(X, out, am, rows, p * rows, int(K), int(Kp));
      return launch_status();
    }
    const dim3 grid{unsigned((rows + 31) / 32), unsigned((Kp + 31) / 32), unsigned(std::min<int64_t>(p, 65535))};
    WP_PROFILE("quant_transpose_fp8", st);
    quant_transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(X, out, am, int(K), int(rows), int(Kp), int(p));
    return launch_status();
  };
  WP_TRY(quant(A, M, !transA, A8, amax));
  WP_TRY(quant(B, N, transB, B8, amax + p));
  CUtensorMap ma, mb;
  constexpr int BN = 256;
  WP_TRY(make_map(&ma, A8, K, Kp, M, p, tc::BM, 1));
  WP_TRY(make_map(&mb, B8, K, Kp, N, p, BN, 1));
  return launch_gemm<BN, 8, 4>(ma, ma, mb, mb, C, M, N, K, p, st, "tc_gemm_fp8", amax, amax + p);
}

int tc_facewise(const float* A, const float* B, float* C, int64_t M, int64_t N, int64_t K, int64_t p, bool transA,
                bool transB, int prec, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (p > 65535 || M > INT32_MAX || N > INT32_MAX || K > INT32_MAX) return WP_ERR_SHAPE;
  if (prec == WP_PREC_FP8) {
    if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return WP_ERR_ALIGN;
    return tc_facewise_fp8(A, B, C, M, N, K, p, transA, transB, ws, ws_bytes, st);
  }
  if (prec != WP_PREC_BF16 && prec != WP_PREC_BF16X3) return WP_ERR_UNSUPPORTED;
  if (p > 65535 || M > INT32_MAX || N > INT32_MAX || K > INT32_MAX) return WP_ERR_SHAPE;
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return WP_ERR_ALIGN;
  const int64_t Kp = pad8(K);
  const bool x3 = (prec == WP_PREC_BF16X3);
  Carver cv(ws, ws_bytes);
  __nv_bfloat16* Ah = cv.take<__nv_bfloat16>(size_t(p) * M * Kp);
  __nv_bfloat16* Bh = cv.take<__nv_bfloat16>(size_t(p) * N * Kp);
  __nv_bfloat16* Al = x3 ? cv.take<__nv_bfloat16>(size_t(p) * M * Kp) : nullptr;
  __nv_bfloat16* Bl = x3 ? cv.take<__nv_bfloat16>(size_t(p) * N * Kp) : nullptr;
  if (!cv.ok) return WP_ERR_WORKSPACE;
  // op(A) is M x K: K-major when A is stored (p, M, K), i.e. not transposed.
  WP_TRY(split_operand(A, M, K, Kp, p, !transA, Ah, Al, st));
  // op(B) is K x N: K-major (N x K storage) when B is stored transposed.
  WP_TRY(split_operand(B, N, K, Kp, p, transB, Bh, Bl, st));
  CUtensorMap mah, mal, mbh, mbl;
  if (x3) {
    constexpr int BN = 128;
    WP_TRY(make_map(&mah, Ah, K, Kp, M, p, tc::BM));
    WP_TRY(make_map(&mal, Al, K, Kp, M, p, tc::BM));
    WP_TRY(make_map(&mbh, Bh, K, Kp, N, p, BN));
    WP_TRY(make_map(&mbl, Bl, K, Kp, N, p, BN));
    return launch_gemm<BN, 3, 3>(mah, mal, mbh, mbl, C, M, N, K, p, st, "tc_gemm_bf16x3");
  }
  constexpr int BN = 256;
  WP_TRY(make_map(&mah, Ah, K, Kp, M, p, tc::BM));
  WP_TRY(make_map(&mbh, Bh, K, Kp, N, p, BN));
  return launch_gemm<BN, 1, 4>(mah, mah, mbh, mbh, C, M, N, K, p, st, "tc_gemm_bf16");
}

}  // namespace wp

namespace wp {

template <int L>
static int launch_lift_split_transpose(const float* B, __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t p, int R, int C,
                                       int Rp, cudaStream_t st) {
  constexpr int G = 1 << L;
  constexpr int E = (G <= 16) ? 2048 : 1024;
  constexpr int TR = (512 / G) < 64 ? (512 / G) : 64;
  constexpr int CW = E / TR;
  const size_t smem = size_t(G) * TR * (CW + 1) * sizeof(float);
  static bool attr = false;
  if (!attr) {
    WP_CUDA_TRY(cudaFuncSetAttribute(lift_split_transpose_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(smem)));
    attr = true;
  }
  const dim3 grid{unsigned((C + CW - 1) / CW), unsigned((Rp + TR - 1) / TR), unsigned(p >> L)};
  WP_PROFILE("lift_split_transpose_bf16", st);
  lift_split_transpose_kernel<L><<<grid, 256, smem, st>>>(B, hi, lo, p, R, C, Rp);
  return launch_status();
}

// Lift + split of A (and B, when given) into K- (resp. N-) contiguous BF16
// hi/lo rows: one launch for both when both allow 16-byte accesses.
template <int L>
static int launch_lift_split_rows(const float* A, __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t p, int R, int C,
                                  int Cp, cudaStream_t st, const float* B = nullptr, __nv_bfloat16* bhi = nullptr,
                                  __nv_bfloat16* blo = nullptr, int RB = 0, int CB = 0, int CBp = 0) {
  auto operand = [&](const float* x, __nv_bfloat16* h, __nv_bfloat16* l, int r, int c, int cp, int vec) {
    return SplitOperand{x, h, l, r, c, cp, (p >> L) * (int64_t(r) * c / vec)};
  };
  auto launch = [&](const SplitOperand& d0, const SplitOperand& d1, bool v4) -> int {
    const int64_t total = d0.items + d1.items;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, int64_t(sm_count()) * 8));
    WP_PROFILE("lift_split_bf16", st);
    if (v4) lift_split_rows_kernel<L, 4><<<unsigned(blocks), 256, 0, st>>>(d0, d1, p);
    else lift_split_rows_kernel<L, 1><<<unsigned(blocks), 256, 0, st>>>(d0, d1, p);
    return launch_status();
  };
  const bool a4 = (C % 4 == 0) && aligned16(A);
  const SplitOperand none{nullptr, nullptr, nullptr, 1, 1, 1, 0};
  if (!B) return launch(operand(A, hi, lo, R, C, Cp, a4 ? 4 : 1), none, a4);
  const bool b4 = (CB % 4 == 0) && aligned16(B);
  if (a4 == b4) return launch(operand(A, hi, lo, R, C, Cp, a4 ? 4 : 1), operand(B, bhi, blo, RB, CB, CBp, a4 ? 4 : 1), a4);
  WP_TRY(launch(operand(A, hi, lo, R, C, Cp, a4 ? 4 : 1), none, a4));
  return launch(operand(B, bhi, blo, RB, CB, CBp, b4 ? 4 : 1), none, b4);
}

// One CTA per SM with all 512 TMEM columns (measured faster at L = 3 than
// two CTAs with 256 columns each: narrower N = 32 tiles, 2-stage rings).
template <int L, int NPROD, bool BMN>
static int launch_fused(const CUtensorMap& ah, const CUtensorMap& al, const CUtensorMap& bh, const CUtensorMap& bl,
                        float* C, int64_t M, int64_t N, int64_t K, int64_t p, cudaStream_t st) {
  constexpr int TMEM = 512;
  using Probe = tc::FusedLayout<L, NPROD, 1, TMEM>;
  constexpr int STAGES = std::min(6, 196608 / Probe::STAGE);
  using Lay = tc::FusedLayout<L, NPROD, STAGES, TMEM>;
  auto kern = tc::tc_gemm_ilift_kernel<L, NPROD, STAGES, TMEM, BMN>;
  static bool attr = false;
  if (!attr) {
    WP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::SMEM));
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned((N + Lay::BN - 1) / Lay::BN), unsigned((M + tc::BM - 1) / tc::BM), unsigned(p >> L));
  cfg.blockDim = dim3(tc::THREADS, 1, 1);
  cfg.dynamicSmemBytes = Lay::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attrs[1];
  // programmatic serialisation: the prologue may overlap the operand
  // preparation kernel; the kernel waits for it before its first load
  attrs[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attrs[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attrs;
  cfg.numAttrs = 1;
  // output tensor map for the TMA-store epilogue: (p, M, N) FP32 with N % 4
  // == 0 (16-byte row stride), boxes of 32 columns x 128 rows x SPP slices
  constexpr int SPP = tc::fused_store_slices(Lay::G, Lay::BN, STAGES * Lay::STAGE);
  CUtensorMap mc = ah;
  int tma_store = 0;
  if (Lay::BN >= 32 && Lay::CH >= 4 && SPP >= 1 && N % 4 == 0 && aligned16(C)) {
    WP_TRY(make_map_f32(&mc, C, N, M, p, 32, tc::BM, SPP));
    tma_store = 1;
  }
  WP_PROFILE(NPROD == 3 ? "tc_gemm_ilift_bf16x3" : "tc_gemm_ilift_bf16", st);
  WP_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, ah, al, bh, bl, mc, tma_store, C, int(M), int(N), int(K), p,
                                 device_status_ptr()));
  return launch_status();
}

// The lifted-operand kernel: no workspace, no preparation launch.
template <int L, int NPROD>
static int launch_lift(const float* A, const float* B, float* C, int64_t M, int64_t N, int64_t K, int64_t p,
                       cudaStream_t st) {
  using Lay = tc::LiftLayout<L, NPROD>;
  auto kern = tc::tc_wprod_lift_kernel<L, NPROD>;
  static bool attr = false;
  if (!attr) {
    WP_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::SMEM));
    attr = true;
  }
  constexpr int SPP = tc::fused_store_slices(Lay::G, Lay::BN, Lay::STAGES * Lay::STAGE);
  CUtensorMap mc;
  WP_TRY(make_map_f32(&mc, C, N, M, p, 32, tc::BM, SPP));
  const dim3 grid(unsigned((N + Lay::BN - 1) / Lay::BN), unsigned((M + tc::BM - 1) / tc::BM), unsigned(p >> L));
  WP_PROFILE(NPROD == 3 ? "tc_wprod_lift_bf16x3" : "tc_wprod_lift_bf16", st);
  kern<<<grid, Lay::THREADS, Lay::SMEM, st>>>(A, B, mc, int(M), int(N), int(K), device_status_ptr());
  return launch_status();
}

template <int L>
static int fused_levels(const float* A, const float* B, float* C, int64_t n1, int64_t n2, int64_t n4, int64_t p,
                        bool x3, __nv_bfloat16* Ah, __nv_bfloat16* Al, __nv_bfloat16* Bh, __nv_bfloat16* Bl,
                        int64_t Kp, float* Chat, cudaStream_t st) {
  CUtensorMap mah, mal, mbh, mbl;
  if (Chat) {
    // lift + split of A and of B (B in its natural layout, MN-major for the
    // MMA) in one launch, the persistent wide-tile GEMM into the
    // wavelet-domain C_hat, then the inverse transform
    const int64_t Np = pad8(n4);
    WP_TRY(launch_lift_split_rows<L>(A, Ah, Al, p, int(n1), int(n2), int(Kp), st, B, Bh, Bl, int(n2), int(n4),
                                     int(Np)));
    WP_TRY(make_map(&mah, Ah, n2, Kp, n1, p, tc::BM));
    WP_TRY(make_map(&mbh, Bh, n4, Np, n2, p, tc::BK));
    if (x3) {
      WP_TRY(make_map(&mal, Al, n2, Kp, n1, p, tc::BM));
      WP_TRY(make_map(&mbl, Bl, n4, Np, n2, p, tc::BK));
      WP_TRY((launch_gemm<128, 3, 3, true>(mah, mal, mbh, mbl, Chat, n1, n4, n2, p, st, "tc_gemm_bf16x3")));
    } else {
      WP_TRY((launch_gemm<256, 1, 4, true>(mah, mah, mbh, mbh, Chat, n1, n4, n2, p, st, "tc_gemm_bf16")));
    }
    return lift_dispatch(LIFT_INV, Chat, C, n1 * n4, p, L, st, true);
  }
  constexpr int BN = tc::FusedLayout<L, 1, 1, 512>::BN;
  constexpr bool BMN = (L <= 3);
  WP_TRY(make_map(&mah, Ah, n2, Kp, n1, p, tc::BM));
  if (x3) WP_TRY(make_map(&mal, Al, n2, Kp, n1, p, tc::BM));
  if constexpr (BMN) {
    // W(B) in its natural layout (K rows of n4 columns), 64-column boxes
    const int64_t Np = pad8(n4);
    WP_TRY(launch_lift_split_rows<L>(A, Ah, Al, p, int(n1), int(n2), int(Kp), st, B, Bh, Bl, int(n2), int(n4),
                                     int(Np)));
    WP_TRY(make_map(&mbh, Bh, n4, Np, n2, p, tc::BK));
    if (x3) WP_TRY(make_map(&mbl, Bl, n4, Np, n2, p, tc::BK));
  } else {
    WP_TRY(launch_lift_split_rows<L>(A, Ah, Al, p, int(n1), int(n2), int(Kp), st));
    WP_TRY(launch_lift_split_transpose<L>(B, Bh, Bl, p, int(n2), int(n4), int(Kp), st));
    WP_TRY(make_map(&mbh, Bh, n2, Kp, n4, p, BN));
    if (x3) WP_TRY(make_map(&mbl, Bl, n2, Kp, n4, p, BN));
  }
  if (x3) return launch_fused<L, 3, BMN>(mah, mal, mbh, mbl, C, n1, n4, n2, p, st);
  return launch_fused<L, 1, BMN>(mah, mah, mbh, mbh, C, n1, n4, n2, p, st);
}

// Elements per thread of the FP8 lift passes: G x VEC values stay in
// registers, so the vector narrows as the group grows (4 up to L = 3, 2 at
// L = 4, 1 at L = 5), as far as the row length and alignment allow.
template <int L>
static int fp8_vec(bool four_ok, bool two_ok) {
  if (L <= 3 && four_ok) return 4;
  if (L <= 4 && two_ok) return 2;
  return 1;
}

// FP8 w-product: amax pass and quantisation passes with the lift folded in,
// the persistent E4M3 GEMM (scales applied in its epilogue) into the
// wavelet-domain C_hat, then the inverse transform.
template <int L>
static int wprod_fp8_levels(const float* A, const float* B, float* C, int64_t n1, int64_t n2, int64_t n4, int64_t p,
                            void* ws, size_t ws_bytes, cudaStream_t st) {
  const int64_t m = p >> L, Kp = pad16(n2);
  Carver cv(ws, ws_bytes);
  float* Chat = cv.take<float>(size_t(p) * n1 * n4);
  uint8_t* A8 = cv.take<uint8_t>(size_t(p) * n1 * Kp);
  uint8_t* B8 = cv.take<uint8_t>(size_t(p) * n4 * Kp);
  uint8_t* B8r = cv.take<uint8_t>(size_t(p) * n2 * n4);   // W(B) codes in row order
  unsigned* amax = cv.take<unsigned>(2 * size_t(p));
  float* inv = cv.take<float>(2 * size_t(p));
  if (!cv.ok) return WP_ERR_WORKSPACE;
  WP_CUDA_TRY(cudaMemsetAsync(amax, 0, 2 * size_t(p) * sizeof(unsigned), st));
  const Fp8Operand da{A, A8, amax, inv, int(n1), int(n2), int(Kp)};
  const Fp8Operand db{B, B8r, amax + p, inv + p, int(n2), int(n4), int(n4)};
  // both operands' rows must allow the vector width (A rows n2, B rows n4)
  const int vec = fp8_vec<L>(n2 % 4 == 0 && n4 % 4 == 0 && aligned16(A) && aligned16(B),
                             n2 % 2 == 0 && n4 % 2 == 0);
  {
    // one CTA row per tube group and operand; about 8 CTAs per SM in all
    const int64_t maxx = (std::max(n1 * n2, n2 * n4) / vec + 255) / 256;
    const int64_t bx = std::max<int64_t>(1, std::min<int64_t>(maxx, (int64_t(sm_count()) * 8 + 2 * m - 1) / (2 * m)));
    const dim3 grid{unsigned(bx), unsigned(2 * m), 1u};
    WP_PROFILE("lift_amax_fp8", st);
    if constexpr (L <= 3) {
      if (vec == 4) lift_amax_kernel<L, 4><<<grid, 256, 0, st>>>(da, db, p, int(m));
    }
    if constexpr (L <= 4) {
      if (vec == 2) lift_amax_kernel<L, 2><<<grid, 256, 0, st>>>(da, db, p, int(m));
    }
    if (vec == 1) lift_amax_kernel<L, 1><<<grid, 256, 0, st>>>(da, db, p, int(m));
    WP_TRY(launch_status());
  }
  {
    WP_PROFILE("fp8_scales", st);
    fp8_inv_scales_kernel<<<unsigned((2 * p + 255) / 256), 256, 0, st>>>(amax, inv, int(2 * p));
    WP_TRY(launch_status());
  }
  {
    // W(A) straight to K-major codes, W(B) to row-order codes (transposed next)
    const int64_t total = m * ((n1 * n2 + n2 * n4) / vec);
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, int64_t(sm_count()) * 8));
    WP_PROFILE("lift_quant_fp8", st);
    if constexpr (L <= 3) {
      if (vec == 4) lift_quant_rows_kernel<L, 4><<<unsigned(blocks), 256, 0, st>>>(da, db, p);
    }
    if constexpr (L <= 4) {
      if (vec == 2) lift_quant_rows_kernel<L, 2><<<unsigned(blocks), 256, 0, st>>>(da, db, p);
    }
    if (vec == 1) lift_quant_rows_kernel<L, 1><<<unsigned(blocks), 256, 0, st>>>(da, db, p);
    WP_TRY(launch_status());
  }
  {
    const dim3 grid{unsigned((n4 + 63) / 64), unsigned((Kp + 63) / 64), unsigned(p)};
    const int vec16 = (n4 % 16 == 0);
    WP_PROFILE("transpose_fp8", st);
    transpose_bytes_kernel<<<grid, 256, 0, st>>>(B8r, B8, int(n2), int(n4), int(Kp), vec16);
    WP_TRY(launch_status());
  }
  CUtensorMap ma, mb;
  constexpr int BN = 256;
  WP_TRY(make_map(&ma, A8, n2, Kp, n1, p, tc::BM, 1));
  WP_TRY(make_map(&mb, B8, n2, Kp, n4, p, BN, 1));
  WP_TRY((launch_gemm<BN, 8, 4>(ma, ma, mb, mb, Chat, n1, n4, n2, p, st, "tc_gemm_fp8", amax, amax + p)));
  return lift_dispatch(LIFT_INV, Chat, C, n1 * n4, p, L, st, true);
}

// Which of the fused-epilogue and persistent BF16 / BF16x3 w-product kernels
// a shape takes when the lifted-operand kernel does not (lift_variant).  The
// inverse-lift epilogue needs all 2^L accumulators of a tile in TMEM, so its
// tile is only 512 / 2^L wide.  Rule of thumb, measured on GB300 (BF16x3,
// the 256 x 256 x 192 L = 3 case and neighbours): the fused kernel wins with
// wide tiles (L <= 2), short K (n2 <= 64, where the wavelet-domain round trip
// of C dominates) and small slices (n1, n4 <= 128); otherwise the persistent
// wide-tile GEMM into C_hat plus a separate inverse lift is faster (88 vs
// 96 us at 256 x 256 x 192).  A choice timed by wp_wprod_tune for the shape
// (plan cache, tune.cu) takes precedence: 1 fused, 2 persistent + inverse
// lift, 3 lifted operands + fused epilogue.
static bool fused_rule(int64_t n1, int64_t n2, int64_t n4, int L) {
  const int64_t bn_fused = 512 >> L;
  return (n4 + bn_fused - 1) / bn_fused <= 4 && (L <= 2 || n2 <= 64 || (n1 <= 128 && n4 <= 128));
}

static bool use_epilogue_fused(int64_t n1, int64_t n2, int64_t n4, int64_t p, int L, int prec) {
  const int v = wprod_plan_lookup(n1, n2, n4, p, L, prec);
  if (v == kVariantFused) return true;
  if (v == kVariantPersistent) return false;
  return fused_rule(n1, n2, n4, L);
}

static bool fused_domain(int64_t n1, int64_t n2, int64_t n4, int64_t p, int L, int prec) {
  if (prec != WP_PREC_BF16 && prec != WP_PREC_BF16X3 && prec != WP_PREC_FP8) return false;
  if (L < 1 || L > 5) return false;
  return !((p >> L) > 65535 || p > 65535 || n1 > INT32_MAX || n2 > INT32_MAX || n4 > INT32_MAX);
}

bool wprod_tunable(int64_t n1, int64_t n2, int64_t n4, int64_t p, int L, int prec) {
  return (prec == WP_PREC_BF16 || prec == WP_PREC_BF16X3) && fused_domain(n1, n2, n4, p, L, prec);
}

// Arguments the lifted-operand kernel takes: L <= 3 (all 2^L slices of a
// K step in one shared-memory stage), rows of A and B in whole float4s,
// 16-byte aligned A, B and C (C is written by TMA stores).
bool wprod_lift_ok(const float* A, const float* B, const float* C, int64_t n1, int64_t n2, int64_t n4, int64_t p,
                   int L, int prec) {
  return wprod_tunable(n1, n2, n4, p, L, prec) && L <= 3 && n2 % 4 == 0 && n4 % 4 == 0 && aligned16(A) &&
         aligned16(B) && aligned16(C) && (n1 + tc::BM - 1) / tc::BM <= 65535;
}

// Whether wp_wprod takes the lifted-operand kernel: the tuned variant if
// there is one for the shape, else at L <= 2 with at most two column tiles
// of 512 / 2^L (each column tile converts the whole row band of A again).
// Measured on GB300, BF16x3: 192 x 256^3 60 / 69 / 91 us at L = 1 / 2 / 3
// against 82 / 78 / 81 us for the best of the other two kernels; 64 x 1024 x
// 256 x 512 at L = 2 (four column tiles) 128 us against 113 us (fused).
static bool use_lift(const float* A, const float* B, const float* C, int64_t n1, int64_t n2, int64_t n4, int64_t p,
                     int L, int prec) {
  if (!wprod_lift_ok(A, B, C, n1, n2, n4, p, L, prec)) return false;
  const int v = wprod_plan_lookup(n1, n2, n4, p, L, prec);
  if (v != 0) return v == kVariantLifted;
  const int64_t bn = 512 >> L;
  return L <= 2 && (n4 + bn - 1) / bn <= 2;
}

// C = A *w B for tensor-core precisions with the transform fused into the
// operand preparation and the GEMM epilogue.  WP_ERR_UNSUPPORTED when the
// arguments fall outside the fused path (the caller then uses the unfused one).
int tc_wprod_fused(const float* A, const float* B, float* C, int64_t n1, int64_t n2, int64_t n4, int64_t p, int L,
                   int prec, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (!fused_domain(n1, n2, n4, p, L, prec)) return WP_ERR_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return WP_ERR_ALIGN;
  if (prec == WP_PREC_FP8) {
    if (2 * (p >> L) > 65535) return WP_ERR_UNSUPPORTED;
    switch (L) {
      case 1: return wprod_fp8_levels<1>(A, B, C, n1, n2, n4, p, ws, ws_bytes, st);
      case 2: return wprod_fp8_levels<2>(A, B, C, n1, n2, n4, p, ws, ws_bytes, st);
      case 3: return wprod_fp8_levels<3>(A, B, C, n1, n2, n4, p, ws, ws_bytes, st);
      case 4: return wprod_fp8_levels<4>(A, B, C, n1, n2, n4, p, ws, ws_bytes, st);
      default: return wprod_fp8_levels<5>(A, B, C, n1, n2, n4, p, ws, ws_bytes, st);
    }
  }
  const bool x3 = (prec == WP_PREC_BF16X3);
  if (use_lift(A, B, C, n1, n2, n4, p, L, prec)) {
    switch (L) {
      case 1: return x3 ? launch_lift<1, 3>(A, B, C, n1, n4, n2, p, st) : launch_lift<1, 1>(A, B, C, n1, n4, n2, p, st);
      case 2: return x3 ? launch_lift<2, 3>(A, B, C, n1, n4, n2, p, st) : launch_lift<2, 1>(A, B, C, n1, n4, n2, p, st);
      default: return x3 ? launch_lift<3, 3>(A, B, C, n1, n4, n2, p, st) : launch_lift<3, 1>(A, B, C, n1, n4, n2, p, st);
    }
  }
  const int64_t Kp = pad8(n2);
  const bool epilogue_fused = use_epilogue_fused(n1, n2, n4, p, L, prec);
  Carver cv(ws, ws_bytes);
  float* Chat = epilogue_fused ? nullptr : cv.take<float>(size_t(p) * n1 * n4);
  // B operand: (p, n2, pad8(n4)) MN-major on the fused-epilogue path at
  // L <= 3, else (p, n4, Kp) K-major; room for the larger of the two
  const size_t bsz = size_t(p) * std::max<int64_t>(n4 * Kp, n2 * pad8(n4));
  __nv_bfloat16* Ah = cv.take<__nv_bfloat16>(size_t(p) * n1 * Kp);
  __nv_bfloat16* Bh = cv.take<__nv_bfloat16>(bsz);
  __nv_bfloat16* Al = x3 ? cv.take<__nv_bfloat16>(size_t(p) * n1 * Kp) : nullptr;
  __nv_bfloat16* Bl = x3 ? cv.take<__nv_bfloat16>(bsz) : nullptr;
  if (!cv.ok) return WP_ERR_WORKSPACE;
  switch (L) {
    case 1: return fused_levels<1>(A, B, C, n1, n2, n4, p, x3, Ah, Al, Bh, Bl, Kp, Chat, st);
    case 2: return fused_levels<2>(A, B, C, n1, n2, n4, p, x3, Ah, Al, Bh, Bl, Kp, Chat, st);
    case 3: return fused_levels<3>(A, B, C, n1, n2, n4, p, x3, Ah, Al, Bh, Bl, Kp, Chat, st);
    case 4: return fused_levels<4>(A, B, C, n1, n2, n4, p, x3, Ah, Al, Bh, Bl, Kp, Chat, st);
    default: return fused_levels<5>(A, B, C, n1, n2, n4, p, x3, Ah, Al, Bh, Bl, Kp, Chat, st);
  }
}

}  // namespace wp
