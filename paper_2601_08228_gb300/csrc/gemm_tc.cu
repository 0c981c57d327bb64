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
//
// Pipeline (one CTA per 128 x BN output tile of one slice, 6 warps):
//   warp 0      TMA producer: loads the K-major BF16 tiles of A (128 x 64)
//               and B (BN x 64) with 128-byte swizzle into a STAGES-deep ring
//   warp 1      allocates TMEM; one lane issues tcgen05.mma (M = 128, N = BN,
//               K = 16) and frees ring slots with tcgen05.commit
//   warps 2-5   epilogue: tcgen05.ld of the accumulator, masked FP32 stores
// Operands are prepared by `split` kernels that round the FP32 wavelet-domain
// slices to BF16 hi (/ lo) and, where the stored layout is not K-major,
// transpose through shared memory.  Every mbarrier wait is bounded.

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "internal.cuh"
#include "tc_ptx.cuh"

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

// ---- the GEMM kernel ---------------------------------------------------------------

namespace tc {

constexpr int BM = 128;
constexpr int BK = 64;          // BF16 elements per 128-byte swizzle row
constexpr int THREADS = 192;

template <int BN, int NPROD, int STAGES>
struct Layout {
  static constexpr int NCOPY = (NPROD == 1) ? 1 : 2;
  static constexpr int A_TILE = BM * BK * 2;
  static constexpr int B_TILE = BN * BK * 2;
  static constexpr int STAGE = NCOPY * (A_TILE + B_TILE);
  static constexpr int BAR_OFF = STAGES * STAGE;
  static constexpr int SMEM = BAR_OFF + (2 * STAGES + 1) * 8 + 16 + 1024;   // + alignment slack
  static constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;
};

template <int BN, int NPROD, int STAGES>
__global__ void __launch_bounds__(THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                   const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                   float* __restrict__ C, int M, int N, int K, int* status) {
  using Lay = Layout<BN, NPROD, STAGES>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + Lay::BAR_OFF);
  uint64_t* empty = full + STAGES;
  uint64_t* accum = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * BM, b = blockIdx.z;
  const int nk = (K + BK - 1) / BK;

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
    int issued = 0;
    for (int kb = 0; kb < nk && ok; ++kb) {
      const int s = kb % STAGES;
      if (kb >= STAGES) ok = ptx::mbar_wait(&empty[s], ((kb / STAGES) - 1) & 1, status);
      if (!ok) break;
      ptx::mbar_arrive_expect_tx(&full[s], Lay::STAGE);
      ptx::tma_load_3d(a_tile(s, 0), &tmAh, kb * BK, m0, b, &full[s]);
      if (NPROD == 3) ptx::tma_load_3d(a_tile(s, 1), &tmAl, kb * BK, m0, b, &full[s]);
      ptx::tma_load_3d(b_tile(s, 0), &tmBh, kb * BK, n0, b, &full[s]);
      if (NPROD == 3) ptx::tma_load_3d(b_tile(s, 1), &tmBl, kb * BK, n0, b, &full[s]);
      ++issued;
    }
    if (!ok) {
      // drain: wait (bounded) for the loads still in flight into this CTA's ring
      for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
        ptx::mbar_wait(&full[kb % STAGES], (kb / STAGES) & 1, nullptr, 100000000ull);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    constexpr uint32_t idesc = ptx::idesc_bf16_f32(BM, BN);
    for (int kb = 0; kb < nk && ok; ++kb) {
      const int s = kb % STAGES;
      ok = ptx::mbar_wait(&full[s], (kb / STAGES) & 1, status);
      if (!ok) break;
      ptx::tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint64_t ah = ptx::sdesc_kmajor_sw128(a_tile(s, 0) + kk * 32);
        const uint64_t bh = ptx::sdesc_kmajor_sw128(b_tile(s, 0) + kk * 32);
        ptx::mma_bf16(tmem, ah, bh, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
        if (NPROD == 3) {
          const uint64_t al = ptx::sdesc_kmajor_sw128(a_tile(s, 1) + kk * 32);
          const uint64_t bl = ptx::sdesc_kmajor_sw128(b_tile(s, 1) + kk * 32);
          ptx::mma_bf16(tmem, ah, bl, idesc, 1u);
          ptx::mma_bf16(tmem, al, bh, idesc, 1u);
        }
      }
      ptx::mma_commit(&empty[s]);
    }
    ptx::mma_commit(accum);   // also on failure: tracks completion of all issued MMAs
  } else if (warp >= 2) {
    // ---- epilogue ----
    ok = ptx::mbar_wait(accum, 0, status);
    ptx::tc_fence_after();
    if (ok) {
      const int quad = warp & 3;               // TMEM lanes this warp may access
      const int row = m0 + quad * 32 + lane;
      float* crow = C + (int64_t(b) * M + row) * N;
      const bool vec = (N % 4) == 0;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        if (n0 + c0 >= N) break;
        float v[32];
        ptx::tmem_ld_32cols(tmem + (uint32_t(quad * 32) << 16) + uint32_t(c0), v);
        if (row < M) {
          const int col = n0 + c0;
          if (vec && col + 32 <= N) {
#pragma unroll
            for (int j = 0; j < 32; j += 4)
              *reinterpret_cast<float4*>(crow + col + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
          } else {
            for (int j = 0; j < 32 && col + j < N; ++j) crow[col + j] = v[j];
          }
        }
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    ptx::tc_fence_after();
    if (!ok) ptx::mbar_wait(accum, 0, nullptr, 100000000ull);   // MMAs finished before TMEM is freed
    __syncwarp();
    ptx::tmem_dealloc(tmem, Lay::TMEM_COLS);
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

// Tensor map of a (batch, rows, Kp) BF16 array, box = (64, box_rows, 1), 128B swizzle.
static int make_map(CUtensorMap* map, const void* base, int64_t K, int64_t Kp, int64_t rows, int64_t batch,
                    int box_rows) {
  auto fn = encode_fn();
  if (!fn) return WP_ERR_CUDA;
  cuuint64_t dims[3] = {cuuint64_t(K), cuuint64_t(rows), cuuint64_t(batch)};
  cuuint64_t strides[2] = {cuuint64_t(Kp * 2), cuuint64_t(rows * Kp * 2)};
  cuuint32_t box[3] = {cuuint32_t(tc::BK), cuuint32_t(box_rows), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? WP_OK : WP_ERR_CUDA;
}

static int64_t pad8(int64_t k) { return (k + 7) / 8 * 8; }

size_t tc_facewise_workspace(int64_t M, int64_t N, int64_t K, int64_t p, int prec) {
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
  const dim3 grid{unsigned((rows + 31) / 32), unsigned((Kp + 31) / 32), unsigned(std::min<int64_t>(p, 65535))};
  WP_PROFILE("split_transpose_bf16", st);
  split_transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(X, hi, lo, int(K), int(rows), int(Kp), int(p));
  return launch_status();
}

template <int BN, int NPROD, int STAGES>
static int launch_gemm(const CUtensorMap& ah, const CUtensorMap& al, const CUtensorMap& bh, const CUtensorMap& bl,
                       float* C, int64_t M, int64_t N, int64_t K, int64_t p, cudaStream_t st, const char* name) {
  using Lay = tc::Layout<BN, NPROD, STAGES>;
  static bool attr = false;
  if (!attr) {
    WP_CUDA_TRY(cudaFuncSetAttribute(tc::tc_gemm_kernel<BN, NPROD, STAGES>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, Lay::SMEM));
    attr = true;
  }
  const dim3 grid{unsigned((N + BN - 1) / BN), unsigned((M + tc::BM - 1) / tc::BM), unsigned(p)};
  WP_PROFILE(name, st);
  tc::tc_gemm_kernel<BN, NPROD, STAGES><<<grid, tc::THREADS, Lay::SMEM, st>>>(ah, al, bh, bl, C, int(M), int(N),
                                                                              int(K), device_status_ptr());
  return launch_status();
}

int tc_facewise(const float* A, const float* B, float* C, int64_t M, int64_t N, int64_t K, int64_t p, bool transA,
                bool transB, int prec, void* ws, size_t ws_bytes, cudaStream_t st) {
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
