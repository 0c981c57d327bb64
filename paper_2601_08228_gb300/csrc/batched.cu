// Batched launch over many uneven tensors: for every item, C = A *w B
// (Def. 2.1, Algorithm 1) and C_r = rank-r w-svd of A (Algorithm 2).
//
// The host builds the work lists once (wp_batched_plan) into the workspace;
// wp_batched_run then issues persistent, grouped kernels whose CTAs loop
// over those lists, so one launch covers every item of a phase whatever its
// shape:
//   1. lifting      every A and B (one descriptor per tensor, CTA-sized
//                   chunks of (tube group, plane range), L dispatched per chunk)
//   2. face-product every wavelet-domain slice A_hat_k B_hat_k (one slice per
//                   CTA iteration, operands staged in shared memory)
//   3. Jacobi SVD   every slice of A_hat (block-cyclic one-sided Jacobi, the
//                   slice's columns in registers, jacobi_block.cuh), the
//                   rank-r slice C_hat_k = U_r U_r^T A_hat_k (or
//                   A_hat_k V_r V_r^T) rebuilt in the same CTA; slices of at
//                   most 32 / 48 columns on 4- / 6-warp CTAs, the rest on CTAs
//                   sized for 64 columns (three launches)
//   4. inverse lifting of every C_hat and C_hat_r
// wp_batched_run performs no allocation, host synchronisation or copy, so it
// can be captured in a CUDA graph.  The CTA sizes of phases 2 and 3 are picked
// by timing candidates on the planned work (wp_batched_plan with tune = 1).

#include <vector>

#include <mutex>

#include "common.cuh"
#include "internal.cuh"
#include "jacobi_block.cuh"
#include "jacobi_group.cuh"
#include "jacobi_common.cuh"
#include "lift_math.cuh"

namespace wp {

struct BItem {
  const float* A;
  const float* B;
  float* C;
  float* Cr;
  float* Ah;    // workspace: wavelet-domain A, B, C, C_r
  float* Bh;
  float* Ch;
  float* Crh;
  int n1, n2, n4, p, L, r;
};

struct LiftDesc {
  const float* src;
  float* dst;
  int64_t first_block;   // first CTA-chunk index of this tensor
  int32_t plane, p, L, op;
  int32_t chunks_per_group;
  int32_t vec;           // plane elements per thread (batched_lift_vec)
};

// Plane elements per thread of the grouped lift: vectors where the plane
// and both pointers allow, narrower as the group grows so that no case of
// the one grouped kernel needs more than 32 live values per thread.
__host__ __device__ constexpr int batched_lift_vec_max(int L) { return L <= 2 ? 4 : (L == 3 ? 2 : 1); }

constexpr int BL_THREADS = 256;

// ---- phase 1 / 4: grouped lifting ---------------------------------------------------

// The wavelet-domain copies of the items never leave the batched launch, so
// they use the group-interleaved slice order (local index t of group g at
// slice g * 2^L + t): both directions stream 2^L consecutive slices.
template <int L, int VEC>
__device__ __forceinline__ void lift_chunk(const LiftDesc& d, int64_t g, int64_t e) {
  constexpr int G = 1 << L;
  const bool fwd = (d.op == LIFT_FWD);
  float v[G][VEC];
#pragma unroll
  for (int t = 0; t < G; ++t) {
    const float* src = d.src + (g * G + t) * d.plane + e;
    if constexpr (VEC == 4) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(src));
      v[t][0] = q.x; v[t][1] = q.y; v[t][2] = q.z; v[t][3] = q.w;
    } else if constexpr (VEC == 2) {
      const float2 q = __ldg(reinterpret_cast<const float2*>(src));
      v[t][0] = q.x; v[t][1] = q.y;
    } else {
      v[t][0] = __ldg(src);
    }
  }
#pragma unroll
  for (int j = 0; j < VEC; ++j) {
    float x[G], y[G];
#pragma unroll
    for (int t = 0; t < G; ++t) x[t] = v[t][j];
    if (fwd) lift_group<L>(x, y);
    else ilift_group<L>(x, y);
#pragma unroll
    for (int t = 0; t < G; ++t) v[t][j] = y[t];
  }
#pragma unroll
  for (int t = 0; t < G; ++t) {
    float* dst = d.dst + (g * G + t) * d.plane + e;
    if constexpr (VEC == 4) *reinterpret_cast<float4*>(dst) = make_float4(v[t][0], v[t][1], v[t][2], v[t][3]);
    else if constexpr (VEC == 2) *reinterpret_cast<float2*>(dst) = make_float2(v[t][0], v[t][1]);
    else *dst = v[t][0];
  }
}

template <int L>
__device__ __forceinline__ void lift_chunk_vec(const LiftDesc& d, int64_t g, int64_t e) {
  constexpr int VM = batched_lift_vec_max(L);
  if (VM >= 4 && d.vec == 4) lift_chunk<L, VM >= 4 ? 4 : 1>(d, g, e);
  else if (VM >= 2 && d.vec == 2) lift_chunk<L, VM >= 2 ? 2 : 1>(d, g, e);
  else lift_chunk<L, 1>(d, g, e);
}

__global__ void __launch_bounds__(BL_THREADS) batched_lift_kernel(const LiftDesc* __restrict__ descs, int ndesc,
                                                                  int64_t total_blocks) {
  for (int64_t b = blockIdx.x; b < total_blocks; b += gridDim.x) {
    // binary search for the descriptor owning CTA-chunk b
    int lo = 0, hi = ndesc - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (descs[mid].first_block <= b) lo = mid;
      else hi = mid - 1;
    }
    const LiftDesc d = descs[lo];
    const int64_t local = b - d.first_block;
    const int64_t g = local / d.chunks_per_group;
    const int64_t e = ((local % d.chunks_per_group) * BL_THREADS + threadIdx.x) * d.vec;
    if (e >= d.plane) continue;
    switch (d.L) {
      case 0: lift_chunk_vec<0>(d, g, e); break;
      case 1: lift_chunk_vec<1>(d, g, e); break;
      case 2: lift_chunk_vec<2>(d, g, e); break;
      case 3: lift_chunk_vec<3>(d, g, e); break;
      case 4: lift_chunk_vec<4>(d, g, e); break;
      default: lift_chunk_vec<5>(d, g, e); break;
    }
  }
}

// ---- phase 2: grouped face-products (n1, n2, n4 <= 64) --------------------------------

constexpr int BMAX = 64;

// One wavelet-domain slice per CTA iteration: A_hat_k staged transposed and
// B_hat_k as is in shared memory (rows of BS floats, 16-byte aligned), then
// 4 x 4 output micro-tiles per thread: two 16-byte shared loads per 16 FMAs.
constexpr int BS = BMAX + 4;

__global__ void batched_facewise_kernel(const BItem* __restrict__ items, const int2* __restrict__ units,
                                        int64_t nunits) {
  __shared__ __align__(16) float At[BMAX * BS];   // At[k][i] = A_hat_k[i][k]
  __shared__ __align__(16) float Bs[BMAX * BS];   // Bs[k][j] = B_hat_k[k][j]
  for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int2 uk = units[u];
    const BItem it = items[uk.x];
    const int n1 = it.n1, n2 = it.n2, n4 = it.n4;
    const float* a = it.Ah + int64_t(uk.y) * n1 * n2;
    const float* bm = it.Bh + int64_t(uk.y) * n2 * n4;
    float* c = it.Ch + int64_t(uk.y) * n1 * n4;
    for (int i = threadIdx.x; i < n1 * n2; i += blockDim.x) {
      const int row = i / n2, col = i - row * n2;
      At[col * BS + row] = __ldg(a + i);
    }
    for (int i = threadIdx.x; i < n2 * n4; i += blockDim.x) {
      const int row = i / n4, col = i - row * n4;
      Bs[row * BS + col] = __ldg(bm + i);
    }
    __syncthreads();
    // micro-tile (ti, tj): rows 4 ti .. 4 ti + 3, columns 4 tj .. 4 tj + 3
    const int mt = (n1 + 3) >> 2, nt = (n4 + 3) >> 2;
    for (int w = threadIdx.x; w < mt * nt; w += blockDim.x) {
      const int ti = w / nt, tj = w - ti * nt;
      float acc[4][4] = {};
      for (int k = 0; k < n2; ++k) {
        const float4 av = *reinterpret_cast<const float4*>(At + k * BS + 4 * ti);
        const float4 bv = *reinterpret_cast<const float4*>(Bs + k * BS + 4 * tj);
        const float ar[4] = {av.x, av.y, av.z, av.w}, br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(ar[x], br[y], acc[x][y]);
      }
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const int row = 4 * ti + x;
        if (row < n1) {
#pragma unroll
          for (int y = 0; y < 4; ++y)
            if (4 * tj + y < n4) c[row * n4 + 4 * tj + y] = acc[x][y];
        }
      }
    }
    __syncthreads();
  }
}

// ---- phase 3: grouped Jacobi SVD + rank-r rebuild ---------------------------------------

// Jacobi phase: the block-cyclic register-resident one-sided Jacobi of
// jacobi_block.cuh on one CTA per wavelet-domain slice (persistent over the
// work list): blocks of PPW columns, NW warps, rows lane and lane + 32 of
// every column in registers (slices up to 64 x 64), then the rank-r rebuild
// from the leading vectors, staged in shared memory.
template <int PPW, int NW, bool GROUP = false>
struct BJ {
  static constexpr int RPL = 2;
  static constexpr size_t BLOCK = GROUP ? jgroup::Lay<NW>::total
                                        : jblock::block_smem<1, PPW, RPL, NW>(BMAX);   // n_pad <= 64
  // + the leading vectors, max(n1, n2) x r floats (at most 64 x 64)
  static size_t smem(int vec_floats) { return BLOCK + (size_t(vec_floats) * sizeof(float) + 15) / 16 * 16; }
};

// 64 registers: 1024 threads per SM's worth of CTAs (8 of 4 warps, 4 of 8)
// when shared memory allows.
// GROUP: the lane-group kernel of jacobi_group.cuh (blocks of 4 columns)
// instead of the block-cyclic one.
template <int PPW, int NW, bool GROUP>
__global__ void __launch_bounds__(NW * 32, 32 / NW) batched_jacobi_kernel(const BItem* __restrict__ items,
                                                                 const int2* __restrict__ units, int64_t nunits,
                                                                 int max_sweeps, int* status,
                                                                 unsigned long long* stats) {
  using L = BJ<PPW, NW, GROUP>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* vec = reinterpret_cast<float*>(smem_raw + L::BLOCK);   // m_len x r
  float* T = reinterpret_cast<float*>(smem_raw);                // rebuild scratch (block area is free by then)
  constexpr int nthr = NW * 32;
  for (int64_t u = blockIdx.x; u < nunits; u += gridDim.x) {
    const int2 uk = units[u];
    const BItem it = items[uk.x];
    const int n1 = it.n1, n2 = it.n2, r = it.r;
    JacobiArgs b{};
    b.n1 = n1;
    b.n2 = n2;
    b.trans = (n1 < n2) ? 1 : 0;
    b.m_len = b.trans ? n2 : n1;
    b.n_vec = b.trans ? n1 : n2;
    b.n_pad = (b.n_vec + 2 * PPW - 1) / (2 * PPW) * (2 * PPW);
    b.rpc = b.m_len;
    b.r = r;
    b.tol = 2.f * sqrtf(float(b.m_len < 16 ? 16 : b.m_len)) * 1.1920929e-7f;
    b.max_sweeps = max_sweeps;
    b.status = status;
    b.stats = stats;
    const float* A = it.Ah + int64_t(uk.y) * n1 * n2;
    if constexpr (GROUP) jgroup::group_jacobi_slice<NW>(b, A, vec);
    else jblock::block_jacobi_slice<1, PPW, L::RPL, NW, false>(b, A, 0, vec, nullptr);
    // rebuild the rank-r slice from the original A_hat_k (still in global memory)
    float* Cr = it.Crh + int64_t(uk.y) * n1 * n2;
    if (!b.trans) {
      // T = U^T A (r x n2), C = U T
      for (int idx = threadIdx.x; idx < r * n2; idx += nthr) {
        const int kq = idx / n2, j = idx % n2;
        float acc = 0.f;
        for (int i = 0; i < n1; ++i) acc = fmaf(vec[i * r + kq], A[i * n2 + j], acc);
        T[idx] = acc;
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < n1 * n2; idx += nthr) {
        const int i = idx / n2, j = idx % n2;
        float acc = 0.f;
        for (int kq = 0; kq < r; ++kq) acc = fmaf(vec[i * r + kq], T[kq * n2 + j], acc);
        Cr[idx] = acc;
      }
    } else {
      // T = A V (n1 x r), C = T V^T
      for (int idx = threadIdx.x; idx < n1 * r; idx += nthr) {
        const int i = idx / r, kq = idx % r;
        float acc = 0.f;
        for (int j = 0; j < n2; ++j) acc = fmaf(A[i * n2 + j], vec[j * r + kq], acc);
        T[idx] = acc;
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < n1 * n2; idx += nthr) {
        const int i = idx / n2, j = idx % n2;
        float acc = 0.f;
        for (int kq = 0; kq < r; ++kq) acc = fmaf(T[i * r + kq], vec[j * r + kq], acc);
        Cr[idx] = acc;
      }
    }
    __syncthreads();
  }
}

// ---- host side --------------------------------------------------------------------------------

static int validate_items(const wp_batch_item* items, int count) {
  if (!items) return WP_ERR_NULL;
  if (count < 1) return WP_ERR_SHAPE;
  for (int i = 0; i < count; ++i) {
    const wp_batch_item& t = items[i];
    if (t.n1 < 1 || t.n2 < 1 || t.n4 < 1 || t.p < 1 || t.n1 > BMAX || t.n2 > BMAX || t.n4 > BMAX)
      return WP_ERR_SHAPE;
    if (t.L < 0 || t.L > 5 || (t.p % (1 << t.L)) != 0) return WP_ERR_LEVELS;
    if (t.r < 1 || t.r > std::min(t.n1, t.n2)) return WP_ERR_RANK;
    if (!t.A || !t.B || !t.C || !t.C_r) return WP_ERR_NULL;
    if (!aligned16(t.A) || !aligned16(t.B) || !aligned16(t.C) || !aligned16(t.C_r)) return WP_ERR_ALIGN;
  }
  return WP_OK;
}

struct BatchLayout {
  size_t items_off, lift1_off, lift2_off, units_off, data_off, total;
  int64_t nunits;
  std::vector<size_t> tensor_off;   // per item: offset (floats) of Ah inside the data region
};

static void batch_layout(const wp_batch_item* items, int count, BatchLayout& lay) {
  Sizer s;
  lay.items_off = 0;
  s.take<BItem>(count);
  lay.lift1_off = s.bytes();
  s.take<LiftDesc>(2 * size_t(count));
  lay.lift2_off = s.bytes();
  s.take<LiftDesc>(2 * size_t(count));
  lay.units_off = s.bytes();
  lay.nunits = 0;
  for (int i = 0; i < count; ++i) lay.nunits += items[i].p;
  s.take<int2>(size_t(lay.nunits));
  lay.data_off = s.bytes();
  size_t floats = 0;
  lay.tensor_off.resize(count);
  for (int i = 0; i < count; ++i) {
    const wp_batch_item& t = items[i];
    lay.tensor_off[i] = floats;
    const size_t p = size_t(t.p);
    floats += p * t.n1 * t.n2;        // A_hat
    floats = align_up(floats, 64);
    floats += p * t.n2 * t.n4;        // B_hat
    floats = align_up(floats, 64);
    floats += p * t.n1 * t.n4;        // C_hat
    floats = align_up(floats, 64);
    floats += p * t.n1 * t.n2;        // C_hat_r
    floats = align_up(floats, 64);
  }
  lay.total = lay.data_off + floats * sizeof(float);
}

static int64_t make_lift_descs(std::vector<LiftDesc>& d, const float* src, float* dst, int plane, int p, int L,
                               int op, int64_t first) {
  LiftDesc x{};
  x.src = src;
  x.dst = dst;
  x.first_block = first;
  x.plane = plane;
  x.p = p;
  x.L = L;
  x.op = op;
  // vectors need a plane of whole vectors and 16- (8-) byte aligned tensors
  const int vm = batched_lift_vec_max(L);
  const bool a16 = aligned16(src) && aligned16(dst);
  const bool a8 = (reinterpret_cast<uintptr_t>(src) & 7u) == 0 && (reinterpret_cast<uintptr_t>(dst) & 7u) == 0;
  x.vec = (vm >= 4 && plane % 4 == 0 && a16) ? 4 : (vm >= 2 && plane % 2 == 0 && a8) ? 2 : 1;
  x.chunks_per_group = (plane + BL_THREADS * x.vec - 1) / (BL_THREADS * x.vec);
  d.push_back(x);
  return first + int64_t(p >> L) * x.chunks_per_group;
}

static int launch_batched_lift(const LiftDesc* d, int ndesc, int64_t blocks, cudaStream_t st) {
  const int64_t grid = std::min<int64_t>(blocks, int64_t(sm_count()) * 8);
  WP_PROFILE("batched_lift", st);
  batched_lift_kernel<<<unsigned(std::max<int64_t>(grid, 1)), BL_THREADS, 0, st>>>(d, ndesc, blocks);
  return launch_status();
}

static int launch_batched_gemm(const BItem* items, const int2* units, int64_t n, int threads, cudaStream_t st) {
  const int64_t grid = std::min<int64_t>(n, int64_t(sm_count()) * (2048 / threads));
  WP_PROFILE("batched_facewise", st);
  batched_facewise_kernel<<<unsigned(std::max<int64_t>(grid, 1)), threads, 0, st>>>(items, units, n);
  return launch_status();
}

template <int PPW, int NW, bool GROUP = false>
static int launch_batched_jacobi_t(const BItem* items, const int2* units, int64_t n, int vec_floats,
                                   cudaStream_t st) {
  using L = BJ<PPW, NW, GROUP>;
  const size_t smem = L::smem(vec_floats);
  static bool attr = false;
  if (!attr) {
    WP_CUDA_TRY(cudaFuncSetAttribute(batched_jacobi_kernel<PPW, NW, GROUP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(L::smem(BMAX * BMAX))));
    attr = true;
  }
  int per_sm = 0;
  WP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_jacobi_kernel<PPW, NW, GROUP>, NW * 32, smem));
  if (per_sm < 1) per_sm = 1;
  const int64_t grid = std::min<int64_t>(n, int64_t(sm_count()) * per_sm);
  WP_PROFILE("batched_jacobi", st);
  batched_jacobi_kernel<PPW, NW, GROUP><<<unsigned(std::max<int64_t>(grid, 1)), NW * 32, smem, st>>>(
      items, units, n, jacobi_max_sweeps(), device_status_ptr(), jacobi_stats_ptr());
  return launch_status();
}

// threads: 128 (4 warps, blocks of 8 columns) or 256 (8 warps, blocks of 4)
// Slices with min(n1, n2) > 32 (up to 64 columns): 8 warps of 4-column
// blocks or 4 warps of 8-column blocks, as tuned.
static int launch_batched_jacobi(const BItem* items, const int2* units, int64_t n, int threads, int vec_floats,
                                 bool group, cudaStream_t st) {
  if (n < 1) return WP_OK;
  if (group) return launch_batched_jacobi_t<4, 8, true>(items, units, n, vec_floats, st);
  if (threads == 256) return launch_batched_jacobi_t<4, 8>(items, units, n, vec_floats, st);
  return launch_batched_jacobi_t<8, 4>(items, units, n, vec_floats, st);
}

// Slices with at most 32 (48) columns: 4 (6) warps of 4-column blocks, so
// that at most one warp of a CTA idles and more slices run per SM than on
// 8-warp CTAs.
static int launch_batched_jacobi_narrow(const BItem* items, const int2* units, int64_t n, int vec_floats,
                                        bool group, cudaStream_t st) {
  if (n < 1) return WP_OK;
  if (group) return launch_batched_jacobi_t<4, 4, true>(items, units, n, vec_floats, st);
  return launch_batched_jacobi_t<4, 4>(items, units, n, vec_floats, st);
}

static int launch_batched_jacobi_mid(const BItem* items, const int2* units, int64_t n, int vec_floats, bool group,
                                     cudaStream_t st) {
  if (n < 1) return WP_OK;
  if (group) return launch_batched_jacobi_t<4, 6, true>(items, units, n, vec_floats, st);
  return launch_batched_jacobi_t<4, 6>(items, units, n, vec_floats, st);
}

// Time one candidate configuration of a phase (median of 3 runs).
template <typename F>
static float time_candidate(F&& fn, cudaStream_t st) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(a, st);
    fn();
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    best = std::min(best, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

}  // namespace wp

using namespace wp;

extern "C" int wp_batched_workspace(const wp_batch_item* items, int count, size_t* bytes) {
  if (!bytes) return WP_ERR_NULL;
  WP_TRY(validate_items(items, count));
  BatchLayout lay;
  batch_layout(items, count, lay);
  *bytes = lay.total;
  return WP_OK;
}

// Second stream and fork / join events of one device (created on first use,
// kept for the life of the process): the face-product phase runs on it beside
// the Jacobi phases, which do not depend on it.
struct BatchFork {
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  bool ok = false;
};

static BatchFork* batch_fork() {
  static std::mutex mu;
  static BatchFork forks[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  BatchFork& f = forks[dev];
  if (!f.ok) {
    if (cudaStreamCreateWithFlags(&f.side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&f.join, cudaEventDisableTiming) != cudaSuccess)
      return nullptr;
    f.ok = true;
  }
  return &f;
}

extern "C" int wp_batched_plan(const wp_batch_item* items, int count, int tune, void* ws, size_t ws_bytes,
                               wp_batch_plan* plan, void* stream) {
  if (!plan) return WP_ERR_NULL;
  // the run's second stream exists before any capture of wp_batched_run
  if (!batch_fork()) return WP_ERR_CUDA;
  WP_TRY(validate_items(items, count));
  BatchLayout lay;
  batch_layout(items, count, lay);
  if (!ws || ws_bytes < lay.total) return WP_ERR_WORKSPACE;
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return WP_ERR_ALIGN;
  char* base = static_cast<char*>(ws);
  float* data = reinterpret_cast<float*>(base + lay.data_off);
  std::vector<BItem> bi(count);
  std::vector<LiftDesc> l1, l2;
  // narrow slices (min(n1, n2) <= 32) first, then mid (<= 48), then wide
  std::vector<int2> units, mid, wide;
  units.reserve(size_t(lay.nunits));
  int64_t b1 = 0, b2 = 0;
  for (int i = 0; i < count; ++i) {
    const wp_batch_item& t = items[i];
    BItem& x = bi[i];
    x.A = t.A; x.B = t.B; x.C = t.C; x.Cr = t.C_r;
    size_t off = lay.tensor_off[i];
    const size_t p = size_t(t.p);
    x.Ah = data + off; off = align_up(off + p * t.n1 * t.n2, 64);
    x.Bh = data + off; off = align_up(off + p * t.n2 * t.n4, 64);
    x.Ch = data + off; off = align_up(off + p * t.n1 * t.n4, 64);
    x.Crh = data + off;
    x.n1 = t.n1; x.n2 = t.n2; x.n4 = t.n4; x.p = t.p; x.L = t.L; x.r = t.r;
    b1 = make_lift_descs(l1, t.A, x.Ah, t.n1 * t.n2, t.p, t.L, LIFT_FWD, b1);
    b1 = make_lift_descs(l1, t.B, x.Bh, t.n2 * t.n4, t.p, t.L, LIFT_FWD, b1);
    b2 = make_lift_descs(l2, x.Ch, t.C, t.n1 * t.n4, t.p, t.L, LIFT_INV, b2);
    b2 = make_lift_descs(l2, x.Crh, t.C_r, t.n1 * t.n2, t.p, t.L, LIFT_INV, b2);
    const int nv = std::min(t.n1, t.n2);
    for (int k = 0; k < t.p; ++k) (nv <= 32 ? units : nv <= 48 ? mid : wide).push_back(make_int2(i, k));
  }
  const int64_t n_narrow = int64_t(units.size()), n_mid = int64_t(mid.size());
  units.insert(units.end(), mid.begin(), mid.end());
  units.insert(units.end(), wide.begin(), wide.end());
  cudaStream_t st = as_stream(stream);
  WP_CUDA_TRY(cudaMemcpyAsync(base + lay.items_off, bi.data(), bi.size() * sizeof(BItem), cudaMemcpyHostToDevice, st));
  WP_CUDA_TRY(cudaMemcpyAsync(base + lay.lift1_off, l1.data(), l1.size() * sizeof(LiftDesc), cudaMemcpyHostToDevice, st));
  WP_CUDA_TRY(cudaMemcpyAsync(base + lay.lift2_off, l2.data(), l2.size() * sizeof(LiftDesc), cudaMemcpyHostToDevice, st));
  WP_CUDA_TRY(cudaMemcpyAsync(base + lay.units_off, units.data(), units.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
  WP_CUDA_TRY(cudaStreamSynchronize(st));   // host vectors go out of scope below
  plan->count = count;
  plan->items_off = lay.items_off;
  plan->lift_fwd_off = lay.lift1_off;
  plan->lift_inv_off = lay.lift2_off;
  plan->units_off = lay.units_off;
  plan->n_lift_fwd = int32_t(l1.size());
  plan->n_lift_inv = int32_t(l2.size());
  plan->lift_fwd_blocks = b1;
  plan->lift_inv_blocks = b2;
  plan->n_units = lay.nunits;
  plan->n_units_narrow = n_narrow;
  plan->n_units_mid = n_mid;
  plan->gemm_threads = 256;
  plan->svd_threads = 128;
  plan->svd_group = 1;
  plan->reserved = 0;
  plan->svd_vec_floats = 1;
  for (int i = 0; i < count; ++i)
    plan->svd_vec_floats = std::max(plan->svd_vec_floats, std::max(items[i].n1, items[i].n2) * items[i].r);
  if (tune) {
    // autotune the CTA sizes of the face-product and Jacobi phases on the
    // planned work (phase 1 first so that the operands are real)
    const BItem* di = reinterpret_cast<const BItem*>(base + lay.items_off);
    const int2* du = reinterpret_cast<const int2*>(base + lay.units_off);
    WP_TRY(launch_batched_lift(reinterpret_cast<const LiftDesc*>(base + lay.lift1_off), plan->n_lift_fwd, b1, st));
    float best = 1e30f;
    for (int thr : {64, 128, 256, 512}) {
      const float t = time_candidate([&] { launch_batched_gemm(di, du, lay.nunits, thr, st); }, st);
      if (t < best) { best = t; plan->gemm_threads = thr; }
    }
    // the whole Jacobi phase: the lane-group kernel, or the block-cyclic one
    // with either CTA size for the widest class
    best = 1e30f;
    for (int cand = 0; cand < 3; ++cand) {
      const bool grp = cand == 0;
      const int thr = cand == 2 ? 256 : 128;
      const float t = time_candidate([&] {
        launch_batched_jacobi_narrow(di, du, n_narrow, plan->svd_vec_floats, grp, st);
        launch_batched_jacobi_mid(di, du + n_narrow, n_mid, plan->svd_vec_floats, grp, st);
        launch_batched_jacobi(di, du + n_narrow + n_mid, lay.nunits - n_narrow - n_mid, thr, plan->svd_vec_floats,
                              grp, st);
      }, st);
      if (t < best) {
        best = t;
        plan->svd_group = grp ? 1 : 0;
        plan->svd_threads = thr;
      }
    }
    WP_CUDA_TRY(cudaGetLastError());
  }
  return WP_OK;
}

extern "C" int wp_batched_run(const wp_batch_plan* plan, void* ws, void* stream) {
  if (!plan || !ws) return WP_ERR_NULL;
  if (plan->count < 1 || plan->n_units < 1) return WP_ERR_SHAPE;
  if (plan->svd_vec_floats < 1 || plan->svd_vec_floats > BMAX * BMAX) return WP_ERR_SHAPE;
  if (plan->svd_group != 0 && plan->svd_group != 1) return WP_ERR_SHAPE;
  if (plan->n_units_narrow < 0 || plan->n_units_mid < 0 ||
      plan->n_units_narrow + plan->n_units_mid > plan->n_units)
    return WP_ERR_SHAPE;
  char* base = static_cast<char*>(ws);
  cudaStream_t st = as_stream(stream);
  const BItem* di = reinterpret_cast<const BItem*>(base + plan->items_off);
  const int2* du = reinterpret_cast<const int2*>(base + plan->units_off);
  BatchFork* f = batch_fork();
  if (!f) return WP_ERR_CUDA;
  WP_TRY(launch_batched_lift(reinterpret_cast<const LiftDesc*>(base + plan->lift_fwd_off), plan->n_lift_fwd,
                             plan->lift_fwd_blocks, st));
  // the face-products (C_hat) and the Jacobi phases (C_r_hat) both read only
  // the lifted operands: the face-products go to the side stream
  WP_CUDA_TRY(cudaEventRecord(f->fork, st));
  WP_CUDA_TRY(cudaStreamWaitEvent(f->side, f->fork, 0));
  WP_TRY(launch_batched_gemm(di, du, plan->n_units, plan->gemm_threads, f->side));
  const int64_t nn = plan->n_units_narrow, nm = plan->n_units_mid;
  const bool grp = plan->svd_group != 0;
  WP_TRY(launch_batched_jacobi_narrow(di, du, nn, plan->svd_vec_floats, grp, st));
  WP_TRY(launch_batched_jacobi_mid(di, du + nn, nm, plan->svd_vec_floats, grp, st));
  WP_TRY(launch_batched_jacobi(di, du + nn + nm, plan->n_units - nn - nm, plan->svd_threads, plan->svd_vec_floats,
                               grp, st));
  WP_CUDA_TRY(cudaEventRecord(f->join, f->side));
  WP_CUDA_TRY(cudaStreamWaitEvent(st, f->join, 0));
  return launch_batched_lift(reinterpret_cast<const LiftDesc*>(base + plan->lift_inv_off), plan->n_lift_inv,
                             plan->lift_inv_blocks, st);
}
