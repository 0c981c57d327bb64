// Batched one-sided Jacobi SVD of wavelet-domain frontal slices (Algorithm 2:
// "svd" of every A_{d_j}[:, :, k] and A_{s_L}[:, :, k]).
//
// One-sided (Hestenes) Jacobi orthogonalises the columns of the working
// matrix X (m_len x n_vec, m_len >= n_vec): for a column pair (a, b) with
// alpha = |x_a|^2, beta = |x_b|^2, gamma = x_a . x_b, the plane rotation
//   zeta = (beta - alpha) / (2 gamma),  t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
//   c = 1 / sqrt(1 + t^2),  s = c t,   x_a <- c x_a - s x_b,  x_b <- s x_a + c x_b
// makes the pair orthogonal; sweeps over all pairs converge to X = U Sigma
// (columns x_i = sigma_i u_i).  X is the slice itself when n1 >= n2 (giving
// U) or its transpose otherwise (giving V); the other factor and the rank-r
// reconstruction are recovered afterwards with small products (svd.cu).
//
// Parallel ordering: round-robin "circle" tournament, n_pad - 1 rounds of
// n_pad / 2 disjoint pairs per sweep.  A slice is held in shared memory,
// split by rows across a thread-block cluster of CL CTAs (CL = 1, 2, 4, 8);
// each warp owns pairs, computes its rows' partial dot product with lane
// strides and a shuffle reduction, and publishes the partial to every CTA of
// the cluster through distributed shared memory (double-buffered per round,
// one cluster barrier per round).  Every CTA then sums the partials in rank
// order -- bit-identical totals, hence identical rotation decisions across
// the cluster -- and rotates its own rows.  Column norms are tracked with
// alpha' = alpha - t gamma, beta' = beta + t gamma and recomputed exactly at
// the start of every sweep.  A sweep with no rotation above the threshold
// |gamma| > tol sqrt(alpha beta) ends the iteration; reaching max_sweeps sets
// WP_ERR_NOT_CONVERGED in the device status word (results are still written).
//
// The rotation angle is computed in FP32 with the stable formula above: on
// GB300 the FP64 pipe is ~64x slower than FP32, and the angle, being
// computed from FP32 inputs, gains nothing measurable from FP64.

#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.cuh"

namespace cg = cooperative_groups;

namespace wp {

constexpr int JAC_THREADS = 256;
constexpr int JAC_WARPS = JAC_THREADS / 32;

struct JacobiArgs {
  const float* X;      // slices (p, n1, n2)
  int n1, n2;
  int trans;           // 1: working columns are the rows of the slice
  int m_len, n_vec, n_pad, rpc;
  int slice0;          // first slice handled by this launch
  int r;
  float* vec_out;      // (p, m_len, r): leading r unit vectors, slice-indexed
  float* sig_out;      // (p, r): leading r singular values, descending
  float tol;
  int max_sweeps;
  int* status;
};

__device__ __forceinline__ void pair_of(int i, int k, int n, int& a, int& b) {
  // circle method: position 0 fixed, positions 1..n-1 rotate by k
  auto elem = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + k) % (n - 1); };
  a = elem(i);
  b = elem(n - 1 - i);
}

template <int CL>
__device__ __forceinline__ void cluster_barrier() {
  if constexpr (CL > 1) cg::this_cluster().sync();
  else __syncthreads();
}

// Publish `val` as this CTA's partial for entry i of buffer `buf`.
template <int CL>
__device__ __forceinline__ void publish(float* part, int buf, int rank, int n_pad, int i, float val, int lane) {
  float* local = part + (size_t(buf) * CL + rank) * n_pad + i;
  if constexpr (CL == 1) {
    if (lane == 0) *local = val;
  } else {
    if (lane < CL) {
      float* remote = cg::this_cluster().map_shared_rank(local, lane);
      *remote = val;
    }
  }
}

template <int CL>
__device__ __forceinline__ float gather(const float* part, int buf, int n_pad, int i) {
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < CL; ++q) s += part[(size_t(buf) * CL + q) * n_pad + i];
  return s;
}

template <int CL>
__global__ void __launch_bounds__(JAC_THREADS) jacobi_kernel(JacobiArgs a) {
  extern __shared__ float sm[];
  const int n_pad = a.n_pad, rpc = a.rpc;
  float* Xs = sm;                                     // [n_pad][rpc], column-major
  float* norms = Xs + size_t(n_pad) * rpc;            // [n_pad]
  float* part = norms + n_pad;                        // [2][CL][n_pad]
  int* order = reinterpret_cast<int*>(part + 2 * CL * n_pad);   // [n_pad]
  __shared__ int rot_count;

  const int rank = (CL > 1) ? int(cg::this_cluster().block_rank()) : 0;
  const int slice = a.slice0 + int(blockIdx.x) / CL;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const float* A = a.X + int64_t(slice) * a.n1 * a.n2;
  const int row0 = rank * rpc;

  // load this CTA's rows of the working matrix (zero padding rows / column)
  for (int idx = threadIdx.x; idx < n_pad * rpc; idx += JAC_THREADS) {
    const int c = idx / rpc, rr = idx % rpc, R = row0 + rr;
    float v = 0.f;
    if (c < a.n_vec && R < a.m_len) v = a.trans ? A[int64_t(c) * a.n2 + R] : A[int64_t(R) * a.n2 + c];
    Xs[idx] = v;
  }
  __syncthreads();

  auto exact_norms = [&](int buf) {
    for (int c = warp; c < n_pad; c += JAC_WARPS) {
      const float* col = Xs + size_t(c) * rpc;
      float s = 0.f;
      for (int rr = lane; rr < rpc; rr += 32) s = fmaf(col[rr], col[rr], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      publish<CL>(part, buf, rank, n_pad, c, s, lane);
    }
    cluster_barrier<CL>();
    for (int c = threadIdx.x; c < n_pad; c += JAC_THREADS) norms[c] = gather<CL>(part, buf, n_pad, c);
    __syncthreads();
  };

  int buf = 0;
  bool converged = false;
  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    exact_norms(buf);
    buf ^= 1;
    if (threadIdx.x == 0) rot_count = 0;
    __syncthreads();
    for (int k = 0; k < n_pad - 1; ++k) {
      // partial dot products of this CTA's rows
      for (int i = warp; i < n_pad / 2; i += JAC_WARPS) {
        int ca, cb;
        pair_of(i, k, n_pad, ca, cb);
        const float* xa = Xs + size_t(ca) * rpc;
        const float* xb = Xs + size_t(cb) * rpc;
        float g = 0.f;
        for (int rr = lane; rr < rpc; rr += 32) g = fmaf(xa[rr], xb[rr], g);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
        publish<CL>(part, buf, rank, n_pad, i, g, lane);
      }
      cluster_barrier<CL>();
      // identical rotation decisions on every CTA; each rotates its own rows
      int local_rot = 0;
      for (int i = warp; i < n_pad / 2; i += JAC_WARPS) {
        int ca, cb;
        pair_of(i, k, n_pad, ca, cb);
        const float g = gather<CL>(part, buf, n_pad, i);
        const float al = norms[ca], be = norms[cb];
        if (g != 0.f && fabsf(g) > a.tol * sqrtf(al) * sqrtf(be)) {
          const float zeta = (be - al) / (2.f * g);
          const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
          const float c = rsqrtf(fmaf(t, t, 1.f));
          const float s = c * t;
          float* xa = Xs + size_t(ca) * rpc;
          float* xb = Xs + size_t(cb) * rpc;
          for (int rr = lane; rr < rpc; rr += 32) {
            const float u = xa[rr], v = xb[rr];
            xa[rr] = fmaf(c, u, -s * v);
            xb[rr] = fmaf(s, u, c * v);
          }
          __syncwarp();
          if (lane == 0) {
            norms[ca] = fmaf(-t, g, al);
            norms[cb] = fmaf(t, g, be);
          }
          ++local_rot;
        }
      }
      if (lane == 0 && local_rot) atomicAdd(&rot_count, local_rot);
      buf ^= 1;
      __syncthreads();
    }
    __syncthreads();
    const int rc = rot_count;
    __syncthreads();
    if (rc == 0) { converged = true; break; }
  }
  if (!converged && threadIdx.x == 0 && rank == 0) report_device_error(a.status, WP_ERR_NOT_CONVERGED);

  // exact final norms -> singular values; rank columns (ties by index)
  exact_norms(buf);
  buf ^= 1;
  for (int c = threadIdx.x; c < a.n_vec; c += JAC_THREADS) {
    const float sc = norms[c];
    int pos = 0;
    for (int q = 0; q < a.n_vec; ++q) {
      const float sq = norms[q];
      pos += (sq > sc) || (sq == sc && q < c);
    }
    if (pos < a.r) order[pos] = c;
  }
  __syncthreads();
  float* vo = a.vec_out + int64_t(slice) * a.m_len * a.r;
  for (int idx = threadIdx.x; idx < a.r * rpc; idx += JAC_THREADS) {
    const int kq = idx / rpc, rr = idx % rpc, R = row0 + rr;
    if (R >= a.m_len) continue;
    const int c = order[kq];
    const float sg = sqrtf(norms[c]);
    vo[int64_t(R) * a.r + kq] = sg > 0.f ? Xs[size_t(c) * rpc + rr] / sg : 0.f;
  }
  if (rank == 0)
    for (int kq = threadIdx.x; kq < a.r; kq += JAC_THREADS)
      a.sig_out[int64_t(slice) * a.r + kq] = sqrtf(norms[order[kq]]);
  // no CTA may leave while a peer can still write into its shared memory
  cluster_barrier<CL>();
}

static size_t jacobi_smem(int n_pad, int rpc, int CL) {
  return (size_t(n_pad) * rpc + n_pad + 2 * size_t(CL) * n_pad) * sizeof(float) + size_t(n_pad) * sizeof(int);
}

constexpr size_t JAC_SMEM_MAX = 200 * 1024;

// Pick the cluster size: the smallest that fits shared memory, grown (while
// every CTA keeps at least 32 rows) until the launch has >= 4 CTAs per SM.
static int pick_cluster(int m_len, int n_pad, int nslices) {
  int chosen = -1;
  for (int CL = 1; CL <= 8; CL *= 2) {
    const int rpc = (m_len + CL - 1) / CL;
    if (jacobi_smem(n_pad, rpc, CL) > JAC_SMEM_MAX) continue;
    if (chosen > 0 && rpc < 32) break;
    chosen = CL;
    if (int64_t(nslices) * CL >= 4 * int64_t(sm_count())) break;
  }
  return chosen;
}

template <int CL>
static int launch_jacobi(const JacobiArgs& args, int nslices, size_t smem, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    WP_CUDA_TRY(cudaFuncSetAttribute(jacobi_kernel<CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     int(JAC_SMEM_MAX + 4096)));
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(nslices * CL), 1, 1);
  cfg.blockDim = dim3(JAC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attrs[1];
  attrs[0].id = cudaLaunchAttributeClusterDimension;
  attrs[0].val.clusterDim.x = CL;
  attrs[0].val.clusterDim.y = 1;
  attrs[0].val.clusterDim.z = 1;
  cfg.attrs = attrs;
  cfg.numAttrs = 1;
  WP_PROFILE("jacobi_svd", st);
  WP_CUDA_TRY(cudaLaunchKernelEx(&cfg, jacobi_kernel<CL>, args));
  return launch_status();
}

// Leading r singular triplets of slices [slice0, slice0 + nslices) of X
// (p, n1, n2).  Writes unit vectors (p, max(n1,n2), r) -- left vectors when
// n1 >= n2, right vectors otherwise -- and singular values (p, r).
int jacobi_svd(const float* X, int n1, int n2, int slice0, int nslices, int r, float* vec_out, float* sig_out,
               cudaStream_t st) {
  if (nslices <= 0) return WP_OK;
  JacobiArgs a{};
  a.X = X;
  a.n1 = n1;
  a.n2 = n2;
  a.trans = (n1 < n2) ? 1 : 0;
  a.m_len = a.trans ? n2 : n1;
  a.n_vec = a.trans ? n1 : n2;
  a.n_pad = a.n_vec + (a.n_vec & 1);
  if (a.n_pad < 2) a.n_pad = 2;
  a.slice0 = slice0;
  a.r = r;
  a.vec_out = vec_out;
  a.sig_out = sig_out;
  a.tol = 2.f * sqrtf(float(std::max(a.m_len, 16))) * 1.1920929e-7f;
  a.max_sweeps = 40;
  a.status = device_status_ptr();
  const int CL = pick_cluster(a.m_len, a.n_pad, nslices);
  if (CL < 0) return WP_ERR_UNSUPPORTED;
  a.rpc = (a.m_len + CL - 1) / CL;
  const size_t smem = jacobi_smem(a.n_pad, a.rpc, CL);
  switch (CL) {
    case 1: return launch_jacobi<1>(a, nslices, smem, st);
    case 2: return launch_jacobi<2>(a, nslices, smem, st);
    case 4: return launch_jacobi<4>(a, nslices, smem, st);
    default: return launch_jacobi<8>(a, nslices, smem, st);
  }
}

bool jacobi_supported(int n1, int n2) {
  const int m_len = std::max(n1, n2), n_vec = std::min(n1, n2);
  const int n_pad = std::max(2, n_vec + (n_vec & 1));
  return pick_cluster(m_len, n_pad, 1) > 0;
}

}  // namespace wp
