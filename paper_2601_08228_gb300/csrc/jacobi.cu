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
// Two kernels share these definitions.  The block-cyclic register-resident
// kernel (jacobi_block.cu) takes every slice with more than 32 columns whose
// rows fit in registers on at most 8 CTAs; the shared-memory kernel below
// takes the rest (narrow slices, very tall ones).  The register-resident
// kernels also end the iteration after a sweep whose largest cosine stays
// below sqrt(tol): by the quadratic convergence of the method the next sweep
// would leave cosines of order tol, so it is not run.
//
// Shared-memory kernel.  Parallel ordering: round-robin "circle" tournament,
// n_pad - 1 rounds of n_pad / 2 disjoint pairs per sweep.  A slice is held in
// shared memory,
// split by rows across a thread-block cluster of CL CTAs (CL = 1, 2, 4, 8);
// each warp computes its pairs' partial dot products over the CTA's rows, and publishes the partial to every CTA of
// the cluster through distributed shared memory (double-buffered per round,
// one cluster barrier per round).  Every CTA then sums the partials in rank
// order -- bit-identical totals, hence identical rotation decisions across
// the cluster -- and rotates its own rows.  Within a CTA a warp owns up to 8
// pairs of a round: its lanes sweep consecutive rows (no shared-memory bank
// conflicts), the pairs are independent instruction streams, and one
// multi-value butterfly reduces all of them.  Column norms are tracked with
// alpha' = alpha - t gamma, beta' = beta + t gamma and recomputed exactly at
// the start of every sweep.  A sweep with no rotation above the threshold
// |gamma| > tol sqrt(alpha beta) (tol = 2 sqrt(m_len) eps, relaxed 8x after
// 20 sweeps) ends the iteration; reaching max_sweeps sets
// WP_ERR_NOT_CONVERGED in the device status word (results are still written).
//
// The rotation angle is computed in FP32 with the stable formula above: on
// GB300 the FP64 pipe is ~64x slower than FP32, and the angle, being
// computed from FP32 inputs, gains nothing measurable from FP64.

#include <atomic>

#include "common.cuh"
#include "internal.cuh"
#include "jacobi_common.cuh"

namespace wp {

// One warp owns PPW column pairs of a round; its 32 lanes sweep consecutive
// rows (conflict-free shared-memory access) and the PPW pairs form
// independent instruction streams.  RPL rows per lane per chunk.
template <int CL, int PPW, int RPL>
__global__ void __launch_bounds__(JAC_THREADS) jacobi_kernel(JacobiArgs a) {
  extern __shared__ float sm[];
  const int n_pad = a.n_pad, rpc = a.rpc, npairs = n_pad / 2;
  float* Xs = sm;                                     // [n_pad][rpc], column-major
  float* norms = Xs + size_t(n_pad) * rpc;            // [n_pad]
  float* part = norms + n_pad;                        // [2][CL][n_pad]
  int* order = reinterpret_cast<int*>(part + 2 * CL * n_pad);   // [n_pad]
  constexpr int NW = JAC_THREADS / 32;
  constexpr int LPP = 32 / PPW;                       // lanes holding one pair's total
  constexpr int SHIFT = (PPW == 1) ? 5 : (PPW == 2) ? 4 : (PPW == 4) ? 3 : (PPW == 8) ? 2 : 1;

  const int rank = (CL > 1) ? int(cg::this_cluster().block_rank()) : 0;
  const int slice = a.slice0 + int(blockIdx.x) / CL;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const float* A = a.X + int64_t(slice) * a.n1 * a.n2;
  const int row0 = rank * rpc;

  for (int idx = threadIdx.x; idx < n_pad * rpc; idx += JAC_THREADS) {
    const int c = idx / rpc, rr = idx % rpc, R = row0 + rr;
    float v = 0.f;
    if (c < a.n_vec && R < a.m_len) v = a.trans ? A[int64_t(c) * a.n2 + R] : A[int64_t(R) * a.n2 + c];
    Xs[idx] = v;
  }
  __syncthreads();

  // publish the warp's PPW totals: lane l holds entry `base + (l >> SHIFT) * stride`
  auto publish_warp = [&](int buf, float total, int first, int stride, int limit) {
    const int j = lane >> SHIFT;
    const int e = first + j * stride;
    if (e < limit) {
      for (int q = lane & (LPP - 1); q < CL; q += LPP) {
        float* local = part + (size_t(buf) * CL + rank) * n_pad + e;
        if constexpr (CL == 1) *local = total;
        else *cg::this_cluster().map_shared_rank(local, q) = total;
      }
    }
  };

  auto exact_norms = [&](int buf) {
    // warp w handles columns w + NW * (j + PPW * it)
    for (int base = 0; base < n_pad; base += NW * PPW) {
      float acc[PPW];
#pragma unroll
      for (int j = 0; j < PPW; ++j) {
        acc[j] = 0.f;
        const int c = base + warp + j * NW;
        if (c < n_pad) {
          const float* col = Xs + size_t(c) * rpc;
          for (int rr = lane; rr < rpc; rr += 32) acc[j] = fmaf(col[rr], col[rr], acc[j]);
        }
      }
      const float t = multi_reduce<PPW>(acc, lane);
      publish_warp(buf, t, base + warp, NW, n_pad);
    }
    cluster_barrier<CL>();
    for (int c = threadIdx.x; c < n_pad; c += JAC_THREADS) norms[c] = gather<CL>(part, buf, n_pad, c);
    __syncthreads();
  };

  int buf = 0;
  bool converged = false;
  int sweeps_done = 0;
  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    sweeps_done = sweep + 1;
    // after kStrictSweeps the threshold is relaxed 8x: rounding noise in the
    // FP32 cosine of nearly orthogonal small columns can sit at the strict
    // threshold and keep a slice rotating forever
    const float tol_eff = sweep < kStrictSweeps ? a.tol : 8.f * a.tol;
    exact_norms(buf);
    buf ^= 1;
    // a column whose squared norm is below (m eps)^2 |X|_max^2 is numerically
    // zero: its direction is rounding noise, so its pairs are not rotated
    // (otherwise a rank-deficient slice would never converge)
    float nmax = 0.f;
    for (int c = 0; c < n_pad; ++c) nmax = fmaxf(nmax, norms[c]);
    const float meps = float(a.m_len) * 1.1920929e-7f;
    const float negligible = nmax * meps * meps;
    int rotated_sweep = 0;
    for (int k = 0; k < n_pad - 1; ++k) {
      int rotated = 0;
      for (int base = 0; base < npairs; base += NW * PPW) {
        // ---- partial dot products of this CTA's rows, PPW independent chains
        int ca[PPW], cb[PPW];
        float acc[PPW];
#pragma unroll
        for (int j = 0; j < PPW; ++j) {
          const int i = base + warp + j * NW;
          acc[j] = 0.f;
          ca[j] = cb[j] = 0;
          if (i < npairs) pair_of(i, k, n_pad, ca[j], cb[j]);
        }
        // RPL > 0: the pair's rows stay in registers from the dot product to
        // the rotation (4 shared-memory accesses per element pair, not 6)
        float ru[PPW][RPL > 0 ? RPL : 1], rv[PPW][RPL > 0 ? RPL : 1];
        if constexpr (RPL > 0) {
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            const int rr = lane + 32 * q;
#pragma unroll
            for (int j = 0; j < PPW; ++j) {
              const bool in = rr < rpc;
              ru[j][q] = in ? Xs[size_t(ca[j]) * rpc + rr] : 0.f;
              rv[j][q] = in ? Xs[size_t(cb[j]) * rpc + rr] : 0.f;
              acc[j] = fmaf(ru[j][q], rv[j][q], acc[j]);
            }
          }
        } else {
          for (int rr = lane; rr < rpc; rr += 32) {
#pragma unroll
            for (int j = 0; j < PPW; ++j)
              acc[j] = fmaf(Xs[size_t(ca[j]) * rpc + rr], Xs[size_t(cb[j]) * rpc + rr], acc[j]);
          }
        }
        const float tot = multi_reduce<PPW>(acc, lane);
        publish_warp(buf, tot, base + warp, NW, npairs);
        cluster_barrier<CL>();
        // ---- rotation: lane quad of pair j computes its angle, then broadcast
        const int jm = lane >> SHIFT;
        const int im = base + warp + jm * NW;
        float cm = 1.f, sm_ = 0.f;
        if (im < npairs) {
          int xa, xb;
          pair_of(im, k, n_pad, xa, xb);
          const float g = gather<CL>(part, buf, n_pad, im);
          const float al = norms[xa], be = norms[xb];
          if (g != 0.f && al > negligible && be > negligible && fabsf(g) > tol_eff * sqrtf(al * be)) {
            // stable angle; c^2 + s^2 = 1 holds whatever the rounding of t
            const float zeta = __fdividef(be - al, 2.f * g);
            const float t = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
            cm = rsqrtf(fmaf(t, t, 1.f));
            sm_ = cm * t;
            rotated = 1;
            if ((lane & (LPP - 1)) == 0) {
              norms[xa] = fmaf(-t, g, al);
              norms[xb] = fmaf(t, g, be);
            }
          }
        }
        float cj[PPW], sj[PPW];
#pragma unroll
        for (int j = 0; j < PPW; ++j) {
          cj[j] = __shfl_sync(0xffffffffu, cm, j << SHIFT);
          sj[j] = __shfl_sync(0xffffffffu, sm_, j << SHIFT);
        }
        if constexpr (RPL > 0) {
#pragma unroll
          for (int j = 0; j < PPW; ++j) {
            if (sj[j] != 0.f) {
#pragma unroll
              for (int q = 0; q < RPL; ++q) {
                const int rr = lane + 32 * q;
                if (rr < rpc) {
                  const float u = ru[j][q], v = rv[j][q];
                  Xs[size_t(ca[j]) * rpc + rr] = fmaf(cj[j], u, -sj[j] * v);
                  Xs[size_t(cb[j]) * rpc + rr] = fmaf(sj[j], u, cj[j] * v);
                }
              }
            }
          }
        } else {
          for (int rr = lane; rr < rpc; rr += 32) {
#pragma unroll
            for (int j = 0; j < PPW; ++j) {
              if (sj[j] != 0.f) {
                float* xa = Xs + size_t(ca[j]) * rpc + rr;
                float* xb = Xs + size_t(cb[j]) * rpc + rr;
                const float u = *xa, v = *xb;
                *xa = fmaf(cj[j], u, -sj[j] * v);
                *xb = fmaf(sj[j], u, cj[j] * v);
              }
            }
          }
        }
        buf ^= 1;
        if (base + NW * PPW < npairs) __syncthreads();
      }
      rotated_sweep |= __syncthreads_or(rotated);
    }
    if (!rotated_sweep) { converged = true; break; }
  }
  if (!converged && threadIdx.x == 0 && rank == 0) report_device_error(a.status, WP_ERR_NOT_CONVERGED);
  if (threadIdx.x == 0 && rank == 0 && a.stats) {
    atomicAdd(&a.stats[0], (unsigned long long)sweeps_done);
    atomicMax(&a.stats[1], (unsigned long long)sweeps_done);
  }

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

// Pick the cluster size: the smallest that fits the slice in shared memory.
// A round is latency-bound (two barriers and a short dependency chain), so
// splitting a slice over more CTAs barely shortens it while multiplying the
// CTAs that must be resident; measured on 256 x 256 slices, 2-CTA clusters
// finish 192 slices twice as fast as 4-CTA clusters.
static int pick_cluster(int m_len, int n_pad, int /*nslices*/) {
  for (int CL = 1; CL <= 8; CL *= 2) {
    const int rpc = (m_len + CL - 1) / CL;
    if (jacobi_smem(n_pad, rpc, CL) <= JAC_SMEM_MAX) return CL;
  }
  return -1;
}

template <int CL, int PPW, int RPL>
static int launch_jacobi(const JacobiArgs& args, int nslices, size_t smem, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    WP_CUDA_TRY(cudaFuncSetAttribute(jacobi_kernel<CL, PPW, RPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
  WP_CUDA_TRY(cudaLaunchKernelEx(&cfg, jacobi_kernel<CL, PPW, RPL>, args));
  return launch_status();
}

template <int CL, int PPW>
static int launch_jacobi_rpl(const JacobiArgs& args, int nslices, size_t smem, cudaStream_t st) {
  // rows per lane kept in registers (RPL * PPW * 2 values); 0 = reload path
  const int rpl = (args.rpc + 31) / 32;
  if (rpl <= 1) return launch_jacobi<CL, PPW, 1>(args, nslices, smem, st);
  if (rpl <= 2) return launch_jacobi<CL, PPW, 2>(args, nslices, smem, st);
  if (rpl <= 4 && PPW <= 8) return launch_jacobi<CL, PPW, 4>(args, nslices, smem, st);
  return launch_jacobi<CL, PPW, 0>(args, nslices, smem, st);
}

template <int CL>
static int launch_jacobi_lg(const JacobiArgs& args, int nslices, size_t smem, cudaStream_t st) {
  // pairs per warp: enough that one pass covers a round (at most 8)
  const int npairs = args.n_pad / 2;
  const int nw = JAC_THREADS / 32;
  if (npairs <= nw) return launch_jacobi_rpl<CL, 1>(args, nslices, smem, st);
  if (npairs <= 2 * nw) return launch_jacobi_rpl<CL, 2>(args, nslices, smem, st);
  if (npairs <= 4 * nw) return launch_jacobi_rpl<CL, 4>(args, nslices, smem, st);
  return launch_jacobi_rpl<CL, 8>(args, nslices, smem, st);
}

// Leading r singular triplets of slices [slice0, slice0 + nslices) of X
// (p, n1, n2).  Writes unit vectors (p, max(n1,n2), r) -- left vectors when
// n1 >= n2, right vectors otherwise -- and singular values (p, r).
int jacobi_svd(const float* X, int n1, int n2, int slice0, int nslices, int r, float* vec_out, float* sig_out,
               cudaStream_t st, void* work, size_t work_bytes) {
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
  a.max_sweeps = jacobi_max_sweeps();
  a.status = device_status_ptr();
  a.stats = jacobi_stats_ptr();
  // block-cyclic register-resident kernel where the slice shape suits it
  {
    const int rc = jacobi_block_launch(a, nslices, st);
    if (rc != WP_ERR_UNSUPPORTED) return rc;
  }
  const int CL = pick_cluster(a.m_len, a.n_pad, nslices);
  if (CL < 0) return jacobi_global_launch(a, nslices, work, work_bytes, st);
  a.rpc = (a.m_len + CL - 1) / CL;
  const size_t smem = jacobi_smem(a.n_pad, a.rpc, CL);
  switch (CL) {
    case 1: return launch_jacobi_lg<1>(a, nslices, smem, st);
    case 2: return launch_jacobi_lg<2>(a, nslices, smem, st);
    case 4: return launch_jacobi_lg<4>(a, nslices, smem, st);
    default: return launch_jacobi_lg<8>(a, nslices, smem, st);
  }
}

static __device__ unsigned long long g_jacobi_stats[2];
static std::atomic<int> g_jacobi_max_sweeps{kJacobiMaxSweeps};

int jacobi_max_sweeps() { return g_jacobi_max_sweeps.load(std::memory_order_relaxed); }

unsigned long long* jacobi_stats_ptr() {
  static unsigned long long* cached[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (!cached[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_jacobi_stats) != cudaSuccess) return nullptr;
    cached[dev] = static_cast<unsigned long long*>(p);
  }
  return cached[dev];
}

// The cluster kernels take the slice when it fits in the shared memory of an
// 8-CTA cluster (the block-cyclic kernel's register shapes are a subset).
static bool cluster_fits(int n1, int n2) {
  const int m_len = std::max(n1, n2), n_vec = std::min(n1, n2);
  const int n_pad = std::max(2, n_vec + (n_vec & 1));
  return pick_cluster(m_len, n_pad, 1) > 0;
}

bool jacobi_supported(int n1, int n2) { return cluster_fits(n1, n2) || jacobi_global_supported(n1, n2); }

size_t jacobi_work_bytes(int n1, int n2, int nslices) {
  return cluster_fits(n1, n2) ? 0 : jacobi_global_work_bytes(n1, n2, nslices);
}

static std::atomic<int> g_jacobi_precondition{1};

bool jacobi_preconditioned(int n1, int n2) {
  const int m_len = std::max(n1, n2), n_vec = std::min(n1, n2);
  return g_jacobi_precondition.load(std::memory_order_relaxed) != 0 && n_vec >= 32 && qr_supported(m_len, n_vec) &&
         cluster_fits(n_vec, n_vec);
}

}  // namespace wp

extern "C" int wp_set_jacobi_max_sweeps(int max_sweeps) {
  if (max_sweeps < 1 || max_sweeps > 1000) return WP_ERR_SHAPE;
  wp::g_jacobi_max_sweeps.store(max_sweeps, std::memory_order_relaxed);
  return WP_OK;
}

extern "C" int wp_set_jacobi_precondition(int on) {
  if (on != 0 && on != 1) return WP_ERR_SHAPE;
  wp::g_jacobi_precondition.store(on, std::memory_order_relaxed);
  return WP_OK;
}

extern "C" int wp_jacobi_stats(int64_t* total_sweeps, int* max_sweeps) {
  if (!total_sweeps || !max_sweeps) return WP_ERR_NULL;
  unsigned long long* p = wp::jacobi_stats_ptr();
  if (!p) return WP_ERR_CUDA;
  unsigned long long h[2] = {0, 0};
  if (cudaDeviceSynchronize() != cudaSuccess) return WP_ERR_CUDA;
  if (cudaMemcpy(h, p, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return WP_ERR_CUDA;
  const unsigned long long z[2] = {0, 0};
  if (cudaMemcpy(p, z, sizeof(z), cudaMemcpyHostToDevice) != cudaSuccess) return WP_ERR_CUDA;
  *total_sweeps = int64_t(h[0]);
  *max_sweeps = int(h[1]);
  return WP_OK;
}
