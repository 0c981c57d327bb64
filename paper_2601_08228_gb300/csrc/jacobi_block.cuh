// Block-cyclic register-resident one-sided Jacobi kernel (see jacobi_block.cu
// for the ordering and the cluster reduction).  Instantiated once per
// cluster size in jacobi_block_cl{1,2,4,8}.cu so that they compile in
// parallel.
#pragma once

#include <utility>

#include "common.cuh"
#include "internal.cuh"
#include "jacobi_common.cuh"
#include "tc_ptx.cuh"

namespace wp {
namespace jblock {

static __device__ __forceinline__ uint32_t mapa_u32(uint32_t addr, int cta) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(cta));
  return r;
}

static __device__ __forceinline__ void st_async_f32(uint32_t remote_addr, float v, uint32_t remote_bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(remote_addr),
               "r"(__float_as_uint(v)), "r"(remote_bar)
               : "memory");
}

static __device__ __forceinline__ void arm_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

static __device__ __forceinline__ bool try_wait_cluster(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred P;\n"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 P, [%1], %2;\n"
      "selp.b32 %0, 1, 0, P;\n"
      "}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the peers' partials; WP_ERR_TIMEOUT after limit_ns (2 s).
static __device__ __noinline__ bool wait_peers(uint32_t bar, uint32_t parity, int* status,
                                               uint64_t limit_ns = ptx::kWaitLimitNs) {
  const uint64_t t0 = ptx::globaltimer();
  while (!try_wait_cluster(bar, parity)) {
    if (ptx::globaltimer() - t0 > limit_ns) {
      report_device_error(status, WP_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

template <typename F, int... I>
__device__ __forceinline__ void static_for_impl(F& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}

// f(integral_constant<int, 0>), ..., f(integral_constant<int, N - 1>)
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// Circle method on P players, round k: the player at position pos.
template <int P>
__host__ __device__ constexpr int circ(int pos, int k) {
  return pos == 0 ? 0 : 1 + (pos - 1 + k) % (P - 1);
}

// Position of player h in round k (inverse of circ).
template <int P>
__device__ __forceinline__ int circ_pos(int h, int k) {
  if (h == 0) return 0;
  int q = (h - 1 - k) % (P - 1);
  q += (q < 0) ? (P - 1) : 0;
  return 1 + q;
}

constexpr int kBlockWarps = JAC_THREADS / 32;

// A lane's RPL values of one column, contiguous in shared memory (16-byte
// accesses for RPL = 4: conflict-free, consecutive lanes 16 bytes apart).
template <int RPL>
__device__ __forceinline__ void store_row(float* p, const float (&x)[RPL]) {
  if constexpr (RPL == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
  } else if constexpr (RPL == 2) {
    *reinterpret_cast<float2*>(p) = make_float2(x[0], x[1]);
  } else {
#pragma unroll
    for (int q = 0; q < RPL; ++q) p[q] = x[q];
  }
}

template <int RPL>
__device__ __forceinline__ void load_row(const float* p, float (&x)[RPL]) {
  if constexpr (RPL == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
  } else if constexpr (RPL == 2) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    x[0] = v.x; x[1] = v.y;
  } else {
#pragma unroll
    for (int q = 0; q < RPL; ++q) x[q] = p[q];
  }
}

// Shared-memory layout: mbarriers [NW][2] | rotations (c, s) [NW][PPW] |
// partials [NW][2][CL][PPW] |
// warp maxima [NW] | block norms in transit [NW][2][PPW] | norms [n_pad] |
// order [n_pad] | rank_of [n_pad] | (16-byte aligned) block mailboxes
// [NW][2][PPW][32][RPL], which first stage the input slice.
template <int CL, int PPW, int NW = kBlockWarps>
__host__ __device__ constexpr size_t block_mail_offset(int n_pad) {
  return ((size_t(16) * NW + sizeof(float) * size_t(NW) * 2 * PPW +
           sizeof(float) * (size_t(NW) * 2 * CL * PPW + NW + size_t(NW) * 2 * PPW + n_pad) +
           sizeof(int) * 2 * size_t(n_pad)) +
          15) /
         16 * 16;
}

template <int CL, int PPW, int RPL, int NW = kBlockWarps>
__host__ __device__ constexpr size_t block_smem(int n_pad) {
  return block_mail_offset<CL, PPW, NW>(n_pad) + sizeof(float) * size_t(n_pad) * 32 * RPL;
}

// Rank-ordered cluster total of a per-pair partial (lane group g holds pair
// g).  Buffer rnd & 1 of this warp's partial slots [2][CL][PPW] receives the
// peers' values; its mbarrier was armed for them one use earlier and is
// re-armed here for the use after next -- the peers can only send that after
// this warp's next partials, which follow this point.  Lane sub of a group
// sends the group's partial to peers sub, sub + 32 / PPW, ...
template <int CL, int PPW>
struct PeerSum {
  static constexpr int LPP = 32 / PPW;
  static constexpr int NSEND = (CL + LPP - 1) / LPP;
  uint32_t bar;                 // this warp's mbarrier pair (local)
  const float* part;            // this warp's partial slots (local)
  uint32_t rdst[NSEND > 0 ? NSEND : 1], rbar[NSEND > 0 ? NSEND : 1];   // peer addresses, buffer 0
  bool send[NSEND > 0 ? NSEND : 1];
  uint32_t rnd;
  bool failed;

  __device__ __forceinline__ void init(uint32_t bar_w, const float* part_w, int rank, int g, int sub) {
    bar = bar_w;
    part = part_w;
    rnd = 0;
    failed = false;
    const uint32_t mine = ptx::smem_u32(part_w + rank * PPW + g);
#pragma unroll
    for (int k = 0; k < NSEND; ++k) {
      const int q = sub + k * LPP;
      send[k] = q < CL && q != rank;
      rdst[k] = send[k] ? mapa_u32(mine, q) : 0u;
      rbar[k] = send[k] ? mapa_u32(bar_w, q) : 0u;
    }
  }

  __device__ __forceinline__ float total(float v, int rank, int g, int lane, int* status) {
    if constexpr (CL == 1) {
      return v;
    } else {
      const uint32_t b = rnd & 1u, parity = (rnd >> 1) & 1u;
      const uint32_t mbar = bar + 8u * b;
      if (!failed) {
#pragma unroll
        for (int k = 0; k < NSEND; ++k)
          if (send[k]) st_async_f32(rdst[k] + b * (CL * PPW * 4), v, rbar[k] + 8u * b);
        if (!try_wait_cluster(mbar, parity) && !wait_peers(mbar, parity, status)) failed = true;
      }
      const float* src = part + b * (CL * PPW) + g;
      float s;
      if constexpr (CL == 2) {
        s = v + src[(rank ^ 1) * PPW];   // a + b == b + a: identical on both CTAs
      } else {
        s = 0.f;
#pragma unroll
        for (int q = 0; q < CL; ++q) s += (q == rank) ? v : src[q * PPW];
      }
      __syncwarp();
      if (lane == 0 && !failed) arm_tx(mbar, (CL - 1) * PPW * 4);
      ++rnd;
      return s;
    }
  }
};

// One slice on a cluster of CL CTAs of NW warps: A is the slice (n1 x n2,
// row-major), this CTA holds working rows [rank * rpc, (rank + 1) * rpc);
// writes the leading r unit vectors to vo (m_len x r, row-major; any
// memory space) and, from rank 0, the r singular values to so (if not
// null).  GRID: the slice is a.slice0 + blockIdx.x / CL of a.X, the outputs
// its rows of a.vec_out and a.sig_out (A, vo, so unused; the addresses are
// formed where they are used, which keeps them out of the sweep loop's
// registers).  Uses the first block_smem<CL, PPW, RPL, NW>(a.n_pad) bytes of
// the kernel's dynamic shared memory.  Ends with a cluster-wide barrier.
template <int CL, int PPW, int RPL, int NW, bool GRID>
__device__ __forceinline__ void block_jacobi_slice(const JacobiArgs& a, const float* A_in, int rank_in,
                                                   float* vo_in, float* so_in) {
  // the kernel's dynamic shared memory, from offset 0
  extern __shared__ __align__(16) unsigned char smem_raw[];
  static_assert(PPW >= 2 && PPW <= 16 && (PPW & (PPW - 1)) == 0, "PPW: 2, 4, 8 or 16");
  static_assert(2 * PPW * RPL <= 64, "register budget: 2 PPW RPL <= 64 values per lane");
  constexpr int NTH = NW * 32;
  constexpr int LPP = 32 / PPW;
  constexpr int SHIFT = (PPW == 2) ? 4 : (PPW == 4) ? 3 : (PPW == 8) ? 2 : 1;
  constexpr int HALF = PPW / 2;
  constexpr int BLK = PPW * RPL * 32;
  const int n_pad = a.n_pad, rpc = a.rpc;
  const int nb = n_pad / PPW, nw = nb / 2;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw);           // [NW][2]
  float* csa = reinterpret_cast<float*>(mbar + 2 * NW);             // [NW][PPW][2]
  float* part = csa + NW * 2 * PPW;                                 // [NW][2][CL][PPW]
  float* red = part + NW * 2 * CL * PPW;                            // [NW]
  float* mnorm = red + NW;                                          // [NW][2][PPW]
  float* norms = mnorm + NW * 2 * PPW;                              // [n_pad]
  int* order = reinterpret_cast<int*>(norms + n_pad);               // [n_pad]
  int* rank_of = order + n_pad;                                     // [n_pad]
  float* mail = reinterpret_cast<float*>(smem_raw + block_mail_offset<CL, PPW, NW>(n_pad));

  const int rank = GRID ? ((CL > 1) ? int(cg::this_cluster().block_rank()) : 0) : rank_in;
  const int slice = GRID ? a.slice0 + int(blockIdx.x) / CL : 0;
  const float* A = GRID ? a.X + int64_t(slice) * a.n1 * a.n2 : A_in;
  const int warp = int(threadIdx.x) >> 5, lane = int(threadIdx.x) & 31;
  const int g = lane >> SHIFT, sub = lane & (LPP - 1);
  const bool active = warp < nw;
  const int row0 = rank * rpc;
  const int topc = warp * PPW, botc = (nb - 1 - warp) * PPW;

  // stage the CTA's rows of the working matrix, column-major, in the mailboxes
  float* Xs = mail;
  for (int idx = threadIdx.x; idx < n_pad * rpc; idx += NTH) {
    const int c = idx / rpc, rr = idx % rpc, R = row0 + rr;
    float v = 0.f;
    if (c < a.n_vec && R < a.m_len) v = a.trans ? A[int64_t(c) * a.n2 + R] : A[int64_t(R) * a.n2 + c];
    Xs[idx] = v;
  }
  if (CL > 1 && threadIdx.x == 0) {
    for (int i = 0; i < 2 * NW; ++i) ptx::mbar_init(&mbar[i], 1);
    for (int i = 0; i < 2 * NW; ++i) arm_tx(ptx::smem_u32(&mbar[i]), (CL - 1) * PPW * 4);
    ptx::fence_mbar_init();
  }
  __syncthreads();
  float T[PPW][RPL], B[PPW][RPL];
#pragma unroll
  for (int j = 0; j < PPW; ++j) {
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const int rr = lane + 32 * q;
      const bool in = active && rr < rpc;
      T[j][q] = in ? Xs[size_t(topc + j) * rpc + rr] : 0.f;
      B[j][q] = in ? Xs[size_t(botc + j) * rpc + rr] : 0.f;
    }
  }
  // peers' mbarriers are armed, and the staging reads finish before the
  // mailboxes are reused
  cluster_barrier<CL>();

  float* cs_w = csa + warp * 2 * PPW;
  PeerSum<CL, PPW> peers;
  peers.init(ptx::smem_u32(mbar + 2 * warp), part + warp * 2 * CL * PPW, rank, g, sub);
  auto total = [&](float v) { return peers.total(v, rank, g, lane, a.status); };

  // squared norms held by lane group g: top column g, and the bottom column
  // currently paired with it ((g + s) mod PPW in column round s)
  float nT = 0.f, nB = 0.f;
  // scales d of the same columns (stored y = x / d): the inter-block rounds
  // defer each rotation's cosine into them; 1 again at every block move
  float dT = 1.f, dB = 1.f;
  auto exact_norms = [&]() {
    float st[PPW], sb[PPW];
#pragma unroll
    for (int j = 0; j < PPW; ++j) {
      st[j] = sb[j] = 0.f;
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        st[j] = fmaf(T[j][q], T[j][q], st[j]);
        sb[j] = fmaf(B[j][q], B[j][q], sb[j]);
      }
    }
    const float pt = multi_reduce<PPW>(st, lane);
    const float pb = multi_reduce<PPW>(sb, lane);
    nT = total(pt);
    nB = total(pb);
  };

  // plane rotation of the lane group's pair; false when below threshold
  // threshold |gamma| > tol sqrt(alpha beta), tested on squares; the angle
  // from the fast reciprocal and reciprocal square root (a few ulp in t
  // changes how far the pair is orthogonalised, not the orthogonality of
  // the rotation: c = 1 / sqrt(1 + t^2), s = c t)
  // `big` records a pair whose cosine exceeds the stopping bound tol2s of
  // the sweep (see the sweep loop)
  int big = 0;
  float tol2s = 0.f;
  auto angle = [&](float gam, float al, float be, float negl, float tol2, float& c, float& s, float& t) {
    const float ab = al * be;
    if (al > negl && be > negl && gam * gam > tol2s * ab) big = 1;
    if (al > negl && be > negl && gam * gam > tol2 * ab) {
      const float zeta = __fdividef(be - al, 2.f * gam);
      const float az = fminf(fabsf(zeta), 1e18f);
      const float h = fmaf(az, az, 1.f);
      t = copysignf(__fdividef(1.f, az + h * rsqrtf(h)), zeta);
      c = rsqrtf(fmaf(t, t, 1.f));
      s = c * t;
      return true;
    }
    c = 1.f;
    s = 0.f;
    t = 0.f;
    return false;
  };

  // plane rotation with the cosine deferred to the column scales
  auto shear = [&](float (&X)[RPL], float (&Y)[RPL], float ta, float tb) {
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const float u = X[q], v = Y[q];
      X[q] = fmaf(-ta, v, u);
      Y[q] = fmaf(tb, u, v);
    }
  };

  auto rotate = [&](float (&X)[RPL], float (&Y)[RPL], float c, float s) {
#pragma unroll
    for (int q = 0; q < RPL; ++q) {
      const float u = X[q], v = Y[q];
      X[q] = fmaf(c, u, -s * v);
      Y[q] = fmaf(s, u, c * v);
    }
  };

  bool converged = false;
  int sweeps_done = 0;
  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    sweeps_done = sweep + 1;
    // after kStrictSweeps the threshold is relaxed 8x (rounding noise in the
    // cosine of nearly orthogonal small columns can sit at the strict one)
    const float tol_eff = sweep < kStrictSweeps ? a.tol : 8.f * a.tol;
    const float tol2 = tol_eff * tol_eff;
    if (active) exact_norms();
    // a column whose squared norm is below (m eps)^2 |X|_max^2 is
    // numerically zero and is not rotated (rank-deficient slices converge)
    float mx = active ? fmaxf(nT, nB) : 0.f;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, d));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    float nmax = 0.f;
#pragma unroll
    for (int w = 0; w < NW; ++w) nmax = fmaxf(nmax, red[w]);
    const float meps = float(a.m_len) * 1.1920929e-7f;
    const float negl = nmax * meps * meps;
    // Stopping rule.  A sweep in which no pair's cosine |gamma| / sqrt(alpha
    // beta) reaches tol ends the iteration.  Jacobi converges quadratically
    // near the end, so a sweep whose largest cosine stays below sqrt(tol)
    // leaves cosines of order tol: it ends the iteration too, without the
    // confirming sweep that would find (next to) nothing to rotate.
    tol2s = tol_eff;
    big = 0;

    if (active) {
      // every block meets itself: circle method inside the block, top block
      // pairs in lane groups [0, HALF), bottom block pairs in [HALF, PPW)
      static_for<PPW - 1>([&](auto K_) {
        constexpr int K = decltype(K_)::value;
        float acc[PPW];
#pragma unroll
        for (int i = 0; i < HALF; ++i) {
          const int pa = circ<PPW>(i, K), pb = circ<PPW>(PPW - 1 - i, K);
          acc[i] = acc[i + HALF] = 0.f;
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            acc[i] = fmaf(T[pa][q], T[pb][q], acc[i]);
            acc[i + HALF] = fmaf(B[pa][q], B[pb][q], acc[i + HALF]);
          }
        }
        const float gam = total(multi_reduce<PPW>(acc, lane));
        const int i = g & (HALF - 1);
        const bool top = g < HALF;
        const int la = circ<PPW>(i, K) << SHIFT, lb = circ<PPW>(PPW - 1 - i, K) << SHIFT;
        const float aT = __shfl_sync(0xffffffffu, nT, la), aB = __shfl_sync(0xffffffffu, nB, la);
        const float bT = __shfl_sync(0xffffffffu, nT, lb), bB = __shfl_sync(0xffffffffu, nB, lb);
        float al = top ? aT : aB, be = top ? bT : bB;
        float c, s, t;
        if (angle(gam, al, be, negl, tol2, c, s, t)) {
          al = fmaf(-t, gam, al);
          be = fmaf(t, gam, be);
        }
#pragma unroll
        for (int i2 = 0; i2 < HALF; ++i2) {
          const int pa = circ<PPW>(i2, K), pb = circ<PPW>(PPW - 1 - i2, K);
          const float cT = __shfl_sync(0xffffffffu, c, i2 << SHIFT);
          const float sT = __shfl_sync(0xffffffffu, s, i2 << SHIFT);
          if (sT != 0.f) rotate(T[pa], T[pb], cT, sT);
          const float cB = __shfl_sync(0xffffffffu, c, (i2 + HALF) << SHIFT);
          const float sB = __shfl_sync(0xffffffffu, s, (i2 + HALF) << SHIFT);
          if (sB != 0.f) rotate(B[pa], B[pb], cB, sB);
        }
        // updated norms back to the groups that own the columns
        const int ph = circ_pos<PPW>(g, K);
        const int ih = ph < HALF ? ph : PPW - 1 - ph;
        const bool first = ph < HALF;
        const float tA = __shfl_sync(0xffffffffu, al, ih << SHIFT);
        const float tB = __shfl_sync(0xffffffffu, be, ih << SHIFT);
        const float uA = __shfl_sync(0xffffffffu, al, (ih + HALF) << SHIFT);
        const float uB = __shfl_sync(0xffffffffu, be, (ih + HALF) << SHIFT);
        nT = first ? tA : tB;
        nB = first ? uA : uB;
      });
    }

    for (int o = 0; o < nb - 1; ++o) {
      if (active) {
        static_for<PPW>([&](auto S_) {
          constexpr int S = decltype(S_)::value;
          float acc[PPW];
#pragma unroll
          for (int j = 0; j < PPW; ++j) {
            acc[j] = 0.f;
#pragma unroll
            for (int q = 0; q < RPL; ++q) acc[j] = fmaf(T[j][q], B[(j + S) % PPW][q], acc[j]);
          }
          // stored columns are x = d y: the dot product of the x's
          const float gam = total(multi_reduce<PPW>(acc, lane)) * (dT * dB);
          // scale ratios, off the angle's dependency chain
          const float rba = __fdividef(dB, dT), rab = __fdividef(dT, dB);
          float c, s, t, ta = 0.f, tb = 0.f;
          if (angle(gam, nT, nB, negl, tol2, c, s, t)) {
            nT = fmaf(-t, gam, nT);
            nB = fmaf(t, gam, nB);
              // x_a' = c (x_a - t x_b), x_b' = c (x_b + t x_a) with the cosine
            // moved into the scales: y_a -= t (d_b / d_a) y_b, y_b += t (d_a / d_b) y_a
            ta = t * rba;
            tb = t * rab;
            dT *= c;
            dB *= c;
          }
          // broadcast the PPW rotations through shared memory
          __syncwarp();
          if (sub == 0) *reinterpret_cast<float2*>(cs_w + 2 * g) = make_float2(ta, tb);
          __syncwarp();
#pragma unroll
          for (int j = 0; j < PPW; j += 2) {
            const float4 r2 = *reinterpret_cast<const float4*>(cs_w + 2 * j);
            if (r2.x != 0.f) shear(T[j], B[(j + S) % PPW], r2.x, r2.y);
            if (r2.z != 0.f) shear(T[j + 1], B[(j + 1 + S) % PPW], r2.z, r2.w);
          }
          // the bottom block advances one column relative to the top one
          nB = __shfl_sync(0xffffffffu, nB, (lane + LPP) & 31);
          dB = __shfl_sync(0xffffffffu, dB, (lane + LPP) & 31);
        });
      }
      if (active) {
        // fold the column scales into the stored rows (d = 1 again)
        __syncwarp();
        if (sub == 0) *reinterpret_cast<float2*>(cs_w + 2 * g) = make_float2(dT, dB);
        __syncwarp();
#pragma unroll
        for (int j = 0; j < PPW; ++j) {
          const float2 d = *reinterpret_cast<const float2*>(cs_w + 2 * j);
#pragma unroll
          for (int q = 0; q < RPL; ++q) {
            T[j][q] *= d.x;
            B[j][q] *= d.y;
          }
        }
        dT = dB = 1.f;
      }
      // block move: positions 1..nb-1 advance by one (position 0 stays):
      // top of warp w -> top of w + 1 (last warp: its own bottom), bottom of
      // w -> bottom of w - 1 (warp 0: top of warp 1)
      __syncthreads();
      if (active && nw > 1) {
        auto post = [&](const float (&X)[PPW][RPL], float nrm, int slot) {
          float* dst = mail + size_t(slot) * BLK;
#pragma unroll
          for (int j = 0; j < PPW; ++j) store_row<RPL>(dst + (j * 32 + lane) * RPL, X[j]);
          if (sub == 0) mnorm[slot * PPW + g] = nrm;
        };
        if (warp >= 1 && warp <= nw - 2) post(T, nT, 2 * warp);
        post(B, nB, 2 * warp + 1);
      }
      __syncthreads();
      if (active && nw > 1) {
        auto fetch = [&](float (&X)[PPW][RPL], float& nrm, int slot) {
          const float* src = mail + size_t(slot) * BLK;
#pragma unroll
          for (int j = 0; j < PPW; ++j) load_row<RPL>(src + (j * 32 + lane) * RPL, X[j]);
          nrm = mnorm[slot * PPW + g];
        };
        if (warp == nw - 1) {
#pragma unroll
          for (int j = 0; j < PPW; ++j)
#pragma unroll
            for (int q = 0; q < RPL; ++q) B[j][q] = T[j][q];
          nB = nT;
        } else {
          fetch(B, nB, 2 * (warp + 1) + 1);
        }
        if (warp >= 1) fetch(T, nT, warp == 1 ? 1 : 2 * (warp - 1));
      }
    }
    if (!__syncthreads_or(big)) {
      converged = true;
      break;
    }
  }
  if (!converged && threadIdx.x == 0 && rank == 0) report_device_error(a.status, WP_ERR_NOT_CONVERGED);
  if (threadIdx.x == 0 && rank == 0 && a.stats) {
    atomicAdd(&a.stats[0], (unsigned long long)sweeps_done);
    atomicMax(&a.stats[1], (unsigned long long)sweeps_done);
  }

  // exact final norms -> singular values; rank the columns (ties by index)
  if (active) {
    exact_norms();
    if (sub == 0) {
      norms[topc + g] = nT;
      norms[botc + g] = nB;
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < n_pad; c += NTH) {
    int pos = a.r;
    if (c < a.n_vec) {
      const float sc = norms[c];
      pos = 0;
      for (int q = 0; q < a.n_vec; ++q) {
        const float sq = norms[q];
        pos += (sq > sc) || (sq == sc && q < c);
      }
      if (pos < a.r) order[pos] = c;
    }
    rank_of[c] = pos < a.r ? pos : -1;
  }
  __syncthreads();
  float* vo = GRID ? a.vec_out + int64_t(slice) * a.m_len * a.r : vo_in;
  if (active) {
#pragma unroll
    for (int j = 0; j < PPW; ++j) {
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int c = (side ? botc : topc) + j;
        const int kq = rank_of[c];
        if (kq < 0) continue;
        const float sg = sqrtf(norms[c]);
        const float inv = sg > 0.f ? 1.f / sg : 0.f;
#pragma unroll
        for (int q = 0; q < RPL; ++q) {
          const int rr = lane + 32 * q, R = row0 + rr;
          if (rr < rpc && R < a.m_len) vo[int64_t(R) * a.r + kq] = (side ? B[j][q] : T[j][q]) * inv;
        }
      }
    }
  }
  float* so = GRID ? a.sig_out + int64_t(slice) * a.r : so_in;
  if (rank == 0 && so)
    for (int kq = threadIdx.x; kq < a.r; kq += NTH) so[kq] = sqrtf(norms[order[kq]]);
  // no CTA may leave while a peer can still write into its shared memory
  cluster_barrier<CL>();
}

template <int CL, int PPW, int RPL>
__global__ void __launch_bounds__(JAC_THREADS, 1) jacobi_block_kernel(JacobiArgs a) {
  block_jacobi_slice<CL, PPW, RPL, kBlockWarps, true>(a, nullptr, 0, nullptr, nullptr);
}

template <int CL, int PPW, int RPL>
int launch_block(const JacobiArgs& a, int nslices, cudaStream_t st) {
  const size_t smem = block_smem<CL, PPW, RPL>(a.n_pad);
  if (smem > 227 * 1024) return WP_ERR_UNSUPPORTED;
  static bool attr = false;
  if (!attr) {
    WP_CUDA_TRY(cudaFuncSetAttribute(jacobi_block_kernel<CL, PPW, RPL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     227 * 1024));
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
  WP_CUDA_TRY(cudaLaunchKernelEx(&cfg, jacobi_block_kernel<CL, PPW, RPL>, a));
  return launch_status();
}

template <int CL, int PPW>
int launch_block_rpl(const JacobiArgs& a, int nslices, int rpl, cudaStream_t st) {
  if (rpl == 1) return launch_block<CL, PPW, 1>(a, nslices, st);
  if (rpl == 2) return launch_block<CL, PPW, 2>(a, nslices, st);
  if constexpr (PPW <= 8) {
    if (rpl == 4) return launch_block<CL, PPW, 4>(a, nslices, st);
  }
  return WP_ERR_UNSUPPORTED;
}

template <int CL>
int launch_block_ppw(const JacobiArgs& a, int nslices, int ppw, int rpl, cudaStream_t st) {
  switch (ppw) {
    case 2: return launch_block_rpl<CL, 2>(a, nslices, rpl, st);
    case 4: return launch_block_rpl<CL, 4>(a, nslices, rpl, st);
    case 8: return launch_block_rpl<CL, 8>(a, nslices, rpl, st);
    case 16: return launch_block_rpl<CL, 16>(a, nslices, rpl, st);
    default: return WP_ERR_UNSUPPORTED;
  }
}

}  // namespace jblock
}  // namespace wp

#define WP_JACOBI_BLOCK_INSTANTIATE(CLV) \
  template int wp::jblock::launch_block_ppw<CLV>(const wp::JacobiArgs&, int, int, int, cudaStream_t);
