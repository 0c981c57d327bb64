// Column-split register-resident one-sided Jacobi SVD of wavelet-domain
// frontal slices (Algorithm 2: the facewise "svd" of every A_{d_j}[:, :, k]
// and A_{s_L}[:, :, k]) for working matrices of at most 256 rows and 192..256
// columns (the 256 x 256 slices of the benchmark cube, and the R^T factors of
// the QR-preconditioned path), on clusters of CL = 2, 3 or 4 CTAs.  Same rotation formula, thresholds, stopping
// rule, outputs and error reporting as the block-cyclic kernel
// (jacobi_block.cuh); only the distribution of the slice differs.
//
// Distribution.  A cluster holds one slice.  The block-cyclic kernel splits
// the ROWS over the CTAs, so every column pair's dot product is a sum of
// partials that cross the cluster every round.  Here the COLUMNS are split:
// each CTA holds about n_pad / CL whole columns, 8 rows per lane (RPL = 8,
// 256 rows), in blocks of PPW = 4 columns; warp w holds a "top" and a
// "bottom" block.  Wider clusters add no per-round traffic (only more block
// transfers at the CTA boundaries) and put fewer warps on each SM, which
// shortens a round: the host runs full waves of 2-CTA clusters and spreads a
// remainder of slices (or a small batch) over 3 or 4 SMs per slice.  A round's 4 dot products per warp are then complete
// after one warp butterfly (no cluster traffic, no wait), and the rotation
// broadcast carries 4 pairs instead of 8.
//
// Ordering.  The same block tournament as the block-cyclic kernel over
// nb = n_pad / 4 block positions, on nb / 2 warps numbered across the
// cluster (CTA r holds warps r nb / (2 CL) .. (r + 1) nb / (2 CL) - 1).  A block move
// sends top blocks one warp up and bottom blocks one warp down, so a warp
// depends only on its two neighbours: inside a CTA each block goes through
// a mailbox slot guarded by a full / empty mbarrier pair (no CTA-wide
// barrier), and warps drift against each other by up to a move.  Exactly
// two blocks cross each CTA boundary per move (the top block of the lower
// CTA's last warp and the bottom block of the upper CTA's first warp).  Each
// goes straight into the neighbour's top or bottom inbox with st.async
// (16-byte vectors), completing transaction bytes on that inbox's mbarrier;
// the receiving warp waits for it (bounded) and re-arms it for the use after
// next.  Inboxes alternate by move, and an edge warp can only write its
// neighbour's inbox again after receiving the neighbour's next block, which
// the neighbour's edge warp sends after emptying that inbox.  Blocks are stored
// as 16-byte vectors of four rows, consecutive lanes 16 bytes apart
// (conflict-free).
//
// Column scales.  As in the block-cyclic kernel each rotation's cosine is
// deferred into per-column scales d (stored y = x / d, two FMAs per row
// pair); here the scales travel with their blocks, and a warp folds them
// into its rows only when one falls below 2^-10 (and at the start of every
// sweep), not at every block move.
//
// Per-sweep cluster agreement (the largest column norm for the
// numerically-zero rule, and whether any pair still rotated) goes through a
// DSMEM exchange and one cluster barrier each.

#include <atomic>
#include <mutex>

#include "jacobi_block.cuh"

namespace wp {
namespace jcols {

using jblock::arm_tx;
using jblock::circ;
using jblock::circ_pos;
using jblock::mapa_u32;
using jblock::st_async_f32;
using jblock::static_for;
using jblock::try_wait_cluster;
using jblock::wait_peers;

constexpr int NW = JAC_THREADS / 32;   // at most 16 warps per CTA
constexpr int kMaxCL = 4;
constexpr int PPW = 4;                 // columns per block
constexpr int RPL = 8;                 // rows per lane: 256 rows
constexpr int HALF = PPW / 2;
constexpr int LPP = 32 / PPW;          // lanes per lane group (one pair each)
constexpr int SHIFT = 3;               // lane >> SHIFT = lane group
constexpr int BLK = PPW * RPL * 32;    // floats per block (4 KB)
constexpr int INBOX = BLK + 2 * PPW;   // block, its norms, its scales
constexpr uint32_t kInboxBytes = INBOX * 4;
constexpr int kStagePitch = 32 * RPL + 1;   // staging column pitch (bank-conflict free)
constexpr float kFoldBelow = 1.f / 1024.f;
constexpr int kMaxRows = 32 * RPL;
constexpr int kMinPad = 192, kMaxPad = 2 * NW * 2 * PPW;   // 256

struct Layout {
  size_t mbar, full, empty, inbox, csa, red, xch, mnorm, mscale, norms, order, rank_of, mail, total;
};

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) / 16 * 16; }

__host__ __device__ constexpr Layout layout(int n_pad) {
  Layout L{};
  L.mbar = 0;                                                     // [2 sides][2] u64: inboxes
  L.full = L.mbar + 4 * 8;                                        // [2 NW] u64: slot filled
  L.empty = L.full + 2 * size_t(NW) * 8;                          // [2 NW] u64: slot emptied
  L.inbox = align16(L.empty + 2 * size_t(NW) * 8);                // [2 sides][2][INBOX]
  L.csa = align16(L.inbox + 4 * size_t(INBOX) * 4);               // [NW][2 PPW]
  L.red = L.csa + size_t(NW) * 2 * PPW * 4;                       // [NW]
  L.xch = L.red + size_t(NW) * 4;                                 // [2][kMaxCL]
  L.mnorm = L.xch + 2 * kMaxCL * 4;                               // [2 NW][PPW]
  L.mscale = L.mnorm + 2 * size_t(NW) * PPW * 4;                  // [2 NW][PPW]
  L.norms = L.mscale + 2 * size_t(NW) * PPW * 4;                  // [n_pad]
  L.order = L.norms + size_t(n_pad) * 4;                          // [n_pad]
  L.rank_of = L.order + size_t(n_pad) * 4;                        // [n_pad]
  L.mail = align16(L.rank_of + size_t(n_pad) * 4);                // mailboxes / staging
  const size_t mail = 2 * size_t(NW) * BLK * 4;
  const size_t stage = size_t(2 * NW * PPW) * kStagePitch * 4;   // up to 16 warps' columns
  L.total = L.mail + (mail > stage ? mail : stage);
  return L;
}

static __device__ __forceinline__ void st_async_v4(uint32_t remote_addr, float a, float b, float c, float d,
                                                   uint32_t remote_bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                   remote_addr),
               "r"(__float_as_uint(a)), "r"(__float_as_uint(b)), "r"(__float_as_uint(c)), "r"(__float_as_uint(d)),
               "r"(remote_bar)
               : "memory");
}

template <int CL>
__global__ void __launch_bounds__(JAC_THREADS, 1) jacobi_cols_kernel(JacobiArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Layout Ly = layout(a.n_pad);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw + Ly.mbar);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + Ly.full);
  uint64_t* empty = reinterpret_cast<uint64_t*>(smem_raw + Ly.empty);
  float* inbox = reinterpret_cast<float*>(smem_raw + Ly.inbox);
  float* csa = reinterpret_cast<float*>(smem_raw + Ly.csa);
  float* red = reinterpret_cast<float*>(smem_raw + Ly.red);
  float* xch = reinterpret_cast<float*>(smem_raw + Ly.xch);
  float* mnorm = reinterpret_cast<float*>(smem_raw + Ly.mnorm);
  float* mscale = reinterpret_cast<float*>(smem_raw + Ly.mscale);
  float* norms = reinterpret_cast<float*>(smem_raw + Ly.norms);
  int* order = reinterpret_cast<int*>(smem_raw + Ly.order);
  int* rank_of = reinterpret_cast<int*>(smem_raw + Ly.rank_of);
  float* mail = reinterpret_cast<float*>(smem_raw + Ly.mail);

  cg::cluster_group cluster = cg::this_cluster();
  const int rank = int(cluster.block_rank());
  const int slice = a.slice0 + int(blockIdx.x) / CL;
  const float* A = a.X + int64_t(slice) * a.n1 * a.n2;
  const int warp = int(threadIdx.x) >> 5, lane = int(threadIdx.x) & 31;
  const int g = lane >> SHIFT, sub = lane & (LPP - 1);
  const int nb = a.n_pad / PPW;   // block positions
  const int nwt = nb / 2;         // warps over the cluster
  const int start = rank * nwt / CL, end = (rank + 1) * nwt / CL;
  const int nwa = end - start;    // warps of this CTA (at least 6)
  const bool active = warp < nwa;
  const int W = start + warp;                          // warp number in the cluster
  const int topc = W * PPW, botc = (nb - 1 - W) * PPW; // first columns of its blocks

  // ---- stage this CTA's columns (two contiguous ranges), column-major with
  // an odd pitch: local column lc < nwa PPW is global topc0 + lc, the rest
  // are global botc0 + (lc - nwa PPW)
  const int nloc = 2 * nwa * PPW;
  const int topc0 = start * PPW, botc0 = (nb - end) * PPW;
  float* stg = mail;
  if (!a.trans) {
    for (int idx = threadIdx.x; idx < nloc * kMaxRows; idx += JAC_THREADS) {
      const int lc = idx % nloc, R = idx / nloc;
      const int c = lc < nwa * PPW ? topc0 + lc : botc0 + (lc - nwa * PPW);
      float v = 0.f;
      if (c < a.n_vec && R < a.m_len) v = A[int64_t(R) * a.n2 + c];
      stg[lc * kStagePitch + R] = v;
    }
  } else {
    for (int idx = threadIdx.x; idx < nloc * kMaxRows; idx += JAC_THREADS) {
      const int R = idx % kMaxRows, lc = idx / kMaxRows;
      const int c = lc < nwa * PPW ? topc0 + lc : botc0 + (lc - nwa * PPW);
      float v = 0.f;
      if (c < a.n_vec && R < a.m_len) v = A[int64_t(c) * a.n2 + R];
      stg[lc * kStagePitch + R] = v;
    }
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < 4; ++i) {   // top inboxes [0, 2), bottom inboxes [2, 4)
      ptx::mbar_init(&mbar[i], 1);
      arm_tx(ptx::smem_u32(&mbar[i]), kInboxBytes);
    }
    for (int i = 0; i < 2 * NW; ++i) {
      ptx::mbar_init(&full[i], 32);    // the posting warp's lanes
      ptx::mbar_init(&empty[i], 32);   // the fetching warp's lanes
    }
    ptx::fence_mbar_init();
  }
  __syncthreads();
  float T[PPW][RPL], B[PPW][RPL];
  {
    const int lt = warp * PPW, lb = nwa * PPW + (nwa - 1 - warp) * PPW;
#pragma unroll
    for (int j = 0; j < PPW; ++j) {
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        T[j][q] = active ? stg[(lt + j) * kStagePitch + lane + 32 * q] : 0.f;
        B[j][q] = active ? stg[(lb + j) * kStagePitch + lane + 32 * q] : 0.f;
      }
    }
  }
  // the peer's inbox barriers are initialised, and every staging read is
  // done before the mailboxes are reused
  cluster.sync();

  // the blocks that cross a CTA boundary per move: a CTA's last warp sends
  // its top block to the next CTA's top inbox and receives a bottom block
  // (edge0); a CTA's first warp sends its bottom block to the previous CTA's
  // bottom inbox and receives a top block (edge1)
  const bool edge0 = active && rank < CL - 1 && warp == nwa - 1;
  const bool edge1 = active && rank > 0 && warp == 0;
  const int nbr = edge0 ? rank + 1 : edge1 ? rank - 1 : rank;
  const uint32_t inbox_nbr = mapa_u32(ptx::smem_u32(inbox + (edge0 ? 0 : 2 * INBOX)), nbr);
  const uint32_t mbar_nbr = mapa_u32(ptx::smem_u32(mbar + (edge0 ? 0 : 2)), nbr);
  uint32_t mv = 0;      // block moves so far (same count on both CTAs)
  bool failed = false;  // a bounded wait ran out: stop waiting
  uint32_t xu = 0;      // cluster exchanges so far

  // largest of a CTA-uniform value over the cluster
  auto cluster_max = [&](float v) {
    const int s = int(xu & 1u) * kMaxCL;
    if (threadIdx.x < CL) cluster.map_shared_rank(xch, int(threadIdx.x))[s + rank] = v;
    cluster.sync();
    ++xu;
    float m = xch[s];
#pragma unroll
    for (int q = 1; q < CL; ++q) m = fmaxf(m, xch[s + q]);
    return m;
  };

  float nT = 0.f, nB = 0.f;   // squared norms of top column g / bottom column paired with it
  float dT = 1.f, dB = 1.f;   // their scales (x = d y)
  float* cs_w = csa + warp * 2 * PPW;

  auto fold = [&]() {
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
  };

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
    nT = multi_reduce<PPW>(st, lane);
    nB = multi_reduce<PPW>(sb, lane);
  };

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

  // block transfer helpers: local mailbox slot, or the peer's inbox.  Rows
  // 4h..4h+3 of column j of a lane sit at float offset ((j RPL/4 + h) 32 +
  // lane) 4 of the block.
  auto wait_bar = [&](uint64_t* bar, uint32_t parity) {
    if (!failed && !ptx::mbar_wait(bar, parity, a.status)) failed = true;
    failed = __any_sync(0xffffffffu, failed);   // one decision per warp
  };
  auto post = [&](const float (&X)[PPW][RPL], float nrm, float d, int slot) {
    if (mv > 0) wait_bar(&empty[slot], (mv - 1) & 1u);   // the previous block was fetched
    float* dst = mail + size_t(slot) * BLK;
#pragma unroll
    for (int j = 0; j < PPW; ++j)
#pragma unroll
      for (int h = 0; h < RPL / 4; ++h)
        *reinterpret_cast<float4*>(dst + ((j * (RPL / 4) + h) * 32 + lane) * 4) =
            make_float4(X[j][4 * h], X[j][4 * h + 1], X[j][4 * h + 2], X[j][4 * h + 3]);
    if (sub == 0) {
      mnorm[slot * PPW + g] = nrm;
      mscale[slot * PPW + g] = d;
    }
    ptx::mbar_arrive(&full[slot]);
  };
  auto unpack = [&](const float* src, float (&X)[PPW][RPL]) {
#pragma unroll
    for (int j = 0; j < PPW; ++j)
#pragma unroll
      for (int h = 0; h < RPL / 4; ++h) {
        const float4 v = *reinterpret_cast<const float4*>(src + ((j * (RPL / 4) + h) * 32 + lane) * 4);
        X[j][4 * h] = v.x;
        X[j][4 * h + 1] = v.y;
        X[j][4 * h + 2] = v.z;
        X[j][4 * h + 3] = v.w;
      }
  };
  auto fetch = [&](float (&X)[PPW][RPL], float& nrm, float& d, int slot) {
    wait_bar(&full[slot], mv & 1u);
    unpack(mail + size_t(slot) * BLK, X);
    nrm = mnorm[slot * PPW + g];
    d = mscale[slot * PPW + g];
    ptx::mbar_arrive(&empty[slot]);
  };
  auto send = [&](const float (&X)[PPW][RPL], float nrm, float d) {
    const uint32_t b = mv & 1u;
    const uint32_t dst = inbox_nbr + b * kInboxBytes, bar = mbar_nbr + 8u * b;
#pragma unroll
    for (int j = 0; j < PPW; ++j)
#pragma unroll
      for (int h = 0; h < RPL / 4; ++h)
        st_async_v4(dst + uint32_t(((j * (RPL / 4) + h) * 32 + lane) * 4) * 4u, X[j][4 * h], X[j][4 * h + 1],
                    X[j][4 * h + 2], X[j][4 * h + 3], bar);
    if (sub == 0) {
      st_async_f32(dst + uint32_t(BLK + g) * 4u, nrm, bar);
      st_async_f32(dst + uint32_t(BLK + PPW + g) * 4u, d, bar);
    }
  };
  // side 0: the top inbox (edge1 receives there), side 1: the bottom inbox (edge0)
  auto receive = [&](float (&X)[PPW][RPL], float& nrm, float& d, int side) {
    const uint32_t b = mv & 1u, parity = (mv >> 1) & 1u;
    const uint32_t bar = ptx::smem_u32(&mbar[2 * side + b]);
    if (!failed && !try_wait_cluster(bar, parity) && !wait_peers(bar, parity, a.status)) failed = true;
    failed = __any_sync(0xffffffffu, failed);   // one decision per warp
    const float* src = inbox + (2 * side + b) * INBOX;
    unpack(src, X);
    nrm = src[BLK + g];
    d = src[BLK + PPW + g];
    __syncwarp();
    if (lane == 0 && !failed) arm_tx(bar, kInboxBytes);
  };

  bool converged = false;
  int sweeps_done = 0;
  for (int sweep = 0; sweep < a.max_sweeps; ++sweep) {
    sweeps_done = sweep + 1;
    const float tol_eff = sweep < kStrictSweeps ? a.tol : 8.f * a.tol;
    const float tol2 = tol_eff * tol_eff;
    if (active) {
      fold();
      exact_norms();
    }
    // numerically zero columns (squared norm below (m eps)^2 |X|_max^2) are
    // not rotated
    float mx = active ? fmaxf(nT, nB) : 0.f;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, d));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    float cmax = 0.f;
#pragma unroll
    for (int w = 0; w < NW; ++w) cmax = fmaxf(cmax, red[w]);
    const float nmax = cluster_max(cmax);
    const float meps = float(a.m_len) * 1.1920929e-7f;
    const float negl = nmax * meps * meps;
    // stopping rule of the block-cyclic kernel: no cosine above tol, or none
    // above sqrt(tol) (the next sweep would find nothing above tol to rotate)
    tol2s = tol_eff;
    big = 0;

    if (active) {
      // every block meets itself (circle method inside the block)
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
        const float gam = multi_reduce<PPW>(acc, lane);
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
            float e0 = 0.f, e1 = 0.f;   // two chains of 4 instead of one of 8
#pragma unroll
            for (int q = 0; q < RPL; q += 2) {
              e0 = fmaf(T[j][q], B[(j + S) % PPW][q], e0);
              e1 = fmaf(T[j][q + 1], B[(j + S) % PPW][q + 1], e1);
            }
            acc[j] = e0 + e1;
          }
          const float gam = multi_reduce<PPW>(acc, lane) * (dT * dB);
          const float rba = __fdividef(dB, dT), rab = __fdividef(dT, dB);
          float c, s, t, ta = 0.f, tb = 0.f;
          if (angle(gam, nT, nB, negl, tol2, c, s, t)) {
            nT = fmaf(-t, gam, nT);
            nB = fmaf(t, gam, nB);
            ta = t * rba;
            tb = t * rab;
            dT *= c;
            dB *= c;
          }
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
        // keep the scales away from underflow
        if (__any_sync(0xffffffffu, dT < kFoldBelow || dB < kFoldBelow)) fold();
      }
      // block move: positions 1..nb-1 advance by one (position 0 stays)
      if (active) {
        if (W >= 1 && W <= nwt - 2) {
          if (edge0) send(T, nT, dT);
          else post(T, nT, dT, 2 * warp);
        }
        if (edge1) send(B, nB, dB);
        else post(B, nB, dB, 2 * warp + 1);
        if (W == nwt - 1) {
#pragma unroll
          for (int j = 0; j < PPW; ++j)
#pragma unroll
            for (int q = 0; q < RPL; ++q) B[j][q] = T[j][q];
          nB = nT;
          dB = dT;
        } else if (edge0) {
          receive(B, nB, dB, 1);
        } else {
          fetch(B, nB, dB, 2 * (warp + 1) + 1);
        }
        if (W >= 1) {
          if (edge1) receive(T, nT, dT, 0);
          else fetch(T, nT, dT, W == 1 ? 1 : 2 * (warp - 1));
        }
      }
      ++mv;
    }
    const int any_big = __syncthreads_or(big);
    if (cluster_max(any_big ? 1.f : 0.f) == 0.f) {
      converged = true;
      break;
    }
  }
  if (!converged && threadIdx.x == 0 && rank == 0) report_device_error(a.status, WP_ERR_NOT_CONVERGED);
  if (threadIdx.x == 0 && rank == 0 && a.stats) {
    atomicAdd(&a.stats[0], (unsigned long long)sweeps_done);
    atomicMax(&a.stats[1], (unsigned long long)sweeps_done);
  }

  // exact final norms of every column on both CTAs; rank them (ties by index)
  if (active) {
    fold();
    exact_norms();
    if (sub == 0) {
#pragma unroll
      for (int q = 0; q < CL; ++q) {
        float* nq = cluster.map_shared_rank(norms, q);
        nq[topc + g] = nT;
        nq[botc + g] = nB;
      }
    }
  }
  cluster.sync();
  for (int c = threadIdx.x; c < a.n_pad; c += JAC_THREADS) {
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
  float* vo = a.vec_out + int64_t(slice) * a.m_len * a.r;
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
          const int R = lane + 32 * q;
          if (R < a.m_len) vo[int64_t(R) * a.r + kq] = (side ? B[j][q] : T[j][q]) * inv;
        }
      }
    }
  }
  if (rank == 0)
    for (int kq = threadIdx.x; kq < a.r; kq += JAC_THREADS) a.sig_out[int64_t(slice) * a.r + kq] = sqrtf(norms[order[kq]]);
  // no CTA may leave while its peer can still read or write its shared memory
  cluster.sync();
}

static std::atomic<int> g_enabled{1};
static std::atomic<int> g_cluster{0};   // 0: automatic, else every launch on clusters of this size

// Clusters of CL CTAs that can be resident at once (0 if the query fails).
template <int CL>
int max_clusters() {
  static int cached = -1;
  if (cached >= 0) return cached;
  if (cudaFuncSetAttribute(jacobi_cols_kernel<CL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(layout(kMaxPad).total)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(CL * 64), 1, 1);
  cfg.blockDim = dim3(JAC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = layout(kMaxPad).total;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, jacobi_cols_kernel<CL>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  cached = n;
  return n;
}

// `timed`: bracket the launch for per-kernel timing (a pair of launches is
// timed as one span by launch_pair instead)
template <int CL>
int launch(const JacobiArgs& a, int nslices, cudaStream_t st, bool timed = true) {
  if (nslices <= 0) return WP_OK;
  if (max_clusters<CL>() <= 0) return WP_ERR_UNSUPPORTED;   // also sets the shared-memory attribute
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(nslices * CL), 1, 1);
  cfg.blockDim = dim3(JAC_THREADS, 1, 1);
  cfg.dynamicSmemBytes = layout(a.n_pad).total;
  cfg.stream = st;
  cudaLaunchAttribute attrs[1];
  attrs[0].id = cudaLaunchAttributeClusterDimension;
  attrs[0].val.clusterDim.x = CL;
  attrs[0].val.clusterDim.y = 1;
  attrs[0].val.clusterDim.z = 1;
  cfg.attrs = attrs;
  cfg.numAttrs = 1;
  if (timed) {
    WP_PROFILE("jacobi_svd", st);
    WP_CUDA_TRY(cudaLaunchKernelEx(&cfg, jacobi_cols_kernel<CL>, a));
  } else {
    WP_CUDA_TRY(cudaLaunchKernelEx(&cfg, jacobi_cols_kernel<CL>, a));
  }
  return launch_status();
}

static int launch_cl(int cl, const JacobiArgs& a, int nslices, cudaStream_t st, bool timed = true) {
  return cl == 4 ? launch<4>(a, nslices, st, timed)
                 : cl == 3 ? launch<3>(a, nslices, st, timed) : launch<2>(a, nslices, st, timed);
}

// Second stream and fork / join events of one device (created on first use,
// kept for the life of the process), for two launches of different cluster
// sizes that run side by side; the mutex keeps concurrent host threads from
// interleaving their record / wait pairs on the shared events.
struct Fork {
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  bool ok = false;
};
static std::mutex g_fork_mu;

static Fork* fork_of_device() {
  static Fork forks[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  Fork& f = forks[dev];
  if (!f.ok) {
    if (cudaStreamCreateWithFlags(&f.side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&f.join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    f.ok = true;
  }
  return &f;
}

// slices [slice0, slice0 + na) on clusters of cla CTAs on `st`, the next nb
// beside them on clusters of clb CTAs on the side stream
static int launch_pair(int cla, const JacobiArgs& a, int na, int clb, int nb, cudaStream_t st) {
  JacobiArgs b = a;
  b.slice0 = a.slice0 + na;
  std::lock_guard<std::mutex> lk(g_fork_mu);
  // one timed span on the call's stream, from before the fork to after the join
  WP_PROFILE("jacobi_svd", st);
  Fork* f = fork_of_device();
  if (!f) {   // no second stream: one after the other
    WP_TRY(launch_cl(cla, a, na, st, false));
    return launch_cl(clb, b, nb, st, false);
  }
  WP_CUDA_TRY(cudaEventRecord(f->fork, st));
  WP_CUDA_TRY(cudaStreamWaitEvent(f->side, f->fork, 0));
  WP_TRY(launch_cl(cla, a, na, st, false));
  WP_TRY(launch_cl(clb, b, nb, f->side, false));
  WP_CUDA_TRY(cudaEventRecord(f->join, f->side));
  WP_CUDA_TRY(cudaStreamWaitEvent(st, f->join, 0));
  return WP_OK;
}

}  // namespace jcols

bool jacobi_cols_fits(int m_len, int n_vec) {
  const int n_pad = (n_vec + 15) / 16 * 16;
  return m_len <= jcols::kMaxRows && n_pad >= jcols::kMinPad && n_pad <= jcols::kMaxPad;
}

bool jacobi_cols_enabled() { return jcols::g_enabled.load(std::memory_order_relaxed) != 0; }

// Cluster sizes.  A slice takes 1, 0.81 and 0.66 of its 2-CTA time on 2-,
// 3- and 4-CTA clusters (256 x 256 R^T factors on GB300), so 2-CTA clusters
// do the most work per SM and wider ones pay off where SMs would otherwise
// idle: (1) every slice in one wave of 4-CTA, else of 3-CTA clusters;
// (2) a wave of 3-CTA clusters plus the few slices beyond its capacity on
// 2-CTA clusters in the SMs it leaves, side by side; (3) full waves of
// 2-CTA clusters and, beside them on the second stream, the remainder on
// 3-CTA clusters (a last wave of a few 2-CTA clusters would leave most SMs
// idle for a whole slice time).  3- and 4-CTA clusters do not share the
// GPCs well (measured), so they are never paired.
int jacobi_cols_launch(const JacobiArgs& a0, int nslices, cudaStream_t st) {
  if (!jacobi_cols_fits(a0.m_len, a0.n_vec)) return WP_ERR_UNSUPPORTED;
  JacobiArgs a = a0;
  a.n_pad = (a0.n_vec + 15) / 16 * 16;
  a.rpc = a0.m_len;
  const int forced = jcols::g_cluster.load(std::memory_order_relaxed);
  if (forced) return jcols::launch_cl(forced, a, nslices, st);
  const int c2 = jcols::max_clusters<2>(), c3 = jcols::max_clusters<3>(), c4 = jcols::max_clusters<4>();
  if (c2 <= 0) return WP_ERR_UNSUPPORTED;
  if (nslices <= c4) return jcols::launch<4>(a, nslices, st);
  if (nslices <= c3) return jcols::launch<3>(a, nslices, st);
  const int spare2 = (sm_count() - 3 * c3) / 2;   // 2-CTA clusters beside a full wave of 3-CTA ones
  if (c3 > 0 && nslices <= c3 + spare2) return jcols::launch_pair(3, a, c3, 2, nslices - c3, st);
  const int full = nslices / c2 * c2, rest = nslices - full;
  if (rest == 0 || c3 <= 0 || rest > c3) return jcols::launch<2>(a, nslices, st);
  return jcols::launch_pair(2, a, full, 3, rest, st);
}

}  // namespace wp

extern "C" int wp_set_jacobi_column_split(int on) {
  if (on != 0 && on != 1) return WP_ERR_SHAPE;
  wp::jcols::g_enabled.store(on, std::memory_order_relaxed);
  return WP_OK;
}

extern "C" int wp_set_jacobi_cluster_size(int cl) {
  if (cl != 0 && (cl < 2 || cl > wp::jcols::kMaxCL)) return WP_ERR_SHAPE;
  wp::jcols::g_cluster.store(cl, std::memory_order_relaxed);
  return WP_OK;
}

extern "C" int wp_jacobi_cluster_capacity(int cl, int* clusters) {
  if (!clusters) return WP_ERR_NULL;
  switch (cl) {
    case 2: *clusters = wp::jcols::max_clusters<2>(); return WP_OK;
    case 3: *clusters = wp::jcols::max_clusters<3>(); return WP_OK;
    case 4: *clusters = wp::jcols::max_clusters<4>(); return WP_OK;
    default: return WP_ERR_SHAPE;
  }
}
