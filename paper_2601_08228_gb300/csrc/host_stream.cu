// w-product of host-resident tensors with the copies overlapped with the
// compute (Def. 2.1, Algorithm 1): chunks of whole tube groups flow through
// a three-stage pipeline -- host-to-device copy, wp_wprod, device-to-host
// copy -- on three streams, with three device buffers per operand (with two,
// the copy of chunk k + 1 would wait for the product and the copy back of
// chunk k - 1, which share the host link with it and take longer).

#include "common.cuh"
#include "internal.cuh"

namespace wp {
namespace {

constexpr int kBufs = 3;

// Streams and events of one device's pipeline (created on first use, kept
// for the life of the process).
struct HostPipe {
  cudaStream_t h2d = nullptr, comp = nullptr, d2h = nullptr;
  cudaEvent_t loaded[kBufs] = {};   // chunk's A, B on the device
  cudaEvent_t done[kBufs] = {};     // chunk's C computed
  cudaEvent_t freed[kBufs] = {};    // chunk's C copied back: buffers reusable
  cudaEvent_t start = nullptr, end = nullptr;
  bool ready = false;
};

HostPipe* host_pipe() {
  static HostPipe pipes[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  HostPipe& hp = pipes[dev];
  if (!hp.ready) {
    const unsigned sf = cudaStreamNonBlocking, ef = cudaEventDisableTiming;
    if (cudaStreamCreateWithFlags(&hp.h2d, sf) != cudaSuccess || cudaStreamCreateWithFlags(&hp.comp, sf) != cudaSuccess ||
        cudaStreamCreateWithFlags(&hp.d2h, sf) != cudaSuccess)
      return nullptr;
    for (int b = 0; b < kBufs; ++b)
      if (cudaEventCreateWithFlags(&hp.loaded[b], ef) != cudaSuccess ||
          cudaEventCreateWithFlags(&hp.done[b], ef) != cudaSuccess ||
          cudaEventCreateWithFlags(&hp.freed[b], ef) != cudaSuccess)
        return nullptr;
    if (cudaEventCreateWithFlags(&hp.start, ef) != cudaSuccess || cudaEventCreateWithFlags(&hp.end, ef) != cudaSuccess)
      return nullptr;
    hp.ready = true;
  }
  return &hp;
}

// Largest chunk (slices): the request, else ~p / 4; whole tube groups.
int64_t chunk_of(int64_t p, int L, int64_t req) {
  const int64_t G = int64_t(1) << L;
  int64_t cs = req > 0 ? req : (p + 3) / 4;
  cs = (cs + G - 1) / G * G;
  return cs < p ? cs : p;
}

// Slices of chunk k starting at slice s0.  A request gives uniform chunks.
// The default ramps: one tube group first (the device starts computing after
// a short copy) and one last (the final copy back is short), chunks of about
// p / 4 in between.
int64_t chunk_at(int64_t p, int L, int64_t req, int64_t k, int64_t s0) {
  const int64_t G = int64_t(1) << L;
  const int64_t cs = chunk_of(p, L, req);
  int64_t ns;
  if (req > 0 || p <= 4 * G) {
    ns = cs;
  } else if (k == 0 || p - s0 <= G) {
    ns = G;
  } else {
    ns = cs < p - s0 - G ? cs : p - s0 - G;   // leave the last group for the last chunk
  }
  return ns < p - s0 ? ns : p - s0;
}

void host_layout(int64_t n1, int64_t n2, int64_t n4, int64_t cs, size_t wsz, Sizer& s) {
  for (int b = 0; b < kBufs; ++b) {
    s.take<float>(size_t(cs) * n1 * n2);
    s.take<float>(size_t(cs) * n2 * n4);
    s.take<float>(size_t(cs) * n1 * n4);
  }
  s.take<char>(wsz);
}

}  // namespace
}  // namespace wp

using namespace wp;

extern "C" int wp_wprod_host_workspace(int64_t n1, int64_t n2, int64_t n4, int64_t p, int L, int prec,
                                       int64_t chunk_slices, size_t* bytes) {
  if (!bytes) return WP_ERR_NULL;
  if (n1 < 1 || n2 < 1 || n4 < 1 || p < 1 || chunk_slices < 0) return WP_ERR_SHAPE;
  if (L < 0 || L > WP_MAX_LEVELS || (p % (int64_t(1) << L)) != 0) return WP_ERR_LEVELS;
  if (chunk_slices > 0 && chunk_slices % (int64_t(1) << L) != 0) return WP_ERR_SHAPE;
  const int64_t cs = chunk_of(p, L, chunk_slices);
  size_t wsz = 0;
  WP_TRY(wp_wprod_workspace(n1, n2, n4, cs, L, prec, &wsz));
  Sizer s;
  host_layout(n1, n2, n4, cs, wsz, s);
  *bytes = s.bytes();
  return WP_OK;
}

extern "C" int wp_wprod_host(const float* A, const float* B, float* C, int64_t n1, int64_t n2, int64_t n4,
                             int64_t p, int L, int prec, int64_t chunk_slices, void* ws, size_t ws_bytes,
                             void* stream) {
  if (!A || !B || !C) return WP_ERR_NULL;
  size_t need = 0;
  WP_TRY(wp_wprod_host_workspace(n1, n2, n4, p, L, prec, chunk_slices, &need));
  if (!ws || ws_bytes < need) return WP_ERR_WORKSPACE;
  const int64_t cs = chunk_of(p, L, chunk_slices);
  size_t wsz = 0;
  WP_TRY(wp_wprod_workspace(n1, n2, n4, cs, L, prec, &wsz));
  Carver cv(ws, ws_bytes);
  float* Ad[kBufs];
  float* Bd[kBufs];
  float* Cd[kBufs];
  for (int b = 0; b < kBufs; ++b) {
    Ad[b] = cv.take<float>(size_t(cs) * n1 * n2);
    Bd[b] = cv.take<float>(size_t(cs) * n2 * n4);
    Cd[b] = cv.take<float>(size_t(cs) * n1 * n4);
  }
  void* wprod_ws = cv.take<char>(wsz);
  if (!cv.ok) return WP_ERR_WORKSPACE;
  HostPipe* hp = host_pipe();
  if (!hp) return WP_ERR_CUDA;
  cudaStream_t caller = as_stream(stream);
  WP_CUDA_TRY(cudaEventRecord(hp->start, caller));
  WP_CUDA_TRY(cudaStreamWaitEvent(hp->h2d, hp->start, 0));
  WP_CUDA_TRY(cudaStreamWaitEvent(hp->comp, hp->start, 0));
  WP_CUDA_TRY(cudaStreamWaitEvent(hp->d2h, hp->start, 0));
  const size_t pa = size_t(n1) * n2, pb = size_t(n2) * n4, pc = size_t(n1) * n4;   // floats per slice
  for (int64_t k = 0, s0 = 0, ns = 0; s0 < p; ++k, s0 += ns) {
    const int b = int(k % kBufs);
    ns = chunk_at(p, L, chunk_slices, k, s0);
    // stage 1: the buffers of chunk k - kBufs are free once its C is back
    if (k >= kBufs) WP_CUDA_TRY(cudaStreamWaitEvent(hp->h2d, hp->freed[b], 0));
    WP_CUDA_TRY(cudaMemcpyAsync(Ad[b], A + size_t(s0) * pa, size_t(ns) * pa * sizeof(float), cudaMemcpyHostToDevice,
                                hp->h2d));
    WP_CUDA_TRY(cudaMemcpyAsync(Bd[b], B + size_t(s0) * pb, size_t(ns) * pb * sizeof(float), cudaMemcpyHostToDevice,
                                hp->h2d));
    WP_CUDA_TRY(cudaEventRecord(hp->loaded[b], hp->h2d));
    // stage 2 (in order on its stream, one workspace)
    WP_CUDA_TRY(cudaStreamWaitEvent(hp->comp, hp->loaded[b], 0));
    WP_TRY(wp_wprod(Ad[b], Bd[b], Cd[b], n1, n2, n4, ns, L, 0, 0, prec, wprod_ws, wsz, hp->comp));
    WP_CUDA_TRY(cudaEventRecord(hp->done[b], hp->comp));
    // stage 3
    WP_CUDA_TRY(cudaStreamWaitEvent(hp->d2h, hp->done[b], 0));
    WP_CUDA_TRY(cudaMemcpyAsync(C + size_t(s0) * pc, Cd[b], size_t(ns) * pc * sizeof(float), cudaMemcpyDeviceToHost,
                                hp->d2h));
    WP_CUDA_TRY(cudaEventRecord(hp->freed[b], hp->d2h));
  }
  WP_CUDA_TRY(cudaEventRecord(hp->end, hp->d2h));
  WP_CUDA_TRY(cudaStreamWaitEvent(caller, hp->end, 0));
  return WP_OK;
}
