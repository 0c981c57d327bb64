// wp_wprod_noalloc: the w-product for callers that cannot allocate device
// memory.
//
// Some callers of this library have no way to provide a device workspace:
// plain C hosts that link libwprod.so without any device allocator of their
// own, and plug-ins running inside an application whose memory manager owns
// every device allocation (allocating behind its back is forbidden, and a
// cudaMalloc there can also synchronise the whole device in the middle of a
// latency-sensitive loop).  For them this entry point takes its scratch space
// from one fixed array in device global memory that belongs to the library
// itself, so the caller passes only inputs and outputs.
//
// The array is a file-scope __device__ variable of WP_NOALLOC_SCRATCH_BYTES
// bytes: every GPU that loads the library holds it until the process exits.
// Host code may not use the array's name as a device address (on the host it
// names a stand-in object), so the device address is looked up once per
// device with cudaGetSymbolAddress, while that device is current, and then
// passed to the kernels as an ordinary pointer.

#include <mutex>

#include "common.cuh"

static __device__ __align__(256) unsigned char g_noalloc_scratch[WP_NOALLOC_SCRATCH_BYTES];

namespace wp {

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {nullptr};

// Device address of the scratch array on the current device (looked up on
// the first call per device).
static int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return WP_ERR_CUDA;
  if (dev < 0 || dev >= 64) return WP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return WP_ERR_CUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return WP_OK;
}

}  // namespace wp

extern "C" int wp_wprod_noalloc(const float* A, const float* B, float* C, int64_t n1, int64_t n2,
                                int64_t n4, int64_t p, int L, int transA, int transB, int prec,
                                void* stream) {
  size_t need = 0;
  WP_TRY(wp_wprod_workspace(n1, n2, n4, p, L, prec, &need));
  if (need > size_t(WP_NOALLOC_SCRATCH_BYTES)) return WP_ERR_WORKSPACE;
  void* scratch = nullptr;
  WP_TRY(wp::noalloc_scratch(&scratch));
  // Every byte of the workspace that the w-product reads is written earlier
  // in the same call (transforms, operand splits, face-products), so nothing
  // left over from a previous call is ever used and nothing needs clearing.
  return wp_wprod(A, B, C, n1, n2, n4, p, L, transA, transB, prec, scratch,
                  size_t(WP_NOALLOC_SCRATCH_BYTES), stream);
}
