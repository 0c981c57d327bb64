// Shared host/device helpers for libwprod.so (no method arithmetic here).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <algorithm>

#include "wprod.h"

namespace wp {

// Device address of the per-device status word (defined in abi.cu) that
// kernels write when they detect a fault (an expired bounded wait, a Jacobi
// sweep limit).  Kernels receive it as a plain pointer argument; it is read
// and cleared by wp_get_device_error.  Returns nullptr if CUDA fails.
int* device_status_ptr();

__device__ __forceinline__ void report_device_error(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline bool overlaps(const void* a, size_t abytes, const void* b, size_t bbytes) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + bbytes && y < x + abytes;
}

inline int check_levels(int64_t p, int L) {
  if (L < 0 || L > WP_MAX_LEVELS) return WP_ERR_LEVELS;
  if (p < 1 || (p % (int64_t(1) << L)) != 0) return WP_ERR_LEVELS;
  return WP_OK;
}

// Number of SMs of the current device (cached per device).
int sm_count();

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Carves sub-buffers out of a caller-supplied workspace, 256-byte aligned.
struct Carver {
  char* base;
  size_t cap;
  size_t off = 0;
  bool ok = true;
  Carver(void* b, size_t c) : base(static_cast<char*>(b)), cap(c) {}
  template <typename T>
  T* take(size_t count) {
    size_t start = align_up(off, 256);
    size_t bytes = count * sizeof(T);
    off = start + bytes;
    if (off > cap || base == nullptr) { ok = false; return nullptr; }
    return reinterpret_cast<T*>(base + start);
  }
};

// Size-only counterpart of Carver, for the *_workspace queries.
struct Sizer {
  size_t off = 0;
  template <typename T>
  void take(size_t count) { off = align_up(off, 256) + count * sizeof(T); }
  size_t bytes() const { return align_up(off, 256); }
};

#define WP_CUDA_TRY(expr)                                  \
  do {                                                     \
    cudaError_t _e = (expr);                               \
    if (_e != cudaSuccess) return WP_ERR_CUDA;             \
  } while (0)

#define WP_TRY(expr)                                       \
  do {                                                     \
    int _s = (expr);                                       \
    if (_s != WP_OK) return _s;                            \
  } while (0)

// Counts every kernel launch the library issues (reported by wp_launch_count).
void count_launch();

// Optional per-kernel timing (wp_profile_begin / wp_profile_end): when
// enabled, a ProfileScope placed right before a kernel launch records a CUDA
// event on the launching stream at construction and another at destruction,
// bracketing exactly that launch.  Disabled: no events, no cost.
bool profiling_enabled();
void profile_record(const char* name, cudaStream_t st, cudaEvent_t* start, cudaEvent_t* stop);
void profile_finish(const char* name, cudaStream_t st, cudaEvent_t start, cudaEvent_t stop);

struct ProfileScope {
  const char* name;
  cudaStream_t st;
  cudaEvent_t start = nullptr, stop = nullptr;
  ProfileScope(const char* n, cudaStream_t s) : name(n), st(s) {
    if (profiling_enabled()) profile_record(name, st, &start, &stop);
  }
  ~ProfileScope() {
    if (start) profile_finish(name, st, start, stop);
  }
};

#define WP_PROFILE(name, stream) ::wp::ProfileScope _wp_prof_scope((name), (stream))

// Call right after each kernel launch: counts it and reports launch errors.
inline int launch_status() {
  count_launch();
  return cudaGetLastError() == cudaSuccess ? WP_OK : WP_ERR_CUDA;
}

}  // namespace wp
