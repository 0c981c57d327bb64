// Library-level entry points: status strings, version, device status word,
// launch counter.

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace wp {

static __device__ int g_device_status = 0;

static std::atomic<unsigned long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// ---- per-kernel profiler --------------------------------------------------
struct ProfRecord { const char* name; cudaEvent_t start, stop; };
struct ProfTotal { std::string name; long launches; double ms; };
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::string g_prof_only;   // record only launches of this name (empty: all)
static std::vector<ProfRecord> g_prof_records;
static std::vector<cudaEvent_t> g_prof_pool;
static std::vector<ProfTotal> g_prof_totals;

bool profiling_enabled() { return g_prof_on; }

static cudaEvent_t prof_event() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void profile_record(const char* name, cudaStream_t st, cudaEvent_t* start, cudaEvent_t* stop) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_only.empty() && g_prof_only != name) return;
  *start = prof_event();
  *stop = prof_event();
  if (*start) cudaEventRecord(*start, st);
}

void profile_finish(const char* name, cudaStream_t st, cudaEvent_t start, cudaEvent_t stop) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (stop) cudaEventRecord(stop, st);
  g_prof_records.push_back({name, start, stop});
}

int* device_status_ptr() {
  static int* cached[64] = {nullptr};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  if (cached[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_device_status) != cudaSuccess) return nullptr;
    cached[dev] = static_cast<int*>(p);
  }
  return cached[dev];
}

int sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (cached[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    cached[dev] = n;
  }
  return cached[dev];
}

}  // namespace wp

extern "C" const char* wp_status_string(int status) {
  switch (status) {
    case WP_OK: return "WP_OK";
    case WP_ERR_NULL: return "WP_ERR_NULL: a required pointer is NULL";
    case WP_ERR_SHAPE: return "WP_ERR_SHAPE: a dimension is out of range";
    case WP_ERR_LEVELS: return "WP_ERR_LEVELS: L out of range or p not a multiple of 2^L";
    case WP_ERR_RANK: return "WP_ERR_RANK: rank r outside [1, min(rows, cols)]";
    case WP_ERR_PREC: return "WP_ERR_PREC: unknown precision mode";
    case WP_ERR_ALIGN: return "WP_ERR_ALIGN: pointer not 16-byte aligned";
    case WP_ERR_WORKSPACE: return "WP_ERR_WORKSPACE: workspace missing or too small";
    case WP_ERR_NOT_CONVERGED: return "WP_ERR_NOT_CONVERGED: Jacobi SVD reached its sweep limit";
    case WP_ERR_TIMEOUT: return "WP_ERR_TIMEOUT: a bounded device-side wait expired";
    case WP_ERR_CUDA: return "WP_ERR_CUDA: a CUDA runtime call failed";
    case WP_ERR_ALIAS: return "WP_ERR_ALIAS: an output overlaps an input";
    case WP_ERR_UNSUPPORTED: return "WP_ERR_UNSUPPORTED: not implemented for these arguments";
    default: return "WP_ERR_UNKNOWN";
  }
}

extern "C" int wp_version(void) { return 100; }

extern "C" int wp_get_device_error(void* stream) {
  if (cudaStreamSynchronize(wp::as_stream(stream)) != cudaSuccess) return WP_ERR_CUDA;
  int code = 0;
  if (cudaMemcpyFromSymbol(&code, wp::g_device_status, sizeof(int)) != cudaSuccess) return WP_ERR_CUDA;
  const int zero = 0;
  if (cudaMemcpyToSymbol(wp::g_device_status, &zero, sizeof(int)) != cudaSuccess) return WP_ERR_CUDA;
  return code;
}

extern "C" uint64_t wp_launch_count(void) {
  return static_cast<uint64_t>(wp::g_launches.load(std::memory_order_relaxed));
}

extern "C" int wp_profile_begin(void) {
  std::lock_guard<std::mutex> lk(wp::g_prof_mu);
  for (auto& r : wp::g_prof_records) {
    wp::g_prof_pool.push_back(r.start);
    wp::g_prof_pool.push_back(r.stop);
  }
  wp::g_prof_records.clear();
  wp::g_prof_totals.clear();
  wp::g_prof_on = true;
  return WP_OK;
}

extern "C" int wp_profile_only(const char* name) {
  std::lock_guard<std::mutex> lk(wp::g_prof_mu);
  wp::g_prof_only = name ? name : "";
  return WP_OK;
}

extern "C" int wp_profile_end(void) {
  std::lock_guard<std::mutex> lk(wp::g_prof_mu);
  wp::g_prof_on = false;
  if (cudaDeviceSynchronize() != cudaSuccess) return WP_ERR_CUDA;
  wp::g_prof_totals.clear();
  for (auto& r : wp::g_prof_records) {
    float ms = 0.f;
    if (!r.start || !r.stop || cudaEventElapsedTime(&ms, r.start, r.stop) != cudaSuccess) return WP_ERR_CUDA;
    bool found = false;
    for (auto& t : wp::g_prof_totals)
      if (t.name == r.name) { t.launches++; t.ms += ms; found = true; break; }
    if (!found) wp::g_prof_totals.push_back({r.name, 1, double(ms)});
    wp::g_prof_pool.push_back(r.start);
    wp::g_prof_pool.push_back(r.stop);
  }
  wp::g_prof_records.clear();
  return int(wp::g_prof_totals.size()) >= 0 ? WP_OK : WP_ERR_CUDA;
}

extern "C" int wp_profile_count(void) {
  std::lock_guard<std::mutex> lk(wp::g_prof_mu);
  return int(wp::g_prof_totals.size());
}

extern "C" int wp_profile_get(int index, char* name, int name_len, int64_t* launches, double* total_ms) {
  std::lock_guard<std::mutex> lk(wp::g_prof_mu);
  if (index < 0 || index >= int(wp::g_prof_totals.size())) return WP_ERR_SHAPE;
  if (!name || name_len < 1 || !launches || !total_ms) return WP_ERR_NULL;
  const auto& t = wp::g_prof_totals[index];
  const int n = std::min<int>(name_len - 1, int(t.name.size()));
  for (int i = 0; i < n; ++i) name[i] = t.name[i];
  name[n] = 0;
  *launches = t.launches;
  *total_ms = t.ms;
  return WP_OK;
}
