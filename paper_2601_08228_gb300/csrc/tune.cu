// Autotuner and plan cache of the tensor-core w-product.
//
// The BF16 / BF16x3 w-product (gemm_tc.cu) has three kernels: one that keeps
// all 2^L wavelet-domain accumulators of a tile in tensor memory and applies
// the inverse lift in its epilogue (narrow tiles, no C_hat round trip), the
// same tile with the forward lift done by its own producer warps on the
// spatial operands (L <= 3: no W(A), W(B) round trip either), and a
// persistent wide-tile GEMM into C_hat followed by a separate inverse lift.
// Which is faster depends on the shape (tile width against 512 / 2^L, K,
// the number of tiles against the SM count), so wp_wprod_tune times them on
// the caller's tensors and keeps the fastest in a process-wide cache keyed by
// (n1, n2, n4, p, L, precision); wp_wprod consults it before its rule of
// thumb.  The cache can be written to and read from a text file of one JSON
// object per line.

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "internal.cuh"

namespace wp {

using PlanKey = std::tuple<int64_t, int64_t, int64_t, int64_t, int, int>;
struct PlanVal {
  int variant;          // kVariantFused, kVariantPersistent or kVariantLifted
  double ms;
};

static std::mutex g_plan_mu;
static std::map<PlanKey, PlanVal> g_plans;

int wprod_plan_lookup(int64_t n1, int64_t n2, int64_t n4, int64_t p, int L, int prec) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  auto it = g_plans.find(PlanKey{n1, n2, n4, p, L, prec});
  return it == g_plans.end() ? 0 : it->second.variant;
}

static void plan_store(const PlanKey& k, int variant, double ms) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  g_plans[k] = PlanVal{variant, ms};
}

static bool valid_variant(int v) { return v == kVariantFused || v == kVariantPersistent || v == kVariantLifted; }

static bool plan_erase(const PlanKey& k, PlanVal* old) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  auto it = g_plans.find(k);
  if (it == g_plans.end()) return false;
  *old = it->second;
  g_plans.erase(it);
  return true;
}

}  // namespace wp

using namespace wp;

extern "C" int wp_plan_set(int64_t n1, int64_t n2, int64_t n4, int64_t p, int L, int prec, int variant) {
  if (n1 < 1 || n2 < 1 || n4 < 1 || p < 1) return WP_ERR_SHAPE;
  WP_TRY(check_levels(p, L));
  if (prec < WP_PREC_FP32 || prec > WP_PREC_FP8) return WP_ERR_PREC;
  const PlanKey k{n1, n2, n4, p, L, prec};
  if (variant <= 0) {
    PlanVal old;
    plan_erase(k, &old);
    return WP_OK;
  }
  if (!valid_variant(variant)) return WP_ERR_SHAPE;
  plan_store(k, variant, -1.0);
  return WP_OK;
}

extern "C" int wp_plan_get(int64_t n1, int64_t n2, int64_t n4, int64_t p, int L, int prec, int* variant) {
  if (!variant) return WP_ERR_NULL;
  *variant = wprod_plan_lookup(n1, n2, n4, p, L, prec);
  return WP_OK;
}

extern "C" int wp_plan_clear(void) {
  std::lock_guard<std::mutex> lk(g_plan_mu);
  g_plans.clear();
  return WP_OK;
}

extern "C" int wp_plan_save(const char* path) {
  if (!path) return WP_ERR_NULL;
  std::lock_guard<std::mutex> lk(g_plan_mu);
  FILE* f = std::fopen(path, "w");
  if (!f) return WP_ERR_SHAPE;
  for (const auto& kv : g_plans) {
    const auto& k = kv.first;
    std::fprintf(f,
                 "{\"op\": \"wprod\", \"n1\": %lld, \"n2\": %lld, \"n4\": %lld, \"p\": %lld, \"L\": %d, "
                 "\"prec\": %d, \"variant\": %d, \"ms\": %.6f}\n",
                 (long long)std::get<0>(k), (long long)std::get<1>(k), (long long)std::get<2>(k),
                 (long long)std::get<3>(k), std::get<4>(k), std::get<5>(k), kv.second.variant, kv.second.ms);
  }
  const bool ok = std::fclose(f) == 0;
  return ok ? WP_OK : WP_ERR_SHAPE;
}

// Value of "key": <number> in one line of the cache file (false if absent).
static bool json_number(const char* line, const char* key, double* out) {
  char pat[32];
  std::snprintf(pat, sizeof(pat), "\"%s\":", key);
  const char* at = std::strstr(line, pat);
  if (!at) return false;
  return std::sscanf(at + std::strlen(pat), " %lf", out) == 1;
}

extern "C" int wp_plan_load(const char* path, int* entries) {
  if (!path) return WP_ERR_NULL;
  FILE* f = std::fopen(path, "r");
  if (!f) return WP_ERR_SHAPE;
  char line[512];
  int n = 0;
  int rc = WP_OK;
  while (std::fgets(line, sizeof(line), f)) {
    if (!std::strstr(line, "\"op\": \"wprod\"")) continue;
    double v[8];
    const char* keys[8] = {"n1", "n2", "n4", "p", "L", "prec", "variant", "ms"};
    bool ok = true;
    for (int i = 0; i < 8 && ok; ++i) ok = json_number(line, keys[i], &v[i]);
    if (!ok) {
      rc = WP_ERR_SHAPE;
      break;
    }
    const int64_t n1 = int64_t(v[0]), n2 = int64_t(v[1]), n4 = int64_t(v[2]), p = int64_t(v[3]);
    const int L = int(v[4]), prec = int(v[5]), cg = int(v[6]);
    if (n1 < 1 || n2 < 1 || n4 < 1 || p < 1 || check_levels(p, L) != WP_OK || !valid_variant(cg) ||
        prec < WP_PREC_FP32 || prec > WP_PREC_FP8) {
      rc = WP_ERR_SHAPE;
      break;
    }
    plan_store(PlanKey{n1, n2, n4, p, L, prec}, cg, v[7]);
    ++n;
  }
  std::fclose(f);
  if (entries) *entries = n;
  return rc;
}

extern "C" int wp_wprod_tune(const float* A, const float* B, float* C, int64_t n1, int64_t n2, int64_t n4,
                             int64_t p, int L, int prec, void* ws, size_t ws_bytes, void* stream, int* variant,
                             double* best_ms) {
  if (!variant) return WP_ERR_NULL;
  *variant = 0;
  if (best_ms) *best_ms = 0.0;
  // validation is wp_wprod's: run it once with the current plan
  WP_TRY(wp_wprod(A, B, C, n1, n2, n4, p, L, 0, 0, prec, ws, ws_bytes, stream));
  if (!wprod_tunable(n1, n2, n4, p, L, prec)) return WP_OK;   // one kernel only: nothing to choose
  const PlanKey key{n1, n2, n4, p, L, prec};
  PlanVal prev{0, 0.0};
  const bool had = plan_erase(key, &prev);
  cudaStream_t st = as_stream(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = WP_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = WP_ERR_CUDA;
  int best = 0;
  float best_t = 0.f;
  const bool lift = wprod_lift_ok(A, B, C, n1, n2, n4, p, L, prec);
  for (int v : {kVariantFused, kVariantPersistent, kVariantLifted}) {
    if (rc != WP_OK) break;
    if (v == kVariantLifted && !lift) continue;
    plan_store(key, v, -1.0);
    // one warm-up call, then the mean of three back-to-back calls
    rc = wp_wprod(A, B, C, n1, n2, n4, p, L, 0, 0, prec, ws, ws_bytes, stream);
    if (rc != WP_OK) break;
    if (cudaEventRecord(e0, st) != cudaSuccess) { rc = WP_ERR_CUDA; break; }
    for (int r = 0; r < 3 && rc == WP_OK; ++r) rc = wp_wprod(A, B, C, n1, n2, n4, p, L, 0, 0, prec, ws, ws_bytes, stream);
    if (rc != WP_OK) break;
    float ms = 0.f;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = WP_ERR_CUDA;
      break;
    }
    ms /= 3.f;
    if (best == 0 || ms < best_t) {
      best = v;
      best_t = ms;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc != WP_OK || best == 0) {
    PlanVal dummy;
    plan_erase(key, &dummy);
    if (had) plan_store(key, prev.variant, prev.ms);
    return rc != WP_OK ? rc : WP_ERR_CUDA;
  }
  plan_store(key, best, double(best_t));
  // C from the chosen kernel
  rc = wp_wprod(A, B, C, n1, n2, n4, p, L, 0, 0, prec, ws, ws_bytes, stream);
  *variant = best;
  if (best_ms) *best_ms = double(best_t);
  return rc;
}
