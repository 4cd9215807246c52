// profile.cu -- kernel launch counting and optional CUDA-event timing of the
// fine-level kernels (the tracing facility behind mgglam_profile_* and
// mgglam_launch_count).  When profiling is off the hooks cost one branch.
#include <string.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "mg_internal.h"

namespace mg {

static const char* kProfNames[PC_COUNT] = {
    "smooth32_fine",     "residual_restrict32_fine", "prolong_correct32_fine", "outer_residual64",
    "apply_correction64", "smooth64_fine",           "residual_restrict64_fine", "prolong_correct64_fine",
    "residual64_fine",   "coarse_levels",            "deposit_cic",            "deposit_finish",
    "field_transform",   "gather_force",             "poisson_fft",            "pm_potential",
    "pm_kick_drift"};

static std::atomic<long long> g_launches{0};
static std::mutex g_pmu;
static bool g_on = false;
struct Rec {
  int cls;
  cudaEvent_t a, b;
  double bytes;
};
static std::vector<Rec> g_recs;
static std::vector<cudaEvent_t> g_pool;
static int g_open = -1;

void note_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(); }

static cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void prof_begin(int cls, cudaStream_t st, double alg_bytes) {
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_pmu);
  Rec r{cls, take_event(), take_event(), alg_bytes};
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  g_open = (int)g_recs.size() - 1;
}

void prof_end(cudaStream_t st) {
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_pmu);
  if (g_open >= 0) cudaEventRecord(g_recs[g_open].b, st);
  g_open = -1;
}

int prof_start() {
  std::lock_guard<std::mutex> lk(g_pmu);
  for (auto& r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  g_open = -1;
  g_on = true;
  return MGGLAM_OK;
}

int prof_stop(mgglam_kernel_profile* out, int max_entries, int* n_entries) {
  std::lock_guard<std::mutex> lk(g_pmu);
  g_on = false;
  if (cudaDeviceSynchronize() != cudaSuccess) return MGGLAM_ERR_CUDA;
  mgglam_kernel_profile acc[PC_COUNT];
  memset(acc, 0, sizeof(acc));
  for (auto& r : g_recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) continue;
    acc[r.cls].launches += 1;
    acc[r.cls].ms += ms;
    acc[r.cls].bytes += r.bytes;
  }
  int n = 0;
  for (int c = 0; c < PC_COUNT; ++c) {
    if (acc[c].launches == 0) continue;
    if (out && n < max_entries) {
      out[n] = acc[c];
      strncpy(out[n].name, kProfNames[c], sizeof(out[n].name) - 1);
    }
    ++n;
  }
  if (n_entries) *n_entries = n;
  return MGGLAM_OK;
}

}  // namespace mg

extern "C" {

int mgglam_profile_start(void) { return mg::prof_start(); }

int mgglam_profile_stop(mgglam_kernel_profile* out, int max_entries, int* n_entries) {
  return mg::prof_stop(out, max_entries, n_entries);
}

long long mgglam_launch_count(void) { return mg::launch_count(); }

}  // extern "C"
