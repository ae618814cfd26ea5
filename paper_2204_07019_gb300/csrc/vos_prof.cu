// Launch counting and optional per-kernel CUDA-event timing.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/vos.h"
#include "vos_internal.cuh"

namespace vos {

std::atomic<unsigned long long> g_launch_count{0};
unsigned long long exec_count_solver();
unsigned long long exec_count_fields();
unsigned long long exec_count_deflate();
unsigned long long exec_count_unet();
unsigned long long exec_count_batch();
unsigned long long exec_count_mgtail();
unsigned long long exec_count_sum() {
  return exec_count_solver() + exec_count_fields() + exec_count_deflate() + exec_count_unet() + exec_count_batch() +
         exec_count_mgtail();
}
bool g_prof_any = false;

namespace {

struct Pending {
  cudaEvent_t a, b;
  int id;
  double bytes;
};
struct Acc {
  std::string name;
  long long n = 0;
  double ms = 0.0, bytes = 0.0;
};

std::mutex g_mu;
std::vector<std::string> g_filters;
std::vector<cudaEvent_t> g_pool;
std::vector<Pending> g_pending;
std::vector<Acc> g_acc;
std::map<std::string, int> g_ids;
constexpr size_t kMaxPending = 4096;

bool matches(const char* name) {
  for (const auto& f : g_filters)
    if (f == "*" || std::strstr(name, f.c_str()) != nullptr) return true;
  return false;
}

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void harvest_locked() {
  for (auto& p : g_pending) {
    cudaEventSynchronize(p.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    Acc& a = g_acc[p.id];
    a.n += 1;
    a.ms += ms;
    a.bytes += p.bytes;
    g_pool.push_back(p.a);
    g_pool.push_back(p.b);
  }
  g_pending.clear();
}

}  // namespace

int prof_before(const char* name, double bytes, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!matches(name)) return -1;
  if (g_pending.size() >= kMaxPending) harvest_locked();
  auto it = g_ids.find(name);
  int id;
  if (it == g_ids.end()) {
    id = (int)g_acc.size();
    g_ids[name] = id;
    g_acc.push_back(Acc{name});
  } else {
    id = it->second;
  }
  Pending p{take_event(), take_event(), id, bytes};
  cudaEventRecord(p.a, st);
  g_pending.push_back(p);
  return (int)g_pending.size() - 1;
}

void prof_after(int slot, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (slot >= 0 && slot < (int)g_pending.size()) cudaEventRecord(g_pending[slot].b, st);
}

}  // namespace vos

extern "C" {

int vos_prof_enable(const char* filter) {
  std::lock_guard<std::mutex> lk(vos::g_mu);
  vos::g_filters.clear();
  if (filter && *filter) {
    std::string f(filter);
    size_t pos = 0;
    while (pos <= f.size()) {
      size_t q = f.find(',', pos);
      if (q == std::string::npos) q = f.size();
      if (q > pos) vos::g_filters.push_back(f.substr(pos, q - pos));
      pos = q + 1;
    }
  }
  vos::g_prof_any = !vos::g_filters.empty();
  return VOS_OK;
}

int vos_prof_report(char* buf, size_t len) {
  std::lock_guard<std::mutex> lk(vos::g_mu);
  vos::harvest_locked();
  std::string out;
  char line[512];
  for (const auto& a : vos::g_acc) {
    std::snprintf(line, sizeof(line), "%s\t%lld\t%.6f\t%.0f\n", a.name.c_str(), a.n, a.ms, a.bytes);
    out += line;
  }
  if (!buf || len == 0) return (int)out.size() + 1;
  std::snprintf(buf, len, "%s", out.c_str());
  return (out.size() + 1 <= len) ? VOS_OK : (int)out.size() + 1;
}

void vos_prof_reset(void) {
  std::lock_guard<std::mutex> lk(vos::g_mu);
  vos::harvest_locked();
  vos::g_acc.clear();
  vos::g_ids.clear();
}

uint64_t vos_kernel_launches(void) {
  // Executions counted on the device: includes kernels replayed by CUDA
  // graphs (synchronises with the device).
  cudaDeviceSynchronize();
  return vos::exec_count_sum();
}

}  // extern "C"
