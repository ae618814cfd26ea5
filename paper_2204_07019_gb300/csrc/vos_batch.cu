// Batched stepping of many independent simulations (e.g. micromodels of
// uneven sizes).  In the default (graph) launch mode a batch step is ONE
// CUDA-graph launch: the steps of all instances are captured once into a
// single graph as parallel branches (each branch the instance's own step,
// with its device-driven refinement and Krylov WHILE loops), forked from and
// joined into one capture stream; the per-instance time steps are scattered
// into the instances' device dt slots by one kernel before the launch.  The
// graph is captured again only when an instance's momentum-preconditioner
// choice (it depends on dt) or its captured parameters (geometry reset by
// vos_set_fields, a network attached) change.  In the eager launch mode, or
// when an instance has a learned preconditioner attached, each instance is
// advanced by one of a pool of host worker threads on its own stream.  A
// batch step is fenced on the caller's stream in both modes, so CUDA events
// on the caller's stream time the whole batch step.
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/vos.h"
#include "vos_internal.cuh"

namespace vos {
void set_global_error(const char* msg);
bool graphs_enabled();
bool batch_graphable(const vos_handle* h);
unsigned batch_generation(const vos_handle* h);
int batch_key(const vos_handle* h, double dt);
double* batch_dt_slot(vos_handle* h);
cudaError_t batch_enqueue(vos_handle* h, int key, cudaEvent_t fork, cudaEvent_t* join);
int batch_finish(vos_handle* h, double dt);

static __device__ unsigned long long vos_exec_count = 0;
__global__ void k_scatter_dt(int n, const double* __restrict__ dt, double* const* __restrict__ slot) {
  VOS_COUNT_EXEC();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) *slot[i] = dt[i];
}
unsigned long long exec_count_batch() {
  unsigned long long v = 0;
  cudaMemcpyFromSymbol(&v, vos_exec_count, sizeof(v));
  return v;
}
}  // namespace vos

using namespace vos;

struct vos_batch {
  int n;
  cudaStream_t main;
  std::vector<cudaStream_t> streams;
  std::vector<vos_handle*> h;
  std::vector<cudaEvent_t> done;
  cudaEvent_t start;
  // worker pool
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::vector<double> dt;
  std::vector<int> status;
  int next = 0, finished = 0;
  bool quit = false;
  // single-graph path
  cudaStream_t cap = nullptr;          // capture / launch stream
  cudaGraphExec_t gexec = nullptr;
  std::vector<int> gkey;               // momentum-preconditioner choice per instance
  std::vector<unsigned> ggen;          // captured generation per instance
  double* h_dt = nullptr;              // pinned, n
  double* d_dt = nullptr;              // device, n
  double** d_slot = nullptr;           // device, n: each instance's dt slot
};

namespace {

void worker(vos_batch* b) {
  std::unique_lock<std::mutex> lk(b->mu);
  for (;;) {
    b->cv_work.wait(lk, [&] { return b->quit || b->next < b->n; });
    if (b->quit) return;
    const int i = b->next++;
    lk.unlock();
    const int rc = vos_step(b->h[i], b->dt[i]);
    cudaEventRecord(b->done[i], b->streams[i]);
    lk.lock();
    b->status[i] = rc;
    if (++b->finished == b->n) b->cv_done.notify_all();
  }
}

void destroy_batch(vos_batch* b) {
  if (!b) return;
  {
    std::lock_guard<std::mutex> lk(b->mu);
    b->quit = true;
  }
  b->cv_work.notify_all();
  for (auto& t : b->workers) t.join();
  if (b->cap) cudaStreamSynchronize(b->cap);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  for (auto* h : b->h) vos_destroy(h);
  for (auto e : b->done) cudaEventDestroy(e);
  for (auto s : b->streams) cudaStreamDestroy(s);
  if (b->start) cudaEventDestroy(b->start);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->h_dt) cudaFreeHost(b->h_dt);
  if (b->d_dt) cudaFree(b->d_dt);
  if (b->d_slot) cudaFree(b->d_slot);
  delete b;
}

// Capture the steps of all instances into one graph (keys: momentum
// preconditioner per instance).
cudaError_t capture_batch(vos_batch* b, const std::vector<int>& key) {
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  VOS_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
  cudaError_t err = cudaEventRecord(b->start, b->cap);
  for (int i = 0; i < b->n && err == cudaSuccess; ++i) {
    cudaEvent_t join = nullptr;
    err = batch_enqueue(b->h[i], key[i], b->start, &join);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(b->cap, join, 0);
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
  if (err == cudaSuccess) err = e2;
  if (err == cudaSuccess && g) err = cudaGraphInstantiate(&b->gexec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (err != cudaSuccess) {
    b->gexec = nullptr;
    cudaGetLastError();
    return err;
  }
  b->gkey = key;
  b->ggen.resize(b->n);
  for (int i = 0; i < b->n; ++i) b->ggen[i] = batch_generation(b->h[i]);
  return cudaSuccess;
}

int batch_step_graph(vos_batch* b, const double* dt) {
  std::vector<int> key(b->n);
  bool same = b->gexec != nullptr && (int)b->gkey.size() == b->n;
  for (int i = 0; i < b->n; ++i) {
    key[i] = batch_key(b->h[i], dt[i]);
    if (same && (key[i] != b->gkey[i] || b->ggen[i] != batch_generation(b->h[i]))) same = false;
  }
  if (!same) {
    cudaError_t e = capture_batch(b, key);
    if (e != cudaSuccess) {
      vos::set_global_error((std::string("vos_batch_step: graph capture failed: ") + cudaGetErrorString(e)).c_str());
      return VOS_ECUDA;
    }
  }
  std::memcpy(b->h_dt, dt, b->n * sizeof(double));
  cudaEventRecord(b->start, b->main);
  cudaStreamWaitEvent(b->cap, b->start, 0);
  cudaMemcpyAsync(b->d_dt, b->h_dt, b->n * sizeof(double), cudaMemcpyHostToDevice, b->cap);
  vlaunch("batch_dt", 0.0, k_scatter_dt, (b->n + 127) / 128, 128, b->cap, b->n, (const double*)b->d_dt,
          (double* const*)b->d_slot);
  cudaGraphLaunch(b->gexec, b->cap);
  cudaEventRecord(b->done[0], b->cap);
  cudaStreamWaitEvent(b->main, b->done[0], 0);
  cudaError_t e = cudaStreamSynchronize(b->cap);
  if (e != cudaSuccess) {
    vos::set_global_error((std::string("vos_batch_step: ") + cudaGetErrorString(e)).c_str());
    return VOS_ECUDA;
  }
  int worst = VOS_OK;
  for (int i = 0; i < b->n; ++i) {
    const int rc = batch_finish(b->h[i], dt[i]);
    if (rc != VOS_OK && (worst == VOS_OK || worst == VOS_ENOCONV)) worst = rc;
  }
  return worst;
}

}  // namespace

extern "C" {

int vos_batch_create(int n, const double* const* eps_s, const vos_params* prm, void* stream, int nthreads,
                     const vos_allocator* alloc, vos_batch** out) {
  if (!out) {
    vos::set_global_error("vos_batch_create: out is NULL");
    return VOS_EINVAL;
  }
  *out = nullptr;
  if (n < 1 || !eps_s || !prm) {
    vos::set_global_error("vos_batch_create: need n >= 1, eps_s and prm");
    return VOS_EINVAL;
  }
  vos_batch* b = new vos_batch();
  b->n = n;
  b->main = (cudaStream_t)stream;
  b->start = nullptr;
  b->dt.assign(n, 0.0);
  b->status.assign(n, 0);
  b->next = n;  // no work until the first vos_batch_step
  if (cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming) != cudaSuccess) {
    vos::set_global_error("vos_batch_create: cudaEventCreate failed");
    destroy_batch(b);
    return VOS_ECUDA;
  }
  for (int i = 0; i < n; ++i) {
    cudaStream_t s;
    cudaEvent_t e;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      vos::set_global_error("vos_batch_create: stream/event creation failed");
      destroy_batch(b);
      return VOS_ECUDA;
    }
    b->streams.push_back(s);
    b->done.push_back(e);
    vos_handle* h = nullptr;
    int rc = vos_create(eps_s[i], &prm[i], s, alloc, &h);
    if (rc != VOS_OK) {
      std::string msg = std::string("vos_batch_create: instance ") + std::to_string(i) + ": " + vos_last_error(nullptr);
      destroy_batch(b);
      vos::set_global_error(msg.c_str());
      return rc;
    }
    b->h.push_back(h);
  }
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost((void**)&b->h_dt, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&b->d_dt, n * sizeof(double)) != cudaSuccess ||
      cudaMalloc((void**)&b->d_slot, n * sizeof(double*)) != cudaSuccess) {
    vos::set_global_error("vos_batch_create: stream or buffer allocation failed");
    destroy_batch(b);
    return VOS_ECUDA;
  }
  {
    std::vector<double*> slots(n);
    for (int i = 0; i < n; ++i) slots[i] = batch_dt_slot(b->h[i]);
    if (cudaMemcpy(b->d_slot, slots.data(), n * sizeof(double*), cudaMemcpyHostToDevice) != cudaSuccess) {
      vos::set_global_error("vos_batch_create: cudaMemcpy failed");
      destroy_batch(b);
      return VOS_ECUDA;
    }
  }
  int nt = nthreads > 0 ? nthreads : 8;
  if (nt > n) nt = n;
  for (int t = 0; t < nt; ++t) b->workers.emplace_back(worker, b);
  *out = b;
  return VOS_OK;
}

int vos_batch_step(vos_batch* b, const double* dt) {
  if (!b || !dt) {
    vos::set_global_error("vos_batch_step: NULL argument");
    return VOS_EINVAL;
  }
  for (int i = 0; i < b->n; ++i)
    if (!(dt[i] > 0.0) || !std::isfinite(dt[i])) {
      vos::set_global_error("vos_batch_step: every dt must be finite and > 0");
      return VOS_EINVAL;
    }
  bool graph = graphs_enabled();
  for (int i = 0; i < b->n && graph; ++i) graph = batch_graphable(b->h[i]);
  if (graph) return batch_step_graph(b, dt);
  cudaEventRecord(b->start, b->main);
  for (int i = 0; i < b->n; ++i) cudaStreamWaitEvent(b->streams[i], b->start, 0);
  {
    std::unique_lock<std::mutex> lk(b->mu);
    for (int i = 0; i < b->n; ++i) b->dt[i] = dt[i];
    b->next = 0;
    b->finished = 0;
    b->cv_work.notify_all();
    b->cv_done.wait(lk, [&] { return b->finished == b->n; });
  }
  for (int i = 0; i < b->n; ++i) cudaStreamWaitEvent(b->main, b->done[i], 0);
  int worst = VOS_OK;
  for (int i = 0; i < b->n; ++i) {
    const int s = b->status[i];
    if (s != VOS_OK && (worst == VOS_OK || worst == VOS_ENOCONV)) worst = s;
  }
  if (worst != VOS_OK && worst != VOS_ENOCONV) vos::set_global_error("vos_batch_step: an instance failed");
  return worst;
}

int vos_batch_handle(vos_batch* b, int i, vos_handle** h) {
  if (!b || !h || i < 0 || i >= b->n) {
    vos::set_global_error("vos_batch_handle: bad argument");
    return VOS_EINVAL;
  }
  *h = b->h[i];
  return VOS_OK;
}

void vos_batch_destroy(vos_batch* b) { destroy_batch(b); }

}  // extern "C"
