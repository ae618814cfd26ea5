// Batched stepping of many independent simulations (e.g. micromodels of
// uneven sizes).  Each instance owns a non-blocking CUDA stream and is
// advanced by one of a pool of host worker threads, so the GPU overlaps the
// instances' (mostly latency-bound) kernels and the host-side solver polls
// of different instances run concurrently.  A batch step is fenced on the
// caller's stream: every instance stream waits for an event recorded there
// first, and the caller's stream waits for every instance at the end, so
// CUDA events on the caller's stream time the whole batch step.
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
}

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
  for (auto* h : b->h) vos_destroy(h);
  for (auto e : b->done) cudaEventDestroy(e);
  for (auto s : b->streams) cudaStreamDestroy(s);
  if (b->start) cudaEventDestroy(b->start);
  delete b;
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
    if (!(dt[i] > 0.0)) {
      vos::set_global_error("vos_batch_step: every dt must be > 0");
      return VOS_EINVAL;
    }
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
