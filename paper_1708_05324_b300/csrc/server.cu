// Request server: continuous batching of propagation requests.
//
// Requests enter a FIFO queue.  A request is admitted when the head of the
// queue fits both the in-flight count and the device-byte budget (its
// workspace size, gmmnlse_request_bytes).  Each admitted request runs on a
// worker thread with its own CUDA stream and its own workspace, so requests
// that arrive while others are running are admitted as soon as a slot and
// memory free up, and their kernels overlap with the running ones on the GPU.
// Workspaces are pooled per (context, M) and reused.
#include <cuda_runtime.h>

#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/gmmnlse.h"
#include "engine.h"

namespace {

struct Request {
  uint64_t ticket = 0;
  gmmnlse_ctx* ctx = nullptr;
  std::vector<double> A0, Aout;
  double L = 0, dz = 0, tol = 0;
  int M = 0;
  size_t bytes = 0;
  int status = GMMNLSE_PENDING;
  gmmnlse_stats st{};
};

struct PooledJob {
  gmmnlse_ctx* ctx;
  int M;
  gm_job* job;
};

constexpr size_t kMaxQueued = 65536;

}  // namespace

struct gmmnlse_server {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::map<uint64_t, Request*> all;
  std::vector<PooledJob> pool;
  std::vector<std::thread> workers;
  size_t budget = 0, inflight_bytes = 0;
  int max_inflight = 1, inflight = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
};

static void worker_main(gmmnlse_server* s) {
  cudaStream_t stream = nullptr;
  int stream_dev = -1;
  for (;;) {
    Request* r = nullptr;
    gm_job* job = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] {
        if (s->stop) return true;
        if (s->queue.empty() || s->inflight >= s->max_inflight) return false;
        return s->inflight_bytes + s->queue.front()->bytes <= s->budget;
      });
      if (s->stop) break;
      r = s->queue.front();
      s->queue.pop_front();
      s->inflight += 1;
      s->inflight_bytes += r->bytes;
      for (size_t i = 0; i < s->pool.size(); ++i)
        if (s->pool[i].ctx == r->ctx && s->pool[i].M >= r->M) {
          job = s->pool[i].job;
          s->pool.erase(s->pool.begin() + i);
          break;
        }
    }
    const int dev = gm_ctx_device(r->ctx);
    int rc = cudaSetDevice(dev) == cudaSuccess ? GMMNLSE_OK : GMMNLSE_E_CUDA;
    if (!rc && stream_dev != dev) {
      if (stream) cudaStreamDestroy(stream);
      stream = nullptr;
      rc = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess ? GMMNLSE_OK : GMMNLSE_E_CUDA;
      stream_dev = rc ? -1 : dev;
    }
    if (!rc && !job) rc = gm_job_create(r->ctx, r->M, &job);
    if (!rc) {
      r->Aout.resize(r->A0.size());
      rc = gm_job_propagate(job, r->A0.data(), false, r->L, r->dz, r->M, r->tol, r->Aout.data(), &r->st, stream);
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      r->status = rc;
      s->inflight -= 1;
      s->inflight_bytes -= r->bytes;
      if (job) {
        if (s->pool.size() < (size_t)s->max_inflight) s->pool.push_back({r->ctx, r->M, job});
        else gm_job_destroy(job);
      }
    }
    s->cv_work.notify_all();
    s->cv_done.notify_all();
  }
  if (stream) cudaStreamDestroy(stream);
}

extern "C" int gmmnlse_server_create(size_t hbm_budget, int max_inflight, gmmnlse_server** out) {
  if (!out || hbm_budget == 0 || max_inflight < 1 || max_inflight > 256) return GMMNLSE_E_INVALID;
  gmmnlse_server* s = new (std::nothrow) gmmnlse_server();
  if (!s) return GMMNLSE_E_NOMEM;
  s->budget = hbm_budget;
  s->max_inflight = max_inflight;
  for (int i = 0; i < max_inflight; ++i) s->workers.emplace_back(worker_main, s);
  *out = s;
  return GMMNLSE_OK;
}

extern "C" int gmmnlse_submit(gmmnlse_server* s, gmmnlse_ctx* ctx, const double* A0, double L, double dz, int M,
                              double tol, uint64_t* ticket) {
  if (!s || !ctx || !A0 || !ticket) return GMMNLSE_E_INVALID;
  long nf;
  int mr;
  int rc = gm_schedule(L, dz, M, &nf, &mr);
  if (rc) return rc;
  const size_t bytes = gmmnlse_request_bytes(ctx, M);
  if (bytes > s->budget) return GMMNLSE_E_NOMEM;
  Request* r = new (std::nothrow) Request();
  if (!r) return GMMNLSE_E_NOMEM;
  const size_t cnt = (size_t)gm_ctx_modes(ctx) * gm_ctx_samples(ctx) * 2;
  r->ctx = ctx;
  r->A0.assign(A0, A0 + cnt);
  r->L = L;
  r->dz = dz;
  r->M = M;
  r->tol = tol;
  r->bytes = bytes;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->queue.size() >= kMaxQueued) {
      delete r;
      return GMMNLSE_E_BUSY;
    }
    r->ticket = s->next_ticket++;
    s->all[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
  }
  s->cv_work.notify_one();
  return GMMNLSE_OK;
}

extern "C" int gmmnlse_poll(gmmnlse_server* s, uint64_t ticket, double* Aout, gmmnlse_stats* st) {
  if (!s) return GMMNLSE_E_INVALID;
  Request* r = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return GMMNLSE_E_INVALID;
    r = it->second;
    if (r->status == GMMNLSE_PENDING) return GMMNLSE_PENDING;
    s->all.erase(it);
  }
  const int status = r->status;
  if (Aout && !r->Aout.empty()) std::memcpy(Aout, r->Aout.data(), r->Aout.size() * sizeof(double));
  if (st) *st = r->st;
  delete r;
  return status;
}

extern "C" int gmmnlse_server_destroy(gmmnlse_server* s) {
  if (!s) return GMMNLSE_OK;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    // cancel what has not started; wait for what runs
    for (Request* r : s->queue) {
      s->all.erase(r->ticket);
      delete r;
    }
    s->queue.clear();
    s->cv_done.wait(lk, [&] { return s->inflight == 0; });
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& kv : s->all) delete kv.second;
  for (auto& pj : s->pool) gm_job_destroy(pj.job);
  delete s;
  return GMMNLSE_OK;
}
