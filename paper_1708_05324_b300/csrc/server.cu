// Request server: continuous batching of propagation requests.
//
// Requests enter a FIFO queue and are admitted while the in-flight count and
// the device-byte budget allow (first fit: a request that does not fit yet
// does not hold back a smaller one behind it).  Two ways to run:
//
//  - Packed (same shape).  Requests with the same context and substeps per
//    long step M that run whole long steps (L a multiple of M dz) and no
//    Sec. IV terms share a packed workspace of several slots: one launch
//    advances every occupied slot by one long step (each kernel of the MPA
//    iteration over all slots at once, captured once as a CUDA graph per
//    workspace), and between launches finished requests leave and waiting
//    ones of that shape join.  Each slot keeps its own field, dz, tolerance
//    and convergence, so a result is the same alone and in the pack.
//  - Single.  Any other request runs alone on a worker thread with its own
//    stream and workspace (the path of gmmnlse_propagate).
//
// Device bytes: every workspace the server holds counts against the budget
// while it exists, in use or kept idle for reuse, at its real size; idle
// workspaces (single ones, or a shape's with no request in it) are freed,
// oldest first, when a new one would not fit otherwise.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/gmmnlse.h"
#include "engine.h"

namespace {

// A workspace the server holds, with what it was made for.  `bytes` is
// charged against the budget from the moment it is reserved; `job` is
// allocated by the thread that runs it.
struct Space {
  gmmnlse_ctx* ctx = nullptr;
  int M = 0;
  int slots = 1;
  size_t bytes = 0;
  gm_job* job = nullptr;
  bool busy = false;  // single: a request runs on it
};

struct Request {
  uint64_t ticket = 0;
  gmmnlse_ctx* ctx = nullptr;
  std::vector<double> A0, Aout;
  double L = 0, dz = 0, tol = 0;
  int M = 0;
  bool packed = false;
  Space* space = nullptr;  // single: reserved for it, waiting for a worker
  int status = GMMNLSE_PENDING;
  gmmnlse_stats st{};
};

// The packed requests of one shape (context, M) and the thread that runs them.
struct Group {
  gmmnlse_ctx* ctx = nullptr;
  int M = 0;
  int slots = 1;
  Space* space = nullptr;          // the packed workspace, or none (freed while idle)
  std::deque<Request*> waiting;    // admitted, not yet in a slot
  std::vector<Request*> in_slot;   // [slots]
  std::thread thread;
  std::condition_variable cv;
  bool stop = false;
  bool idle() const {
    if (!waiting.empty()) return false;
    for (Request* r : in_slot)
      if (r) return false;
    return true;
  }
};

constexpr size_t kMaxQueued = 65536;

}  // namespace

struct gmmnlse_server {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;  // not yet admitted, or single and waiting for a worker
  std::map<uint64_t, Request*> all;
  std::list<Space> spaces;     // every workspace held (oldest first)
  std::map<std::pair<gmmnlse_ctx*, int>, std::unique_ptr<Group>> groups;
  std::vector<std::thread> workers;
  std::vector<gm_job*> graveyard;  // released workspaces, freed outside the lock
  size_t budget = 0, resident = 0, peak = 0;
  int max_inflight = 1, inflight = 0, pack_slots = 1;
  uint64_t next_ticket = 1;
  bool stop = false;
};

static size_t space_bytes(gmmnlse_ctx* c, int M, int slots) { return gmmnlse_request_bytes(c, M) * (size_t)slots; }

static Space* reserve(gmmnlse_server* s, gmmnlse_ctx* c, int M, int slots, bool busy) {
  const size_t b = space_bytes(c, M, slots);
  s->spaces.push_back(Space{c, M, slots, b, nullptr, busy});
  s->resident += b;
  s->peak = std::max(s->peak, s->resident);
  return &s->spaces.back();
}

// Lock held: the workspace's memory is freed by drain() after the lock is
// let go (freeing waits for the device).
static void release(gmmnlse_server* s, Space* sp) {
  if (sp->job) s->graveyard.push_back(sp->job);
  s->resident -= sp->bytes;
  for (auto it = s->spaces.begin(); it != s->spaces.end(); ++it)
    if (&*it == sp) {
      s->spaces.erase(it);
      return;
    }
}

// Free the released workspaces (lock not held).
static void drain(gmmnlse_server* s) {
  std::vector<gm_job*> dead;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    dead.swap(s->graveyard);
  }
  for (gm_job* j : dead) gm_job_destroy(j);
}

// Make room for `need` more bytes by freeing idle workspaces, oldest first;
// true if they fit.  Lock held.
static bool make_room(gmmnlse_server* s, size_t need) {
  if (s->resident + need <= s->budget) return true;
  std::vector<Space*> order;
  for (auto& sp : s->spaces) order.push_back(&sp);
  for (Space* sp : order) {
    if (s->resident + need <= s->budget) break;
    Group* owner = nullptr;
    for (auto& kv : s->groups)
      if (kv.second->space == sp) owner = kv.second.get();
    if (owner) {
      if (!owner->idle()) continue;
      owner->space = nullptr;  // (its thread uses the workspace only while it holds requests)
    } else if (sp->busy) {
      continue;
    }
    release(s, sp);
  }
  return s->resident + need <= s->budget;
}

static void group_main(gmmnlse_server* s, Group* gp);

// Admit what the in-flight count and the budget allow, first fit.  Lock held.
static void dispatch(gmmnlse_server* s) {
  for (auto it = s->queue.begin(); it != s->queue.end() && s->inflight < s->max_inflight;) {
    Request* r = *it;
    if (r->space) {  // single, already admitted
      ++it;
      continue;
    }
    bool admitted = false;
    if (r->packed) {
      const auto key = std::make_pair(r->ctx, r->M);
      auto g = s->groups.find(key);
      if (g == s->groups.end()) {
        std::unique_ptr<Group> gp(new Group());
        gp->ctx = r->ctx;
        gp->M = r->M;
        gp->slots = s->pack_slots;
        gp->in_slot.assign(gp->slots, nullptr);
        Group* raw = gp.get();
        g = s->groups.emplace(key, std::move(gp)).first;
        raw->thread = std::thread(group_main, s, raw);
      }
      Group* gp = g->second.get();
      if (!gp->space && make_room(s, space_bytes(r->ctx, r->M, gp->slots)))
        gp->space = reserve(s, r->ctx, r->M, gp->slots, false);
      if (gp->space) {
        gp->waiting.push_back(r);
        gp->cv.notify_one();
        it = s->queue.erase(it);
        admitted = true;
      }
    } else {
      // an idle workspace of the same context with M' >= M, or a new one
      for (auto& sp : s->spaces) {
        bool owned = false;
        for (auto& kv : s->groups)
          if (kv.second->space == &sp) owned = true;
        if (!owned && !sp.busy && sp.slots == 1 && sp.ctx == r->ctx && sp.M >= r->M) {
          sp.busy = true;
          r->space = &sp;
          break;
        }
      }
      if (!r->space && make_room(s, space_bytes(r->ctx, r->M, 1))) r->space = reserve(s, r->ctx, r->M, 1, true);
      admitted = r->space != nullptr;
      ++it;  // stays queued until a worker takes it
    }
    if (admitted) s->inflight += 1;
    else if (r->packed) ++it;
  }
}

// Single requests: a worker takes the first queued request with a reserved
// workspace, runs it, and keeps the workspace for reuse.
static void worker_main(gmmnlse_server* s) {
  cudaStream_t stream = nullptr;
  int stream_dev = -1;
  for (;;) {
    Request* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      auto ready = [&] {
        for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
          if ((*it)->space) return it;
        return s->queue.end();
      };
      s->cv_work.wait(lk, [&] { return s->stop || ready() != s->queue.end(); });
      if (s->stop) break;
      auto it = ready();
      r = *it;
      s->queue.erase(it);
    }
    Space* sp = r->space;
    const int dev = gm_ctx_device(r->ctx);
    int rc = cudaSetDevice(dev) == cudaSuccess ? GMMNLSE_OK : GMMNLSE_E_CUDA;
    if (!rc && stream_dev != dev) {
      if (stream) cudaStreamDestroy(stream);
      stream = nullptr;
      rc = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess ? GMMNLSE_OK : GMMNLSE_E_CUDA;
      stream_dev = rc ? -1 : dev;
    }
    if (!rc && !sp->job) rc = gm_job_create(r->ctx, sp->M, &sp->job);
    if (!rc) {
      r->Aout.resize(r->A0.size());
      rc = gm_job_propagate(sp->job, r->A0.data(), false, r->L, r->dz, r->M, r->tol, r->Aout.data(), &r->st, stream);
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      r->status = rc;
      r->space = nullptr;
      s->inflight -= 1;
      if (!sp->job) release(s, sp);  // its allocation failed
      else sp->busy = false;
      dispatch(s);
    }
    drain(s);
    s->cv_work.notify_all();
    s->cv_done.notify_all();
  }
  if (stream) cudaStreamDestroy(stream);
}

// The thread of one shape: fill free slots from the waiting requests, run one
// packed long step, hand back the requests that ended, repeat.
static void group_main(gmmnlse_server* s, Group* gp) {
  cudaStream_t stream = nullptr;
  int srs = cudaSetDevice(gm_ctx_device(gp->ctx)) == cudaSuccess ? GMMNLSE_OK : GMMNLSE_E_CUDA;
  if (!srs) srs = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) == cudaSuccess ? GMMNLSE_OK : GMMNLSE_E_CUDA;
  std::vector<int> finished(gp->slots, 0);
  for (;;) {
    std::vector<std::pair<int, Request*>> joining;
    Space* sp = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      gp->cv.wait(lk, [&] { return gp->stop || !gp->idle(); });
      if (gp->idle()) break;  // stopping, nothing left
      sp = gp->space;
      for (int b = 0; b < gp->slots && !gp->waiting.empty(); ++b)
        if (!gp->in_slot[b]) {
          gp->in_slot[b] = gp->waiting.front();
          gp->waiting.pop_front();
          joining.push_back({b, gp->in_slot[b]});
        }
    }
    int rc = srs;
    if (!rc && !sp->job) rc = gm_job_create_slots(gp->ctx, gp->M, gp->slots, &sp->job);
    std::vector<std::pair<Request*, int>> ended;
    for (auto& jr : joining) {
      const int e = rc ? rc
                       : gm_pack_admit(sp->job, jr.first, jr.second->A0.data(), jr.second->L, jr.second->dz,
                                       jr.second->tol, stream);
      if (e) {
        ended.push_back({jr.second, e});
        gp->in_slot[jr.first] = nullptr;
      }
    }
    bool any = false;
    for (Request* q : gp->in_slot)
      if (q) any = true;
    if (any) {
      const int e = rc ? rc : gm_pack_step(sp->job, stream, finished.data());
      for (int b = 0; b < gp->slots; ++b) {
        Request* q = gp->in_slot[b];
        if (!q || (!finished[b] && !e)) continue;
        q->Aout.resize(q->A0.size());
        const int st = rc ? rc : gm_pack_retire(sp->job, b, q->Aout.data(), &q->st, stream);
        ended.push_back({q, e ? e : st});
        gp->in_slot[b] = nullptr;
      }
    }
    if (!ended.empty()) {
      {
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto& er : ended) {
          er.first->status = er.second;
          s->inflight -= 1;
        }
        dispatch(s);
      }
      drain(s);
      s->cv_done.notify_all();
      s->cv_work.notify_all();
    }
  }
  if (stream) cudaStreamDestroy(stream);
}

extern "C" int gmmnlse_server_create(size_t hbm_budget, int max_inflight, gmmnlse_server** out) {
  if (!out || hbm_budget == 0 || max_inflight < 1 || max_inflight > 256) return GMMNLSE_E_INVALID;
  gmmnlse_server* s = new (std::nothrow) gmmnlse_server();
  if (!s) return GMMNLSE_E_NOMEM;
  s->budget = hbm_budget;
  s->max_inflight = max_inflight;
  s->pack_slots = std::min(max_inflight, 16);
  // GMMNLSE_PACK_SLOTS overrides the slots of a packed workspace (1: no packing)
  if (const char* v = getenv("GMMNLSE_PACK_SLOTS")) s->pack_slots = std::max(1, std::min(16, atoi(v)));
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
  bool packed = s->pack_slots > 1 && gm_packable(ctx, L, dz, M);
  // a packed workspace that does not fit the budget: run it alone
  if (packed && space_bytes(ctx, M, s->pack_slots) > s->budget) packed = false;
  if (space_bytes(ctx, M, 1) > s->budget) return GMMNLSE_E_NOMEM;
  Request* r = new (std::nothrow) Request();
  if (!r) return GMMNLSE_E_NOMEM;
  const size_t cnt = (size_t)gm_ctx_modes(ctx) * gm_ctx_samples(ctx) * 2;
  r->ctx = ctx;
  r->A0.assign(A0, A0 + cnt);
  r->L = L;
  r->dz = dz;
  r->M = M;
  r->tol = tol;
  r->packed = packed;
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
    dispatch(s);
  }
  drain(s);
  s->cv_work.notify_all();
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

extern "C" int gmmnlse_cancel(gmmnlse_server* s, uint64_t ticket) {
  if (!s) return GMMNLSE_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return GMMNLSE_E_INVALID;
  Request* r = it->second;
  if (r->status != GMMNLSE_PENDING) return GMMNLSE_OK;  // finished: its poll reports the result
  for (auto q = s->queue.begin(); q != s->queue.end(); ++q)
    if (*q == r && !r->space) {  // not admitted yet
      s->queue.erase(q);
      r->status = GMMNLSE_E_CANCELLED;
      return GMMNLSE_OK;
    }
  for (auto& kv : s->groups) {
    auto& w = kv.second->waiting;
    for (auto q = w.begin(); q != w.end(); ++q)
      if (*q == r) {  // admitted, not in a slot yet
        w.erase(q);
        s->inflight -= 1;
        r->status = GMMNLSE_E_CANCELLED;
        dispatch(s);
        return GMMNLSE_OK;
      }
  }
  return GMMNLSE_E_BUSY;  // running: it completes normally
}

extern "C" int gmmnlse_server_resident_bytes(gmmnlse_server* s, size_t* now, size_t* peak) {
  if (!s) return GMMNLSE_E_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  if (now) *now = s->resident;
  if (peak) *peak = s->peak;
  return GMMNLSE_OK;
}

extern "C" int gmmnlse_server_destroy(gmmnlse_server* s) {
  if (!s) return GMMNLSE_OK;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    // cancel what has not started; wait for what runs
    for (auto it = s->queue.begin(); it != s->queue.end();) {
      Request* r = *it;
      if (r->space) {  // admitted: a worker runs it
        ++it;
        continue;
      }
      s->all.erase(r->ticket);
      delete r;
      it = s->queue.erase(it);
    }
    for (auto& kv : s->groups) {
      for (Request* r : kv.second->waiting) {
        s->all.erase(r->ticket);
        s->inflight -= 1;
        delete r;
      }
      kv.second->waiting.clear();
    }
    s->cv_done.wait(lk, [&] { return s->inflight == 0; });
    s->stop = true;
    for (auto& kv : s->groups) {
      kv.second->stop = true;
      kv.second->cv.notify_all();
    }
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& kv : s->groups)
    if (kv.second->thread.joinable()) kv.second->thread.join();
  for (auto& kv : s->all) delete kv.second;
  for (auto& sp : s->spaces)
    if (sp.job) gm_job_destroy(sp.job);
  for (gm_job* j : s->graveyard) gm_job_destroy(j);
  delete s;
  return GMMNLSE_OK;
}
