// qp_serve.cu -- continuous-batching request server (host runtime of the
// qp_serve_* calls in qp.h), in two modes.
//
// Launches (QP_SERVE_LAUNCHES).  Requests of any supported size arrive one at
// a time (qp_serve_submit copies their data).  A scheduler thread turns the
// queue into ragged launches: the oldest waiting request picks the kernel
// class (shared-memory kernel with 128 or 512 threads, or the large-problem
// variant) and the launch takes every waiting request of that class, up to
// max_batch and up to the free device memory, in arrival order.  A class may
// occupy the last free stream only while it has fewer than
// max(1, max_inflight / 3) launches in flight, so requests of another class
// always find a stream even while long launches of one class run.  Each
// launch owns one stream and one block of the device arena laid out as
// [inputs | outputs | caches, workspaces]: one upload, the forward kernel over
// all requests (one CTA each, sizes from a descriptor table), the backward
// kernel over those that asked for gradients, one download.  Up to
// max_inflight launches run at once.  A request's arithmetic does not depend
// on the launch it lands in (one CTA per instance, the same kernel class and
// size-derived configuration as a qp_solve_batch of that size), so served
// results equal solo results bit for bit.
//
// Persistent (QP_SERVE_PERSISTENT).  Each admitted request gets its own arena
// block [inputs | outputs | cache, workspace]; its inputs are uploaded (one
// stream, one event per scheduler pass) and, once they are on the device,
// its descriptor is published in a ring in mapped host memory (descriptor
// first, then the tail with release semantics).  The resident CTAs of
// qp_serve_persist.cu claim descriptors in order and write each request's
// outputs into the mapped host mirror of its block, then its completion word;
// the scheduler collects completed requests in any order.  A ring slot is
// reused only after its previous request completed.  The scheduler keeps one
// CTA per SM resident while work is queued, published or uploading: CTAs
// count themselves out in the control block when they leave (idle, lifetime,
// stop), and the scheduler launches as many as are missing.
//
// Memory admission (both modes): a request reserves its
// qp_serve_footprint_bytes in the arena (first fit); a request larger than
// the arena is refused at submit.  The scheduler detects completion by
// polling events or completion words (no host callbacks) and never holds its
// lock while it calls into CUDA, so nothing the runtime does (for example
// loading a module on a kernel's first launch) can wait on this file's lock.
// Every wait here is bounded.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "qp.h"
#include "qp_internal.h"

using namespace qpgpu;

namespace {

constexpr size_t kAlign = 256;  // arena granularity in bytes

long long r4(long long v) { return (v + 3) & ~3LL; }

// Kernel configuration of one problem size.
struct SizeCfg {
  int nt = 0, amax = 0, bnt = 0;
  bool split = false;
  size_t fsmem = 0, bsmem = 0;
  long long ws = 0, cache = 0;  // floats per instance
  int cls() const { return split ? 2 : (nt == 128 ? 0 : 1); }
};

// persistent: every size at 512 threads (the resident kernel's width; the
// amax, so the cache layout, is the default's), within its shared memory
bool size_cfg(int n, int m, int p, SizeCfg* c, bool persistent = false) {
  if (n < 1 || p < 0 || p > n || m < 0) return false;
  long long ws = 0;
  c->fsmem = forward_config(n, m, p, &c->nt, &c->amax, &ws, false, 512, persistent);
  if (c->fsmem == 0) return false;
  c->split = ws > 0;
  c->ws = ws;
  c->bsmem = backward_smem_bytes(n, m, p, c->amax, c->split, &c->bnt);
  if (c->bsmem == 0) return false;
  if (persistent && (c->fsmem > serve_kernel_smem() || c->bsmem > serve_kernel_smem()))
    return false;
  c->cache = cache_layout(n, m, p, c->amax, c->split).stride;
  return true;
}

// Floats of one request's three regions.
struct Footprint {
  long long in, out, dev;
};

Footprint footprint(int n, int m, int p, bool grad, const SizeCfg& c) {
  Footprint f;
  f.in = r4((long long)n * n) + r4(n) + r4((long long)p * n) + r4(p) + r4((long long)m * n) +
         r4(m) + (grad ? r4(n) : 0);
  f.out = r4(n) + r4(p) + 2 * r4(m) + 4 +
          (grad ? r4((long long)n * n) + r4(n) + r4((long long)p * n) + r4(p) +
                      r4((long long)m * n) + r4(m)
                : 0);
  f.dev = (grad ? r4(c.cache) : 0) + (c.split ? r4(c.ws) : 0);
  return f;
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// First-fit allocator over [0, size) in kAlign units.
class Arena {
 public:
  explicit Arena(size_t size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = round_up(bytes, kAlign);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = round_up(bytes, kAlign);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t largest() const {
    size_t b = 0;
    for (const auto& kv : free_) b = kv.second > b ? kv.second : b;
    return b;
  }

 private:
  std::map<size_t, size_t> free_;
};

enum State { kQueued, kLaunched, kDone, kFailed };

struct Req {
  uint64_t ticket = 0;
  int n = 0, m = 0, p = 0;
  bool grad = false;
  SizeCfg cfg;
  Footprint fp{};
  std::vector<float> in;   // Q, q, A, b, G, h (, g) as submitted, packed
  std::vector<float> out;  // x, y, z, s, status, iters, kkt (, gradients) after completion
  float *x = nullptr, *y = nullptr, *z = nullptr, *s = nullptr;
  float *dQ = nullptr, *dq = nullptr, *dA = nullptr, *db = nullptr, *dG = nullptr,
        *dh = nullptr;
  State state = kQueued;
  int err = QP_OK;
  double t_submit = 0, t_launch = 0, t_done = 0;
  // persistent mode: the request's own arena block and ring sequence number
  size_t off = 0, bytes = 0;
  uint32_t seq = 0;
};

// Persistent mode: inputs uploaded in one scheduler pass, published when the
// pass's event has completed.
struct Upload {
  cudaEvent_t ev = nullptr;
  std::vector<Req*> reqs;
};

struct Launch {
  bool busy = false;
  int cls = 0;  // kernel class of the requests in flight
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;  // recorded after the launch's download
  ReqDesc* hdesc = nullptr;  // pinned: forward descriptors, then backward ones
  ReqDesc* ddesc = nullptr;  // device copy
  size_t off = 0, bytes = 0;
  long long in_floats = 0, out_floats = 0;
  std::vector<Req*> reqs;
  std::vector<long long> out_off;  // floats from the block start
};

}  // namespace

struct qp_server {
  qp_serve_config cfg;
  FwdParams base;  // settings of every launch
  int device = 0;
  float* dmem = nullptr;  // device arena
  float* hmem = nullptr;  // pinned mirror of the arena (inputs and outputs)
  std::unique_ptr<Arena> arena;
  std::vector<Launch> launches;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> pending;
  std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
  std::deque<uint64_t> done_fifo;
  uint64_t next_ticket = 1;
  bool stop = false;
  int fatal = QP_OK;
  std::thread worker;
  std::chrono::steady_clock::time_point t0;

  // persistent mode (mapped host memory: ring, done, ctl; device: head)
  bool persistent = false;
  ServeParams sp{};        // kernel parameters (device views of the above)
  ReqDesc* ring = nullptr;
  uint32_t* done = nullptr;
  ServeCtl* ctl = nullptr;
  uint32_t* head = nullptr;
  float* hmem_dev = nullptr;  // device view of hmem (outputs are written there)
  uint32_t cap = 0;
  uint32_t next_seq = 0;   // next ring sequence number to publish
  uint32_t launched = 0;   // CTAs started so far
  int target = 0;          // CTAs resident at most (one per SM)
  cudaStream_t up_stream = nullptr;
  // resident CTAs are started on an idle stream of this pool, so that CTAs
  // topped up while earlier ones still run start at once instead of queueing
  // behind the earlier kernel on its stream
  std::vector<cudaStream_t> k_streams;
  std::deque<Upload> uploads;         // inputs in flight, publication order
  std::vector<cudaEvent_t> ev_pool;   // free upload events
  std::vector<Req*> published;        // published, not yet complete
  size_t inflight_reqs = 0;           // uploading + published

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
        .count();
  }
  void run();
  bool take_group(Launch& L);
  cudaError_t issue(Launch& L);
  void finish_launch(Launch& L);
  void fail_launch(Launch& L);
  void fail_pending();
  // persistent mode
  void run_persistent();
  void fail_all_persistent();
};


// Select the next group and reserve its arena block (called with mu held):
// the oldest waiting request whose class may take a stream picks the class.
bool qp_server::take_group(Launch& L) {
  if (pending.empty()) return false;
  int inflight[3] = {0, 0, 0}, nfree = 0;
  for (const Launch& o : launches) {
    if (o.busy) ++inflight[o.cls];
    else ++nfree;
  }
  const int cap = cfg.max_inflight / 3 > 1 ? cfg.max_inflight / 3 : 1;
  int cls = -1;
  for (const Req* r : pending) {
    const int c = r->cfg.cls();
    if (inflight[c] < cap || nfree > 1) {
      cls = c;
      break;
    }
  }
  if (cls < 0) return false;
  const size_t room = arena->largest();
  std::vector<Req*> take;
  long long in_f = 0, out_f = 0, dev_f = 0;
  for (Req* r : pending) {
    if ((int)take.size() >= cfg.max_batch) break;
    if (r->cfg.cls() != cls) continue;
    const size_t need =
        (size_t)(in_f + out_f + dev_f + r->fp.in + r->fp.out + r->fp.dev) * sizeof(float);
    if (round_up(need, kAlign) > room) break;
    take.push_back(r);
    in_f += r->fp.in;
    out_f += r->fp.out;
    dev_f += r->fp.dev;
  }
  if (take.empty()) return false;  // waits for memory
  size_t off = 0;
  const size_t bytes = (size_t)(in_f + out_f + dev_f) * sizeof(float);
  if (!arena->alloc(bytes, &off)) return false;
  // remove the taken requests from the queue, keeping the others in order
  std::deque<Req*> rest;
  size_t k = 0;
  for (Req* r : pending) {
    if (k < take.size() && r == take[k]) ++k;
    else rest.push_back(r);
  }
  pending.swap(rest);

  L.busy = true;
  L.cls = cls;
  L.off = off;
  L.bytes = bytes;
  L.in_floats = in_f;
  L.out_floats = out_f;
  L.reqs = take;
  L.out_off.assign(take.size(), 0);
  const double t = now_ms();
  for (Req* r : take) {
    r->state = kLaunched;
    r->t_launch = t;
  }
  return true;
}

// Stage the group's inputs and issue its work on its stream (called without
// mu: only the scheduler thread touches a busy launch and its requests).
cudaError_t qp_server::issue(Launch& L) {
  const std::vector<Req*>& take = L.reqs;
  const long long in_f = L.in_floats, out_f = L.out_floats;
  float* hb = hmem + L.off / sizeof(float);
  float* db = dmem + L.off / sizeof(float);
  long long io = 0, oo = in_f, dv = in_f + out_f;
  size_t fsmem = 0, bsmem = 0;
  int nb = 0;
  const int R = (int)take.size();
  for (int i = 0; i < R; ++i) {
    Req* r = take[i];
    const int n = r->n, m = r->m, p = r->p;
    memcpy(hb + io, r->in.data(), r->in.size() * sizeof(float));
    ReqDesc d;
    memset(&d, 0, sizeof(d));
    d.n = n; d.m = m; d.p = p; d.amax = r->cfg.amax;
    long long o = io;
    d.Q = db + o; o += r4((long long)n * n);
    d.q = db + o; o += r4(n);
    d.A = db + o; o += r4((long long)p * n);
    d.b = db + o; o += r4(p);
    d.G = db + o; o += r4((long long)m * n);
    d.h = db + o; o += r4(m);
    if (r->grad) { d.g = db + o; o += r4(n); }
    io += r->fp.in;
    L.out_off[i] = oo;
    o = oo;
    d.x = db + o; o += r4(n);
    d.y = db + o; o += r4(p);
    d.z = db + o; o += r4(m);
    d.s = db + o; o += r4(m);
    d.status = reinterpret_cast<int32_t*>(db + o);
    d.iters = reinterpret_cast<int32_t*>(db + o + 1);
    d.kkt = db + o + 2;
    o += 4;
    if (r->grad) {
      d.dQ = db + o; o += r4((long long)n * n);
      d.dq = db + o; o += r4(n);
      d.dA = db + o; o += r4((long long)p * n);
      d.db = db + o; o += r4(p);
      d.dG = db + o; o += r4((long long)m * n);
      d.dh = db + o; o += r4(m);
    }
    oo += r->fp.out;
    o = dv;
    if (r->grad) { d.cache = db + o; o += r4(r->cfg.cache); }
    if (r->cfg.split) { d.ws = db + o; o += r4(r->cfg.ws); }
    dv += r->fp.dev;
    L.hdesc[i] = d;
    if (r->grad) L.hdesc[R + nb++] = d;
    fsmem = r->cfg.fsmem > fsmem ? r->cfg.fsmem : fsmem;
    if (r->grad) bsmem = r->cfg.bsmem > bsmem ? r->cfg.bsmem : bsmem;
  }
  cudaError_t e = cudaMemcpyAsync(db, hb, (size_t)in_f * sizeof(float), cudaMemcpyHostToDevice,
                                  L.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(L.ddesc, L.hdesc, (size_t)(R + nb) * sizeof(ReqDesc),
                        cudaMemcpyHostToDevice, L.stream);
  if (e == cudaSuccess) {
    FwdParams P = base;
    P.batch = R;
    P.desc = L.ddesc;
    const SizeCfg& c0 = take[0]->cfg;
    P.ws = c0.split ? db : nullptr;  // selects the large variant; CTAs use their descriptor's
    if (!c0.split) P.gwg = 0;  // tensor-core G'WG: large variant only
    e = launch_forward(P, c0.nt, fsmem, R, L.stream);
  }
  if (e == cudaSuccess && nb > 0) {
    BwdParams B;
    memset(&B, 0, sizeof(B));
    B.batch = nb;
    B.split = take[0]->cfg.split ? 1 : 0;
    B.desc = L.ddesc + R;
    e = launch_backward(B, backward_threads(take[0]->n, take[0]->cfg.split), bsmem,
                        L.stream);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hb + in_f, db + in_f, (size_t)out_f * sizeof(float),
                        cudaMemcpyDeviceToHost, L.stream);
  if (e == cudaSuccess) e = cudaEventRecord(L.done, L.stream);
  return e;
}

// After a device error no request is admitted any more: the ones still
// queued fail too (they hold no arena block yet), so that their callers get
// QP_ECUDA instead of waiting out their timeouts (called with mu held).
void qp_server::fail_pending() {
  const double t = now_ms();
  for (Req* r : pending) {
    r->state = kFailed;
    r->err = QP_ECUDA;
    r->t_done = t;
    done_fifo.push_back(r->ticket);
  }
  pending.clear();
}

// A launch whose issue or execution failed: drain its stream (without mu),
// then fail its requests and release its block (with mu).
void qp_server::fail_launch(Launch& L) {
  cudaGetLastError();
  for (Req* r : L.reqs) {
    r->state = kFailed;
    r->err = QP_ECUDA;
    r->t_done = now_ms();
    done_fifo.push_back(r->ticket);
  }
  arena->release(L.off, L.bytes);
  L.reqs.clear();
  L.busy = false;
  fatal = QP_ECUDA;
  fail_pending();
  cv_done.notify_all();
}

// Collect the results of a finished launch (called with mu held).
void qp_server::finish_launch(Launch& L) {
  const float* hb = hmem + L.off / sizeof(float);
  const double t = now_ms();
  for (size_t i = 0; i < L.reqs.size(); ++i) {
    Req* r = L.reqs[i];
    r->out.assign(hb + L.out_off[i], hb + L.out_off[i] + r->fp.out);
    r->state = kDone;
    r->t_done = t;
    r->in.clear();
    r->in.shrink_to_fit();
    done_fifo.push_back(r->ticket);
  }
  arena->release(L.off, L.bytes);
  L.reqs.clear();
  L.busy = false;
  cv_done.notify_all();
}

void qp_server::run() {
  cudaSetDevice(device);
  if (persistent) {
    run_persistent();
    return;
  }
  std::unique_lock<std::mutex> lock(mu);
  while (!stop) {
    bool progress = false, inflight = false;
    for (Launch& L : launches) {
      if (!L.busy) continue;
      const cudaError_t q = cudaEventQuery(L.done);
      if (q == cudaSuccess) {
        finish_launch(L);
        progress = true;
      } else if (q != cudaErrorNotReady) {
        lock.unlock();
        cudaStreamSynchronize(L.stream);
        lock.lock();
        fail_launch(L);
        progress = true;
      } else {
        inflight = true;
      }
    }
    for (Launch& L : launches) {
      if (fatal != QP_OK || L.busy || pending.empty()) continue;
      if (!take_group(L)) break;  // waits for arena memory or a stream of its class
      lock.unlock();
      const cudaError_t e = issue(L);
      if (e != cudaSuccess) cudaStreamSynchronize(L.stream);  // drain what was issued
      lock.lock();
      if (e != cudaSuccess) fail_launch(L);
      progress = true;
      inflight = true;
    }
    if (!progress)
      cv_work.wait_for(lock, inflight ? std::chrono::microseconds(100)
                                      : std::chrono::microseconds(20000));
  }
}

// ---- persistent mode ------------------------------------------------------

namespace {

// Lay out a request's block [inputs | outputs | cache, workspace] and fill
// its descriptor: inputs, cache and workspace in the device arena, outputs in
// the mapped host mirror.
ReqDesc persistent_desc(const Req* r, float* db, float* hb_dev) {
  const int n = r->n, m = r->m, p = r->p;
  ReqDesc d;
  memset(&d, 0, sizeof(d));
  d.n = n; d.m = m; d.p = p; d.amax = r->cfg.amax; d.bnt = r->cfg.bnt;
  long long o = 0;
  d.Q = db + o; o += r4((long long)n * n);
  d.q = db + o; o += r4(n);
  d.A = db + o; o += r4((long long)p * n);
  d.b = db + o; o += r4(p);
  d.G = db + o; o += r4((long long)m * n);
  d.h = db + o; o += r4(m);
  if (r->grad) { d.g = db + o; o += r4(n); }
  o = r->fp.in;
  d.x = hb_dev + o; o += r4(n);
  d.y = hb_dev + o; o += r4(p);
  d.z = hb_dev + o; o += r4(m);
  d.s = hb_dev + o; o += r4(m);
  d.status = reinterpret_cast<int32_t*>(hb_dev + o);
  d.iters = reinterpret_cast<int32_t*>(hb_dev + o + 1);
  d.kkt = hb_dev + o + 2;
  o += 4;
  if (r->grad) {
    d.dQ = hb_dev + o; o += r4((long long)n * n);
    d.dq = hb_dev + o; o += r4(n);
    d.dA = hb_dev + o; o += r4((long long)p * n);
    d.db = hb_dev + o; o += r4(p);
    d.dG = hb_dev + o; o += r4((long long)m * n);
    d.dh = hb_dev + o; o += r4(m);
  }
  o = r->fp.in + r->fp.out;
  if (r->grad) { d.cache = db + o; o += r4(r->cfg.cache); }
  if (r->cfg.split) { d.ws = db + o; o += r4(r->cfg.ws); }
  return d;
}

}  // namespace

// After a device error: every request in flight fails (called with mu held).
void qp_server::fail_all_persistent() {
  cudaGetLastError();
  const double t = now_ms();
  auto fail = [&](Req* r) {
    r->state = kFailed;
    r->err = QP_ECUDA;
    r->t_done = t;
    arena->release(r->off, r->bytes);
    done_fifo.push_back(r->ticket);
  };
  for (Upload& u : uploads) {
    for (Req* r : u.reqs) fail(r);
    ev_pool.push_back(u.ev);
  }
  uploads.clear();
  for (Req* r : published) fail(r);
  published.clear();
  inflight_reqs = 0;
  fatal = QP_ECUDA;
  fail_pending();
  cv_done.notify_all();
}

void qp_server::run_persistent() {
  std::unique_lock<std::mutex> lock(mu);
  while (!stop) {
    bool progress = false;
    // 1. completions, in any order: the outputs are in the mapped mirror
    if (!published.empty()) {
      const double t = now_ms();
      for (size_t i = 0; i < published.size();) {
        Req* r = published[i];
        if (__atomic_load_n(done + (r->seq % cap), __ATOMIC_ACQUIRE) != r->seq + 1u) {
          ++i;
          continue;
        }
        const float* hb = hmem + r->off / sizeof(float) + r->fp.in;
        r->out.assign(hb, hb + r->fp.out);
        r->state = kDone;
        r->t_done = t;
        r->in.clear();
        r->in.shrink_to_fit();
        arena->release(r->off, r->bytes);
        done_fifo.push_back(r->ticket);
        published[i] = published.back();
        published.pop_back();
        --inflight_reqs;
        progress = true;
      }
      if (progress) cv_done.notify_all();
    }
    // 2. uploads that have landed: publish their descriptors in order, each
    //    into a ring slot whose previous request is complete
    while (!uploads.empty() && fatal == QP_OK) {
      const cudaError_t q = cudaEventQuery(uploads.front().ev);
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) {
        fail_all_persistent();
        break;
      }
      uint32_t oldest = next_seq;
      for (const Req* r : published)
        if ((int32_t)(r->seq - oldest) < 0) oldest = r->seq;
      Upload& u = uploads.front();
      if ((uint32_t)(next_seq + (uint32_t)u.reqs.size() - oldest) > cap) break;  // ring full
      const double t = now_ms();
      for (Req* r : u.reqs) {
        r->seq = next_seq++;
        ring[r->seq % cap] = persistent_desc(r, dmem + r->off / sizeof(float),
                                             hmem_dev + r->off / sizeof(float));
        r->state = kLaunched;
        r->t_launch = t;
        published.push_back(r);
      }
      __atomic_store_n(&ctl->tail, next_seq, __ATOMIC_RELEASE);
      ev_pool.push_back(u.ev);
      uploads.pop_front();
      progress = true;
    }
    // 3. admission: reserve blocks, stage and upload the inputs (one event)
    if (fatal == QP_OK && !pending.empty() && !ev_pool.empty()) {
      std::vector<Req*> batch;
      while (!pending.empty() && inflight_reqs + batch.size() < cap) {
        Req* r = pending.front();
        size_t off = 0;
        const size_t bytes = (size_t)(r->fp.in + r->fp.out + r->fp.dev) * sizeof(float);
        if (!arena->alloc(bytes, &off)) break;  // waits for memory
        r->off = off;
        r->bytes = bytes;
        batch.push_back(r);
        pending.pop_front();
      }
      if (!batch.empty()) {
        cudaEvent_t ev = ev_pool.back();
        ev_pool.pop_back();
        inflight_reqs += batch.size();
        lock.unlock();
        cudaError_t e = cudaSuccess;
        for (Req* r : batch) {
          float* hb = hmem + r->off / sizeof(float);
          memcpy(hb, r->in.data(), r->in.size() * sizeof(float));
          if (e == cudaSuccess)
            e = cudaMemcpyAsync(dmem + r->off / sizeof(float), hb, r->in.size() * sizeof(float),
                                cudaMemcpyHostToDevice, up_stream);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev, up_stream);
        if (e != cudaSuccess) cudaStreamSynchronize(up_stream);
        lock.lock();
        Upload u;
        u.ev = ev;
        u.reqs = std::move(batch);
        uploads.push_back(std::move(u));
        if (e != cudaSuccess) fail_all_persistent();
        progress = true;
      }
    }
    // 4. resident CTAs: while there is work, keep one per SM, topping up on
    //    an idle stream; a kernel that failed on the device leaves its stream
    //    in error
    const bool work = fatal == QP_OK && (!uploads.empty() || !published.empty());
    if (work) {
      const uint32_t gone = __atomic_load_n(&ctl->exited, __ATOMIC_ACQUIRE);
      const int live = (int)(launched - gone);
      lock.unlock();
      cudaStream_t idle = nullptr;
      bool broken = false;
      for (cudaStream_t st : k_streams) {
        const cudaError_t q = cudaStreamQuery(st);
        if (q == cudaSuccess) {
          if (!idle) idle = st;
        } else if (q != cudaErrorNotReady) {
          broken = true;
        }
      }
      cudaError_t e = cudaSuccess;
      int grid = 0;
      if (!broken && live < target && idle) {
        grid = target - live;
        e = launch_serve_kernel(sp, grid, idle);
      }
      lock.lock();
      if (broken || e != cudaSuccess) {
        fail_all_persistent();
      } else if (grid > 0) {
        launched += (uint32_t)grid;
        progress = true;
      }
    }
    if (!progress)
      cv_work.wait_for(lock, work ? std::chrono::microseconds(20)
                                  : std::chrono::microseconds(20000));
  }
}

namespace {

int fill_result(qp_server* sv, Req* r, qp_result* res) {
  if (res) {
    memset(res, 0, sizeof(*res));
    res->ticket = r->ticket;
    res->t_submit_ms = r->t_submit;
    res->t_launch_ms = r->t_launch;
    res->t_done_ms = r->t_done;
  }
  const int rc = r->state == kFailed ? r->err : QP_OK;
  if (r->state == kDone) {
    const int n = r->n, m = r->m, p = r->p;
    const float* o = r->out.data();
    auto put = [&](float* dst, long long cnt, long long adv) {
      if (dst && cnt) memcpy(dst, o, (size_t)cnt * sizeof(float));
      o += adv;
    };
    put(r->x, n, r4(n));
    put(r->y, p, r4(p));
    put(r->z, m, r4(m));
    put(r->s, m, r4(m));
    if (res) {
      res->status = reinterpret_cast<const int32_t*>(o)[0];
      res->iters = reinterpret_cast<const int32_t*>(o)[1];
      res->kkt_res = o[2];
    }
    o += 4;
    if (r->grad) {
      put(r->dQ, (long long)n * n, r4((long long)n * n));
      put(r->dq, n, r4(n));
      put(r->dA, (long long)p * n, r4((long long)p * n));
      put(r->db, p, r4(p));
      put(r->dG, (long long)m * n, r4((long long)m * n));
      put(r->dh, m, r4(m));
    }
  }
  sv->reqs.erase(r->ticket);
  return rc;
}

}  // namespace

namespace {

void free_persistent(qp_server* sv) {
  for (cudaEvent_t ev : sv->ev_pool) cudaEventDestroy(ev);
  sv->ev_pool.clear();
  for (Upload& u : sv->uploads)
    if (u.ev) cudaEventDestroy(u.ev);
  sv->uploads.clear();
  if (sv->up_stream) cudaStreamDestroy(sv->up_stream);
  for (cudaStream_t st : sv->k_streams) cudaStreamDestroy(st);
  sv->k_streams.clear();
  if (sv->ring) cudaFreeHost(sv->ring);
  if (sv->done) cudaFreeHost(sv->done);
  if (sv->ctl) cudaFreeHost(sv->ctl);
  if (sv->head) cudaFree(sv->head);
  sv->up_stream = nullptr;
  sv->ring = nullptr;
  sv->done = nullptr;
  sv->ctl = nullptr;
  sv->head = nullptr;
}

}  // namespace

extern "C" {

void qp_serve_config_default(qp_serve_config* c) {
  if (!c) return;
  memset(c, 0, sizeof(*c));
  c->hbm_budget_bytes = (size_t)1 << 30;
  c->max_inflight = 8;
  c->max_batch = 1024;
  c->max_queue = 1 << 20;
  qp_settings_default(&c->settings);
  c->mode = QP_SERVE_PERSISTENT;
  c->idle_ms = 50;
}

size_t qp_serve_footprint_bytes(int32_t n, int32_t n_eq, int32_t n_ineq, int32_t want_grad) {
  SizeCfg c;
  if (!size_cfg(n, n_ineq, n_eq, &c)) return 0;
  const Footprint f = footprint(n, n_ineq, n_eq, want_grad != 0, c);
  return round_up((size_t)(f.in + f.out + f.dev) * sizeof(float), kAlign);
}

int qp_serve_create(const qp_serve_config* cfg, qp_server** out) {
  if (!cfg || !out) return QP_EINVAL;
  *out = nullptr;
  if (cfg->hbm_budget_bytes < (1u << 20) || cfg->max_inflight < 1 || cfg->max_inflight > 64 ||
      cfg->max_batch < 1 || cfg->max_queue < 1 ||
      (cfg->mode != QP_SERVE_LAUNCHES && cfg->mode != QP_SERVE_PERSISTENT) ||
      (cfg->mode == QP_SERVE_PERSISTENT && (cfg->idle_ms < 1 || cfg->idle_ms > 10000)))
    return QP_EINVAL;
  std::unique_ptr<qp_server> sv(new qp_server());
  sv->cfg = *cfg;
  memset(&sv->base, 0, sizeof(sv->base));
  int rc = settings_to_params(&cfg->settings, &sv->base);
  if (rc != QP_OK) return rc;
  if (cfg->settings.warm_start) return QP_EINVAL;  // requests carry no starting point
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    cudaGetLastError();
    return QP_ECUDA;
  }
  sv->persistent = cfg->mode == QP_SERVE_PERSISTENT;
  if (sv->persistent) {
    int atomics = 0, sms = 0;
    if (cudaDeviceGetAttribute(&atomics, cudaDevAttrHostNativeAtomicSupported, sv->device) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, sv->device) !=
            cudaSuccess) {
      cudaGetLastError();
      return QP_ECUDA;
    }
    if (!atomics) return QP_ENOTSUP;  // CTAs count themselves out in host memory
    const int per_sm = serve_kernel_blocks_per_sm();
    if (per_sm < 1) {
      cudaGetLastError();
      return QP_ECUDA;
    }
    sv->target = sms * per_sm;
  }
  const size_t budget = round_up(cfg->hbm_budget_bytes, kAlign);
  bool ok = cudaMalloc((void**)&sv->dmem, budget) == cudaSuccess &&
            cudaHostAlloc((void**)&sv->hmem, budget,
                          sv->persistent ? cudaHostAllocMapped : cudaHostAllocDefault) ==
                cudaSuccess;
  if (ok && sv->persistent) {
    // the ring, its completion words and the control block in mapped host
    // memory; the claim counter on the device
    sv->cap = 4096;
    void *rd = nullptr, *dd = nullptr, *cd = nullptr, *hd = nullptr;
    ok = cudaHostAlloc((void**)&sv->ring, sv->cap * sizeof(ReqDesc), cudaHostAllocMapped) ==
             cudaSuccess &&
         cudaHostAlloc((void**)&sv->done, sv->cap * sizeof(uint32_t), cudaHostAllocMapped) ==
             cudaSuccess &&
         cudaHostAlloc((void**)&sv->ctl, sizeof(ServeCtl), cudaHostAllocMapped) == cudaSuccess &&
         cudaMalloc((void**)&sv->head, sizeof(uint32_t)) == cudaSuccess &&
         cudaMemset(sv->head, 0, sizeof(uint32_t)) == cudaSuccess &&
         cudaHostGetDevicePointer(&rd, sv->ring, 0) == cudaSuccess &&
         cudaHostGetDevicePointer(&dd, sv->done, 0) == cudaSuccess &&
         cudaHostGetDevicePointer(&cd, sv->ctl, 0) == cudaSuccess &&
         cudaHostGetDevicePointer(&hd, sv->hmem, 0) == cudaSuccess &&
         cudaStreamCreateWithFlags(&sv->up_stream, cudaStreamNonBlocking) == cudaSuccess &&
         cudaDeviceSynchronize() == cudaSuccess;
    for (int i = 0; ok && i < 8; ++i) {
      cudaStream_t st = nullptr;
      ok = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
      if (ok) sv->k_streams.push_back(st);
    }
    for (int i = 0; ok && i < 16; ++i) {
      cudaEvent_t ev = nullptr;
      ok = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
      if (ok) sv->ev_pool.push_back(ev);
    }
    if (ok) {
      memset(sv->ring, 0, sv->cap * sizeof(ReqDesc));
      memset(sv->done, 0, sv->cap * sizeof(uint32_t));
      memset(sv->ctl, 0, sizeof(ServeCtl));
      sv->hmem_dev = static_cast<float*>(hd);
      ServeParams& P = sv->sp;
      memset(&P, 0, sizeof(P));
      P.base = sv->base;
      P.ring = static_cast<const ReqDesc*>(rd);
      P.done = static_cast<uint32_t*>(dd);
      P.ctl = static_cast<ServeCtl*>(cd);
      P.head = sv->head;
      P.cap = sv->cap;
      P.idle_ns = (unsigned long long)cfg->idle_ms * 1000000ull;
      P.life_ns = 10000000000ull;  // a CTA takes no new request after 10 s
    }
  }
  sv->launches.resize(sv->persistent ? 0 : cfg->max_inflight);
  const size_t dbytes = (size_t)2 * cfg->max_batch * sizeof(ReqDesc);
  for (Launch& L : sv->launches) {
    if (!ok) break;
    ok = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) == cudaSuccess &&
         cudaHostAlloc((void**)&L.hdesc, dbytes, cudaHostAllocDefault) == cudaSuccess &&
         cudaMalloc((void**)&L.ddesc, dbytes) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    for (Launch& L : sv->launches) {
      if (L.stream) cudaStreamDestroy(L.stream);
      if (L.done) cudaEventDestroy(L.done);
      if (L.hdesc) cudaFreeHost(L.hdesc);
      if (L.ddesc) cudaFree(L.ddesc);
    }
    free_persistent(sv.get());
    if (sv->dmem) cudaFree(sv->dmem);
    if (sv->hmem) cudaFreeHost(sv->hmem);
    cudaGetLastError();
    return QP_ENOMEM;
  }
  // load every kernel variant now, not on the first request of its class
  preload_forward_kernels();
  preload_backward_kernels();
  sv->arena.reset(new Arena(budget));
  sv->t0 = std::chrono::steady_clock::now();
  qp_server* raw = sv.get();
  sv->worker = std::thread([raw] { raw->run(); });
  *out = sv.release();
  return QP_OK;
}

int qp_serve_submit(qp_server* sv, const qp_request* rq, uint64_t* ticket) {
  if (!sv || !rq || !ticket) return QP_EINVAL;
  const int n = rq->n, m = rq->n_ineq, p = rq->n_eq;
  const bool grad = rq->want_grad != 0;
  if (n < 1 || p < 0 || p > n || m < 0) return QP_EINVAL;
  if (!rq->Q || !rq->q || (p > 0 && (!rq->A || !rq->b)) || (m > 0 && (!rq->G || !rq->h)) ||
      (grad && !rq->dl_dx))
    return QP_EINVAL;
  std::unique_ptr<Req> r(new Req());
  if (!size_cfg(n, m, p, &r->cfg, sv->persistent)) return QP_ENOTSUP;
  r->n = n; r->m = m; r->p = p; r->grad = grad;
  r->fp = footprint(n, m, p, grad, r->cfg);
  if ((size_t)(r->fp.in + r->fp.out + r->fp.dev) * sizeof(float) >
      round_up(sv->cfg.hbm_budget_bytes, kAlign))
    return QP_ENOTSUP;
  r->in.assign((size_t)r->fp.in, 0.0f);
  float* o = r->in.data();
  auto take = [&](const float* src, long long cnt, long long adv) {
    if (cnt) memcpy(o, src, (size_t)cnt * sizeof(float));
    o += adv;
  };
  take(rq->Q, (long long)n * n, r4((long long)n * n));
  take(rq->q, n, r4(n));
  take(rq->A, (long long)p * n, r4((long long)p * n));
  take(rq->b, p, r4(p));
  take(rq->G, (long long)m * n, r4((long long)m * n));
  take(rq->h, m, r4(m));
  if (grad) take(rq->dl_dx, n, r4(n));
  r->x = rq->x; r->y = rq->y; r->z = rq->z; r->s = rq->s;
  if (grad) {
    r->dQ = rq->dQ; r->dq = rq->dq; r->dA = rq->dA; r->db = rq->db; r->dG = rq->dG;
    r->dh = rq->dh;
  }
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    if (sv->fatal != QP_OK) return sv->fatal;
    if ((int64_t)sv->pending.size() >= sv->cfg.max_queue) return QP_EAGAIN;
    r->ticket = sv->next_ticket++;
    r->t_submit = sv->now_ms();
    *ticket = r->ticket;
    sv->pending.push_back(r.get());
    sv->reqs.emplace(r->ticket, std::move(r));
  }
  sv->cv_work.notify_one();
  return QP_OK;
}

int qp_serve_poll(qp_server* sv, uint64_t ticket, qp_result* res) {
  if (!sv) return QP_EINVAL;
  std::lock_guard<std::mutex> lock(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return QP_EINVAL;
  Req* r = it->second.get();
  if (r->state != kDone && r->state != kFailed) return QP_PENDING;
  return fill_result(sv, r, res);
}

int qp_serve_poll_any(qp_server* sv, qp_result* res) {
  if (!sv) return QP_EINVAL;
  std::lock_guard<std::mutex> lock(sv->mu);
  while (!sv->done_fifo.empty()) {
    const uint64_t t = sv->done_fifo.front();
    sv->done_fifo.pop_front();
    auto it = sv->reqs.find(t);
    if (it == sv->reqs.end()) continue;  // already collected by qp_serve_poll
    return fill_result(sv, it->second.get(), res);
  }
  return QP_PENDING;
}

int qp_serve_wait(qp_server* sv, uint64_t ticket, int32_t timeout_ms, qp_result* res) {
  if (!sv || timeout_ms < 0) return QP_EINVAL;
  std::unique_lock<std::mutex> lock(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return QP_EINVAL;
  Req* r = it->second.get();
  const bool ready = sv->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), [&] {
    return r->state == kDone || r->state == kFailed;
  });
  if (!ready) return QP_ETIMEOUT;
  return fill_result(sv, r, res);
}

int qp_serve_destroy(qp_server* sv) {
  if (!sv) return QP_EINVAL;
  {
    std::lock_guard<std::mutex> lock(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  if (sv->persistent && sv->ctl) {
    // resident CTAs leave after the request they hold (each bounded by its
    // iteration limits); requests not yet claimed are dropped
    __atomic_store_n(&sv->ctl->stop, 1u, __ATOMIC_RELEASE);
    for (cudaStream_t st : sv->k_streams) cudaStreamSynchronize(st);
    if (sv->up_stream) cudaStreamSynchronize(sv->up_stream);
  }
  free_persistent(sv);
  for (Launch& L : sv->launches) {
    if (L.stream) {
      cudaStreamSynchronize(L.stream);
      cudaStreamDestroy(L.stream);
    }
    if (L.done) cudaEventDestroy(L.done);
    if (L.hdesc) cudaFreeHost(L.hdesc);
    if (L.ddesc) cudaFree(L.ddesc);
  }
  cudaFree(sv->dmem);
  cudaFreeHost(sv->hmem);
  cudaGetLastError();
  delete sv;
  return QP_OK;
}

}  // extern "C"
