// Continuous-batching server for heat-conduction solves.
//
// Requests (an n x n conductivity and right-hand side, copied in at submit)
// wait in a FIFO.  A worker thread admits the oldest requests whenever the
// batch has a free slot and the device pool has room for their arrays
// (admission by HBM footprint), adds them to the running CgBatch, advances
// every admitted solve by a few CG iterations per round, and retires the
// finished ones -- so requests that arrive while others run join the batch
// as soon as memory frees up, and their work overlaps on the GPU.  The pool
// and the batch's device tables are allocated at open; the serving loop
// never calls cudaMalloc, and the batch's captured tick graph is reused
// whatever requests come and go.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "cg.h"
#include "internal.h"
#include "opstile.h"

using namespace opstile;

namespace {

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// First-fit sub-allocator over one device region (256-byte granules).
class Pool {
 public:
  void init(char* base, size_t bytes) {
    base_ = base;
    free_.clear();
    free_[0] = bytes;
  }
  // returns offset or (size_t)-1
  size_t take(size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it)
      if (it->second >= bytes) {
        const size_t off = it->first, len = it->second;
        free_.erase(it);
        if (len > bytes) free_[off + bytes] = len - bytes;
        return off;
      }
    return (size_t)-1;
  }
  void give(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
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
  char* base() const { return base_; }

 private:
  char* base_ = nullptr;
  std::map<size_t, size_t> free_;
};

enum ReqState { RQ_QUEUED, RQ_RUNNING, RQ_DONE, RQ_FAILED };

struct Request {
  uint64_t id;
  int n, units = 0;
  double tol = 0.0;
  int prec = 0;
  std::vector<double> kappa, rhs, x;
  int state = RQ_QUEUED;
  int slot = -1;
  size_t off = 0, bytes = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  ops_cg_stats stats{};
};

}  // namespace

struct ops_server_s {
  ops_ctx ctx = nullptr;
  ops_serve_config cfg;
  std::unique_ptr<CgBatch> batch;
  void* region = nullptr;
  size_t region_bytes = 0;
  Pool pool;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::map<uint64_t, std::unique_ptr<Request>> reqs;
  std::map<int, Request*> by_slot;
  int max_units = 0, live_units = 0;  // work units the batch's fixed tables hold / the admitted solves use
  uint64_t next_id = 1;
  bool stop = false;
  int error = OPS_OK;
  std::thread worker;
};

namespace {

void worker_loop(ops_server s) {
  std::vector<int> done;
  std::vector<Request*> admit;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // admit the oldest requests while a slot, pool memory and unit-table
      // room are free
      admit.clear();
      while (!s->queue.empty() && s->batch->live() + (int)admit.size() < s->cfg.max_batch) {
        Request* r = s->queue.front();
        if (s->live_units + r->units > s->max_units) break;
        const size_t off = s->pool.take(r->bytes);
        if (off == (size_t)-1) break;
        s->queue.pop_front();
        r->off = off;
        s->live_units += r->units;
        admit.push_back(r);
      }
      if (admit.empty() && s->batch->live() == 0) {
        if (s->stop) return;
        s->cv_work.wait_for(lk, std::chrono::milliseconds(1));
        continue;
      }
    }
    // uploads happen outside the lock, so submitters never wait on them
    // (only this thread touches the batch)
    const ops_cg_params& P = s->cfg.params;
    for (Request* r : admit) {
      const int slot = s->batch->add(r->n, r->kappa.data(), r->rhs.data(), r->tol, r->prec,
                                     P.inner_tol > 0 ? P.inner_tol : 1e-4, P.maxit, P.maxouter > 0 ? P.maxouter : 100,
                                     s->pool.base() + r->off);
      std::lock_guard<std::mutex> lk(s->mu);
      r->slot = slot;
      r->state = RQ_RUNNING;
      r->t_admit = now_ms();
      s->by_slot[slot] = r;
    }
    cudaError_t e = s->batch->run(s->cfg.ticks_per_poll);
    if (e == cudaSuccess) e = s->batch->poll(done);
    std::unique_lock<std::mutex> lk(s->mu);
    if (e != cudaSuccess) {
      s->error = OPS_ERR_CUDA;
      for (auto& kv : s->by_slot) kv.second->state = RQ_FAILED;
      s->by_slot.clear();
      s->cv_done.notify_all();
      return;
    }
    for (int slot : done) {
      Request* r = s->by_slot[slot];
      CgProb info;
      r->x.resize((size_t)r->n * r->n);
      lk.unlock();
      e = s->batch->fetch(slot, r->x.data(), &info);
      lk.lock();
      r->stats.iterations = info.it;
      r->stats.outer = info.outer;
      r->stats.converged = info.conv;
      r->stats.relres = info.rel;
      r->state = e == cudaSuccess ? RQ_DONE : RQ_FAILED;
      r->t_done = now_ms();
      s->batch->remove(slot);
      s->pool.give(r->off, r->bytes);
      s->live_units -= r->units;
      s->by_slot.erase(slot);
      std::vector<double>().swap(r->kappa);
      std::vector<double>().swap(r->rhs);
    }
    if (!done.empty()) s->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

int ops_serve_open(ops_server* out, const ops_serve_config* cfg) {
  if (!out || !cfg) return OPS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!(cfg->params.tol > 0.0) || cfg->params.maxit < 1 || cfg->hbm_budget <= 0 ||
      (cfg->params.precision != OPS_PREC_FP64 && cfg->params.precision != OPS_PREC_MIXED))
    return OPS_ERR_INVALID_ARG;
  std::unique_ptr<ops_server_s> s(new ops_server_s);
  s->cfg = *cfg;
  if (s->cfg.max_batch <= 0) s->cfg.max_batch = 1024;
  if (s->cfg.ticks_per_poll <= 0) s->cfg.ticks_per_poll = 4;
  ops_config c;
  ops_config_default(&c);
  c.device = cfg->device;
  int rc = ops_init(&s->ctx, &c);
  if (rc) return rc;
  s->region_bytes = (size_t)cfg->hbm_budget;
  rc = ctx_alloc(s->ctx, &s->region, s->region_bytes);
  if (rc) {
    ops_finalize(s->ctx);
    return rc;
  }
  s->pool.init((char*)s->region, s->region_bytes);
  // the batch's tables, sized once for the most work units the pool can
  // hold: problems hold at least min_bpu pool bytes per unit
  double min_bpu = 1e30;
  for (int n = 1; n <= 4096; ++n) min_bpu = std::min(min_bpu, (double)cg_problem_bytes(n) / cg_unit_count(n));
  s->max_units = (int)std::min<double>(1 << 30, (double)s->region_bytes / min_bpu + s->cfg.max_batch);
  s->batch.reset(new CgBatch(ctx_stream(s->ctx), ctx_num_sms(s->ctx), s->cfg.max_batch, s->max_units));
  if (s->batch->init_status() != cudaSuccess) {
    s->batch.reset();
    ctx_free(s->ctx, s->region, s->region_bytes);
    ops_finalize(s->ctx);
    return OPS_ERR_NOMEM;
  }
  ops_server raw = s.get();
  s->worker = std::thread(worker_loop, raw);
  *out = s.release();
  return OPS_OK;
}

int ops_serve_submit(ops_server s, int n, const double* host_kappa, const double* host_rhs, double tol, int precision,
                     uint64_t* id) {
  if (!s || !host_kappa || !host_rhs || !id || n < 1 || n > 46000) return OPS_ERR_INVALID_ARG;
  if (precision >= 0 && precision != OPS_PREC_FP64 && precision != OPS_PREC_MIXED) return OPS_ERR_INVALID_ARG;
  const size_t bytes = (size_t)cg_problem_bytes(n);
  if (bytes > s->region_bytes || cg_unit_count(n) > s->max_units) return OPS_ERR_NOMEM;  // could never be admitted
  std::unique_ptr<Request> r(new Request);
  r->n = n;
  r->units = cg_unit_count(n);
  r->tol = tol > 0.0 ? tol : s->cfg.params.tol;
  r->prec = precision >= 0 ? precision : s->cfg.params.precision;
  r->bytes = bytes;
  r->kappa.assign(host_kappa, host_kappa + (size_t)n * n);
  r->rhs.assign(host_rhs, host_rhs + (size_t)n * n);
  r->t_submit = now_ms();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->error) return s->error;
  r->id = s->next_id++;
  *id = r->id;
  s->queue.push_back(r.get());
  s->reqs[r->id] = std::move(r);
  s->cv_work.notify_one();
  return OPS_OK;
}

int ops_serve_poll(ops_server s, uint64_t id, int wait, double* host_x, ops_solve_stats* st) {
  if (!s) return OPS_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return OPS_ERR_INVALID_ARG;
  Request* r = it->second.get();
  while (wait && r->state != RQ_DONE && r->state != RQ_FAILED && !s->error)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(5));
  if (r->state == RQ_FAILED || (s->error && r->state != RQ_DONE)) return OPS_ERR_CUDA;
  if (r->state != RQ_DONE) return OPS_ERR_STATE;
  if (host_x) std::memcpy(host_x, r->x.data(), sizeof(double) * r->x.size());
  if (st) {
    st->iterations = r->stats.iterations;
    st->outer = r->stats.outer;
    st->converged = r->stats.converged;
    st->relres = r->stats.relres;
    st->queue_ms = r->t_admit - r->t_submit;
    st->service_ms = r->t_done - r->t_admit;
    st->latency_ms = r->t_done - r->t_submit;
    st->submit_ms = r->t_submit;
    st->done_ms = r->t_done;
  }
  s->reqs.erase(it);
  return OPS_OK;
}

int ops_serve_close(ops_server s) {
  if (!s) return OPS_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    // drop requests not admitted yet; running ones finish first
    for (Request* r : s->queue) r->state = RQ_FAILED;
    s->queue.clear();
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  s->batch.reset();
  ctx_free(s->ctx, s->region, s->region_bytes);
  ops_finalize(s->ctx);
  delete s;
  return OPS_OK;
}

}  // extern "C"
