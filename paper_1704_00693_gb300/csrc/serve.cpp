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
// whatever requests come and go.  Finished solutions are copied to the host
// by a second thread on a stream of its own while the worker keeps running
// rounds (a finished problem is no longer written by any kernel); the
// worker frees a problem's slot and memory once its copy is done.
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

// memcpy of n doubles, split over up to 8 host threads when large (one
// host thread copies at about 12 GB/s on the Grace host, the arrays here
// reach 32 MB)
void copy_doubles(double* dst, const double* src, size_t n) {
  const size_t chunk = (size_t)1 << 20;  // doubles per thread at least
  const int nt = (int)std::min<size_t>(8, (n + chunk - 1) / chunk);
  if (nt <= 1) {
    if (n) std::memcpy(dst, src, sizeof(double) * n);
    return;
  }
  std::vector<std::thread> th;
  const size_t per = (n + nt - 1) / nt;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([=] {
      const size_t a = (size_t)t * per, b = std::min(n, a + per);
      if (b > a) std::memcpy(dst + a, src + a, sizeof(double) * (b - a));
    });
  for (std::thread& t : th) t.join();
}

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
  std::unique_ptr<double[]> kappa, rhs;  // copies of the submitted arrays until admission
  std::unique_ptr<double[]> x;  // the solution (cells doubles), not zero-filled first
  size_t cells = 0;
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
  ops_serve_counters counters{};  // updated by the worker under mu
  std::thread worker;
  // finished solves waiting for their copy to the host, and slots whose copy
  // is done (the worker removes them from the batch)
  // A retired slot carries its pool memory and work units: once a request
  // is done the client may poll it, which frees the Request.
  struct Retired {
    int slot;
    size_t off, bytes;
    int units;
  };
  struct FetchJob {
    Request* r;
    const double* dx;
    size_t cells;
    CgProb info;
    Retired ret;
  };
  std::deque<FetchJob> fetch_q;
  std::vector<Retired> retire;
  int pending = 0;  // finished solves not retired yet
  bool fetch_stop = false;
  std::condition_variable cv_fetch;
  cudaStream_t fstream = nullptr;
  std::thread fetcher;
};

namespace {

// Copies finished solutions to host memory on its own stream.
void fetch_loop(ops_server s) {
  for (;;) {
    ops_server_s::FetchJob job;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      while (s->fetch_q.empty() && !s->fetch_stop) s->cv_fetch.wait(lk);
      if (s->fetch_q.empty()) return;
      job = s->fetch_q.front();
      s->fetch_q.pop_front();
    }
    Request* r = job.r;
    const double t0 = now_ms();
    r->x.reset(new double[job.cells]);
    r->cells = job.cells;
    cudaError_t e = cudaMemcpyAsync(r->x.get(), job.dx, sizeof(double) * job.cells, cudaMemcpyDeviceToHost,
                                    s->fstream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->fstream);
    const double t1 = now_ms();
    std::lock_guard<std::mutex> lk(s->mu);
    r->stats.iterations = job.info.it;
    r->stats.outer = job.info.outer;
    r->stats.converged = job.info.conv;
    r->stats.relres = job.info.rel;
    r->state = e == cudaSuccess ? RQ_DONE : RQ_FAILED;
    r->t_done = t1;
    s->counters.fetch_ms += t1 - t0;
    ++s->counters.completed;
    s->retire.push_back(job.ret);  // r may be freed by a poll from here on
    s->cv_done.notify_all();
    s->cv_work.notify_one();
  }
}

void worker_loop(ops_server s) {
  std::vector<int> done;
  std::vector<CgProb> infos;
  std::vector<Request*> admit;
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      // slots whose solutions reached the host go back to the batch and the pool
      for (const ops_server_s::Retired& t : s->retire) {
        s->batch->remove(t.slot);
        s->pool.give(t.off, t.bytes);
        s->live_units -= t.units;
        s->by_slot.erase(t.slot);
        --s->pending;
      }
      s->retire.clear();
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
      if (admit.empty() && s->batch->live() - s->pending == 0) {
        if (s->stop && s->batch->live() == 0) return;
        const double t = now_ms();
        s->cv_work.wait_for(lk, std::chrono::milliseconds(1));
        s->counters.idle_ms += now_ms() - t;
        continue;
      }
    }
    const double t_up = now_ms();
    // uploads happen outside the lock, so submitters never wait on them
    // (only this thread touches the batch)
    const ops_cg_params& P = s->cfg.params;
    for (Request* r : admit) {
      const int slot = s->batch->add(r->n, r->kappa.get(), r->rhs.get(), r->tol, r->prec,
                                     P.inner_tol > 0 ? P.inner_tol : 1e-4, P.maxit, P.maxouter > 0 ? P.maxouter : 100,
                                     s->pool.base() + r->off);
      // copies from pageable memory have read their source when they return
      r->kappa.reset();
      r->rhs.reset();
      std::lock_guard<std::mutex> lk(s->mu);
      r->slot = slot;
      r->state = RQ_RUNNING;
      r->t_admit = now_ms();
      s->by_slot[slot] = r;
    }
    const double t_run = now_ms();
    cudaError_t e = s->batch->run(s->cfg.ticks_per_poll);
    if (e == cudaSuccess) e = s->batch->poll(done, &infos);
    const double t_end = now_ms();
    std::unique_lock<std::mutex> lk(s->mu);
    s->counters.admitted += (int64_t)admit.size();
    s->counters.upload_ms += t_run - t_up;
    s->counters.run_ms += t_end - t_run;
    ++s->counters.rounds;
    if (e != cudaSuccess) {
      s->error = OPS_ERR_CUDA;
      // requests already done may have been polled and freed: drop their
      // slots first, then fail every other admitted request
      for (const ops_server_s::Retired& t : s->retire) s->by_slot.erase(t.slot);
      s->retire.clear();
      for (auto& kv : s->by_slot)
        if (kv.second->state != RQ_DONE) kv.second->state = RQ_FAILED;
      s->by_slot.clear();
      s->cv_done.notify_all();
      return;
    }
    for (size_t k = 0; k < done.size(); ++k) {
      const int slot = done[k];
      Request* r = s->by_slot[slot];
      const size_t cells = (size_t)s->batch->side(slot) * s->batch->side(slot);
      s->fetch_q.push_back(ops_server_s::FetchJob{r, s->batch->solution(slot), cells, infos[k],
                                                  ops_server_s::Retired{slot, r->off, r->bytes, r->units}});
      ++s->pending;
    }
    if (!done.empty()) s->cv_fetch.notify_one();
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
  if (cudaStreamCreateWithFlags(&s->fstream, cudaStreamNonBlocking) != cudaSuccess) {
    s->batch.reset();
    ctx_free(s->ctx, s->region, s->region_bytes);
    ops_finalize(s->ctx);
    return OPS_ERR_CUDA;
  }
  ops_server raw = s.get();
  s->fetcher = std::thread(fetch_loop, raw);
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
  r->t_submit = now_ms();
  const size_t cells = (size_t)n * n;
  r->kappa.reset(new double[cells]);
  r->rhs.reset(new double[cells]);
  copy_doubles(r->kappa.get(), host_kappa, cells);
  copy_doubles(r->rhs.get(), host_rhs, cells);
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
  std::unique_ptr<double[]> x;
  size_t cells = 0;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return OPS_ERR_INVALID_ARG;
    Request* r = it->second.get();
    while (wait && r->state != RQ_DONE && r->state != RQ_FAILED && !s->error)
      s->cv_done.wait_for(lk, std::chrono::milliseconds(5));
    if (r->state == RQ_FAILED || (s->error && r->state != RQ_DONE)) return OPS_ERR_CUDA;
    if (r->state != RQ_DONE) return OPS_ERR_STATE;
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
    x = std::move(r->x);
    cells = r->cells;
    s->reqs.erase(it);
  }
  // the copy runs outside the server's lock
  if (host_x && cells) copy_doubles(host_x, x.get(), cells);
  return OPS_OK;
}

int ops_serve_stats(ops_server s, ops_serve_counters* out) {
  if (!s || !out) return OPS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->counters;
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
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->fetch_stop = true;
  }
  s->cv_fetch.notify_all();
  if (s->fetcher.joinable()) s->fetcher.join();
  if (s->fstream) cudaStreamDestroy(s->fstream);
  s->batch.reset();
  ctx_free(s->ctx, s->region, s->region_bytes);
  ops_finalize(s->ctx);
  delete s;
  return OPS_OK;
}

}  // extern "C"
