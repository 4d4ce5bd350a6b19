// Serving loop: continuous batching of lattice problems on one GPU.
//
// Requests are deep-copied at submission, checked and sized (the same
// planner that lays out a batch's device slab), and queued FIFO.  `slots`
// worker threads each own a private context (its own CUDA stream); a free
// worker admits the queue's head request and, in queue order, the following
// requests of the same kind -- periodic (one pass: Fourier blocks) or
// structured (an iteration: box chains and defects) -- while they fit the
// server's HBM budget (bytes reserved by the batches already on the device
// are subtracted) and the batch cap, solves them as one batch, publishes
// the per-request results and releases its reservation.  A structured
// request is published as soon as it leaves the block iteration, not when
// its batch's slowest problem does.  A batch holds its reservation until its
// slowest problem ends, so one-pass problems are not batched with iterated
// ones; the head of the queue is always admitted first, so neither kind
// waits more than the batches ahead of it.  Requests arriving
// while batches run are admitted by the next free worker, so their work
// overlaps on the device with the batches in flight.  Batch slabs come from
// one stream-ordered memory pool owned by the server (no device-wide
// synchronisation from allocation or release).
//
// A request's result does not depend on the batch it lands in: every
// reduction order and the block iteration's start vectors are fixed per
// problem (the batched planner's invariance), which the tests check.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/fock.h"
#include "admission.h"

namespace fock {
int detail_estimate(const fock_problem& p, size_t* bytes, int* n_evals, std::string& why);
fock_ctx* detail_worker_ctx(int device, cudaMemPool_t pool, size_t budget);
const char* detail_ctx_error(const fock_ctx* c);
cudaStream_t detail_ctx_stream(const fock_ctx* c);
int detail_solve(fock_ctx* w, int n, const fock_problem* probs, fock_output* outs, double tol, int maxit,
                 const std::function<void(int, const fock_output&)>* release);
}  // namespace fock

namespace {

using Clock = std::chrono::steady_clock;

// A problem whose arrays are owned by the request (the caller's may be freed
// as soon as submit returns).
struct OwnedProblem {
  fock_problem p{};
  std::vector<double> Z, frac, exps, t, c;
  std::vector<int> ang, centre;
  std::vector<fock_defect> defects;

  void copy_from(const fock_problem& s) {
    p = s;
    Z.assign(s.Z, s.Z + s.M0);
    frac.assign(s.frac, s.frac + 3 * s.M0);
    exps.assign(s.exps, s.exps + s.m0);
    ang.assign(s.ang, s.ang + s.m0);
    centre.assign(s.centre, s.centre + s.m0);
    if (s.sinc_t && s.sinc_c) {
      t.assign(s.sinc_t, s.sinc_t + s.R);
      c.assign(s.sinc_c, s.sinc_c + s.R);
    }
    if (s.ndef > 0 && s.defects) defects.assign(s.defects, s.defects + s.ndef);
    p.Z = Z.data();
    p.frac = frac.data();
    p.exps = exps.data();
    p.ang = ang.data();
    p.centre = centre.data();
    p.sinc_t = t.empty() ? nullptr : t.data();
    p.sinc_c = c.empty() ? nullptr : c.data();
    p.defects = defects.empty() ? nullptr : defects.data();
  }
};

struct Req {
  uint64_t ticket = 0;
  OwnedProblem op;
  size_t bytes = 0;
  int n_evals = 0;
  int64_t t_submit = 0, t_admit = -1, t_done = -1;
  int status = FOCK_EAGAIN;
  std::vector<double> ev;
  std::vector<int> blk;
  int iters = 0;
  double resid = 0.0;
  int batch_id = -1, batch_size = 0;
  bool done = false;
};

bool structured(const fock_problem& p) {
  for (int a = 0; a < 3; ++a)
    if (p.L[a] > 1 && !p.periodic[a]) return true;
  return p.ndef > 0;
}

}  // namespace

struct fock_server {
  int device = 0;
  fock_serve_config cfg{};
  size_t reserved = 0, peak_reserved = 0;
  cudaMemPool_t pool = nullptr;
  std::mutex m;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> pending;
  std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
  uint64_t next_ticket = 1;
  int next_batch = 0;
  bool stopping = false;
  int inflight = 0, max_inflight = 0;
  uint64_t completed = 0;
  std::vector<std::thread> workers;
  std::vector<fock_ctx*> wctx;
  Clock::time_point t0;
  std::string err;

  int64_t now_ns() const {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - t0).count();
  }
  void worker(int slot);
};

void fock_server::worker(int slot) {
  cudaSetDevice(device);
  fock_ctx* w = wctx[slot];
  for (;;) {
    std::vector<Req*> batch;
    size_t bytes = 0;
    int bid = 0;
    {
      std::unique_lock<std::mutex> lk(m);
      for (;;) {
        if (!pending.empty()) {
          // the head request, then the later ones of its kind in queue order,
          // up to the first of that kind that does not fit the free budget
          const size_t free_bytes = cfg.hbm_budget_bytes > reserved ? cfg.hbm_budget_bytes - reserved : 0;
          batch = fock::admit_batch(
              pending, [](const Req* r) { return structured(r->op.p); },
              [](const Req* r) { return r->bytes; }, free_bytes, cfg.max_batch, &bytes);
          if (!batch.empty()) break;
        } else if (stopping) {
          return;
        }
        cv_work.wait(lk);   // new requests, or memory released by another slot
      }
      reserved += bytes;
      peak_reserved = std::max(peak_reserved, reserved);
      ++inflight;
      max_inflight = std::max(max_inflight, inflight);
      bid = next_batch++;
      const int64_t ta = now_ns();
      for (Req* r : batch) {
        r->t_admit = ta;
        r->batch_id = bid;
        r->batch_size = (int)batch.size();
      }
      // requests left behind (the other kind, or beyond the cap): wake an idle slot
      if (!pending.empty()) cv_work.notify_one();
    }
    const int n = (int)batch.size();
    std::vector<fock_problem> probs(n);
    std::vector<fock_output> outs(n);
    for (int i = 0; i < n; ++i) {
      Req* r = batch[i];
      probs[i] = r->op.p;
      r->ev.assign(r->n_evals, 0.0);
      if (!structured(r->op.p)) r->blk.assign(r->n_evals, 0);
      std::memset(&outs[i], 0, sizeof(fock_output));
      outs[i].evals = r->ev.data();
      outs[i].block_of = r->blk.empty() ? nullptr : r->blk.data();
      outs[i].status = FOCK_EAGAIN;
    }
    // a structured request is published as soon as it leaves the block
    // iteration (its result is final then); the batch's end publishes the rest.
    // A published request may be released by its client at once, so nothing
    // below touches it again.
    std::vector<char> published(n, 0);
    int n_published = 0;
    const std::function<void(int, const fock_output&)> publish = [&](int i, const fock_output& o) {
      std::lock_guard<std::mutex> lk(m);
      Req* r = batch[i];
      r->status = o.status;
      r->iters = o.iters;
      r->resid = o.resid;
      r->t_done = now_ns();
      r->done = true;
      published[i] = 1;
      ++n_published;
      ++completed;
      cv_done.notify_all();
    };
    int rc = fock::detail_solve(w, n, probs.data(), outs.data(), cfg.tol, cfg.maxit, &publish);
    {
      std::lock_guard<std::mutex> lk(m);
      const int64_t td = now_ns();
      for (int i = 0; i < n; ++i) {
        if (published[i]) continue;
        Req* r = batch[i];
        r->status = (outs[i].status == FOCK_EAGAIN) ? (rc ? rc : FOCK_ECUDA) : outs[i].status;
        r->iters = outs[i].iters;
        r->resid = outs[i].resid;
        r->t_done = td;
        r->done = true;
      }
      if (rc && rc != FOCK_ENOCONV && rc != FOCK_EINVAL) err = fock::detail_ctx_error(w);
      reserved -= bytes;
      --inflight;
      completed += n - n_published;
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }
}

extern "C" {

int fock_serve_start(int device, const fock_serve_config* cfg, fock_server** out) {
  if (!out) return FOCK_EINVAL;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return FOCK_ECUDA;
  fock_server* S = new fock_server();
  S->device = device;
  if (cfg) S->cfg = *cfg;
  if (S->cfg.max_batch <= 0) S->cfg.max_batch = 256;
  if (S->cfg.slots <= 0) S->cfg.slots = 2;
  if (S->cfg.slots > 16) S->cfg.slots = 16;
  if (!(S->cfg.tol > 0.0)) S->cfg.tol = 1e-10;
  if (S->cfg.maxit <= 0) S->cfg.maxit = FOCK_DEFAULT_MAXIT;
  if (S->cfg.hbm_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    S->cfg.hbm_budget_bytes = (size_t)(0.8 * (double)fr);
  }
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof(props));
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  if (cudaMemPoolCreate(&S->pool, &props) != cudaSuccess) { delete S; return FOCK_ECUDA; }
  uint64_t keep = (uint64_t)S->cfg.hbm_budget_bytes;   // freed blocks stay cached in the pool
  cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  S->t0 = Clock::now();
  for (int s = 0; s < S->cfg.slots; ++s) {
    fock_ctx* w = fock::detail_worker_ctx(device, S->pool, S->cfg.hbm_budget_bytes);
    if (!w) {
      for (fock_ctx* x : S->wctx) fock_destroy(x);
      cudaMemPoolDestroy(S->pool);
      delete S;
      return FOCK_ECUDA;
    }
    S->wctx.push_back(w);
  }
  for (int s = 0; s < S->cfg.slots; ++s) S->workers.emplace_back(&fock_server::worker, S, s);
  *out = S;
  return FOCK_OK;
}

int fock_serve_submit(fock_server* S, const fock_problem* p, uint64_t* ticket) {
  if (!S || !p || !ticket) return FOCK_EINVAL;
  std::unique_ptr<Req> r(new Req());
  r->op.copy_from(*p);
  std::string why;
  int rc = fock::detail_estimate(r->op.p, &r->bytes, &r->n_evals, why);
  std::lock_guard<std::mutex> lk(S->m);
  if (rc) { S->err = why; return rc; }
  if (S->stopping) { S->err = "server is stopping"; return FOCK_EINVAL; }
  if (r->bytes > S->cfg.hbm_budget_bytes) {
    S->err = "request needs " + std::to_string(r->bytes) + " bytes, budget " +
             std::to_string(S->cfg.hbm_budget_bytes);
    return FOCK_ENOMEM;
  }
  r->ticket = S->next_ticket++;
  r->t_submit = S->now_ns();
  *ticket = r->ticket;
  S->pending.push_back(r.get());
  S->reqs.emplace(r->ticket, std::move(r));
  S->cv_work.notify_one();
  return FOCK_OK;
}

int fock_serve_poll(fock_server* S, uint64_t ticket, fock_result* out, int timeout_ms) {
  if (!S || !out) return FOCK_EINVAL;
  std::unique_lock<std::mutex> lk(S->m);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return FOCK_EINVAL;
  Req* r = it->second.get();
  if (!r->done) {
    if (timeout_ms < 0)
      S->cv_done.wait(lk, [&] { return r->done; });
    else if (timeout_ms > 0)
      S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; });
    if (!r->done) return FOCK_EAGAIN;
  }
  out->evals = r->ev.data();
  out->block_of = r->blk.empty() ? nullptr : r->blk.data();
  out->n_evals = r->n_evals;
  out->status = r->status;
  out->iters = r->iters;
  out->resid = r->resid;
  out->t_submit_ns = r->t_submit;
  out->t_admit_ns = r->t_admit;
  out->t_done_ns = r->t_done;
  out->batch_id = r->batch_id;
  out->batch_size = r->batch_size;
  return FOCK_OK;
}

int fock_result_release(fock_server* S, uint64_t ticket) {
  if (!S) return FOCK_EINVAL;
  std::lock_guard<std::mutex> lk(S->m);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return FOCK_EINVAL;
  if (!it->second->done) return FOCK_EAGAIN;
  S->reqs.erase(it);
  return FOCK_OK;
}

int fock_serve_stats(fock_server* S, fock_serve_stats_t* st) {
  if (!S || !st) return FOCK_EINVAL;
  std::lock_guard<std::mutex> lk(S->m);
  st->completed = S->completed;
  st->pending = (uint64_t)S->pending.size();
  st->batches = (uint64_t)S->next_batch;
  st->inflight = S->inflight;
  st->max_inflight = S->max_inflight;
  st->reserved_bytes = S->reserved;
  st->peak_reserved_bytes = S->peak_reserved;
  st->budget_bytes = S->cfg.hbm_budget_bytes;
  return FOCK_OK;
}

const char* fock_serve_last_error(const fock_server* S) { return S ? S->err.c_str() : "null server"; }

int fock_serve_stop(fock_server* S) {
  if (!S) return FOCK_EINVAL;
  {
    std::lock_guard<std::mutex> lk(S->m);
    S->stopping = true;
  }
  S->cv_work.notify_all();
  for (auto& th : S->workers) th.join();
  int rc = FOCK_OK;
  for (fock_ctx* w : S->wctx) {
    if (cudaStreamSynchronize(fock::detail_ctx_stream(w)) != cudaSuccess) rc = FOCK_ECUDA;
    fock_destroy(w);
  }
  cudaMemPoolDestroy(S->pool);
  delete S;
  return rc;
}

}  // extern "C"
