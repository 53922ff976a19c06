// Continuous-batching server for smoothing and solve requests (not in the
// paper; it serves the smoothers to many concurrent users of one GPU).
//
// Two threads own the GPU work.  The copy thread admits waiting requests in
// arrival order while their device memory fits the HBM budget and a slot is
// free, takes their grids from a stream-ordered memory pool and copies them
// to the device on a copy stream, and hands finished grids back the same way;
// the compute thread runs rounds over the requests on the device: up to
// `sweeps_per_round` sweeps of every smoothing request, all requests of one
// (smoother, dtype) class in ONE persistent batched launch
// (stencil_batched), and one multigrid V-cycle (red-black Gauss-Seidel
// smoother) of every solve request.
// Copies of requests arriving or leaving overlap the rounds' kernels.
// A request's result does not depend on the other requests in the mix: the
// batched kernel is exact per grid, sweeps split into rounds compose exactly,
// and a solve request's cycles and residual tests are its own.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

struct stencil_server;

namespace stn {

using Clock = std::chrono::steady_clock;

struct Req {
  uint64_t ticket;
  stencil_request r;
  Clock::time_point t_submit, t_admit, t_done;
  size_t bytes = 0;
  void* du = nullptr;
  void* df = nullptr;
  int done_sweeps = 0;
  int state = 0;  // 0 waiting, 3 uploading, 1 on the device, 4 finished on the device, 2 reported
  bool failed = false;
  double last_rel = -1.0;
  stencil_result res{};
};

}  // namespace stn

using namespace stn;

struct stencil_server {
  stencil_ctx* ctx = nullptr;
  size_t budget = 0;
  int quantum = 10;
  int max_active = 0;  // slots: admitted requests at most (0 = memory bound only)
  std::mutex mu;
  std::condition_variable cv_work, cv_done, cv_copy;
  std::deque<uint64_t> waiting;
  std::deque<uint64_t> to_download;
  std::map<uint64_t, Req*> reqs;
  std::vector<uint64_t> active;
  int admitted_live = 0;  // admitted and not yet handed back
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker, copier;
  cudaMemPool_t pool = nullptr;
  cudaStream_t cstream = nullptr;
  size_t in_use = 0, peak = 0;
  stencil_server_stats st{};
  std::vector<double> lat;
  double busy_s = 0.0, lup = 0.0;
  std::string err;
};

namespace stn {

static size_t req_bytes(const stencil_request& r) {
  const size_t n = (size_t)(r.dims[0] + 2) * (size_t)(r.dims[1] + 2) * (size_t)(r.dims[2] + 2);
  const size_t esz = r.dtype == STENCIL_F64 ? 8 : 4;
  size_t b = n * esz;                      // u
  if (r.f_in) b += n * esz;                // f
  if (r.kind == STENCIL_REQ_JACOBI) b += n * esz;  // second Jacobi grid (batch workspace)
  return b;
}

static void finish(stencil_server* s, Req* q, int status, double rel) {
  q->t_done = Clock::now();
  q->res.status = status;
  q->res.sweeps_done = q->done_sweeps;
  q->res.rel_residual = rel;
  q->res.queue_s = std::chrono::duration<double>(q->t_admit - q->t_submit).count();
  q->res.latency_s = std::chrono::duration<double>(q->t_done - q->t_submit).count();
  q->state = 2;
}

// --- copy thread: admission, uploads, downloads -----------------------------
//
// Admits waiting requests in arrival order while their memory fits the budget
// and a slot is free, takes their grids from the server's stream-ordered
// memory pool (no cudaMalloc / cudaFree per request) and copies them to the
// device on the copy stream; hands finished grids back (device -> host) and
// returns their memory to the pool.  It runs beside the compute thread, so a
// round's kernels overlap the next requests' copies.
static bool copy_step(stencil_server* s) {
  std::vector<Req*> down, admit;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    while (!s->to_download.empty()) {
      down.push_back(s->reqs[s->to_download.front()]);
      s->to_download.pop_front();
    }
    while (!s->waiting.empty()) {
      Req* q = s->reqs[s->waiting.front()];
      if (s->budget && q->bytes > s->budget) {  // can never fit
        s->waiting.pop_front();
        q->t_admit = Clock::now();
        finish(s, q, STENCIL_ERR_OOM, -1.0);
        s->cv_done.notify_all();
        continue;
      }
      if (s->budget && s->in_use + q->bytes > s->budget) break;  // wait, in arrival order, for memory
      if (s->max_active && s->admitted_live >= s->max_active) break;  // ... or for a free slot
      s->waiting.pop_front();
      s->in_use += q->bytes;
      s->peak = std::max(s->peak, s->in_use);
      s->admitted_live++;
      q->t_admit = Clock::now();
      q->state = 3;
      admit.push_back(q);
      s->st.admitted++;
    }
  }
  if (down.empty() && admit.empty()) return false;
  const auto tc0 = Clock::now();
  double nbytes = 0.0;
  cudaStream_t cs = s->cstream;
  for (Req* q : down) {
    const size_t n = (size_t)(q->r.dims[0] + 2) * (size_t)(q->r.dims[1] + 2) * (size_t)(q->r.dims[2] + 2);
    const size_t esz = q->r.dtype == STENCIL_F64 ? 8 : 4;
    if (q->r.u_out && q->du && (q->res.status == STENCIL_OK || q->res.status == STENCIL_ERR_NOT_CONVERGED)) {
      cudaMemcpyAsync(q->r.u_out, q->du, n * esz, cudaMemcpyDeviceToHost, cs);
      nbytes += (double)(n * esz);
    }
    if (q->du) cudaFreeAsync(q->du, cs);
    if (q->df) cudaFreeAsync(q->df, cs);
  }
  for (Req* q : admit) {
    const size_t n = (size_t)(q->r.dims[0] + 2) * (size_t)(q->r.dims[1] + 2) * (size_t)(q->r.dims[2] + 2);
    const size_t esz = q->r.dtype == STENCIL_F64 ? 8 : 4;
    cudaError_t e = cudaMallocFromPoolAsync(&q->du, n * esz, s->pool, cs);
    if (e == cudaSuccess && q->r.f_in) e = cudaMallocFromPoolAsync(&q->df, n * esz, s->pool, cs);
    if (e == cudaSuccess) e = cudaMemcpyAsync(q->du, q->r.u_in, n * esz, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && q->df) e = cudaMemcpyAsync(q->df, q->r.f_in, n * esz, cudaMemcpyHostToDevice, cs);
    nbytes += (double)(n * esz) * (q->df ? 2.0 : 1.0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      q->failed = true;
    }
  }
  cudaStreamSynchronize(cs);  // downloads landed, uploads on the device
  std::lock_guard<std::mutex> lk(s->mu);
  s->st.copy_bytes += nbytes;
  s->st.copy_s += std::chrono::duration<double>(Clock::now() - tc0).count();
  for (Req* q : down) {
    q->du = q->df = nullptr;
    s->in_use -= q->bytes;
    s->admitted_live--;
    q->t_done = Clock::now();
    q->res.latency_s = std::chrono::duration<double>(q->t_done - q->t_submit).count();
    s->lat.push_back(q->res.latency_s);
    s->st.completed++;
    q->state = 2;
  }
  for (Req* q : admit) {
    if (q->failed) {
      if (q->du) cudaFreeAsync(q->du, cs);
      if (q->df) cudaFreeAsync(q->df, cs);
      q->du = q->df = nullptr;
      s->in_use -= q->bytes;
      s->admitted_live--;
      finish(s, q, STENCIL_ERR_OOM, -1.0);
      q->state = 2;
      continue;
    }
    q->state = 1;
    s->active.push_back(q->ticket);
  }
  s->cv_done.notify_all();
  s->cv_work.notify_all();
  return true;
}

// Requests finished on the device (state 2) leave the active list for the copy
// thread, which reads them back.  handoff_locked: the caller holds s->mu.
static void handoff_locked(stencil_server* s) {
  std::vector<uint64_t> keep;
  bool any = false;
  for (uint64_t t : s->active) {
    Req* q = s->reqs[t];
    if (q->state == 2) {
      q->state = 4;
      s->to_download.push_back(t);
      any = true;
    } else {
      keep.push_back(t);
    }
  }
  s->active.swap(keep);
  if (any) s->cv_copy.notify_all();
}

static void handoff_finished(stencil_server* s) {
  std::lock_guard<std::mutex> lk(s->mu);
  handoff_locked(s);
}

// --- compute thread: one round over the requests on the device --------------
//
// Smoothing requests: up to `quantum` sweeps each, all requests of one
// (smoother, dtype) class in one batched launch; the finished ones are handed
// to the copy thread at once.  Solve requests: up to quantum / 4 multigrid
// V(2,2) cycles each (red-black Gauss-Seidel smoother; FP32 cycles inside
// FP64 defect correction for the mixed kind; plain lexicographic sweeps when
// an extent cannot coarsen), the residual tested after every cycle.  Requests
// that finish are handed to the copy thread.
static bool compute_round(stencil_server* s) {
  std::vector<Req*> act;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (uint64_t t : s->active) act.push_back(s->reqs[t]);
  }
  if (act.empty()) return false;
  stencil_ctx* ctx = s->ctx;
  cudaStream_t st = ctx->gstream;
  const auto t0 = Clock::now();
  double lup = 0.0, smooth_lup = 0.0, cycles = 0.0;
  for (int cls = 0; cls < 4; ++cls) {
    const int smoother = cls / 2 == 0 ? STENCIL_JACOBI : STENCIL_GS;
    const int dtype = cls % 2 == 0 ? STENCIL_F64 : STENCIL_F32;
    std::vector<Req*> grp;
    for (Req* q : act)
      if (q->r.kind < STENCIL_REQ_SOLVE && q->r.dtype == dtype &&
          (q->r.kind == STENCIL_REQ_JACOBI ? STENCIL_JACOBI : STENCIL_GS) == smoother)
        grp.push_back(q);
    if (grp.empty()) continue;
    std::vector<void*> u;
    std::vector<const void*> f;
    std::vector<int64_t> dims;
    std::vector<double> h;
    std::vector<int> ns;
    for (Req* q : grp) {
      u.push_back(q->du);
      f.push_back(q->df);
      dims.insert(dims.end(), q->r.dims, q->r.dims + 3);
      h.push_back(q->r.h);
      ns.push_back(std::min(s->quantum, q->r.nsweeps - q->done_sweeps));
    }
    const int rc = stencil_batched(ctx, (int)grp.size(), u.data(), f.data(), dims.data(), h.data(), ns.data(),
                                   smoother, dtype, nullptr, st);
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.launches++;
    for (size_t i = 0; i < grp.size(); ++i) {
      Req* q = grp[i];
      if (rc != STENCIL_OK) {
        finish(s, q, rc, -1.0);
        continue;
      }
      q->done_sweeps += ns[i];
      lup += (double)q->r.dims[0] * q->r.dims[1] * q->r.dims[2] * ns[i];
      if (q->done_sweeps >= q->r.nsweeps) finish(s, q, STENCIL_OK, -1.0);
    }
  }
  cudaStreamSynchronize(st);
  const auto t1 = Clock::now();
  smooth_lup = lup;
  handoff_finished(s);  // finished smoothing requests go back before the solve cycles run
  for (Req* q : act) {
    if (q->r.kind < STENCIL_REQ_SOLVE) continue;
    const bool odd = q->r.dims[0] % 2 && q->r.dims[1] % 2 && q->r.dims[2] % 2 && q->r.dims[0] >= 3 &&
                     q->r.dims[1] >= 3 && q->r.dims[2] >= 3;
    const int rem = q->r.nsweeps - q->done_sweeps;
    // a V(2,2) cycle counts four fine-grid sweeps: up to quantum / 4 cycles per round (at least one), within
    // the cap; one level: min(quantum, rem) sweeps per round
    const int levels = odd && rem >= 4 ? 32 : 1;
    const int per = levels > 1 ? 4 : std::min(s->quantum, rem);
    const int maxc = levels > 1 ? std::max(1, std::min(s->quantum / 4, rem / 4)) : 1;
    double rel = -1.0;
    int cyc = 0;
    int rc = STENCIL_OK;
    if (per > 0 && levels > 1 && q->r.kind == STENCIL_REQ_SOLVE_MIXED)  // FP32 cycles, FP64 residual and update
      rc = stencil_solve_mixed_mg(ctx, (double*)q->du, (const double*)q->df, q->r.dims, q->r.h, STENCIL_GS_RB, 2, 2,
                                  s->quantum, levels, q->r.rtol, maxc, 1, &rel, &cyc, st);
    else if (per > 0)
      rc = stencil_mg_solve(ctx, (double*)q->du, (const double*)q->df, q->r.dims, q->r.h,
                            levels > 1 ? STENCIL_GS_RB : STENCIL_GS, 2, 2, levels > 1 ? s->quantum : per, levels,
                            q->r.rtol, maxc, &rel, &cyc, st);
    std::lock_guard<std::mutex> lk(s->mu);
    if (rc != STENCIL_OK && rc != STENCIL_ERR_NOT_CONVERGED) {
      finish(s, q, rc, -1.0);
      continue;
    }
    if (per == 0) {  // the cap is spent: the residual after the last round decides
      finish(s, q, q->last_rel >= 0 && q->last_rel <= q->r.rtol ? STENCIL_OK : STENCIL_ERR_NOT_CONVERGED,
             q->last_rel);
      continue;
    }
    q->done_sweeps += per * cyc;
    q->last_rel = rel;
    cycles += cyc;
    lup += (double)q->r.dims[0] * q->r.dims[1] * q->r.dims[2] * per * cyc;
    if (rel <= q->r.rtol)
      finish(s, q, STENCIL_OK, rel);
    else if (q->done_sweeps + (levels > 1 ? 4 : 1) > q->r.nsweeps)
      finish(s, q, STENCIL_ERR_NOT_CONVERGED, rel);
  }
  cudaStreamSynchronize(st);
  std::lock_guard<std::mutex> lk(s->mu);
  const auto t2 = Clock::now();
  s->busy_s += std::chrono::duration<double>(t2 - t0).count();
  s->lup += lup;
  s->st.smooth_lup += smooth_lup;
  s->st.smooth_s += std::chrono::duration<double>(t1 - t0).count();
  s->st.solve_cycles += cycles;
  s->st.solve_s += std::chrono::duration<double>(t2 - t1).count();
  handoff_locked(s);
  return true;
}

static void compute_main(stencil_server* s) {
  cudaSetDevice(s->ctx->device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait_for(lk, std::chrono::milliseconds(50), [&] { return s->stop || !s->active.empty(); });
      if (s->stop) break;
      if (s->active.empty()) continue;
    }
    compute_round(s);
  }
}

static void copy_main(stencil_server* s) {
  cudaSetDevice(s->ctx->device);
  for (;;) {
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_copy.wait_for(lk, std::chrono::milliseconds(20),
                          [&] { return s->stop || !s->to_download.empty() || !s->waiting.empty(); });
      if (s->stop) break;
    }
    while (copy_step(s)) {
    }
  }
}

}  // namespace stn

extern "C" {

int stencil_server_create(stencil_server** out, int device, size_t hbm_budget_bytes, int sweeps_per_round,
                          int max_active) {
  if (!out || sweeps_per_round < 0 || max_active < 0) return STENCIL_ERR_ARG;
  *out = nullptr;
  stencil_ctx* ctx = nullptr;
  int rc = stencil_create(&ctx, device, 0);
  if (rc) return rc;
  cudaError_t e = cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking);
  cudaStream_t cs = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  // the requests' grids come from a pool of their own that keeps what it has taken (no release to the
  // device between requests); the budget is enforced on admission
  cudaMemPool_t pool = nullptr;
  if (e == cudaSuccess) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    e = cudaMemPoolCreate(&pool, &props);
  }
  if (e == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  if (e != cudaSuccess) {
    if (pool) cudaMemPoolDestroy(pool);
    if (cs) cudaStreamDestroy(cs);
    stencil_destroy(ctx);
    return set_err(nullptr, STENCIL_ERR_CUDA, "server set-up: %s", cudaGetErrorString(e));
  }
  ctx->df_direct_first = true;  // a round's batch shape rarely recurs: no graph capture for one-off shapes
  stencil_server* s = new stencil_server();
  s->ctx = ctx;
  s->budget = hbm_budget_bytes;
  s->quantum = sweeps_per_round > 0 ? sweeps_per_round : 10;
  s->max_active = max_active;
  s->pool = pool;
  s->cstream = cs;
  s->worker = std::thread(compute_main, s);
  s->copier = std::thread(copy_main, s);
  *out = s;
  return STENCIL_OK;
}

int stencil_server_submit(stencil_server* s, const stencil_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket) return STENCIL_ERR_ARG;
  if (r->kind < STENCIL_REQ_JACOBI || r->kind > STENCIL_REQ_SOLVE_MIXED) return STENCIL_ERR_ARG;
  if (r->dtype != STENCIL_F64 && r->dtype != STENCIL_F32) return STENCIL_ERR_ARG;
  if (r->kind >= STENCIL_REQ_SOLVE && (r->dtype != STENCIL_F64 || !(r->rtol > 0.0))) return STENCIL_ERR_ARG;
  if (!r->u_in || r->nsweeps < 0 || !(r->h > 0.0)) return STENCIL_ERR_ARG;
  for (int d = 0; d < 3; ++d)
    if (r->dims[d] < 1 || r->dims[d] > (1 << 20)) return STENCIL_ERR_ARG;
  Req* q = new Req();
  q->r = *r;
  q->t_submit = Clock::now();
  q->bytes = req_bytes(*r);
  q->res.rel_residual = -1.0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    q->ticket = s->next_ticket++;
    s->reqs[q->ticket] = q;
    s->waiting.push_back(q->ticket);
    s->st.submitted++;
    *ticket = q->ticket;
  }
  s->cv_copy.notify_one();
  return STENCIL_OK;
}

int stencil_server_poll(stencil_server* s, uint64_t ticket, stencil_result* out) {
  if (!s || !out) return STENCIL_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return STENCIL_ERR_ARG;
  Req* q = it->second;
  if (q->state != 2 || q->du) return STENCIL_PENDING;
  *out = q->res;
  return STENCIL_OK;
}

int stencil_server_wait(stencil_server* s, uint64_t ticket, double timeout_s, stencil_result* out) {
  if (!s || !out) return STENCIL_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return STENCIL_ERR_ARG;
  Req* q = it->second;
  const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
  while (q->state != 2 || q->du) {
    if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout && (q->state != 2 || q->du)) return STENCIL_PENDING;
  }
  *out = q->res;
  return STENCIL_OK;
}

int stencil_server_cancel(stencil_server* s, uint64_t ticket) {
  if (!s) return STENCIL_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return STENCIL_ERR_ARG;
  Req* q = it->second;
  if (q->state != 0) return STENCIL_ERR_ARG;  // already admitted
  s->waiting.erase(std::remove(s->waiting.begin(), s->waiting.end(), ticket), s->waiting.end());
  q->t_admit = Clock::now();
  finish(s, q, STENCIL_ERR_CANCELLED, -1.0);
  s->st.cancelled++;
  s->cv_done.notify_all();
  return STENCIL_OK;
}

int stencil_server_stats_get(stencil_server* s, stencil_server_stats* out) {
  if (!s || !out) return STENCIL_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  std::vector<double> l = s->lat;
  std::sort(l.begin(), l.end());
  auto pct = [&](double p) { return l.empty() ? 0.0 : l[std::min(l.size() - 1, (size_t)(p * (l.size() - 1) + 0.5))]; };
  out->p50_s = pct(0.50);
  out->p99_s = pct(0.99);
  double sum = 0.0;
  for (double x : l) sum += x;
  out->mean_s = l.empty() ? 0.0 : sum / l.size();
  out->lup_total = s->lup;
  out->busy_s = s->busy_s;
  out->glups = s->busy_s > 0 ? s->lup / s->busy_s / 1e9 : 0.0;
  out->hbm_in_use = s->in_use;
  out->hbm_peak = s->peak;
  out->queue_depth = (int)s->waiting.size();
  out->active = s->admitted_live;
  return STENCIL_OK;
}

void stencil_server_destroy(stencil_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->cv_copy.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (s->copier.joinable()) s->copier.join();
  cudaSetDevice(s->ctx->device);
  for (auto& kv : s->reqs) {
    Req* q = kv.second;
    if (q->du) cudaFreeAsync(q->du, s->cstream);
    if (q->df) cudaFreeAsync(q->df, s->cstream);
    delete q;
  }
  cudaStreamSynchronize(s->cstream);
  cudaStreamDestroy(s->cstream);
  cudaMemPoolDestroy(s->pool);
  stencil_destroy(s->ctx);
  delete s;
}

}  // extern "C"
