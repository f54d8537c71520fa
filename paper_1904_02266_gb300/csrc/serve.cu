// Request loop behind cvo_submit / cvo_poll: continuous batching of
// frame-pair solves on one GPU.
//
// One host thread per context runs the loop:
//   admit    take queued requests in arrival order while the HBM budget and
//            the in-flight limit allow; upload the frame (centre, pack, Morton
//            order), build its clusters and solve plan against the resident
//            keyframe's cell lists, and stage its start pose;
//   publish  append the request to a queue in host-mapped memory (entry,
//            then entry count, then slot count, each store a release) that a
//            persistent cooperative kernel (queue_kernel) reads while it runs;
//            its blocks claim the request's team of slots as they come free;
//   collect  read each request's done flag (host-mapped, written last by the
//            last block of its team), copy the result out and free the
//            request's device memory, stream-ordered, while the kernel runs.
// The kernel is launched when work arrives and no kernel is up, and told to
// leave (stop flag) once the loop has been idle for linger_ms or its entry
// table is full; the next request starts a new kernel. The kernel runs with
// fewer blocks per SM than the solve kernel's occupancy, so that the frame
// preparation kernels of new requests find room on every SM beside it.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

#include "runtime.h"

namespace cvo {

namespace {

constexpr int kEntryCap = 16384;                       // entries per kernel epoch

double now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

}  // namespace

struct Req {
  uint64_t ticket = 0;
  int32_t target = -1;
  int64_t n = 0;
  std::vector<float> xyz, feat;   // the caller's frame, copied at submit
  double P0[16];
  double ell0 = 0.0;
  double work = 0.0;              // estimated kept pairs of the solve
  double t_submit = 0.0, t_admit = 0.0;
  Cloud* src = nullptr;
  Plan* plan = nullptr;
  int entry = -1;
  bool done = false;
  cvo_result res{};
};

struct Serve {
  cvo_serve_params prm{};
  std::thread th;
  std::atomic<bool> running{false};
  // shared with the API threads (under mu)
  std::mutex mu;
  std::condition_variable cv;
  bool quit = false;
  uint64_t next_ticket = 1;
  std::deque<Req*> pending;
  double pending_work = 0.0;
  std::unordered_map<uint64_t, Req*> tickets;
  // owned by the loop thread
  std::vector<Req*> inflight;
  double inflight_work = 0.0;
  cudaStream_t stream = nullptr;
  cudaEvent_t epoch_done = nullptr;
  bool epoch = false, stopping = false;
  double idle_since = -1.0;
  int nblocks = 0, dp = 0, color_mode = 0;
  QueueEntry* h_entries = nullptr;
  QueueEntry* d_entries = nullptr;
  PairResult* h_results = nullptr;
  PairResult* d_results = nullptr;
  QueueCtl* h_ctl = nullptr;
  QueueCtl* d_ctl = nullptr;
  unsigned long long* d_head = nullptr;   // slot counter, then the kernel status word
  int n_entries = 0;
  unsigned long long tail = 0;
  int* h_kstatus = nullptr;               // pinned: the last kernel's status word
  // counters (stats_mu)
  std::mutex stats_mu;
  cvo_serve_stats stats{};
};

namespace {

// Result of a finished (or failed) request; frees its device memory.
void finish(cvo_ctx* ctx, Serve* sv, Req* r, int code) {
  cvo_result& out = r->res;
  if (code == CVO_OK && r->entry >= 0) {
    const PairResult& pr = sv->h_results[r->entry];
    std::memcpy(out.P, pr.P, sizeof(out.P));
    cvo_stats& st = out.stats;
    st.iters = pr.iters;
    st.converged = pr.converged;
    st.fallback_steps = pr.fallback_steps;
    st.no_ascent_steps = pr.no_ascent_steps;
    st.final_ell = pr.ell;
    st.F_last = pr.F;
    st.t_last = pr.t;
    st.pair_evals = pr.pair_evals;
    st.candidates = pr.candidates;
    st.device_ms = pr.device_ms;
    st.status = status_code(pr.status);
  } else {
    std::memcpy(out.P, r->P0, sizeof(out.P));
    out.stats.status = code;
  }
  const double t = now_ms();
  out.queue_ms = (r->t_admit > 0.0 ? r->t_admit : t) - r->t_submit;
  out.latency_ms = t - r->t_submit;
  if (r->plan) free_plan(ctx, r->plan);
  if (r->src) free_cloud(ctx, r->src);
  r->plan = nullptr;
  r->src = nullptr;
  r->xyz.clear();
  r->xyz.shrink_to_fit();
  r->feat.clear();
  r->feat.shrink_to_fit();
  if (Cloud* t_cloud = get_cloud(ctx, r->target)) t_cloud->refs -= 1;
  {
    std::lock_guard<std::mutex> lk(sv->stats_mu);
    sv->stats.completed += 1;
    if (out.stats.status != CVO_OK) sv->stats.failed += 1;
  }
  std::lock_guard<std::mutex> lk(sv->mu);
  r->done = true;
}

// Upload the frame and build its plan against the keyframe (context lock
// held). On failure nothing of the request stays allocated.
int prepare(cvo_ctx* ctx, Serve* sv, Req* r) {
  Cloud* t = get_cloud(ctx, r->target);
  if (!t) return fail(ctx, CVO_ERR_NOT_FOUND, "keyframe was released");
  Cloud* s = nullptr;
  int rc = create_cloud(ctx, r->xyz.data(), r->feat.empty() ? nullptr : r->feat.data(), r->n,
                        false, nullptr, &s);
  if (rc != CVO_OK) return rc;
  cvo_params prm = ctx->prm;
  if (r->ell0 > 0.0) prm.ell0 = r->ell0;
  const std::vector<double> ells = ell_schedule(prm, std::max(1, prm.max_iters));
  Plan* p = new Plan();
  p->tgt = r->target;
  rc = configure_plan(ctx, p, t, s, ells, kModeAlign);
  if (rc == CVO_OK) {
    SolveState st;
    std::memset(&st, 0, sizeof(st));
    std::memcpy(st.P0, r->P0, sizeof(st.P0));
    cudaError_t e = cudaMemcpyAsync(p->d_state, &st, sizeof(st), cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) rc = fail(ctx, CVO_ERR_CUDA, cudaGetErrorString(e));
  }
  if (rc != CVO_OK) {
    free_plan(ctx, p);
    free_cloud(ctx, s);
    return rc;
  }
  r->src = s;
  r->plan = p;
  (void)sv;
  return CVO_OK;
}

int launch_epoch(cvo_ctx* ctx, Serve* sv) {
  CK(cudaMemsetAsync(sv->d_head, 0, 2 * sizeof(unsigned long long), sv->stream));
  const unsigned long long idle_ns = (unsigned long long)(sv->prm.idle_limit_ms * 1e6);
  CK(launch_queue(sv->dp, sv->color_mode, sv->nblocks, sv->d_entries, sv->d_ctl, sv->d_head,
                  reinterpret_cast<int*>(sv->d_head + 1), idle_ns, sv->stream));
  CK(cudaMemcpyAsync(sv->h_kstatus, sv->d_head + 1, sizeof(int), cudaMemcpyDeviceToHost,
                     sv->stream));
  CK(cudaEventRecord(sv->epoch_done, sv->stream));
  {
    std::lock_guard<std::mutex> lk(sv->stats_mu);
    sv->stats.kernels_launched += 1;
  }
  sv->epoch = true;
  sv->stopping = false;
  sv->idle_since = -1.0;
  return CVO_OK;
}

// Hand a prepared request to the kernel (starting one when none is up).
int publish(cvo_ctx* ctx, Serve* sv, Req* r) {
  if (!sv->epoch) {   // a fresh epoch: empty queue
    sv->n_entries = 0;
    sv->tail = 0;
    sv->h_ctl->tail = 0;
    sv->h_ctl->n_entries = 0;
    sv->h_ctl->stop = 0;
    std::atomic_thread_fence(std::memory_order_seq_cst);
  }
  const double share = r->work / std::max(r->work, sv->inflight_work + sv->pending_work + r->work);
  const double g = std::ceil(sv->prm.team_factor * share * sv->nblocks);
  const int team = (int)std::max(1.0, std::min((double)sv->nblocks, g));
  const int e = sv->n_entries;
  QueueEntry en;
  en.cfg = r->plan->d_cfg;
  en.st = r->plan->d_state;
  en.partials = r->plan->d_partials;
  en.out = sv->d_results + e;
  en.team = team;
  en.slot0 = (int)sv->tail;
  std::memset(&sv->h_results[e], 0, sizeof(PairResult));
  sv->h_entries[e] = en;
  std::atomic_thread_fence(std::memory_order_release);
  __atomic_store_n(&sv->h_ctl->n_entries, (unsigned long long)(e + 1), __ATOMIC_RELEASE);
  sv->tail += (unsigned long long)team;
  __atomic_store_n(&sv->h_ctl->tail, sv->tail, __ATOMIC_RELEASE);
  sv->n_entries = e + 1;
  r->entry = e;
  if (!sv->epoch) return launch_epoch(ctx, sv);
  return CVO_OK;
}

void collect(cvo_ctx* ctx, Serve* sv) {
  bool ended = false;
  int kernel_err = CVO_OK;
  if (sv->epoch) {
    const cudaError_t q = cudaEventQuery(sv->epoch_done);
    if (q == cudaSuccess) {
      ended = true;
    } else if (q != cudaErrorNotReady) {
      ended = true;
      kernel_err = fail(ctx, CVO_ERR_CUDA, std::string("serving kernel: ") + cudaGetErrorString(q));
    }
  }
  for (size_t i = 0; i < sv->inflight.size();) {
    Req* r = sv->inflight[i];
    const bool done = __atomic_load_n(&sv->h_results[r->entry].done, __ATOMIC_ACQUIRE) != 0;
    if (done || ended) {
      // a request still open when its kernel has ended never assembled or
      // finished its team: a bounded device wait gave up
      sv->inflight_work -= r->work;
      finish(ctx, sv, r, done ? CVO_OK : (kernel_err != CVO_OK ? kernel_err : CVO_ERR_TIMEOUT));
      sv->inflight[i] = sv->inflight.back();
      sv->inflight.pop_back();
    } else {
      ++i;
    }
  }
  if (ended) {
    sv->epoch = false;
    sv->stopping = false;
    sv->inflight_work = 0.0;
    if (kernel_err == CVO_OK && (*sv->h_kstatus & kStatusIdleTimeout)) {
      std::lock_guard<std::mutex> lk(sv->stats_mu);
      sv->stats.idle_exits += 1;
    }
  }
}

void admit(cvo_ctx* ctx, Serve* sv) {
  for (;;) {
    Req* r = nullptr;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      if (sv->pending.empty()) return;
      r = sv->pending.front();
    }
    if ((int)sv->inflight.size() >= sv->prm.max_inflight) return;
    if (sv->epoch && sv->stopping) return;   // wait for the leaving kernel
    if (sv->epoch && sv->n_entries >= kEntryCap) {
      __atomic_store_n(&sv->h_ctl->stop, 1ull, __ATOMIC_RELEASE);
      sv->stopping = true;
      return;
    }
    const int rc = prepare(ctx, sv, r);
    if (rc == CVO_ERR_OUT_OF_BUDGET && !sv->inflight.empty()) return;   // retry as memory frees
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->pending.pop_front();
      sv->pending_work -= r->work;
    }
    if (rc != CVO_OK) {
      finish(ctx, sv, r, rc);
      continue;
    }
    r->t_admit = now_ms();
    const int pc = publish(ctx, sv, r);
    if (pc != CVO_OK) {
      finish(ctx, sv, r, pc);
      continue;
    }
    sv->inflight.push_back(r);
    sv->inflight_work += r->work;
  }
}

void loop(cvo_ctx* ctx) {
  Serve* sv = ctx->serve;
  cudaSetDevice(ctx->device);
  for (;;) {
    bool idle;
    {
      std::lock_guard<std::mutex> lk(ctx->mu);
      collect(ctx, sv);
      admit(ctx, sv);
      bool quit, empty;
      {
        std::lock_guard<std::mutex> lk2(sv->mu);
        quit = sv->quit;
        empty = sv->pending.empty();
      }
      idle = empty && sv->inflight.empty();
      if (sv->epoch && !sv->stopping && idle) {
        const double t = now_ms();
        if (sv->idle_since < 0.0) sv->idle_since = t;
        if (quit || t - sv->idle_since >= sv->prm.linger_ms) {
          __atomic_store_n(&sv->h_ctl->stop, 1ull, __ATOMIC_RELEASE);
          sv->stopping = true;
        }
      } else if (!idle) {
        sv->idle_since = -1.0;
      }
      if (quit && idle && !sv->epoch) break;
    }
    std::unique_lock<std::mutex> lk(sv->mu);
    if (idle && !sv->epoch) {
      sv->cv.wait(lk, [&] { return sv->quit || !sv->pending.empty(); });
    } else {
      sv->cv.wait_for(lk, std::chrono::microseconds(20));
    }
  }
  sv->running.store(false);
}

void release_device(Serve* sv) {
  if (sv->epoch_done) cudaEventDestroy(sv->epoch_done);
  if (sv->stream) cudaStreamDestroy(sv->stream);
  if (sv->h_entries) cudaFreeHost(sv->h_entries);
  if (sv->h_results) cudaFreeHost(sv->h_results);
  if (sv->h_ctl) cudaFreeHost(sv->h_ctl);
  if (sv->h_kstatus) cudaFreeHost(sv->h_kstatus);
  sv->h_kstatus = nullptr;
  if (sv->d_head) cudaFree(sv->d_head);
  sv->epoch_done = nullptr;
  sv->stream = nullptr;
  sv->h_entries = nullptr;
  sv->h_results = nullptr;
  sv->h_ctl = nullptr;
  sv->d_head = nullptr;
}

// Start the loop (context lock held).
int start_locked(cvo_ctx* ctx, const cvo_serve_params& prm) {
  if (!ctx->serve) ctx->serve = new Serve();
  Serve* sv = ctx->serve;
  if (sv->running.load()) return fail(ctx, CVO_ERR_BUSY, "the request loop is already running");
  if (sv->th.joinable()) sv->th.join();
  const int dp = [&] {
    const cvo_params& p = ctx->prm;
    if (p.color_mode == CVO_COLOR_NONE || p.feat_dim == 0) return 0;
    return p.feat_dim <= 3 ? 3 : p.feat_dim <= 5 ? 5 : 8;
  }();
  const int per_sm = solve_blocks_per_sm(dp, kernel_mode(ctx->prm));
  if (per_sm <= 0) return fail(ctx, CVO_ERR_CUDA, "solve kernel cannot be resident");
  // block slots left free: the frame preparation kernels (at most 32
  // registers x 1024 threads a block, which fit in the SM a solve block slot
  // stands for) must find room while the serving kernel holds every other slot
  const int slots = std::min(per_sm * ctx->sms, 512);
  if (prm.reserve_blocks < 1 || prm.reserve_blocks >= slots || prm.max_inflight < 1 ||
      prm.max_inflight > 65536 || !(prm.linger_ms >= 0.0) || !std::isfinite(prm.linger_ms) ||
      !(prm.idle_limit_ms > 0.0) || !(prm.idle_limit_ms <= 3.6e6) || !(prm.team_factor > 0.0) ||
      !(prm.team_factor <= 1024.0))
    return fail(ctx, CVO_ERR_INVALID_ARG, "bad serve parameters");
  sv->prm = prm;
  sv->dp = dp;
  sv->color_mode = kernel_mode(ctx->prm);
  sv->nblocks = slots - prm.reserve_blocks;
  if (!sv->h_entries) {
    cudaError_t e = cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sv->epoch_done, cudaEventDisableTiming);
    if (e == cudaSuccess)
      e = cudaHostAlloc((void**)&sv->h_entries, sizeof(QueueEntry) * kEntryCap, cudaHostAllocMapped);
    if (e == cudaSuccess)
      e = cudaHostAlloc((void**)&sv->h_results, sizeof(PairResult) * kEntryCap, cudaHostAllocMapped);
    if (e == cudaSuccess)
      e = cudaHostAlloc((void**)&sv->h_ctl, sizeof(QueueCtl), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&sv->d_entries, sv->h_entries, 0);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&sv->d_results, sv->h_results, 0);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&sv->d_ctl, sv->h_ctl, 0);
    if (e == cudaSuccess) e = cudaMalloc((void**)&sv->d_head, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&sv->h_kstatus, sizeof(int));
    if (e != cudaSuccess) {
      release_device(sv);
      return fail(ctx, CVO_ERR_CUDA, std::string("request loop setup: ") + cudaGetErrorString(e));
    }
    std::memset(sv->h_ctl, 0, sizeof(QueueCtl));
  }
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->quit = false;
  }
  sv->epoch = false;
  sv->stopping = false;
  sv->running.store(true);
  sv->th = std::thread(loop, ctx);
  return CVO_OK;
}

}  // namespace

bool serve_active(cvo_ctx* ctx) { return ctx->serve && ctx->serve->running.load(); }

void serve_shutdown(cvo_ctx* ctx) {
  Serve* sv = ctx->serve;
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->quit = true;
  }
  sv->cv.notify_all();
  if (sv->th.joinable()) sv->th.join();
  for (auto& kv : sv->tickets) delete kv.second;
  sv->tickets.clear();
  release_device(sv);
  delete sv;
  ctx->serve = nullptr;
}

}  // namespace cvo

using namespace cvo;

extern "C" {

void cvo_serve_params_default(cvo_serve_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->reserve_blocks = 4;
  p->max_inflight = 1024;
  p->linger_ms = 0.5;
  p->idle_limit_ms = 10000.0;
  p->team_factor = 6.0;
}

int cvo_serve_start(cvo_ctx* ctx, const cvo_serve_params* params) {
  if (!ctx) return CVO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cvo_serve_params p;
  if (params) p = *params;
  else cvo_serve_params_default(&p);
  CK(cudaSetDevice(ctx->device));
  return start_locked(ctx, p);
}

int cvo_submit(cvo_ctx* ctx, const cvo_request* req, uint64_t* ticket) {
  if (!ctx) return CVO_ERR_INVALID_ARG;
  if (!req || !ticket) return CVO_ERR_INVALID_ARG;
  const int D = ctx->prm.color_mode == CVO_COLOR_NONE ? 0 : ctx->prm.feat_dim;
  Req* r = new Req();
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!req->xyz || req->n <= 0 || req->n > kMaxPoints || (D > 0 && !req->feat) ||
        !(req->ell0 >= 0.0) || !std::isfinite(req->ell0)) {
      delete r;
      return fail(ctx, CVO_ERR_INVALID_ARG, "bad request fields");
    }
    if (check_pose(ctx, req->P0) != CVO_OK) {
      delete r;
      return CVO_ERR_INVALID_ARG;
    }
    Cloud* t = get_cloud(ctx, req->target);
    if (!t) {
      delete r;
      return fail(ctx, CVO_ERR_NOT_FOUND, "unknown keyframe handle");
    }
    if (!serve_active(ctx)) {
      cvo_serve_params p;
      cvo_serve_params_default(&p);
      if (ctx->serve) p = ctx->serve->prm.max_inflight > 0 ? ctx->serve->prm : p;
      const cudaError_t e = cudaSetDevice(ctx->device);
      const int rc = e == cudaSuccess ? start_locked(ctx, p) : CVO_ERR_CUDA;
      if (rc != CVO_OK) {
        delete r;
        return rc;
      }
    }
    t->refs += 1;
    r->target = req->target;
    r->n = req->n;
    r->xyz.assign(req->xyz, req->xyz + 3 * req->n);
    if (D > 0) r->feat.assign(req->feat, req->feat + (size_t)D * req->n);
    std::memcpy(r->P0, req->P0, sizeof(r->P0));
    r->ell0 = req->ell0;
    cvo_params prm = ctx->prm;
    if (r->ell0 > 0.0) prm.ell0 = r->ell0;
    // work estimate with a stand-in source of the frame's size
    Cloud s_est;
    s_est.n = r->n;
    r->work = pair_work(prm, t, &s_est, ell_schedule(prm, std::max(1, prm.max_iters)));
  }
  Serve* sv = ctx->serve;
  r->t_submit = now_ms();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    r->ticket = sv->next_ticket++;
    sv->tickets[r->ticket] = r;
    {
      std::lock_guard<std::mutex> lk2(sv->stats_mu);
      sv->stats.submitted += 1;
    }
    sv->pending.push_back(r);
    sv->pending_work += r->work;
    *ticket = r->ticket;
  }
  sv->cv.notify_all();
  return CVO_OK;
}

int cvo_poll(cvo_ctx* ctx, uint64_t ticket, cvo_result* out, int* done) {
  if (!ctx || !done) return CVO_ERR_INVALID_ARG;
  *done = 0;
  Serve* sv = ctx->serve;
  if (!sv) return CVO_ERR_NOT_FOUND;
  Req* r = nullptr;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->tickets.find(ticket);
    if (it == sv->tickets.end()) return CVO_ERR_NOT_FOUND;
    if (!it->second->done) return CVO_OK;
    r = it->second;
    sv->tickets.erase(it);
  }
  if (out) *out = r->res;
  *done = 1;
  delete r;
  return CVO_OK;
}

int cvo_serve_stop(cvo_ctx* ctx) {
  if (!ctx) return CVO_ERR_INVALID_ARG;
  Serve* sv = ctx->serve;
  if (!sv) return CVO_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->quit = true;
  }
  sv->cv.notify_all();
  if (sv->th.joinable()) sv->th.join();
  return CVO_OK;
}

int cvo_serve_get_stats(cvo_ctx* ctx, cvo_serve_stats* out) {
  if (!ctx || !out) return CVO_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  Serve* sv = ctx->serve;
  if (!sv) return CVO_OK;
  std::lock_guard<std::mutex> lk(sv->stats_mu);
  *out = sv->stats;
  return CVO_OK;
}

}  // extern "C"
