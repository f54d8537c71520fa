// Host-side runtime types behind the C ABI (include/cvo.h), shared by the
// translation units that implement it: clouds with their cached cell lists
// and clusters, solve plans, batches, and the context.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/cvo.h"
#include "cvo_internal.cuh"

namespace cvo {
struct Serve;   // serve.cu
}

namespace cvo {

struct Grid {
  double h_req = 0.0;   // requested cell edge (cache key)
  GridView view{};
  float4* xyz = nullptr;
  float* feat = nullptr;
  int* cell_start = nullptr;
  size_t bytes = 0;
};

struct Clusters {
  float max_edge = 0.f;  // cache key
  int* cstart = nullptr;
  int ncl = 0;
  size_t bytes = 0;
};

struct Cloud {
  int64_t n = 0;
  int n_pad = 0;
  int D = 0, dp = 0;
  int fbytes = 4;         // bytes per stored feature value: 4 (FP32) or 2 (BF16)
  double c[3] = {0, 0, 0};
  float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};  // bounding box, centred frame
  MortonFrame mf{};
  float4* xyz = nullptr;  // packed, original order
  float* feat = nullptr;
  float4* zs = nullptr;   // Morton order (source role, and input of the cell lists)
  float* zf = nullptr;
  double radius = 0.0;    // max |x'| over the centred cloud (from its bounding box)
  std::vector<Grid> grids;
  std::vector<Clusters> clusters;
  size_t bytes = 0;
  int refs = 0;           // batches that use the cloud
};

struct Plan {
  int tgt = -1, src = -1;
  SolveCfg h_cfg{};
  SolveCfg* d_cfg = nullptr;
  IterConst* d_iters = nullptr;
  SolveState* d_state = nullptr;
  double* d_partials = nullptr;
  IterRecord* d_records = nullptr;
  int* seg_xs = nullptr;
  int* seg_pref = nullptr;
  int* cl_nseg = nullptr;
  int* cl_cand = nullptr;
  int* seg_fpref = nullptr;
  int* cl_fcand = nullptr;
  float4* cl_box = nullptr;
  int* cl_kept = nullptr;
  unsigned* ch_act = nullptr;
  int* cl_act = nullptr;
  long long* group_agg = nullptr;
  int cap_iters = 0, cap_ncl = 0;
  int nblocks = 0;
  int n_iters = 0;
  int dp = 0, color_mode = 0;
  size_t bytes = 0;
};

// Queue control of a batch launch (device memory): the control words, the
// slot counter and the kernel status, the last two zeroed before each launch.
struct BatchCtl {
  QueueCtl q;
  unsigned long long head;
  int kstatus;
  int pad;
};

}  // namespace cvo

struct cvo_batch {
  int n = 0;
  int nblocks = 0;
  int dp = 0, color_mode = 0;
  std::vector<cvo::Plan*> plans;  // caller order
  std::vector<int32_t> tgt, src;  // caller order
  std::vector<int> team;          // caller order
  std::vector<int> order;         // queue position -> caller index (largest work first)
  cvo::SolveState* d_states = nullptr; // queue order
  cvo::SolveState* h_states = nullptr; // pinned, queue order
  cvo::QueueEntry* d_entries = nullptr;
  cvo::BatchCtl* d_ctl = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  size_t bytes = 0;
};

struct cvo_ctx {
  cudaMemPool_t pool = nullptr;   // every long-lived device allocation (stream-ordered)
  cvo::Serve* serve = nullptr;    // request loop (cvo_submit / cvo_poll), started on demand
  int device = 0;
  int sms = 0;
  cvo_params prm{};
  size_t budget = 0, used = 0;
  cudaStream_t stream = nullptr;
  std::vector<cvo::Cloud*> clouds;
  std::map<std::pair<int, int>, cvo::Plan*> plans;
  std::vector<cvo_batch*> batches;
  cvo::Plan* eval_plan = nullptr;      // reused by cvo_eval
  cvo::SolveState* h_state = nullptr;  // pinned
  cvo::CloudStats* d_stats = nullptr;
  cvo::CloudStats* h_stats = nullptr;  // pinned
  int* h_int = nullptr;           // pinned scratch for small read-backs
  std::string err;
  std::mutex mu;
};


namespace cvo {

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(ctx, CVO_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// api.cu
int fail(cvo_ctx* ctx, int code, const std::string& msg);
int dev_alloc(cvo_ctx* ctx, void** p, size_t bytes, size_t* acct);   // budgeted, pool, ctx stream
void dev_free(cvo_ctx* ctx, void* p);                                 // stream-ordered on ctx stream
void release_bytes(cvo_ctx* ctx, size_t bytes);
Cloud* get_cloud(cvo_ctx* ctx, int32_t h);
int32_t add_cloud(cvo_ctx* ctx, Cloud* c);
int create_cloud(cvo_ctx* ctx, const float* xyz, const float* feat, int64_t n, bool on_dev,
                 cudaStream_t us, Cloud** out,
                 bool wait = true);
void free_cloud(cvo_ctx* ctx, Cloud* c);
void free_plan(cvo_ctx* ctx, Plan* p);
std::vector<double> ell_schedule(const cvo_params& p, int n);
int configure_plan(cvo_ctx* ctx, Plan* p, Cloud* t, Cloud* s, const std::vector<double>& ells,
                   int mode);
double pair_work(const cvo_params& prm, const Cloud* t, const Cloud* s,
                 const std::vector<double>& ells);
void fill_stats(const SolveState* hs, cvo_stats* stats);
int status_code(int bits);
int check_pose(cvo_ctx* ctx, const double* P);
int kernel_mode(const cvo_params& p);   // label product | kFeatBf16

// serve.cu
void serve_shutdown(cvo_ctx* ctx);   // drain and stop the request loop (no lock held)
bool serve_active(cvo_ctx* ctx);     // the request loop runs: whole-GPU solves must wait

}  // namespace cvo
