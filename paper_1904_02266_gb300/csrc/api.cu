// Host runtime behind the C ABI in include/cvo.h: contexts, clouds, cached
// target cell lists, solve plans, and the launches that run a whole solve on
// the device (Problem 1 iterated inside one persistent kernel, no host round
// trip per iteration): one pair per launch, or many uneven pairs in one
// queue-driven launch replayed from a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/cvo.h"
#include "cvo_internal.cuh"
#include "runtime.h"

using namespace cvo;

const char* cvo_static_last_error();   // noalloc.cu

namespace cvo {

int fail(cvo_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int dev_alloc(cvo_ctx* ctx, void** p, size_t bytes, size_t* acct) {
  *p = nullptr;
  if (ctx->budget > 0 && ctx->used + bytes > ctx->budget)
    return fail(ctx, CVO_ERR_OUT_OF_BUDGET, "HBM budget exhausted");
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, ctx->stream);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail(ctx, CVO_ERR_CUDA, std::string("cudaMallocFromPoolAsync: ") + cudaGetErrorString(e));
  }
  ctx->used += bytes;
  if (acct) *acct += bytes;
  return CVO_OK;
}

void dev_free(cvo_ctx* ctx, void* p) {
  if (p) cudaFreeAsync(p, ctx->stream);
}

void release_bytes(cvo_ctx* ctx, size_t bytes) { ctx->used -= bytes <= ctx->used ? bytes : ctx->used; }

int padded_dim(const cvo_params& p) {
  if (p.color_mode == CVO_COLOR_NONE || p.feat_dim == 0) return 0;
  if (p.feat_dim <= 3) return 3;
  if (p.feat_dim <= 5) return 5;
  return 8;
}

// Mode the kernels are instantiated for: the label product, with kFeatBf16
// when the feature planes hold BF16 values.
int kernel_mode(const cvo_params& p) {
  if (p.color_mode == CVO_COLOR_NONE || p.feat_dim == 0) return kColorNone;
  return p.color_mode | (p.feat_bf16 ? kFeatBf16 : 0);
}

// Feature pre-scale: for the appearance kernel, sqrt(log2(e) / (2 ell_c^2)) so
// that |f'_i - g'_j|^2 is the base-2 exponent; for the dot product, sqrt(s).
float feature_scale(const cvo_params& p) {
  if (p.color_mode == CVO_COLOR_KERNEL)
    return (float)std::sqrt(1.4426950408889634 / (2.0 * p.ell_color * p.ell_color));
  if (p.color_mode == CVO_COLOR_DOT) return (float)std::sqrt(p.color_scale);
  return 1.0f;
}

double cutoff_radius(const cvo_params& p, double ell) {
  return ell * std::sqrt(2.0 * std::log(1.0 / p.kcut));
}

Cloud* get_cloud(cvo_ctx* ctx, int32_t h) {
  if (h < 0 || h >= (int32_t)ctx->clouds.size()) return nullptr;
  return ctx->clouds[h];
}

void free_grid(cvo_ctx* ctx, Grid& g) {
  dev_free(ctx, g.xyz);
  dev_free(ctx, g.feat);
  dev_free(ctx, g.cell_start);
  release_bytes(ctx, g.bytes);
  g = Grid();
}

void free_plan_buffers(cvo_ctx* ctx, Plan* p) {
  dev_free(ctx, p->d_cfg);
  dev_free(ctx, p->d_iters);
  dev_free(ctx, p->d_state);
  dev_free(ctx, p->d_partials);
  dev_free(ctx, p->d_records);
  dev_free(ctx, p->seg_xs);
  dev_free(ctx, p->seg_pref);
  dev_free(ctx, p->cl_nseg);
  dev_free(ctx, p->cl_cand);
  dev_free(ctx, p->seg_fpref);
  dev_free(ctx, p->cl_fcand);
  dev_free(ctx, p->cl_box);
  dev_free(ctx, p->cl_kept);
  dev_free(ctx, p->ch_act);
  dev_free(ctx, p->cl_act);
  dev_free(ctx, p->group_agg);
  release_bytes(ctx, p->bytes);
  p->d_cfg = nullptr;
  p->d_iters = nullptr;
  p->d_state = nullptr;
  p->d_partials = nullptr;
  p->d_records = nullptr;
  p->seg_xs = p->seg_pref = p->cl_nseg = p->cl_cand = p->cl_kept = nullptr;
  p->seg_fpref = p->cl_fcand = nullptr;
  p->cl_box = nullptr;
  p->ch_act = nullptr;
  p->cl_act = nullptr;
  p->group_agg = nullptr;
  p->bytes = 0;
  p->cap_iters = p->cap_ncl = 0;
}

void free_plan(cvo_ctx* ctx, Plan* p) {
  if (!p) return;
  free_plan_buffers(ctx, p);
  delete p;
}

void free_cloud(cvo_ctx* ctx, Cloud* c) {
  if (!c) return;
  for (Grid& g : c->grids) free_grid(ctx, g);
  for (Clusters& k : c->clusters) {
    dev_free(ctx, k.cstart);
    release_bytes(ctx, k.bytes);
  }
  dev_free(ctx, c->xyz);
  dev_free(ctx, c->feat);
  dev_free(ctx, c->zs);
  dev_free(ctx, c->zf);
  release_bytes(ctx, c->bytes);
  delete c;
}

// Cell list of edge >= h_req over target cloud c (cached per requested edge).
int ensure_grid(cvo_ctx* ctx, Cloud* c, double h_req, int* index_out) {
  for (size_t i = 0; i < c->grids.size(); ++i)
    if (c->grids[i].h_req == h_req) {
      *index_out = (int)i;
      return CVO_OK;
    }
  Grid g;
  g.h_req = h_req;
  double h = h_req;
  int nx, ny, nz;
  for (;;) {
    nx = (int)std::floor((c->hi[0] - c->lo[0]) / h) + 1;
    ny = (int)std::floor((c->hi[1] - c->lo[1]) / h) + 1;
    nz = (int)std::floor((c->hi[2] - c->lo[2]) / h) + 1;
    if ((double)nx * ny * nz <= (double)kMaxCells) break;
    h *= 1.25;  // a coarser grid visits more candidates but stays exact
  }
  const int ncells = nx * ny * nz;
  const int n = (int)c->n;
  int rc = dev_alloc(ctx, (void**)&g.xyz, sizeof(float4) * c->n_pad, &g.bytes);
  if (rc == CVO_OK && c->dp > 0)
    rc = dev_alloc(ctx, (void**)&g.feat, (size_t)c->fbytes * c->dp * c->n_pad, &g.bytes);
  if (rc == CVO_OK) rc = dev_alloc(ctx, (void**)&g.cell_start, sizeof(int) * (ncells + 1), &g.bytes);
  if (rc != CVO_OK) {
    free_grid(ctx, g);
    return rc;
  }
  const float hf = (float)h;
  // built from the Morton-ordered copy: the stable cell sort keeps each cell's
  // points in Morton order, so consecutive candidates are spatially compact
  cudaError_t e = build_grid(c->zs, c->zf, n, c->dp, c->n_pad, c->fbytes == 2, nx, ny, nz,
                             c->lo[0], c->lo[1],
                             c->lo[2], hf, g.xyz, g.feat, g.cell_start, ctx->pool, ctx->stream);
  if (e != cudaSuccess) {
    free_grid(ctx, g);
    return fail(ctx, CVO_ERR_CUDA, std::string("build_grid: ") + cudaGetErrorString(e));
  }
  GridView& v = g.view;
  v.xyz = g.xyz;
  v.feat = g.feat;
  v.cell_start = g.cell_start;
  v.n = n;
  v.n_pad = c->n_pad;
  v.nx = nx;
  v.ny = ny;
  v.nz = nz;
  v.ox = c->lo[0];
  v.oy = c->lo[1];
  v.oz = c->lo[2];
  v.h = hf;
  v.inv_h = 1.0f / hf;
  c->grids.push_back(g);
  *index_out = (int)c->grids.size() - 1;
  return CVO_OK;
}

// Source clusters whose octree nodes have edge <= max_edges[l], one set per
// level (cached per edge). Missing sets are built back to back and their
// counts read with one synchronisation.
int ensure_clusters(cvo_ctx* ctx, Cloud* c, const std::vector<float>& max_edges,
                    std::vector<int>* index_out) {
  index_out->assign(max_edges.size(), -1);
  std::vector<size_t> built;   // indices into c->clusters built by this call
  std::vector<float> edges;
  std::vector<int*> starts, counts;
  for (size_t l = 0; l < max_edges.size(); ++l) {
    for (size_t i = 0; i < c->clusters.size(); ++i)
      if (c->clusters[i].max_edge == max_edges[l]) (*index_out)[l] = (int)i;
    if ((*index_out)[l] >= 0) continue;
    if ((int)built.size() >= kMaxLevels) return fail(ctx, CVO_ERR_INTERNAL, "too many levels");
    Clusters k;
    k.max_edge = max_edges[l];
    int rc = dev_alloc(ctx, (void**)&k.cstart, sizeof(int) * (c->n + 2), &k.bytes);
    if (rc != CVO_OK) return rc;
    k.ncl = -1;   // filled after the synchronisation
    edges.push_back(k.max_edge);
    starts.push_back(k.cstart);
    counts.push_back(k.cstart + c->n + 1);
    c->clusters.push_back(k);
    built.push_back(c->clusters.size() - 1);
    (*index_out)[l] = (int)c->clusters.size() - 1;
  }
  if (built.empty()) return CVO_OK;
  // every missing level in one launch, their counts read with one synchronisation
  cudaError_t e = build_clusters(c->zs, (int)c->n, c->mf, edges.data(), starts.data(),
                                 counts.data(), (int)built.size(), ctx->stream);
  for (size_t j = 0; j < built.size() && e == cudaSuccess; ++j)
    e = cudaMemcpyAsync(ctx->h_int + j, counts[j], sizeof(int), cudaMemcpyDeviceToHost,
                        ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    for (size_t j = built.size(); j-- > 0;) {
      Clusters& k = c->clusters[built[j]];
      dev_free(ctx, k.cstart);
      release_bytes(ctx, k.bytes);
      c->clusters.erase(c->clusters.begin() + built[j]);
    }
    return fail(ctx, CVO_ERR_CUDA, std::string("build_clusters: ") + cudaGetErrorString(e));
  }
  for (size_t j = 0; j < built.size(); ++j) c->clusters[built[j]].ncl = ctx->h_int[j];
  return CVO_OK;
}

std::vector<double> ell_schedule(const cvo_params& p, int n) {
  std::vector<double> out;
  out.reserve(n);
  if (p.schedule == CVO_SCHEDULE_TABLE1) {
    for (int k = 0; k < n; ++k) {
      const int it = k + 1;
      out.push_back(it <= 3 ? 0.15 : it <= 10 ? 0.10 : it <= 20 ? 0.06 : 0.03);
    }
    return out;
  }
  double ell = p.ell0;
  for (int k = 0; k < n; ++k) {
    out.push_back(ell);
    ell = std::max(ell * p.ell_decay, p.ell_min);
  }
  return out;
}

double ell_floor(const cvo_params& p) {
  return p.schedule == CVO_SCHEDULE_TABLE1 ? 0.03 : p.ell_min;
}

// Grow the plan's device buffers to the given capacities.
int reserve_plan(cvo_ctx* ctx, Plan* p, int iters, int ncl, int nblocks) {
  if (p->d_cfg && iters <= p->cap_iters && ncl <= p->cap_ncl && nblocks == p->nblocks)
    return CVO_OK;
  free_plan_buffers(ctx, p);
  iters = std::max(iters, 1);
  ncl = std::max(ncl, 1);
  const int ng = (ncl + 31) / 32;
  int rc = dev_alloc(ctx, (void**)&p->d_cfg, sizeof(SolveCfg), &p->bytes);
  if (rc == CVO_OK) rc = dev_alloc(ctx, (void**)&p->d_iters, sizeof(IterConst) * iters, &p->bytes);
  if (rc == CVO_OK) rc = dev_alloc(ctx, (void**)&p->d_state, sizeof(SolveState), &p->bytes);
  if (rc == CVO_OK)
    rc = dev_alloc(ctx, (void**)&p->d_partials, sizeof(double) * 2 * kPartialStride * nblocks,
                   &p->bytes);
  if (rc == CVO_OK)
    rc = dev_alloc(ctx, (void**)&p->d_records, sizeof(IterRecord) * iters, &p->bytes);
  if (rc == CVO_OK) rc = dev_alloc(ctx, (void**)&p->seg_xs, sizeof(int) * (size_t)ncl * kMaxSeg, &p->bytes);
  if (rc == CVO_OK) rc = dev_alloc(ctx, (void**)&p->seg_pref, sizeof(int) * (size_t)ncl * kMaxSeg, &p->bytes);
  if (rc == CVO_OK) rc = dev_alloc(ctx, (void**)&p->cl_nseg, sizeof(int) * ncl, &p->bytes);
  if (rc == CVO_OK) rc = dev_alloc(ctx, (void**)&p->cl_cand, sizeof(int) * ncl, &p->bytes);
  if (rc == CVO_OK) rc = dev_alloc(ctx, (void**)&p->seg_fpref, sizeof(int) * (size_t)ncl * kMaxSeg, &p->bytes);
  if (rc == CVO_OK) rc = dev_alloc(ctx, (void**)&p->cl_fcand, sizeof(int) * ncl, &p->bytes);
  if (rc == CVO_OK) rc = dev_alloc(ctx, (void**)&p->cl_box, sizeof(float4) * 2 * (size_t)ncl, &p->bytes);
  if (rc == CVO_OK) rc = dev_alloc(ctx, (void**)&p->cl_kept, sizeof(int) * ncl, &p->bytes);
  if (rc == CVO_OK) rc = dev_alloc(ctx, (void**)&p->ch_act, sizeof(unsigned) * 32 * (size_t)ncl, &p->bytes);
  if (rc == CVO_OK) rc = dev_alloc(ctx, (void**)&p->cl_act, sizeof(int) * ncl, &p->bytes);
  if (rc == CVO_OK) rc = dev_alloc(ctx, (void**)&p->group_agg, sizeof(long long) * ng, &p->bytes);
  if (rc != CVO_OK) {
    free_plan_buffers(ctx, p);
    return rc;
  }
  p->cap_iters = iters;
  p->cap_ncl = ncl;
  p->nblocks = nblocks;
  return CVO_OK;
}

// Configure a plan for target t, source s and the lengthscales of its
// iterations: cell lists and clusters per level (a finer level whenever the
// cutoff radius has shrunk to half the current cell edge), work buffers, the
// per-iteration constants and the solve configuration on the device.
int configure_plan(cvo_ctx* ctx, Plan* p, Cloud* t, Cloud* s, const std::vector<double>& ells,
                   int mode) {
  const cvo_params& prm = ctx->prm;
  const double f = prm.cell_factor;
  std::vector<double> hs;
  std::vector<int> level_of(ells.size(), 0);
  double h_cur = -1.0;
  for (size_t k = 0; k < ells.size(); ++k) {
    const double rc = cutoff_radius(prm, ells[k]);
    if (h_cur < 0.0 || (f * rc <= CVO_LEVEL_RATIO * h_cur && (int)hs.size() < kMaxLevels)) {
      h_cur = f * rc;
      hs.push_back(h_cur);
    }
    level_of[k] = (int)hs.size() - 1;
  }
  SolveCfg cfg{};
  int ncl_max = 0;
  std::vector<float> edges(hs.size());
  for (size_t l = 0; l < hs.size(); ++l) {
    int gi = 0;
    int rc = ensure_grid(ctx, t, hs[l], &gi);
    if (rc != CVO_OK) return rc;
    cfg.grids[l] = t->grids[gi].view;
    // cluster edge: cluster_factor cells, capped so that the cluster's rotated
    // bounding box widened by the plan radius (<= 2.21 r_c) spans <= 6 cells,
    // i.e. at most 8 x 8 = kMaxSeg cell rows
    const double hh = t->grids[gi].view.h;
    const double rc_level = hs[l] / f;
    edges[l] = (float)std::min(prm.cluster_factor * hh,
                               (6.0 * hh - 2.21 * rc_level) / std::sqrt(3.0));
  }
  std::vector<int> ki;
  int rc = ensure_clusters(ctx, s, edges, &ki);
  if (rc != CVO_OK) return rc;
  for (size_t l = 0; l < hs.size(); ++l) {
    cfg.clusters[l].cstart = s->clusters[ki[l]].cstart;
    cfg.clusters[l].ncl = s->clusters[ki[l]].ncl;
    ncl_max = std::max(ncl_max, s->clusters[ki[l]].ncl);
  }
  const int per_sm = solve_blocks_per_sm(s->dp, kernel_mode(prm));
  if (per_sm <= 0) return fail(ctx, CVO_ERR_CUDA, "solve kernel cannot be resident");
  const int nblocks = std::min(per_sm * ctx->sms, 512);   // the tail reduction covers 512
  rc = reserve_plan(ctx, p, (int)ells.size(), ncl_max, nblocks);
  if (rc != CVO_OK) return rc;
  std::vector<IterConst> ic(ells.size());
  const double log2e = 1.4426950408889634073599246810019;
  for (size_t k = 0; k < ells.size(); ++k) {
    const double ell = ells[k], ell2 = ell * ell;
    const double rc2 = 2.0 * ell2 * std::log(1.0 / prm.kcut);
    ic[k].ell = ell;
    ic[k].inv_l2 = 1.0 / ell2;
    ic[k].A = (float)(log2e / (2.0 * ell2));
    ic[k].rc2 = (float)rc2;
    ic[k].rprune = (float)(std::sqrt(rc2) * 1.001);
    ic[k].level = level_of[k];
    ic[k].at_floor = ell == ell_floor(prm) ? 1 : 0;
    ic[k].kf_rot = prm.sigma * prm.sigma / (ell2 * prm.a2);
    ic[k].kf_tr = prm.sigma * prm.sigma / (ell2 * prm.b2);
    ic[k].filter = (mode == kModeEval ||
                    (k + 1 < ells.size() && ells[k + 1] == ell && level_of[k + 1] == level_of[k]))
                       ? 1 : 0;
  }
  cfg.src.xyz = s->zs;
  cfg.src.feat = s->zf;
  cfg.src.m = (int)s->n;
  cfg.src.m_pad = s->n_pad;
  cfg.iters = p->d_iters;
  cfg.seg_xs = p->seg_xs;
  cfg.seg_pref = p->seg_pref;
  cfg.cl_nseg = p->cl_nseg;
  cfg.cl_cand = p->cl_cand;
  cfg.seg_fpref = p->seg_fpref;
  cfg.cl_fcand = p->cl_fcand;
  cfg.cl_box = p->cl_box;
  cfg.cl_kept = p->cl_kept;
  cfg.ch_act = p->ch_act;
  cfg.cl_act = p->cl_act;
  cfg.group_agg = p->group_agg;
  cfg.src_radius = s->radius;
  cfg.cost_chunk = prm.cost_chunk;
  cfg.cost_cluster = prm.cost_cluster;
  cfg.cost_kept = (float)prm.cost_kept;
  for (int a = 0; a < 3; ++a) {
    cfg.cX[a] = t->c[a];
    cfg.cZ[a] = s->c[a];
  }
  cfg.sigma2 = prm.sigma * prm.sigma;
  cfg.a2 = prm.a2;
  cfg.b2 = prm.b2;
  cfg.ell_floor = ell_floor(prm);
  cfg.eps_pose = prm.eps_pose;
  cfg.eps_grad = prm.eps_grad;
  cfg.max_iters = mode == kModeEval ? 1 : prm.max_iters;
  cfg.step_order = prm.step_order;
  cfg.reduce_fp32 = prm.reduce_fp32;
  cfg.wait_polls = (unsigned)prm.wait_polls;
  cfg.join_limit_ns = (unsigned long long)(prm.join_limit_ms * 1e6);
  cfg.mode = mode;
  // pageable sources: the copies complete before the calls return
  CK(cudaMemcpyAsync(p->d_iters, ic.data(), sizeof(IterConst) * ic.size(), cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaMemcpyAsync(p->d_cfg, &cfg, sizeof(SolveCfg), cudaMemcpyHostToDevice, ctx->stream));
  p->h_cfg = cfg;
  p->n_iters = (int)ells.size();
  p->dp = s->dp;
  p->color_mode = kernel_mode(prm);
  return CVO_OK;
}

int build_plan(cvo_ctx* ctx, int tgt, int src, Plan** out) {
  Cloud* t = get_cloud(ctx, tgt);
  Cloud* s = get_cloud(ctx, src);
  Plan* p = new Plan();
  p->tgt = tgt;
  p->src = src;
  const int max_iters = std::max(0, ctx->prm.max_iters);
  std::vector<double> ells = ell_schedule(ctx->prm, std::max(1, max_iters));
  int rc = configure_plan(ctx, p, t, s, ells, kModeAlign);
  if (rc != CVO_OK) {
    free_plan(ctx, p);
    return rc;
  }
  *out = p;
  return CVO_OK;
}

// Stage P0 (and a zeroed state, which also resets the grid barrier) and run
// the solve kernel.
int run_solve(cvo_ctx* ctx, Plan* p, const double P0[16], bool records) {
  SolveState* hs = ctx->h_state;
  std::memset(hs, 0, sizeof(SolveState));
  std::memcpy(hs->P0, P0, sizeof(double) * 16);
  CK(cudaMemcpyAsync(p->d_state, hs, sizeof(SolveState), cudaMemcpyHostToDevice, ctx->stream));
  CK(launch_solve(p->dp, p->color_mode, p->nblocks, p->d_cfg, p->d_state, p->d_partials,
                  records ? p->d_records : nullptr, ctx->stream));
  CK(cudaMemcpyAsync(hs, p->d_state, sizeof(SolveState), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (hs->status & kStatusTimeout) return fail(ctx, CVO_ERR_TIMEOUT, "grid barrier timed out");
  if (hs->status != 0) return fail(ctx, CVO_ERR_INTERNAL, "cell-row segment overflow");
  return CVO_OK;
}

void destroy_batch(cvo_ctx* ctx, cvo_batch* b);

int check_pose(cvo_ctx* ctx, const double* P) {
  if (!P) return fail(ctx, CVO_ERR_INVALID_ARG, "pose pointer is NULL");
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(P[i])) return fail(ctx, CVO_ERR_INVALID_ARG, "pose has a non-finite entry");
  return CVO_OK;
}

}  // namespace cvo

namespace cvo {

// Upload, check, centre, pack and Morton-order one cloud (the caller holds
// the context lock). xyz / feat are host arrays, or device arrays read on
// stream us when on_dev. The input is read before it returns (the statistics
// are waited for); with wait the packing and ordering have finished too, else
// they finish in order on the context stream, ahead of any later use.
int create_cloud(cvo_ctx* ctx, const float* xyz, const float* feat, int64_t n, bool on_dev,
                 cudaStream_t us, Cloud** out, bool wait) {
  *out = nullptr;
  if (!xyz) return fail(ctx, CVO_ERR_INVALID_ARG, "NULL xyz pointer");
  if (n <= 0 || n > kMaxPoints) return fail(ctx, CVO_ERR_INVALID_ARG, "point count out of range");
  const int D = ctx->prm.color_mode == CVO_COLOR_NONE ? 0 : ctx->prm.feat_dim;
  if (D > 0 && !feat) return fail(ctx, CVO_ERR_INVALID_ARG, "NULL feature pointer");
  CK(cudaSetDevice(ctx->device));
  if (!us) us = ctx->stream;
  Cloud* c = new Cloud();
  c->n = n;
  c->n_pad = (int)((n + 31) / 32 * 32);
  c->D = D;
  c->dp = padded_dim(ctx->prm);
  c->fbytes = (c->dp > 0 && ctx->prm.feat_bf16) ? 2 : 4;
  float *raw_xyz = nullptr, *raw_feat = nullptr;
  int rc = CVO_OK;
  auto cleanup = [&](int code) {
    if (raw_xyz) cudaFreeAsync(raw_xyz, ctx->stream);
    if (raw_feat) cudaFreeAsync(raw_feat, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    free_cloud(ctx, c);
    return code;
  };
  // staging copy of the raw input (library-owned)
  cudaError_t e = cudaMallocFromPoolAsync((void**)&raw_xyz, sizeof(float) * 3 * n, ctx->pool, ctx->stream);
  if (e == cudaSuccess && D > 0)
    e = cudaMallocFromPoolAsync((void**)&raw_feat, sizeof(float) * D * n, ctx->pool, ctx->stream);
  if (e != cudaSuccess) return cleanup(fail(ctx, CVO_ERR_CUDA, cudaGetErrorString(e)));
  if (on_dev && us != ctx->stream) {
    // order the caller's stream before our copies
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, us);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ev, 0);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return cleanup(fail(ctx, CVO_ERR_CUDA, cudaGetErrorString(e)));
  }
  const cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  e = cudaMemcpyAsync(raw_xyz, xyz, sizeof(float) * 3 * n, kind, ctx->stream);
  if (e == cudaSuccess && D > 0)
    e = cudaMemcpyAsync(raw_feat, feat, sizeof(float) * D * n, kind, ctx->stream);
  if (e == cudaSuccess) e = cloud_stats(raw_xyz, raw_feat, (int)n, D, ctx->d_stats, ctx->pool, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->h_stats, ctx->d_stats, sizeof(CloudStats), cudaMemcpyDeviceToHost,
                        ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cleanup(fail(ctx, CVO_ERR_CUDA, cudaGetErrorString(e)));
  const CloudStats st = *ctx->h_stats;
  if (st.bad) return cleanup(fail(ctx, CVO_ERR_INVALID_ARG, "cloud has a non-finite value"));
  for (int a = 0; a < 3; ++a) {
    c->c[a] = st.sum[a] / (double)n;
    // bounding box in the centred frame, widened by a few ulps
    const double lo = (double)st.lo[a] - c->c[a], hi = (double)st.hi[a] - c->c[a];
    const double pad = 1e-6 * (1.0 + std::fabs(lo) + std::fabs(hi));
    c->lo[a] = (float)(lo - pad);
    c->hi[a] = (float)(hi + pad);
  }
  c->mf = morton_frame(c->lo, c->hi);
  for (int cx = 0; cx < 2; ++cx)
    for (int cy = 0; cy < 2; ++cy)
      for (int cz = 0; cz < 2; ++cz) {
        const double x = cx ? c->hi[0] : c->lo[0], y = cy ? c->hi[1] : c->lo[1],
                     z = cz ? c->hi[2] : c->lo[2];
        c->radius = std::max(c->radius, std::sqrt(x * x + y * y + z * z));
      }
  rc = dev_alloc(ctx, (void**)&c->xyz, sizeof(float4) * c->n_pad, &c->bytes);
  if (rc == CVO_OK) rc = dev_alloc(ctx, (void**)&c->zs, sizeof(float4) * c->n_pad, &c->bytes);
  if (rc == CVO_OK && c->dp > 0)
    rc = dev_alloc(ctx, (void**)&c->feat, (size_t)c->fbytes * c->dp * c->n_pad, &c->bytes);
  if (rc == CVO_OK && c->dp > 0)
    rc = dev_alloc(ctx, (void**)&c->zf, (size_t)c->fbytes * c->dp * c->n_pad, &c->bytes);
  if (rc != CVO_OK) return cleanup(rc);
  e = pack_cloud(raw_xyz, raw_feat, (int)n, D, c->dp, c->n_pad, c->c[0], c->c[1], c->c[2],
                 feature_scale(ctx->prm), c->fbytes == 2, c->xyz, c->feat, ctx->stream);
  if (e == cudaSuccess)
    e = morton_order(c->xyz, c->feat, (int)n, c->dp, c->n_pad, c->fbytes == 2, c->mf, c->zs, c->zf,
                     ctx->pool,
                     ctx->stream);
  if (raw_xyz) cudaFreeAsync(raw_xyz, ctx->stream);
  if (raw_feat) cudaFreeAsync(raw_feat, ctx->stream);
  raw_xyz = raw_feat = nullptr;
  if (e == cudaSuccess && wait) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cleanup(fail(ctx, CVO_ERR_CUDA, cudaGetErrorString(e)));
  *out = c;
  return CVO_OK;
}

// Register a cloud under a handle (reusing a free slot).
int32_t add_cloud(cvo_ctx* ctx, Cloud* c) {
  int32_t h = -1;
  for (size_t i = 0; i < ctx->clouds.size(); ++i)
    if (!ctx->clouds[i]) {
      h = (int32_t)i;
      break;
    }
  if (h < 0) {
    h = (int32_t)ctx->clouds.size();
    ctx->clouds.push_back(nullptr);
  }
  ctx->clouds[h] = c;
  return h;
}


}  // namespace cvo

extern "C" {

void cvo_params_default(cvo_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->ell0 = 0.15;
  p->ell_decay = 0.9;
  p->ell_min = 0.02;
  p->schedule = CVO_SCHEDULE_DECAY;
  p->sigma = 1.0;
  p->kcut = 1e-3;
  p->color_mode = CVO_COLOR_KERNEL;
  p->ell_color = 0.1;
  p->color_scale = 1e-5;
  p->a2 = 1.0;
  p->b2 = 1.0;
  p->max_iters = 200;
  p->eps_pose = 1e-5;
  p->eps_grad = 5e-5;
  p->step_order = 4;
  p->feat_dim = 5;
  p->cell_factor = 0.7;
  p->cluster_factor = 2.0;
  p->cost_chunk = 48;
  p->cost_cluster = 32;
  p->cost_kept = 0.0;
  p->team_factor = 4.0;
  p->wait_polls = 1 << 22;
  p->join_limit_ms = 60000.0;
}

const char* cvo_strerror(int s) {
  switch (s) {
    case CVO_OK: return "CVO_OK";
    case CVO_ERR_INVALID_ARG: return "CVO_ERR_INVALID_ARG";
    case CVO_ERR_OUT_OF_BUDGET: return "CVO_ERR_OUT_OF_BUDGET";
    case CVO_ERR_CUDA: return "CVO_ERR_CUDA";
    case CVO_ERR_TIMEOUT: return "CVO_ERR_TIMEOUT";
    case CVO_ERR_BUSY: return "CVO_ERR_BUSY";
    case CVO_ERR_NOT_FOUND: return "CVO_ERR_NOT_FOUND";
    case CVO_ERR_INTERNAL: return "CVO_ERR_INTERNAL";
    default: return "CVO_ERR_UNKNOWN";
  }
}

const char* cvo_last_error(cvo_ctx* ctx) { return ctx ? ctx->err.c_str() : cvo_static_last_error(); }

int cvo_create(const cvo_params* params, int device, size_t hbm_budget_bytes, cvo_ctx** out) {
  if (!out) return CVO_ERR_INVALID_ARG;
  *out = nullptr;
  cvo_params p;
  if (params) p = *params;
  else cvo_params_default(&p);
  const bool ok = p.ell0 > 0 && p.ell_min > 0 && p.ell_decay > 0 && p.ell_decay <= 1 &&
                  p.sigma > 0 && p.kcut > 0 && p.kcut < 1 && p.a2 > 0 && p.b2 > 0 &&
                  p.max_iters >= 0 && p.max_iters <= 100000 && p.feat_dim >= 0 &&
                  p.feat_dim <= CVO_MAX_FEAT && (p.step_order == 2 || p.step_order == 4) &&
                  (p.schedule == CVO_SCHEDULE_DECAY || p.schedule == CVO_SCHEDULE_TABLE1) &&
                  (p.color_mode >= CVO_COLOR_NONE && p.color_mode <= CVO_COLOR_DOT) &&
                  (p.color_mode != CVO_COLOR_KERNEL || p.ell_color > 0) &&
                  (p.color_mode != CVO_COLOR_DOT || p.color_scale > 0) &&
                  p.cell_factor >= 0.5 && p.cell_factor <= 8.0 && std::isfinite(p.ell0) &&
                  p.cluster_factor > 0.0 && p.cluster_factor <= 8.0 && p.cost_chunk >= 0 &&
                  p.cost_chunk <= 4096 && p.cost_cluster >= 0 && p.cost_cluster <= 65536 &&
                  p.team_factor > 0.0 && p.team_factor <= 1024.0 && p.cost_kept >= 0.0 &&
                  p.cost_kept <= 1024.0 && (p.feat_bf16 == 0 || p.feat_bf16 == 1) &&
                  (p.reduce_fp32 == 0 || p.reduce_fp32 == 1) && p.wait_polls >= 1 &&
                  p.wait_polls <= (1 << 30) && p.join_limit_ms > 0.0 && p.join_limit_ms <= 1e7;
  if (!ok) return CVO_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return CVO_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return CVO_ERR_CUDA;
  cvo_ctx* ctx = new cvo_ctx();
  ctx->device = device;
  ctx->prm = p;
  if (p.feat_dim == 0) ctx->prm.color_mode = CVO_COLOR_NONE;
  ctx->budget = hbm_budget_bytes;
  if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost((void**)&ctx->h_state, sizeof(SolveState)) != cudaSuccess ||
      cudaMallocHost((void**)&ctx->h_stats, sizeof(CloudStats)) != cudaSuccess ||
      cudaMallocHost((void**)&ctx->h_int, sizeof(int) * 2 * kMaxLevels) != cudaSuccess ||
      cudaMalloc((void**)&ctx->d_stats, sizeof(CloudStats)) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cvo_destroy(ctx);
    return CVO_ERR_CUDA;
  }
  // a private stream-ordered pool that keeps freed memory for reuse: frees
  // never wait for kernels on other streams (the request loop frees while its
  // persistent kernel runs)
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  uint64_t keep = ~0ull;
  if (cudaMemPoolCreate(&ctx->pool, &props) != cudaSuccess ||
      cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
    ctx->pool = nullptr;
    cvo_destroy(ctx);
    return CVO_ERR_CUDA;
  }
  *out = ctx;
  return CVO_OK;
}

int cvo_destroy(cvo_ctx* ctx) {
  if (!ctx) return CVO_ERR_INVALID_ARG;
  cudaSetDevice(ctx->device);
  serve_shutdown(ctx);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  while (!ctx->batches.empty()) destroy_batch(ctx, ctx->batches.back());
  for (auto& kv : ctx->plans) free_plan(ctx, kv.second);
  ctx->plans.clear();
  free_plan(ctx, ctx->eval_plan);
  for (Cloud* c : ctx->clouds) free_cloud(ctx, c);
  ctx->clouds.clear();
  if (ctx->d_stats) cudaFree(ctx->d_stats);
  if (ctx->h_stats) cudaFreeHost(ctx->h_stats);
  if (ctx->h_int) cudaFreeHost(ctx->h_int);
  if (ctx->h_state) cudaFreeHost(ctx->h_state);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);   // stream-ordered frees complete
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return CVO_OK;
}

int cvo_set_cloud(cvo_ctx* ctx, const float* xyz, const float* feat, int64_t n, uint32_t flags,
                  void* stream, int32_t* handle_out) {
  if (!ctx) return CVO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!handle_out) return fail(ctx, CVO_ERR_INVALID_ARG, "NULL handle pointer");
  Cloud* c = nullptr;
  // the caller's arrays are read before this returns; the packing and ordering
  // complete on the context stream, ahead of every later use of the cloud
  const int rc = create_cloud(ctx, xyz, feat, n, (flags & CVO_DEVICE_PTR) != 0,
                              (cudaStream_t)stream, &c, false);
  if (rc != CVO_OK) return rc;
  *handle_out = add_cloud(ctx, c);
  return CVO_OK;
}

int cvo_release_cloud(cvo_ctx* ctx, int32_t handle) {
  if (!ctx) return CVO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  Cloud* c = get_cloud(ctx, handle);
  if (!c) return fail(ctx, CVO_ERR_NOT_FOUND, "unknown cloud handle");
  if (c->refs > 0) return fail(ctx, CVO_ERR_BUSY, "cloud is used by a batch");
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto it = ctx->plans.begin(); it != ctx->plans.end();) {
    if (it->first.first == handle || it->first.second == handle) {
      free_plan(ctx, it->second);
      it = ctx->plans.erase(it);
    } else {
      ++it;
    }
  }
  free_cloud(ctx, c);
  ctx->clouds[handle] = nullptr;
  return CVO_OK;
}

int cvo_eval(cvo_ctx* ctx, int32_t target, int32_t source, const double P[16], double ell,
             cvo_eval_result* out) {
  if (!ctx) return CVO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (serve_active(ctx))
    return fail(ctx, CVO_ERR_BUSY, "the request loop is running (cvo_serve_stop ends it)");
  Cloud* t = get_cloud(ctx, target);
  Cloud* s = get_cloud(ctx, source);
  if (!t || !s) return fail(ctx, CVO_ERR_NOT_FOUND, "unknown cloud handle");
  if (!out) return fail(ctx, CVO_ERR_INVALID_ARG, "NULL result pointer");
  if (!(ell > 0) || !std::isfinite(ell)) return fail(ctx, CVO_ERR_INVALID_ARG, "ell must be > 0");
  int rc = check_pose(ctx, P);
  if (rc != CVO_OK) return rc;
  CK(cudaSetDevice(ctx->device));
  if (!ctx->eval_plan) ctx->eval_plan = new Plan();
  Plan* p = ctx->eval_plan;
  rc = configure_plan(ctx, p, t, s, std::vector<double>(1, ell), kModeEval);
  if (rc != CVO_OK) return rc;
  rc = run_solve(ctx, p, P, false);
  if (rc != CVO_OK) return rc;
  const SolveState* hs = ctx->h_state;
  out->F = hs->F;
  for (int a = 0; a < 6; ++a) out->grad6[a] = hs->xi[a];
  for (int m = 0; m < 5; ++m) out->S[m] = hs->S[m];
  out->nnz = (int64_t)hs->nnz_eval;
  out->candidates = (int64_t)hs->cand_eval;
  return CVO_OK;
}

}  // extern "C"

namespace cvo {

// Look up (or build) the solve plan of (target, source) and stage P0.
int prepare_solve(cvo_ctx* ctx, int32_t target, int32_t source, const double P0[16],
                  double P_out[16], Plan** out) {
  Cloud* t = get_cloud(ctx, target);
  Cloud* s = get_cloud(ctx, source);
  if (!t || !s) return fail(ctx, CVO_ERR_NOT_FOUND, "unknown cloud handle");
  if (!P_out) return fail(ctx, CVO_ERR_INVALID_ARG, "NULL output pose");
  int rc = check_pose(ctx, P0);
  if (rc != CVO_OK) return rc;
  CK(cudaSetDevice(ctx->device));
  Plan* p = nullptr;
  auto key = std::make_pair((int)target, (int)source);
  auto it = ctx->plans.find(key);
  if (it != ctx->plans.end()) {
    p = it->second;
  } else {
    rc = build_plan(ctx, target, source, &p);
    if (rc != CVO_OK) return rc;
    ctx->plans[key] = p;
  }
  *out = p;
  return CVO_OK;
}

void fill_stats(const SolveState* hs, cvo_stats* stats) {
  if (stats) {
    stats->iters = hs->iter;
    stats->converged = hs->converged;
    stats->fallback_steps = hs->fallback_steps;
    stats->no_ascent_steps = hs->no_ascent_steps;
    stats->final_ell = hs->ell;
    stats->F_last = hs->F;
    stats->t_last = hs->t;
    stats->pair_evals = (int64_t)hs->nnz_total;
    stats->candidates = (int64_t)hs->cand_total;
    stats->status = hs->status;
    stats->device_ms = (double)(hs->t_end_ns - hs->t_begin_ns) * 1e-6;
  }
}

}  // namespace cvo

extern "C" {

int cvo_align(cvo_ctx* ctx, int32_t target, int32_t source, const double P0[16], double P_out[16],
              cvo_stats* stats) {
  if (!ctx) return CVO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (serve_active(ctx))
    return fail(ctx, CVO_ERR_BUSY, "the request loop is running (cvo_serve_stop ends it)");
  Plan* p = nullptr;
  int rc = prepare_solve(ctx, target, source, P0, P_out, &p);
  if (rc != CVO_OK) return rc;
  rc = run_solve(ctx, p, P0, false);
  const SolveState* hs = ctx->h_state;
  std::memcpy(P_out, hs->P, sizeof(double) * 16);
  fill_stats(hs, stats);
  if (stats) stats->status = rc;
  return rc;
}

int cvo_set_wait_limits(cvo_ctx* ctx, int wait_polls, double join_limit_ms) {
  if (!ctx) return CVO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!(wait_polls >= 1 && wait_polls <= (1 << 30) && join_limit_ms > 0.0 && join_limit_ms <= 1e7))
    return fail(ctx, CVO_ERR_INVALID_ARG, "wait_polls outside [1, 2^30] or join_limit_ms "
                                          "outside (0, 1e7]");
  if (serve_active(ctx))
    return fail(ctx, CVO_ERR_BUSY, "the request loop is running (cvo_serve_stop ends it)");
  CK(cudaSetDevice(ctx->device));
  ctx->prm.wait_polls = wait_polls;
  ctx->prm.join_limit_ms = join_limit_ms;
  // every configuration already on the device: cached plans, the evaluation
  // plan and the plans of live batches (a batch's graph reads its plans'
  // configurations at run time)
  std::vector<Plan*> all;
  for (auto& kv : ctx->plans) all.push_back(kv.second);
  if (ctx->eval_plan) all.push_back(ctx->eval_plan);
  for (cvo_batch* b : ctx->batches)
    for (Plan* p : b->plans) all.push_back(p);
  for (Plan* p : all) {
    p->h_cfg.wait_polls = (unsigned)wait_polls;
    p->h_cfg.join_limit_ns = (unsigned long long)(join_limit_ms * 1e6);
    CK(cudaMemcpyAsync(p->d_cfg, &p->h_cfg, sizeof(SolveCfg), cudaMemcpyHostToDevice,
                       ctx->stream));
    // the copy reads h_cfg: wait before the next plan's fields change
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return CVO_OK;
}

int cvo_align_profile(cvo_ctx* ctx, int32_t target, int32_t source, const double P0[16],
                      double P_out[16], cvo_stats* stats, cvo_iter_profile* records,
                      int max_records, int* n_records) {
  if (!ctx) return CVO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (serve_active(ctx))
    return fail(ctx, CVO_ERR_BUSY, "the request loop is running (cvo_serve_stop ends it)");
  if (max_records > 0 && !records) return fail(ctx, CVO_ERR_INVALID_ARG, "NULL records");
  Plan* p = nullptr;
  int rc = prepare_solve(ctx, target, source, P0, P_out, &p);
  if (rc != CVO_OK) return rc;
  rc = run_solve(ctx, p, P0, true);
  const SolveState* hs = ctx->h_state;
  std::memcpy(P_out, hs->P, sizeof(double) * 16);
  fill_stats(hs, stats);
  if (stats) stats->status = rc;
  if (rc != CVO_OK) return rc;
  const int nrec = std::min(hs->iter, max_records);
  if (nrec > 0) {
    std::vector<IterRecord> rec(nrec);
    CK(cudaMemcpy(rec.data(), p->d_records, sizeof(IterRecord) * nrec, cudaMemcpyDeviceToHost));
    for (int i = 0; i < nrec; ++i) {
      cvo_iter_profile& r = records[i];
      r.ell = rec[i].ell;
      r.plan_ms = rec[i].t_plan_ns * 1e-6f;
      r.grad_ms = rec[i].t_grad_ns * 1e-6f;
      r.step_ms = rec[i].t_step_ns * 1e-6f;
      r.grad_pass_ms = rec[i].t_grad_pass_ns * 1e-6f;
      r.grad_sync_ms = rec[i].t_grad_sync_ns * 1e-6f;
      r.step_pass_ms = rec[i].t_step_pass_ns * 1e-6f;
      r.step_sync_ms = rec[i].t_step_sync_ns * 1e-6f;
      r.replanned = rec[i].replanned;
      r.grad_pairs = rec[i].grad_pairs;
      r.step_pairs = rec[i].step_pairs;
      r.grad_candidates = rec[i].grad_candidates;
      r.step_candidates = rec[i].grad_candidates;
    }
  }
  if (n_records) *n_records = nrec;
  return CVO_OK;
}

void* cvo_stream(cvo_ctx* ctx) { return ctx ? (void*)ctx->stream : nullptr; }

}  // extern "C"

namespace cvo {

// Estimated kept pairs of a whole solve, for team sizing: the source points
// times the target's points per unit area (its bounding box read as a
// surface: the sum of the products of pairs of extents) times the cutoff
// disc area, summed over the schedule, two passes per iteration.
double pair_work(const cvo_params& prm, const Cloud* t, const Cloud* s,
                 const std::vector<double>& ells) {
  double e[3];
  for (int a = 0; a < 3; ++a) e[a] = std::max(0.0, (double)t->hi[a] - (double)t->lo[a]);
  const double emax = std::max(e[0], std::max(e[1], e[2]));
  const double area = std::max(e[0] * e[1] + e[0] * e[2] + e[1] * e[2],
                               std::max(1e-3 * emax * emax, 1e-6));
  const double dens = (double)t->n / area;
  const double pi = 3.14159265358979323846;
  double disc = 0.0;
  for (double ell : ells) {
    const double rc = cutoff_radius(prm, ell);
    disc += pi * rc * rc;
  }
  return 2.0 * (double)s->n * std::min((double)t->n, dens * disc / (double)ells.size()) *
         (double)ells.size();
}

// The device work of one batch run on stream st: poses and zeroed states up,
// queue counters reset, the persistent launch, states down.
cudaError_t record_batch_launch(cvo_batch* b, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(b->d_states, b->h_states, sizeof(SolveState) * b->n,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(&b->d_ctl->head, 0, sizeof(unsigned long long) + sizeof(int), st);
  if (e == cudaSuccess)
    e = launch_queue(b->dp, b->color_mode, b->nblocks, b->d_entries, &b->d_ctl->q,
                     &b->d_ctl->head, &b->d_ctl->kstatus, 0ull, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->h_states, b->d_states, sizeof(SolveState) * b->n,
                        cudaMemcpyDeviceToHost, st);
  return e;
}

void destroy_batch(cvo_ctx* ctx, cvo_batch* b) {
  if (!b) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (Plan* p : b->plans) free_plan(ctx, p);
  for (size_t i = 0; i < b->tgt.size(); ++i) {
    if (Cloud* c = get_cloud(ctx, b->tgt[i])) c->refs -= 1;
    if (Cloud* c = get_cloud(ctx, b->src[i])) c->refs -= 1;
  }
  dev_free(ctx, b->d_states);
  dev_free(ctx, b->d_entries);
  dev_free(ctx, b->d_ctl);
  if (b->h_states) cudaFreeHost(b->h_states);
  release_bytes(ctx, b->bytes);
  ctx->batches.erase(std::remove(ctx->batches.begin(), ctx->batches.end(), b),
                     ctx->batches.end());
  delete b;
}

int status_code(int bits) {
  if (bits & kStatusTimeout) return CVO_ERR_TIMEOUT;
  if (bits != 0) return CVO_ERR_INTERNAL;
  return CVO_OK;
}

}  // namespace cvo

extern "C" {

int cvo_batch_create(cvo_ctx* ctx, int n, const int32_t* targets, const int32_t* sources,
                     const double* ell0, const int32_t* team_sizes, cvo_batch** out) {
  if (!ctx) return CVO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!out) return fail(ctx, CVO_ERR_INVALID_ARG, "NULL batch pointer");
  *out = nullptr;
  if (n < 1 || !targets || !sources)
    return fail(ctx, CVO_ERR_INVALID_ARG, "a batch needs n >= 1 and target/source arrays");
  for (int i = 0; i < n; ++i) {
    if (!get_cloud(ctx, targets[i]) || !get_cloud(ctx, sources[i]))
      return fail(ctx, CVO_ERR_NOT_FOUND, "unknown cloud handle in batch");
    if (ell0 && !(ell0[i] > 0.0 && std::isfinite(ell0[i])))
      return fail(ctx, CVO_ERR_INVALID_ARG, "ell0 must be > 0");
  }
  CK(cudaSetDevice(ctx->device));
  const Cloud* s0 = get_cloud(ctx, sources[0]);
  const int per_sm = solve_blocks_per_sm(s0->dp, kernel_mode(ctx->prm));
  if (per_sm <= 0) return fail(ctx, CVO_ERR_CUDA, "solve kernel cannot be resident");
  const int nblocks = std::min(per_sm * ctx->sms, 512);
  if (team_sizes)
    for (int i = 0; i < n; ++i)
      if (team_sizes[i] < 1 || team_sizes[i] > nblocks)
        return fail(ctx, CVO_ERR_INVALID_ARG, "team size outside [1, blocks]");
  cvo_batch* b = new cvo_batch();
  b->n = n;
  b->nblocks = nblocks;
  b->dp = s0->dp;
  b->color_mode = kernel_mode(ctx->prm);
  b->plans.assign(n, nullptr);
  b->tgt.assign(targets, targets + n);
  b->src.assign(sources, sources + n);
  for (int i = 0; i < n; ++i) {
    get_cloud(ctx, targets[i])->refs += 1;
    get_cloud(ctx, sources[i])->refs += 1;
  }
  ctx->batches.push_back(b);
  auto bail = [&](int rc) {
    destroy_batch(ctx, b);
    return rc;
  };
  // one plan per pair: the teams run at the same time, so no two pairs may
  // share work buffers even when they name the same clouds
  std::vector<double> work(n);
  const int iters = std::max(1, ctx->prm.max_iters);
  for (int i = 0; i < n; ++i) {
    cvo_params prm = ctx->prm;
    if (ell0) prm.ell0 = ell0[i];
    std::vector<double> ells = ell_schedule(prm, iters);
    Cloud* t = get_cloud(ctx, targets[i]);
    Cloud* s = get_cloud(ctx, sources[i]);
    Plan* p = new Plan();
    p->tgt = targets[i];
    p->src = sources[i];
    b->plans[i] = p;
    int rc = configure_plan(ctx, p, t, s, ells, kModeAlign);
    if (rc != CVO_OK) return bail(rc);
    work[i] = pair_work(ctx->prm, t, s, ells);
  }
  double total = 0.0;
  for (double w : work) total += w;
  b->team.resize(n);
  for (int i = 0; i < n; ++i) {
    if (team_sizes) {
      b->team[i] = team_sizes[i];
    } else {
      const double share = total > 0.0 ? work[i] / total : 1.0 / n;
      const double g = std::ceil(ctx->prm.team_factor * share * nblocks);
      b->team[i] = (int)std::max(1.0, std::min((double)nblocks, g));
    }
  }
  b->order.resize(n);
  for (int i = 0; i < n; ++i) b->order[i] = i;
  std::stable_sort(b->order.begin(), b->order.end(),
                   [&](int a, int c) { return work[a] > work[c]; });
  // The last pairs of the queue (the last 10% of the estimated work) get
  // teams four times larger: a pair takes about as long as the others on its
  // team (sizes follow the work), so when the queue runs dry the blocks would
  // otherwise wait up to one pair's time for the last teams to finish; larger
  // teams finish those pairs sooner (256-pair batch: 527 -> 570
  // frame-pairs/s; 5% x 2: 528, 10% x 2: 561, 15% x 3: 567, 20% x 4: 562,
  // 20% x 8: 557, 30% x 4: 556)
  if (!team_sizes) {
    constexpr double kTailWork = 0.10;
    constexpr int kTailBoost = 4;
    double tail = 0.0;
    for (int q = n - 1; q >= 0; --q) {
      const int i = b->order[q];
      tail += work[i];
      if (tail > kTailWork * total) break;
      b->team[i] = std::min(nblocks, b->team[i] * kTailBoost);
    }
  }
  int rc = dev_alloc(ctx, (void**)&b->d_states, sizeof(SolveState) * n, &b->bytes);
  if (rc == CVO_OK) rc = dev_alloc(ctx, (void**)&b->d_entries, sizeof(QueueEntry) * n, &b->bytes);
  if (rc == CVO_OK) rc = dev_alloc(ctx, (void**)&b->d_ctl, sizeof(BatchCtl), &b->bytes);
  if (rc != CVO_OK) return bail(rc);
  if (cudaMallocHost((void**)&b->h_states, sizeof(SolveState) * n) != cudaSuccess)
    return bail(fail(ctx, CVO_ERR_CUDA, "cudaMallocHost of batch states failed"));
  std::memset(b->h_states, 0, sizeof(SolveState) * n);
  std::vector<QueueEntry> ent(n);
  long long slot = 0;
  for (int q = 0; q < n; ++q) {
    const int i = b->order[q];
    ent[q].cfg = b->plans[i]->d_cfg;
    ent[q].st = b->d_states + q;
    ent[q].partials = b->plans[i]->d_partials;
    ent[q].out = nullptr;
    ent[q].team = b->team[i];
    ent[q].slot0 = (int)slot;
    slot += b->team[i];
  }
  BatchCtl ctl{};
  ctl.q.tail = (unsigned long long)slot;
  ctl.q.n_entries = (unsigned long long)n;
  ctl.q.stop = 1;
  CK(cudaMemcpyAsync(b->d_entries, ent.data(), sizeof(QueueEntry) * n, cudaMemcpyHostToDevice,
                     ctx->stream));
  CK(cudaMemcpyAsync(b->d_ctl, &ctl, sizeof(BatchCtl), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  // capture the launch once; a batch whose capture fails runs the same
  // operations directly on the stream
  if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    const cudaError_t e = record_batch_launch(b, ctx->stream);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
    if (e == cudaSuccess && e2 == cudaSuccess && g &&
        cudaGraphInstantiate(&b->exec, g, 0) == cudaSuccess) {
      b->graph = g;
    } else {
      if (g) cudaGraphDestroy(g);
      b->exec = nullptr;
    }
    (void)cudaGetLastError();
  }
  *out = b;
  return CVO_OK;
}

int cvo_batch_run(cvo_ctx* ctx, cvo_batch* b, const double* P0, double* P_out,
                  cvo_stats* stats) {
  if (!ctx) return CVO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!b || std::find(ctx->batches.begin(), ctx->batches.end(), b) == ctx->batches.end())
    return fail(ctx, CVO_ERR_NOT_FOUND, "unknown batch");
  if (serve_active(ctx))
    return fail(ctx, CVO_ERR_BUSY, "the request loop is running (cvo_serve_stop ends it)");
  if (!P0 || !P_out) return fail(ctx, CVO_ERR_INVALID_ARG, "NULL pose array");
  for (int i = 0; i < b->n; ++i) {
    const int rc = check_pose(ctx, P0 + 16 * (size_t)i);
    if (rc != CVO_OK) return rc;
  }
  CK(cudaSetDevice(ctx->device));
  for (int q = 0; q < b->n; ++q) {
    SolveState& hs = b->h_states[q];
    std::memset(&hs, 0, sizeof(SolveState));
    std::memcpy(hs.P0, P0 + 16 * (size_t)b->order[q], sizeof(double) * 16);
  }
  if (b->exec) {
    CK(cudaGraphLaunch(b->exec, ctx->stream));
  } else {
    CK(record_batch_launch(b, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  int first = CVO_OK;
  for (int q = 0; q < b->n; ++q) {
    const int i = b->order[q];
    const SolveState& hs = b->h_states[q];
    std::memcpy(P_out + 16 * (size_t)i, hs.P, sizeof(double) * 16);
    const int code = status_code(hs.status);
    if (stats) {
      fill_stats(&hs, &stats[i]);
      stats[i].status = code;
    }
    if (code != CVO_OK && first == CVO_OK) first = code;
  }
  if (first != CVO_OK) fail(ctx, first, "a pair of the batch failed (see its stats)");
  return first;
}

int cvo_batch_get_info(cvo_ctx* ctx, const cvo_batch* b, cvo_batch_info* info,
                       int32_t* team_sizes) {
  if (!ctx) return CVO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!b || std::find(ctx->batches.begin(), ctx->batches.end(), b) == ctx->batches.end())
    return fail(ctx, CVO_ERR_NOT_FOUND, "unknown batch");
  if (info) {
    info->pairs = b->n;
    info->blocks = b->nblocks;
    info->graph = b->exec ? 1 : 0;
    info->max_team = *std::max_element(b->team.begin(), b->team.end());
    size_t bytes = b->bytes;
    for (const Plan* p : b->plans) bytes += p->bytes;
    info->bytes = (int64_t)bytes;
  }
  if (team_sizes)
    for (int i = 0; i < b->n; ++i) team_sizes[i] = b->team[i];
  return CVO_OK;
}

int cvo_batch_destroy(cvo_ctx* ctx, cvo_batch* b) {
  if (!ctx) return CVO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!b || std::find(ctx->batches.begin(), ctx->batches.end(), b) == ctx->batches.end())
    return fail(ctx, CVO_ERR_NOT_FOUND, "unknown batch");
  destroy_batch(ctx, b);
  return CVO_OK;
}

}  // extern "C"

namespace cvo {

namespace {

// Cached structures of a cloud that the tuning changes: its cell lists and
// clusters, and every plan that uses it.
void drop_cloud_caches(cvo_ctx* ctx, int32_t h) {
  for (auto it = ctx->plans.begin(); it != ctx->plans.end();) {
    if (it->first.first == h || it->first.second == h) {
      free_plan(ctx, it->second);
      it = ctx->plans.erase(it);
    } else {
      ++it;
    }
  }
  if (ctx->eval_plan) {
    free_plan(ctx, ctx->eval_plan);
    ctx->eval_plan = nullptr;
  }
  Cloud* c = get_cloud(ctx, h);
  if (!c) return;
  for (Grid& g : c->grids) {
    dev_free(ctx, g.xyz);
    dev_free(ctx, g.feat);
    dev_free(ctx, g.cell_start);
    release_bytes(ctx, g.bytes);
  }
  c->grids.clear();
  for (Clusters& k : c->clusters) {
    dev_free(ctx, k.cstart);
    release_bytes(ctx, k.bytes);
  }
  c->clusters.clear();
}

// Device time of the fastest of reps solves with parameters prm (after one
// untimed solve that builds the plan and its cell lists).
int time_solves(cvo_ctx* ctx, int32_t t, int32_t s, const cvo_params& prm, int reps, double* ms) {
  ctx->prm = prm;
  drop_cloud_caches(ctx, t);
  drop_cloud_caches(ctx, s);
  Plan* p = nullptr;
  int rc = build_plan(ctx, t, s, &p);
  if (rc != CVO_OK) return rc;
  const double I[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double best = 1e300;
  rc = run_solve(ctx, p, I, false);
  if (rc == CVO_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    rc = fail(ctx, CVO_ERR_CUDA, "cudaEventCreate failed");
  for (int r = 0; r < reps && rc == CVO_OK; ++r) {
    SolveState* hs = ctx->h_state;
    std::memset(hs, 0, sizeof(SolveState));
    std::memcpy(hs->P0, I, sizeof(I));
    cudaError_t e = cudaMemcpyAsync(p->d_state, hs, sizeof(SolveState), cudaMemcpyHostToDevice,
                                    ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
    if (e == cudaSuccess)
      e = launch_solve(p->dp, p->color_mode, p->nblocks, p->d_cfg, p->d_state, p->d_partials,
                       nullptr, ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float f = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&f, e0, e1);
    if (e != cudaSuccess) rc = fail(ctx, CVO_ERR_CUDA, cudaGetErrorString(e));
    best = std::min(best, (double)f);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  free_plan(ctx, p);
  *ms = best;
  return rc;
}

}  // namespace

}  // namespace cvo

extern "C" {

int cvo_autotune(cvo_ctx* ctx, int32_t target, int32_t source, const cvo_tune_space* space,
                 cvo_tune_report* report) {
  if (!ctx) return CVO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  Cloud* t = get_cloud(ctx, target);
  Cloud* s = get_cloud(ctx, source);
  if (!t || !s) return fail(ctx, CVO_ERR_NOT_FOUND, "unknown cloud handle");
  if (serve_active(ctx))
    return fail(ctx, CVO_ERR_BUSY, "the request loop is running (cvo_serve_stop ends it)");
  if (t->refs > 0 || s->refs > 0) return fail(ctx, CVO_ERR_BUSY, "a batch uses the clouds");
  CK(cudaSetDevice(ctx->device));
  cvo_tune_space sp{};
  if (space) sp = *space;
  const double cells[] = {0.5, 0.6, 0.7, 0.85, 1.0, 1.25};
  const double clus[] = {1.0, 1.5, 2.0, 2.5, 3.0};
  const int chunks[] = {16, 32, 48, 64, 96};
  const int ccl[] = {0, 32, 64, 128};
  if (sp.n_cell <= 0) {
    sp.n_cell = 6;
    std::copy(cells, cells + 6, sp.cell_factor);
  }
  if (sp.n_cluster <= 0) {
    sp.n_cluster = 5;
    std::copy(clus, clus + 5, sp.cluster_factor);
  }
  if (sp.n_chunk <= 0) {
    sp.n_chunk = 5;
    std::copy(chunks, chunks + 5, sp.cost_chunk);
  }
  if (sp.n_cluster_cost <= 0) {
    sp.n_cluster_cost = 4;
    std::copy(ccl, ccl + 4, sp.cost_cluster);
  }
  if (sp.reps <= 0) sp.reps = 3;
  if (sp.n_cell > 8 || sp.n_cluster > 8 || sp.n_chunk > 8 || sp.n_cluster_cost > 8 || sp.reps > 100)
    return fail(ctx, CVO_ERR_INVALID_ARG, "at most 8 candidates per dimension, 100 repetitions");
  for (int i = 0; i < sp.n_cell; ++i)
    if (!(sp.cell_factor[i] >= 0.5 && sp.cell_factor[i] <= 8.0))
      return fail(ctx, CVO_ERR_INVALID_ARG, "cell_factor candidate outside [0.5, 8]");
  for (int i = 0; i < sp.n_cluster; ++i)
    if (!(sp.cluster_factor[i] > 0.0 && sp.cluster_factor[i] <= 8.0))
      return fail(ctx, CVO_ERR_INVALID_ARG, "cluster_factor candidate outside (0, 8]");
  for (int i = 0; i < sp.n_chunk; ++i)
    if (sp.cost_chunk[i] < 0 || sp.cost_chunk[i] > 4096)
      return fail(ctx, CVO_ERR_INVALID_ARG, "cost_chunk candidate outside [0, 4096]");
  for (int i = 0; i < sp.n_cluster_cost; ++i)
    if (sp.cost_cluster[i] < 0 || sp.cost_cluster[i] > 65536)
      return fail(ctx, CVO_ERR_INVALID_ARG, "cost_cluster candidate outside [0, 65536]");
  const cvo_params start = ctx->prm;
  cvo_params best = start;
  double best_ms = 0.0, start_ms = 0.0;
  int tried = 0;
  int rc = time_solves(ctx, target, source, start, sp.reps, &start_ms);
  best_ms = start_ms;
  ++tried;
  for (int dim = 0; dim < 4 && rc == CVO_OK; ++dim) {
    const int n = dim == 0 ? sp.n_cell : dim == 1 ? sp.n_cluster : dim == 2 ? sp.n_chunk
                                                                           : sp.n_cluster_cost;
    cvo_params base = best;
    for (int i = 0; i < n && rc == CVO_OK; ++i) {
      cvo_params c = base;
      if (dim == 0) c.cell_factor = sp.cell_factor[i];
      else if (dim == 1) c.cluster_factor = sp.cluster_factor[i];
      else if (dim == 2) c.cost_chunk = sp.cost_chunk[i];
      else c.cost_cluster = sp.cost_cluster[i];
      double ms = 0.0;
      rc = time_solves(ctx, target, source, c, sp.reps, &ms);
      ++tried;
      if (rc == CVO_OK && ms < best_ms) {
        best_ms = ms;
        best = c;
      }
    }
  }
  ctx->prm = rc == CVO_OK ? best : start;
  drop_cloud_caches(ctx, target);
  drop_cloud_caches(ctx, source);
  if (rc != CVO_OK) return rc;
  if (report) {
    report->start_ms = start_ms;
    report->best_ms = best_ms;
    report->candidates = tried;
    report->cell_factor = best.cell_factor;
    report->cluster_factor = best.cluster_factor;
    report->cost_chunk = best.cost_chunk;
    report->cost_cluster = best.cost_cluster;
  }
  return CVO_OK;
}

}  // extern "C"
