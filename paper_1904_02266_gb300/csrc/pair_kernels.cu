// The CVO hot path on sm_103a: the cutoff-truncated all-pairs kernel
// reductions behind one gradient-ascent iteration, plus the FP64 tail.
//
//  gradient pass  F = sum c_ij k(x_i, z~_j)                         (Eq. scalar)
//                 dF/domega = (1/ell^2) sum w_ij (z~_j x e_ij)      (Eq. 3_gradient,
//                 dF/dv     = (1/ell^2) sum w_ij e_ij                left-update signs)
//  step pass      S0..S4 = sum w_ij g^m_ij along xi                  (Eq. fourth)
//  tail (FP64)    xi = metric gradient (Eq. metric), t* = first maximiser of the
//                 quartic, P <- exp(t* xi) P (Eqs. newstep, step), lengthscale
//                 schedule and the Table 1 convergence test.
//
// One iteration is four kernels:
//  plan        one warp per source cluster (an octree node of the source, at
//              most 32 points): transform the points, take their bounding box
//              and record the rows of target cells (contiguous runs of the
//              cell-sorted target) that lie within the cutoff radius of it.
//  chunk_scan  cut every cluster's candidate list into 32-candidate chunks and
//              split the chunks evenly over all warps of the pair passes.
//  pair passes each lane owns one candidate target point (coalesced load into
//              registers) and loops over the cluster's source points, which the
//              warp keeps in shared memory and reads as broadcasts. Pair
//              arithmetic is FP32 with one ex2.approx per kept pair. Per-lane
//              FP32 sums are reduced in a fixed tree, blocks in FP64 by the
//              last block to finish, so results are bitwise reproducible.
// The static, even split keeps every SM busy to the end of the pass however
// uneven the clusters are.
#include <cuda_runtime.h>
#include <stdint.h>

#include "cvo_internal.cuh"

namespace cvo {

namespace {

constexpr float kFar = 1.0e18f;   // coordinate of padding points: never within any cutoff
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ int cell_floor(float v, float o, float inv_h, int n) {
  float q = floorf((v - o) * inv_h);
  q = fminf(fmaxf(q, -1.0f), (float)n);
  return (int)q;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(kFull, v, off);
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(kFull, v, off);
  return v;
}

// ---------------------------------------------------------------------------
// FP64 tail
// ---------------------------------------------------------------------------

__device__ __forceinline__ void cross3d(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

// Constants of iteration k (from the host table) and the FP32 pose.
__device__ void load_iteration(const SolveCfg* cfg, SolveState* st, const IterConst& ic) {
  st->ell = ic.ell;
  st->level = ic.level;
  st->A = ic.A;
  st->rc2 = ic.rc2;
  st->rprune = ic.rprune;
  st->inv_l2f = (float)ic.inv_l2;
}

__device__ void set_pose_constants(const SolveCfg* cfg, SolveState* st) {
  const double* P = st->P;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    double tr = P[4 * r + 3] - cfg->cX[r];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      st->R[3 * r + c] = (float)P[4 * r + c];
      tr = fma(P[4 * r + c], cfg->cZ[c], tr);
    }
    st->T[r] = (float)tr;
  }
}

// Smallest positive t at which G'(t) = c0 + c1 t + c2 t^2 + c3 t^3 changes sign
// from + to - (the first local maximum of the quartic model, Sec. 4 "Step
// size"), given c0 = S1 > 0. With three real roots r1 < r2 < r3 the sign
// pattern of G' decides: for c3 < 0 the + -> - crossings are r1 and r3, for
// c3 > 0 only r2; with one real root r, only c3 < 0 gives a crossing.
__device__ bool first_maximiser(double c0, double c1, double c2, double c3, double* t_out) {
  const double s = fmax(fmax(fabs(c0), fabs(c1)), fmax(fabs(c2), fabs(c3)));
  double t = -1.0;
  if (fabs(c3) <= 1e-12 * s) {
    // quadratic c2 t^2 + c1 t + c0 (or linear)
    if (fabs(c2) <= 1e-12 * s) {
      if (c1 < 0.0) t = -c0 / c1;
    } else {
      const double disc = c1 * c1 - 4.0 * c2 * c0;
      if (disc >= 0.0) {
        const double q = -0.5 * (c1 + copysign(sqrt(disc), c1));
        const double ra = q / c2, rb = c0 / q;
        const double lo = fmin(ra, rb), hi = fmax(ra, rb);
        // c2 < 0: + between the roots; crossing + -> - at the larger root.
        // c2 > 0: crossing + -> - at the smaller root.
        t = (c2 < 0.0) ? hi : lo;
        if (!(t > 0.0)) t = -1.0;
      }
    }
  } else {
    const double B = c2 / c3, C = c1 / c3, D = c0 / c3;
    const double B3 = B * (1.0 / 3.0);
    const double p = C - B * B3;
    const double q = (2.0 / 27.0) * B * B * B - B3 * C + D;
    const double disc = 0.25 * q * q + (1.0 / 27.0) * p * p * p;
    if (disc > 0.0) {
      if (c3 < 0.0) {
        const double u = -copysign(cbrt(0.5 * fabs(q) + sqrt(disc)), q);
        t = (u != 0.0 ? u - p / (3.0 * u) : 0.0) - B3;
      }
    } else if (p < 0.0) {
      // roots m cos(phi - 2 pi k / 3) - B/3: k = 0 largest, k = 1 middle, k = 2 smallest
      const double m = 2.0 * sqrt(-p * (1.0 / 3.0));
      const double arg = fmin(1.0, fmax(-1.0, 3.0 * q / (p * m)));
      const double phi = acos(arg) * (1.0 / 3.0);
      const double two_pi_3 = 2.0943951023931954923084289221863;
      if (c3 < 0.0) {
        const double r1 = m * cos(phi - 2.0 * two_pi_3) - B3;
        t = r1 > 0.0 ? r1 : m * cos(phi) - B3;
      } else {
        t = m * cos(phi - two_pi_3) - B3;   // k = 1: middle root
      }
    } else {
      t = -1.0;   // triple root: G'' vanishes there, so it is not a strict maximum
    }
    if (t > 0.0) {  // one Newton polish on the original cubic
      const double f = ((c3 * t + c2) * t + c1) * t + c0;
      const double fp = (3.0 * c3 * t + 2.0 * c2) * t + c1;
      if (fp != 0.0) {
        const double tn = t - f / fp;
        if (tn > 0.0 && isfinite(tn)) t = tn;
      }
    }
  }
  if (t > 0.0 && isfinite(t)) {
    *t_out = t;
    return true;
  }
  return false;
}

// exp of the twist tw = t (omega, v) in SE(3), Eq. step. The coefficients
// sin(th)/th, (1 - cos th)/th^2 and (th - sin th)/th^3 are even functions of
// th; below th = 0.5 they are summed as Taylor series in th^2 (truncation
// error < 1e-16), above it from sin and cos.
__device__ void exp_se3(const double tw[6], double dR[9], double dT[3]) {
  const double* phi = tw;
  const double* rho = tw + 3;
  const double x = phi[0] * phi[0] + phi[1] * phi[1] + phi[2] * phi[2];
  double A, B, C;
  if (x < 0.25) {
    A = 1.0 + x * (-1.0 / 6 + x * (1.0 / 120 + x * (-1.0 / 5040 + x * (1.0 / 362880 +
        x * (-1.0 / 39916800 + x * (1.0 / 6227020800.0))))));
    B = 0.5 + x * (-1.0 / 24 + x * (1.0 / 720 + x * (-1.0 / 40320 + x * (1.0 / 3628800 +
        x * (-1.0 / 479001600 + x * (1.0 / 87178291200.0))))));
    C = 1.0 / 6 + x * (-1.0 / 120 + x * (1.0 / 5040 + x * (-1.0 / 362880 + x * (1.0 / 39916800 +
        x * (-1.0 / 6227020800.0 + x * (1.0 / 1307674368000.0))))));
  } else {
    const double th = sqrt(x);
    const double s = sin(th), hs = sin(0.5 * th);
    A = s / th;
    B = 2.0 * hs * hs / x;
    C = (th - s) / (x * th);
  }
  const double W[9] = {0.0, -phi[2], phi[1], phi[2], 0.0, -phi[0], -phi[1], phi[0], 0.0};
  double W2[9];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      W2[3 * i + j] = W[3 * i] * W[j] + W[3 * i + 1] * W[3 + j] + W[3 * i + 2] * W[6 + j];
  double V[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const double I = (i % 4 == 0) ? 1.0 : 0.0;
    dR[i] = I + A * W[i] + B * W2[i];
    V[i] = I + B * W[i] + C * W2[i];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
    dT[i] = V[3 * i] * rho[0] + V[3 * i + 1] * rho[1] + V[3 * i + 2] * rho[2];
}

// Gradient-pass finaliser: sums -> F, metric gradient, unit step direction.
__device__ void finish_gradient(const SolveCfg* cfg, SolveState* st, const double sums[7]) {
  const double inv_l2 = cfg->iters[cfg->mode == kModeEval ? 0 : st->iter].inv_l2;
  const double s2 = cfg->sigma2;
  const double v[3] = {sums[4], sums[5], sums[6]};
  double cxv[3];
  cross3d(cfg->cX, v, cxv);
  const double ka = s2 * inv_l2 / cfg->a2, kb = s2 * inv_l2 / cfg->b2;
  double xi[6];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    xi[a] = (sums[1 + a] + cxv[a]) * ka;
    xi[3 + a] = v[a] * kb;
  }
  double nrm2 = 0.0;
#pragma unroll
  for (int a = 0; a < 6; ++a) nrm2 += xi[a] * xi[a];
  const double nrm = sqrt(nrm2);
#pragma unroll
  for (int a = 0; a < 6; ++a) st->xi[a] = xi[a];
  st->xi_norm = nrm;
  st->F = s2 * sums[0];
  // direction for the step pass in the centred frame: omega, v + omega x cX
  double wxc[3];
  cross3d(xi, cfg->cX, wxc);
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    st->om[a] = (float)(xi[a] * inv);
    st->vc[a] = (float)((xi[3 + a] + wxc[a]) * inv);
  }
  // counters were bumped by other blocks of this kernel: read past L1
  st->nnz_eval = __ldcg(&st->nnz_pass[0]);
  st->cand_eval = __ldcg(&st->cand_pass[0]);
}

// Step-pass finaliser: S0..S4, step length, pose update, schedule, stop test.
__device__ void finish_step(const SolveCfg* cfg, SolveState* st, const double sums[5],
                            cudaGraphConditionalHandle cond, int use_cond) {
  const double nxi = st->xi_norm;
  double S[5];
  double pw = cfg->sigma2;
#pragma unroll
  for (int m = 0; m < 5; ++m) {  // the sums were taken along xi / |xi|
    S[m] = sums[m] * pw;
    pw *= nxi;
  }
#pragma unroll
  for (int m = 0; m < 5; ++m) st->S[m] = S[m];
  st->nnz_total += __ldcg(&st->nnz_pass[0]) + __ldcg(&st->nnz_pass[1]);
  st->cand_total += __ldcg(&st->cand_pass[0]) + __ldcg(&st->cand_pass[1]);
  if (cfg->mode == kModeEval) {
    st->done = 1;
    if (use_cond) cudaGraphSetConditional(cond, 0u);
    return;
  }
  double t;
  if (!(nxi > 0.0) || !(S[1] > 0.0)) {
    t = 0.0;
    st->no_ascent_steps += 1;
  } else {
    bool ok;
    if (cfg->step_order == 2) {
      ok = S[2] < 0.0;
      t = ok ? -S[1] / (2.0 * S[2]) : 0.0;
    } else {
      ok = first_maximiser(S[1], 2.0 * S[2], 3.0 * S[3], 4.0 * S[4], &t);
    }
    if (!ok) {
      st->fallback_steps += 1;
      t = st->have_t_prev ? 0.5 * st->t_prev : 1e-3 / nxi;
    }
  }
  // P <- exp(t xi) P
  double tw[6], dR[9], dT[3];
#pragma unroll
  for (int a = 0; a < 6; ++a) tw[a] = t * st->xi[a];
  exp_se3(tw, dR, dT);
  double Pn[16];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
      Pn[4 * r + c] = dR[3 * r] * st->P[c] + dR[3 * r + 1] * st->P[4 + c] + dR[3 * r + 2] * st->P[8 + c];
    Pn[4 * r + 3] += dT[r];
  }
#pragma unroll
  for (int i = 0; i < 12; ++i) st->P[i] = Pn[i];
  st->t = t;
  st->t_prev = t;
  st->have_t_prev = 1;
  const int k = st->iter;
  st->iter = k + 1;
  const bool conv = (st->ell == cfg->ell_floor) &&
                    (fabs(t) * nxi < cfg->eps_pose || nxi < cfg->eps_grad);
  if (conv || st->iter >= cfg->max_iters) {
    st->done = 1;
    st->converged = conv ? 1 : 0;
  } else {
    load_iteration(cfg, st, cfg->iters[st->iter]);
    set_pose_constants(cfg, st);
  }
  if (use_cond) cudaGraphSetConditional(cond, st->done ? 0u : 1u);
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

__global__ void init_kernel(const SolveCfg* __restrict__ cfg, SolveState* __restrict__ st,
                            cudaGraphConditionalHandle cond, int use_cond) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < 16; ++i) st->P[i] = st->P0[i];
  st->iter = 0;
  st->done = 0;
  st->converged = 0;
  st->fallback_steps = 0;
  st->no_ascent_steps = 0;
  st->have_t_prev = 0;
  st->status = 0;
  st->t = 0.0;
  st->t_prev = 0.0;
  st->nnz_total = 0;
  st->cand_total = 0;
  st->nnz_pass[0] = st->nnz_pass[1] = 0;
  st->cand_pass[0] = st->cand_pass[1] = 0;
  st->nnz_eval = st->cand_eval = 0;
  st->ticket[0] = st->ticket[1] = 0;
  if (cfg->max_iters <= 0) st->done = 1;
  load_iteration(cfg, st, cfg->iters[0]);
  set_pose_constants(cfg, st);
  if (use_cond) cudaGraphSetConditional(cond, st->done ? 0u : 1u);
}

// One warp per source cluster: transform its points, and list the target
// cell rows within the cutoff of its bounding box as (first index, offset)
// segments of the cell-sorted target.
__global__ void __launch_bounds__(kThreads)
plan_kernel(const SolveCfg* __restrict__ cfg, SolveState* __restrict__ st) {
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int level = st->level;
  const ClusterView cv = cfg->clusters[level];
  if (c >= cv.ncl) return;
  const GridView g = cfg->grids[level];
  const int p0 = cv.cstart[c];
  const int cs = cv.cstart[c + 1] - p0;
  const bool zv = lane < cs;
  float zx = 0.f, zy = 0.f, zz = 0.f;
  if (zv) {
    const float4 p = cfg->src.xyz[p0 + lane];
    zx = fmaf(st->R[0], p.x, fmaf(st->R[1], p.y, fmaf(st->R[2], p.z, st->T[0])));
    zy = fmaf(st->R[3], p.x, fmaf(st->R[4], p.y, fmaf(st->R[5], p.z, st->T[1])));
    zz = fmaf(st->R[6], p.x, fmaf(st->R[7], p.y, fmaf(st->R[8], p.z, st->T[2])));
    cfg->zt[p0 + lane] = make_float4(zx, zy, zz, 0.f);
  }
  float blo[3] = {zv ? zx : INFINITY, zv ? zy : INFINITY, zv ? zz : INFINITY};
  float bhi[3] = {zv ? zx : -INFINITY, zv ? zy : -INFINITY, zv ? zz : -INFINITY};
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      blo[a] = fminf(blo[a], __shfl_xor_sync(kFull, blo[a], off));
      bhi[a] = fmaxf(bhi[a], __shfl_xor_sync(kFull, bhi[a], off));
    }
  }
  const float rp = st->rprune;
  const float rp2 = rp * rp;
  const int cx0 = max(0, cell_floor(blo[0] - rp, g.ox, g.inv_h, g.nx));
  const int cx1 = min(g.nx - 1, cell_floor(bhi[0] + rp, g.ox, g.inv_h, g.nx));
  const int cy0 = max(0, cell_floor(blo[1] - rp, g.oy, g.inv_h, g.ny));
  const int cy1 = min(g.ny - 1, cell_floor(bhi[1] + rp, g.oy, g.inv_h, g.ny));
  const int cz0 = max(0, cell_floor(blo[2] - rp, g.oz, g.inv_h, g.nz));
  const int cz1 = min(g.nz - 1, cell_floor(bhi[2] + rp, g.oz, g.inv_h, g.nz));
  const int nyr = cy1 - cy0 + 1, nzr = cz1 - cz0 + 1;
  const int nrows = (cx0 <= cx1 && nyr > 0 && nzr > 0) ? nyr * nzr : 0;
  int* sxs = cfg->seg_xs + (size_t)c * kMaxSeg;
  int* spf = cfg->seg_pref + (size_t)c * kMaxSeg;
  const unsigned lt = (1u << lane) - 1u;
  int nseg = 0, total = 0;
  bool overflow = false;
  for (int rb = 0; rb < nrows; rb += 32) {
    const int r = rb + lane;
    int len = 0, xs = 0;
    if (r < nrows) {
      const int cy = cy0 + r % nyr, cz = cz0 + r / nyr;
      const float ylo = g.oy + cy * g.h, yhi = ylo + g.h;
      const float zlo = g.oz + cz * g.h, zhi = zlo + g.h;
      const float dy = fmaxf(0.f, fmaxf(ylo - bhi[1], blo[1] - yhi));
      const float dz = fmaxf(0.f, fmaxf(zlo - bhi[2], blo[2] - zhi));
      const float rem = rp2 - dy * dy - dz * dz;
      if (rem >= 0.f) {
        const float rx = sqrtf(rem);
        const int a0 = max(cx0, cell_floor(blo[0] - rx, g.ox, g.inv_h, g.nx));
        const int a1 = min(cx1, cell_floor(bhi[0] + rx, g.ox, g.inv_h, g.nx));
        if (a0 <= a1) {
          const int base = g.nx * (cy + g.ny * cz);
          xs = g.cell_start[base + a0];
          len = g.cell_start[base + a1 + 1] - xs;
        }
      }
    }
    const unsigned m = __ballot_sync(kFull, len > 0);
    const int idx = nseg + __popc(m & lt);
    const int keep = (len > 0 && idx < kMaxSeg) ? len : 0;
    if (len > 0 && idx >= kMaxSeg) overflow = true;
    int incl = keep;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(kFull, incl, off);
      if (lane >= off) incl += v;
    }
    if (keep > 0) {
      sxs[idx] = xs;
      spf[idx] = total + incl - keep;
    }
    nseg += __popc(m);
    total += __shfl_sync(kFull, incl, 31);
  }
  if (__any_sync(kFull, overflow) && lane == 0) atomicOr(&st->status, kStatusSegOverflow);
  if (lane == 0) {
    cfg->cl_nseg[c] = min(nseg, kMaxSeg);
    cfg->cl_cand[c] = total;
  }
}

// Exclusive prefix of 32-candidate chunks over the clusters, and the first
// cluster of every pair-pass warp (warp w owns chunks
// [floor(w TC / NW), floor((w + 1) TC / NW))).
__global__ void __launch_bounds__(1024)
chunk_scan_kernel(const SolveCfg* __restrict__ cfg, SolveState* __restrict__ st) {
  __shared__ int s_sum[1024];
  const int tid = threadIdx.x;
  const int ncl = cfg->clusters[st->level].ncl;
  const int per = (ncl + 1023) / 1024;
  const int b = min(ncl, tid * per), e = min(ncl, b + per);
  int local = 0;
  for (int c = b; c < e; ++c) local += (__ldcg(&cfg->cl_cand[c]) + 31) >> 5;
  s_sum[tid] = local;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int v = tid >= off ? s_sum[tid - off] : 0;
    __syncthreads();
    s_sum[tid] += v;
    __syncthreads();
  }
  const long long TC = s_sum[1023];
  const long long NW = cfg->nwarps;
  int run = s_sum[tid] - local;
  for (int c = b; c < e; ++c) {
    const int ch = (__ldcg(&cfg->cl_cand[c]) + 31) >> 5;
    cfg->chunk_pref[c] = run;
    if (ch > 0) {
      const long long g0 = ((long long)run * NW + TC - 1) / TC;
      const long long g1 = ((long long)(run + ch) * NW + TC - 1) / TC;
      for (long long w = g0; w < g1; ++w) cfg->warp_start[w] = c;
    }
    run += ch;
  }
  if (tid == 1023) cfg->chunk_pref[ncl] = (int)TC;
}

template <bool STEP, int DP, int MODE>
__global__ void __launch_bounds__(kThreads)
pair_pass_kernel(const SolveCfg* __restrict__ cfg, SolveState* __restrict__ st,
                 double* __restrict__ partials, cudaGraphConditionalHandle cond, int use_cond) {
  constexpr int NACC = STEP ? 5 : 7;
  constexpr int DPS = DP > 0 ? DP : 1;
  constexpr int NU = STEP ? 4 : 1;
  __shared__ float4 s_z[kWarps][kClusterMax];
  __shared__ float s_zf[kWarps][DPS][kClusterMax];
  __shared__ float4 s_u[kWarps][NU][kClusterMax];
  __shared__ int s_xs[kWarps][kMaxSeg];
  __shared__ int s_pf[kWarps][kMaxSeg + 1];
  __shared__ float s_red[kWarps][NACC];
  __shared__ double s_fin[kWarps][NACC];
  __shared__ int s_last;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long gw = (long long)blockIdx.x * kWarps + warp;
  const int level = st->level;
  const GridView g = cfg->grids[level];
  const ClusterView cv = cfg->clusters[level];
  const float rc2 = st->rc2, A = st->A;
  float om[3] = {0.f, 0.f, 0.f}, vc[3] = {0.f, 0.f, 0.f};
  float inv_l2 = 0.f;
  if (STEP) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      om[i] = st->om[i];
      vc[i] = st->vc[i];
    }
    inv_l2 = st->inv_l2f;
  }

  float acc[NACC];
#pragma unroll
  for (int i = 0; i < NACC; ++i) acc[i] = 0.f;
  unsigned int nnz = 0, cand = 0;

  const long long TC = __ldcg(&cfg->chunk_pref[cv.ncl]);
  const long long NW = cfg->nwarps;
  const int ch0 = (int)((gw * TC) / NW), ch1 = (int)(((gw + 1) * TC) / NW);
  int c = 0, loaded = -1, cs4 = 0, tc = 0, nseg = 0, cpref = 0, cnext = 0;
  if (ch0 < ch1) {
    c = __ldcg(&cfg->warp_start[gw]);
    cpref = __ldcg(&cfg->chunk_pref[c]);
    cnext = __ldcg(&cfg->chunk_pref[c + 1]);
  }
  for (int ch = ch0; ch < ch1; ++ch) {
    while (ch >= cnext) {
      ++c;
      cpref = cnext;
      cnext = __ldcg(&cfg->chunk_pref[c + 1]);
    }
    if (c != loaded) {
      // stage cluster c: its transformed points, features, step vectors, segments
      __syncwarp();   // every lane is done with the previous cluster
      const int p0 = cv.cstart[c];
      const int cs = cv.cstart[c + 1] - p0;
      const bool zv = lane < cs;
      float4 z = make_float4(kFar, kFar, kFar, 0.f);
      if (zv) z = __ldcg(&cfg->zt[p0 + lane]);
      s_z[warp][lane] = z;
#pragma unroll
      for (int d = 0; d < DP; ++d) s_zf[warp][d][lane] = zv ? cfg->src.feat[d * cfg->src.m_pad + p0 + lane] : 0.f;
      if (STEP) {
        const float zt[3] = {zv ? z.x : 0.f, zv ? z.y : 0.f, zv ? z.z : 0.f};
        float u1[3], u2[3], u3[3], u4[3];
        u1[0] = om[1] * zt[2] - om[2] * zt[1] + vc[0];
        u1[1] = om[2] * zt[0] - om[0] * zt[2] + vc[1];
        u1[2] = om[0] * zt[1] - om[1] * zt[0] + vc[2];
        u2[0] = om[1] * u1[2] - om[2] * u1[1];
        u2[1] = om[2] * u1[0] - om[0] * u1[2];
        u2[2] = om[0] * u1[1] - om[1] * u1[0];
        u3[0] = om[1] * u2[2] - om[2] * u2[1];
        u3[1] = om[2] * u2[0] - om[0] * u2[2];
        u3[2] = om[0] * u2[1] - om[1] * u2[0];
        u4[0] = om[1] * u3[2] - om[2] * u3[1];
        u4[1] = om[2] * u3[0] - om[0] * u3[2];
        u4[2] = om[0] * u3[1] - om[1] * u3[0];
        const float u11 = u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2];
        const float u12 = u1[0] * u2[0] + u1[1] * u2[1] + u1[2] * u2[2];
        const float u13 = u1[0] * u3[0] + u1[1] * u3[1] + u1[2] * u3[2];
        const float u22 = u2[0] * u2[0] + u2[1] * u2[1] + u2[2] * u2[2];
        // beta = e.U1; gamma = e.U2 - k2; delta = e.U3 - k3; eps = e.U4 - k4
        const float c1 = inv_l2, c2 = 0.5f * inv_l2, c3 = inv_l2 * (1.0f / 6.0f),
                    c4 = inv_l2 * (1.0f / 24.0f);
        s_u[warp][0][lane] = make_float4(u1[0] * c1, u1[1] * c1, u1[2] * c1, 0.5f * u11 * inv_l2);
        s_u[warp][1 % NU][lane] = make_float4(u2[0] * c2, u2[1] * c2, u2[2] * c2, 0.5f * u12 * inv_l2);
        s_u[warp][2 % NU][lane] = make_float4(u3[0] * c3, u3[1] * c3, u3[2] * c3,
                                              (u13 * (1.0f / 6.0f) + u22 * 0.125f) * inv_l2);
        s_u[warp][3 % NU][lane] = make_float4(u4[0] * c4, u4[1] * c4, u4[2] * c4, 0.f);
      }
      nseg = __ldcg(&cfg->cl_nseg[c]);
      tc = __ldcg(&cfg->cl_cand[c]);
      for (int i = lane; i < nseg; i += 32) {
        s_xs[warp][i] = __ldcg(&cfg->seg_xs[(size_t)c * kMaxSeg + i]);
        s_pf[warp][i] = __ldcg(&cfg->seg_pref[(size_t)c * kMaxSeg + i]);
      }
      if (lane == 0) s_pf[warp][nseg] = tc;
      cs4 = (cs + 3) & ~3;
      loaded = c;
      __syncwarp();
    }
    // this lane's candidate
    const int q = (ch - cpref) * 32 + lane;
    float4 xp = make_float4(-kFar, -kFar, -kFar, 0.f);
    float xf[DPS];
#pragma unroll
    for (int d = 0; d < DPS; ++d) xf[d] = 0.f;
    if (q < tc) {
      int lo = 0, hi = nseg;  // s_pf[lo] <= q < s_pf[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_pf[warp][mid] <= q) lo = mid;
        else hi = mid;
      }
      const int xi = s_xs[warp][lo] + (q - s_pf[warp][lo]);
      xp = g.xyz[xi];
#pragma unroll
      for (int d = 0; d < DP; ++d) xf[d] = g.feat[d * g.n_pad + xi];
      cand += (unsigned)(cv.cstart[c + 1] - cv.cstart[c]);
    }
    float W = 0.f, Ex = 0.f, Ey = 0.f, Ez = 0.f;
    for (int j0 = 0; j0 < cs4; j0 += 4) {
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int j = j0 + jj;
        const float4 z = s_z[warp][j];
        const float ex = xp.x - z.x, ey = xp.y - z.y, ez = xp.z - z.z;
        const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
        if (d2 <= rc2) {
          float w;
          if (MODE == kColorKernel) {
            float qf = 0.f;
#pragma unroll
            for (int d = 0; d < DP; ++d) {
              const float df = xf[d] - s_zf[warp][d][j];
              qf = fmaf(df, df, qf);
            }
            w = ex2_approx(-fmaf(A, d2, qf));
          } else if (MODE == kColorDot) {
            float cdot = 0.f;
#pragma unroll
            for (int d = 0; d < DP; ++d) cdot = fmaf(xf[d], s_zf[warp][d][j], cdot);
            w = ex2_approx(-A * d2) * cdot;
          } else {
            w = ex2_approx(-A * d2);
          }
          ++nnz;
          if (!STEP) {
            W += w;
            Ex = fmaf(w, ex, Ex);
            Ey = fmaf(w, ey, Ey);
            Ez = fmaf(w, ez, Ez);
          } else {
            const float4 U1 = s_u[warp][0][j], U2 = s_u[warp][1 % NU][j];
            const float4 U3 = s_u[warp][2 % NU][j], U4 = s_u[warp][3 % NU][j];
            const float beta = fmaf(ex, U1.x, fmaf(ey, U1.y, ez * U1.z));
            const float gam = fmaf(ex, U2.x, fmaf(ey, U2.y, fmaf(ez, U2.z, -U1.w)));
            const float del = fmaf(ex, U3.x, fmaf(ey, U3.y, fmaf(ez, U3.z, -U2.w)));
            const float eps = fmaf(ex, U4.x, fmaf(ey, U4.y, fmaf(ez, U4.z, -U3.w)));
            const float b2 = beta * beta;
            const float g2 = fmaf(0.5f, b2, gam);
            const float g3 = fmaf(beta, fmaf(b2, 1.0f / 6.0f, gam), del);
            const float g4 = fmaf(b2 * b2, 1.0f / 24.0f,
                                  fmaf(0.5f * gam, b2 + gam, fmaf(beta, del, eps)));
            acc[0] += w;
            acc[1] = fmaf(w, beta, acc[1]);
            acc[2] = fmaf(w, g2, acc[2]);
            acc[3] = fmaf(w, g3, acc[3]);
            acc[4] = fmaf(w, g4, acc[4]);
          }
        }
      }
    }
    if (!STEP) {
      // x' fixed per lane: sum_j w (z~'_j x e_ij) = x' x E_i
      acc[0] += W;
      acc[1] += xp.y * Ez - xp.z * Ey;
      acc[2] += xp.z * Ex - xp.x * Ez;
      acc[3] += xp.x * Ey - xp.y * Ex;
      acc[4] += Ex;
      acc[5] += Ey;
      acc[6] += Ez;
    }
  }

  // ---- block reduction in a fixed order ----
#pragma unroll
  for (int i = 0; i < NACC; ++i) {
    const float v = warp_sum_f(acc[i]);
    if (lane == 0) s_red[warp][i] = v;
  }
  unsigned long long wn = nnz, wc = cand;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    wn += __shfl_down_sync(kFull, wn, off);
    wc += __shfl_down_sync(kFull, wc, off);
  }
  if (lane == 0 && (wn | wc)) {
    atomicAdd(&st->nnz_pass[STEP ? 1 : 0], wn);
    atomicAdd(&st->cand_pass[STEP ? 1 : 0], wc);
  }
  __syncthreads();
  if (warp == 0) {
    if (lane < NACC) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) s += (double)s_red[w][lane];
      partials[(size_t)blockIdx.x * kPartialStride + lane] = s;
      __threadfence();
    }
    __syncwarp();
    if (lane == 0) {
      const unsigned t = atomicAdd(&st->ticket[STEP ? 1 : 0], 1u);
      s_last = (t == gridDim.x - 1) ? 1 : 0;
    }
  }
  __syncthreads();
  if (!s_last) return;

  // ---- last block: fixed-order FP64 reduction of all block partials ----
  __threadfence();
  double fin[NACC];
#pragma unroll
  for (int i = 0; i < NACC; ++i) fin[i] = 0.0;
  for (int b = tid; b < (int)gridDim.x; b += kThreads) {
#pragma unroll
    for (int i = 0; i < NACC; ++i) fin[i] += __ldcg(&partials[(size_t)b * kPartialStride + i]);
  }
#pragma unroll
  for (int i = 0; i < NACC; ++i) {
    const double v = warp_sum_d(fin[i]);
    if (lane == 0) s_fin[warp][i] = v;
  }
  __syncthreads();
  if (warp == 0) {
    if (lane < NACC) {
      double s = 0.0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) s += s_fin[w][lane];
      s_fin[0][lane] = s;
    }
    __syncwarp();
    if (lane == 0) {
      double sums[NACC];
#pragma unroll
      for (int i = 0; i < NACC; ++i) sums[i] = s_fin[0][i];
      st->ticket[STEP ? 1 : 0] = 0;
      if (!STEP) {
        finish_gradient(cfg, st, sums);
      } else {
        finish_step(cfg, st, sums, cond, use_cond);
        st->nnz_pass[0] = st->nnz_pass[1] = 0;
        st->cand_pass[0] = st->cand_pass[1] = 0;
      }
    }
  }
}

template <bool STEP>
cudaError_t launch_dispatch(int dp, int color_mode, int nblocks, const SolveCfg* cfg,
                            SolveState* st, double* partials, cudaGraphConditionalHandle cond,
                            int use_cond, cudaStream_t s) {
  dim3 grid(nblocks), block(kThreads);
  if (color_mode == kColorNone || dp == 0) {
    pair_pass_kernel<STEP, 0, kColorNone><<<grid, block, 0, s>>>(cfg, st, partials, cond, use_cond);
  } else if (color_mode == kColorKernel) {
    if (dp == 3) pair_pass_kernel<STEP, 3, kColorKernel><<<grid, block, 0, s>>>(cfg, st, partials, cond, use_cond);
    else if (dp == 5) pair_pass_kernel<STEP, 5, kColorKernel><<<grid, block, 0, s>>>(cfg, st, partials, cond, use_cond);
    else pair_pass_kernel<STEP, 8, kColorKernel><<<grid, block, 0, s>>>(cfg, st, partials, cond, use_cond);
  } else {
    if (dp == 3) pair_pass_kernel<STEP, 3, kColorDot><<<grid, block, 0, s>>>(cfg, st, partials, cond, use_cond);
    else if (dp == 5) pair_pass_kernel<STEP, 5, kColorDot><<<grid, block, 0, s>>>(cfg, st, partials, cond, use_cond);
    else pair_pass_kernel<STEP, 8, kColorDot><<<grid, block, 0, s>>>(cfg, st, partials, cond, use_cond);
  }
  return cudaGetLastError();
}

// Sleeps about ns nanoseconds (bounded; used only to line up profiling events).
__global__ void delay_kernel(unsigned ns) {
  for (unsigned waited = 0; waited < ns; waited += 1000) __nanosleep(1000);
}

}  // namespace

cudaError_t launch_delay(unsigned ns, cudaStream_t s) {
  delay_kernel<<<1, 1, 0, s>>>(ns);
  return cudaGetLastError();
}

cudaError_t launch_init(const SolveCfg* cfg, SolveState* st, cudaGraphConditionalHandle cond,
                        int use_cond, cudaStream_t s) {
  init_kernel<<<1, 32, 0, s>>>(cfg, st, cond, use_cond);
  return cudaGetLastError();
}

cudaError_t launch_plan(const SolveCfg* cfg, SolveState* st, int ncl_launch, cudaStream_t s) {
  const int blocks = (ncl_launch + kWarps - 1) / kWarps;
  plan_kernel<<<blocks > 0 ? blocks : 1, kThreads, 0, s>>>(cfg, st);
  chunk_scan_kernel<<<1, 1024, 0, s>>>(cfg, st);
  return cudaGetLastError();
}

cudaError_t launch_pair_pass(bool step, int dp, int color_mode, int nblocks, const SolveCfg* cfg,
                             SolveState* st, double* partials, cudaGraphConditionalHandle cond,
                             int use_cond, cudaStream_t s) {
  if (step) return launch_dispatch<true>(dp, color_mode, nblocks, cfg, st, partials, cond, use_cond, s);
  return launch_dispatch<false>(dp, color_mode, nblocks, cfg, st, partials, cond, use_cond, s);
}

}  // namespace cvo
