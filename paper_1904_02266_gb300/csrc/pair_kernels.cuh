// The CVO hot path on sm_103a: the cutoff-truncated all-pairs kernel
// reductions behind each gradient-ascent iteration, plus the FP64 tail, all in
// one persistent cooperative kernel per solve.
//
//  gradient pass  F = sum c_ij k(x_i, z~_j)                         (Eq. scalar)
//                 dF/domega = (1/ell^2) sum w_ij (z~_j x e_ij)      (Eq. 3_gradient,
//                 dF/dv     = (1/ell^2) sum w_ij e_ij                left-update signs)
//  step pass      S0..S4 = sum w_ij g^m_ij along xi                  (Eq. fourth)
//  tail (FP64)    xi = metric gradient (Eq. metric), t* = first maximiser of the
//                 quartic, P <- exp(t* xi) P (Eqs. newstep, step), lengthscale
//                 schedule and the Table 1 convergence test.
//
// One iteration (every block runs the same sequence; phases are separated by
// a grid barrier whose spin is bounded):
//  plan        (only when needed) one warp per source cluster (an octree node
//              of the source, at most 32 points): transform, bounding box, the
//              rows of target cells within the plan radius, stored as segments
//              of the cell-sorted target, and (clusters with at most
//              kFilterMax candidates) the count of candidates within the plan
//              radius of the box, per segment.                         barrier
//              work totals of groups of 32 clusters.                    barrier
//              every block scans the group totals and places its own warps on
//              an even split of the work, cut at groups of four source points
//              (no further barrier).
//  gradient    each warp walks its share of chunks of 32 filtered candidates:
//  pass        one lane per candidate target point against the cluster's
//              source points staged in shared memory (broadcast reads). FP32
//              pairs, one ex2.approx per kept pair, per-lane FP32 sums,
//              fixed-order reductions.                                 barrier
//  tail        every block reduces all block partials (value-major) in FP64
//              in the same fixed order and runs the same FP64 tail, so
//              nothing is published or broadcast.
//  step pass   as above along the unit direction.                      barrier
//  tail        step length, exponential-map update, next iteration.
// The plan is reused while it still covers the cutoff: it is built with a
// radius 10% wider than the cutoff and rebuilt when the grid level changes,
// when the pose has drifted by more than that margin (an FP64 bound over the
// whole source cloud), or when it has become much wider than needed. A warp
// whose share of a reused plan fits its cache slots also lists, once per
// plan, the (candidate, source point) pairs of each cached cluster within the
// plan radius, and its passes evaluate the lists instead of whole chunks.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "cvo_internal.cuh"

// Resident blocks per SM the solve kernel is compiled for (register budget).
#ifndef CVO_SOLVE_MIN_BLOCKS
#define CVO_SOLVE_MIN_BLOCKS 1
#endif

namespace cvo {

namespace {

constexpr float kFar = 1.0e18f;   // coordinate of padding points: never within any cutoff
constexpr unsigned kFull = 0xffffffffu;
constexpr double kSkin = 0.10;              // plan radius margin (fraction of the cutoff)
constexpr double kLoose = 1.25;             // replan when the plan radius exceeds this factor
constexpr int kFilterMax = 1024;            // candidates of a cluster the plan filters at most
constexpr int kActChunks = 32;              // chunks per cluster whose source-group activity is kept
// teams of at most this many blocks box-test the candidates of unfiltered
// clusters in the streamed passes (their warps' shares are long runs of
// chunks); larger teams, whose shares are short and whose work split counts
// unfiltered candidates, stream them unfiltered
constexpr int kCompactTeamMax = 32;
#ifndef CVO_COST_ACTIVE
#define CVO_COST_ACTIVE 12
#endif
// work model: the pair bodies of a source group that kept a pair, in pair-test units
constexpr int kCostActive = CVO_COST_ACTIVE;

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// One feature value: FP32 planes, or BF16 planes widened to FP32 (FB).
template <bool FB>
__device__ __forceinline__ float load_feat(const float* planes, size_t idx) {
  if constexpr (FB) {
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(planes)[idx]);
  } else {
    return planes[idx];
  }
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
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
// per-block iteration state (identical in every block of a team)
// ---------------------------------------------------------------------------

// The blocks that solve one pair together: the whole grid for a single
// solve, a contiguous run of claimed slots for a queued one.
struct Team {
  int rank, size;
};

// Scalars of the solve configuration that the FP64 tail reads every
// iteration, copied once per solve so that the tail issues no dependent
// global loads.
struct TailConst {
  double cX[3], cZ[3];
  double sigma2, inv_a2, inv_b2;
  double ell_floor, eps_pose, eps_grad, src_radius;
  int mode, step_order, max_iters;
  int reduce_fp32;   // precision study: block and cross-block sums in FP32
  unsigned wait_polls;                 // barrier polls before a block gives up
  unsigned long long join_limit_ns;    // longest wait of a queued team's join
  float cXf[3], inv_a2f, inv_b2f, src_radius_f;   // FP32 copies for the FP32 parts of the tail
};

struct BlockCtx {
  TailConst tc;
  double P[16];           // current pose
  double Rp[9], Tp[3];    // centred pose at the last plan
  double xi[6];           // metric gradient (Eq. metric)
  double x0[6];           // its components before the metric factors (FP64 pair sums, centring
                          // back-map applied)
  double u64[6];          // xi / |xi|
  double xi_norm, xi_inv, F;
  double S[5];            // S0..S4 of the last step pass (formed when published)
  double s_raw[5];        // the step pass's sums along xi / |xi| (S_m = s_m sigma^2 |xi|^m)
  double kf_rot, kf_tr;   // this iteration's metric factors
  int small_grad;         // |xi| below the gradient threshold (or zero): no step, stop test
  int at_floor;           // this iteration's ell is the schedule's floor
  int fin;                // step pass: warps done with their share (the first does the FP64
                          // gradient)
  double t, t_prev;
  double ell, inv_l2, r_plan, plan_ell;
  int k, level, plan_level, plan_filter;
  int need_plan, done, converged, fallback, no_ascent, have_t_prev;
  int use_kept, collect_kept, rebalance;   // kept-pair weighting of the work split
  int use_act;                             // the split weighs source groups by their activity
  int compact;                             // streamed passes box-test unfiltered clusters
  int team_rank, team_size;                // this block's place in its team (read after a pass
                                           // from shared memory rather than kept in registers)
  unsigned long long nnz_total, cand_total, nnz_grad, cand_grad;
  float R[9], T[3];       // FP32 centred pose: z~' = R z' + T
  float om[3], vc[3];     // unit step direction (centred frame)
  float A, rc2, rplan_f, inv_l2f;
  // warp ranges: from group g0 of chunk j0 of cluster c0 up to (not
  // including) group g1 of chunk j1 of cluster c1
  int w_c0[kWarps], w_j0[kWarps], w_g0[kWarps], w_c1[kWarps], w_j1[kWarps], w_g1[kWarps];
  double dR[9], V[9];     // tail scratch: exp map rotation and its V matrix
};

// ---- the FP64 tail, one warp wide -----------------------------------------
// On GB300 a warp's FP64 instruction holds the FP64 pipe about as long as a
// full warp's (about 64 cycles) whatever the number of active lanes, so the
// tail costs what its count of FP64 instructions costs. It runs on warp 0 of
// every block with independent components on separate lanes (the 3 x 4 pose
// product is three instructions, not thirty-six); scalar steps run on every
// lane at the cost of one. Lanes exchange values by shuffles, or through the
// block context (shared memory) between __syncwarp()s.

__device__ __forceinline__ double flip_sign(double v, bool neg) {
  return __longlong_as_double(__double_as_longlong(v) ^
                              (neg ? (long long)0x8000000000000000ull : 0ll));
}

// Conversions and power-of-two scalings by integer operations on the bit
// patterns. On GB300 every FP64 warp instruction (conversions and compares
// included) holds the FP64 pipe for about 64 cycles, so the tails keep their
// FP64 instruction count low and leave the rest to the integer and FP32 pipes.

// x 2^shift truncated to FP32 (toward zero); magnitudes below FP32's normal
// range give a signed zero, above it a signed infinity, a NaN stays a NaN.
__device__ __forceinline__ float f64_to_f32_shift(double x, int shift) {
  const int hi = __double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const int e = (hi >> 20) & 0x7ff;
  const unsigned sign = (unsigned)hi & 0x80000000u;
  const unsigned m = ((unsigned)(hi & 0xfffff) << 3) | (lo >> 29);
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (m != 0u || lo != 0u ? 0x400000u : 0u));
  const int e32 = e - 1023 + 127 + shift;
  if (e == 0 || e32 <= 0) return __uint_as_float(sign);
  if (e32 >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned)e32 << 23) | m);
}

__device__ __forceinline__ float f64_to_f32(double x) { return f64_to_f32_shift(x, 0); }

// The exact FP64 value of an FP32 number (FP32 subnormals as zero).
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned sign = u & 0x80000000u;
  if (e == 0u) return __hiloint2double((int)sign, 0);
  const unsigned e64 = e == 0xffu ? 0x7ffu : e - 127u + 1023u;
  return __hiloint2double((int)(sign | (e64 << 20) | ((u & 0x7fffffu) >> 3)), (int)((u & 7u) << 29));
}

// x 2^k for k in [0, 8]: an exponent increment when x is normal and stays so.
__device__ __forceinline__ double mul_pow2(double x, int k) {
  const int hi = __double2hiint(x);
  const int e = (hi >> 20) & 0x7ff;
  if (e > 0 && e + k < 0x7ff) return __hiloint2double(hi + (k << 20), __double2loint(x));
  return x * (double)(1 << k);
}

// x > 0 (false for zero, negative values and NaN), from the bit pattern.
__device__ __forceinline__ bool is_pos(double x) {
  const int hi = __double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  if (hi < 0) return false;
  if (((hi >> 20) & 0x7ff) == 0x7ff && ((hi & 0xfffff) != 0 || lo != 0u)) return false;
  return hi != 0 || lo != 0u;
}

// Iteration k's constants (ic = the host table's entry k), the FP32 pose, and
// whether the traversal plan must be rebuilt. Warp 0, every lane.
__device__ __noinline__ void begin_iteration(const IterConst& ic, BlockCtx& b, int lane) {
  // centred pose [R T'] on lanes 0..11, element (r, c) = (l / 4, l % 4):
  // R = the pose's rotation, T' = R cZ + T - cX
  const int l = min(lane, 11), r = l >> 2, c = l & 3;
  const double t3 = fma(b.P[4 * r + 2], b.tc.cZ[2],
                        fma(b.P[4 * r + 1], b.tc.cZ[1],
                            fma(b.P[4 * r], b.tc.cZ[0], b.P[4 * r + 3] - b.tc.cX[r])));
  const double v = c == 3 ? t3 : b.P[4 * r + c];
  // is the current plan still a superset of the pairs within the cutoff?
  const float need = ic.rprune;   // 1.001 r_c
  // reuse only at an unchanged lengthscale (the floor of the schedule): while
  // ell shrinks a fresh, tighter plan costs less than the extra candidates
  bool replan = b.need_plan || ic.level != b.plan_level ||
                __double_as_longlong(ic.ell) != __double_as_longlong(b.plan_ell);
  if (!replan) {
    // the differences in FP64, the rest in FP32: the 2e-5 relative and
    // 1e-6 r_c margins below cover its rounding
    const float d = f64_to_f32(v - (c == 3 ? b.Tp[r] : b.Rp[3 * r + c]));
    const float sq = lane < 12 ? d * d : 0.0f;
    float sr = c < 3 ? sq : 0.0f, st = c == 3 ? sq : 0.0f;
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) {
      sr += __shfl_xor_sync(kFull, sr, off);
      st += __shfl_xor_sync(kFull, st, off);
    }
    sr = __shfl_sync(kFull, sr, 0);
    st = __shfl_sync(kFull, st, 0);
    // |dR z + dT| <= |dR|_F |z| + |dT| for every source point, |z| <= r_src
    const float drift = fmaf(sqrtf(sr), b.tc.src_radius_f, sqrtf(st)) * (1.0f + 2e-5f) + 1e-6f * need;
    const float rp = b.rplan_f;
    replan = (need + drift > rp) || (rp > (float)kLoose * (need + drift));
  }
  __syncwarp();   // every lane has read the old plan pose
  if (lane < 12) {
    // rounded to nearest: the passes' pose
    if (c < 3) b.R[3 * r + c] = __double2float_rn(v);
    else b.T[r] = __double2float_rn(v);
    if (replan) {
      if (c < 3) b.Rp[3 * r + c] = v;
      else b.Tp[r] = v;
    }
  }
  if (lane == 0) {
    b.ell = ic.ell;
    b.inv_l2 = ic.inv_l2;
    b.A = ic.A;
    b.rc2 = ic.rc2;
    b.inv_l2f = (float)ic.inv_l2;
    b.level = ic.level;
    b.kf_rot = ic.kf_rot;
    b.kf_tr = ic.kf_tr;
    b.at_floor = ic.at_floor;
    if (replan) {
      b.need_plan = 1;
      b.plan_level = ic.level;
      b.plan_ell = ic.ell;
      b.plan_filter = ic.filter;
      // the radius is FP32 throughout: (float)(need (1 + skin)) is what the
      // plan and the passes use. A plan used for one iteration sees only
      // that iteration's pose (the pose moves at its end and the next
      // iteration re-plans at a new lengthscale), so it needs no skin
      b.r_plan = (double)need * (ic.filter ? 1.0 + kSkin : 1.0);
      b.rplan_f = (float)b.r_plan;
    }
  }
  __syncwarp();
}

// FP64 reciprocal from the FP32 one and a Newton step r <- r (2 - x r) (which
// squares the relative error: 1e-7 -> 1e-14). Finite, nonzero x within FP32
// range.
__device__ __forceinline__ double recip_refined(double x) {
  double r = (double)(1.0f / (float)x);
  r = r * fma(-x, r, 2.0);
  return r;
}

// FP64 reciprocal and square root of any finite x != 0 (x > 0): the
// refined FP32 forms inside FP32's range, the FP64 operations outside it.
__device__ __forceinline__ double rcp64(double x) {
  const double ax = fabs(x);
  return (ax > 1e-30 && ax < 1e30) ? recip_refined(x) : 1.0 / x;
}

__device__ __forceinline__ double sqrt64(double x) {
  if (!(x > 1e-30 && x < 1e30)) return sqrt(x);
  // y ~ 1/sqrt(x) from FP32, two FP64 Newton steps y <- y (1.5 - 0.5 x y^2)
  double y = (double)rsqrtf((float)x);
  y = y * fma(-0.5 * x, y * y, 1.5);
  y = y * fma(-0.5 * x, y * y, 1.5);
  return x * y;
}

// Smallest positive t at which G'(t) = c0 + c1 t + c2 t^2 + c3 t^3 changes sign
// from + to - (the first local maximum of the quartic model, Sec. 4 "Step
// size"), given c0 = S1 > 0. The coefficients are first scaled by a power of
// two (exact) so that the largest has magnitude in [0.5, 1). The critical
// points of G' (the real roots of G'' = c1 + 2 c2 t + 3 c3 t^2) cut t > 0 into
// pieces on which G' is monotone; the first piece whose right end has G' < 0
// (for the last piece, the sign of the leading coefficient) holds the answer,
// which a Newton iteration kept inside the shrinking bracket finds in FP64.
// Its start is the root of the closed-form cubic evaluated in FP32 (cbrt /
// acos / cos, no FP64 transcendentals), or the bracket's midpoint: a close
// start takes two steps; a far one (the FP32 form loses the small roots of a
// cubic whose roots differ by orders of magnitude) a few more.
__device__ bool first_maximiser(double c0, double c1, double c2, double c3, double* t_out) {
  // the largest exponent field among the coefficients (integer work: FP64
  // instructions are the scarce resource here)
  const int e_max = max(max((__double2hiint(c0) >> 20) & 0x7ff, (__double2hiint(c1) >> 20) & 0x7ff),
                        max((__double2hiint(c2) >> 20) & 0x7ff, (__double2hiint(c3) >> 20) & 0x7ff));
  if (e_max == 0x7ff) return false;   // an infinity or a NaN
  // start: a root of the cubic from the closed form, all in FP32 on the
  // coefficients scaled by 2^(1022 - e_max) (the largest has magnitude in
  // [0.5, 1); formed from the bit patterns, truncated: a start needs no
  // more), refined by two FP32 Newton steps; a negligible cubic term is left
  // out of the start only
  const int shift = 1022 - e_max;
  const float f0 = f64_to_f32_shift(c0, shift), f1 = f64_to_f32_shift(c1, shift);
  const float f2 = f64_to_f32_shift(c2, shift), f3 = f64_to_f32_shift(c3, shift);
  float ts = -1.0f;
  if (fabsf(f3) <= 1e-12f) {
    if (fabsf(f2) <= 1e-12f) {
      if (f1 < 0.0f) ts = -f0 / f1;
    } else {
      const float disc = fmaf(f1, f1, -4.0f * f2 * f0);
      if (disc >= 0.0f) {
        const float qf = -0.5f * (f1 + copysignf(sqrtf(disc), f1));
        const float ra = qf / f2, rb = f0 / qf;
        ts = (f2 < 0.0f) ? fmaxf(ra, rb) : fminf(ra, rb);
      }
    }
  } else {
    const float r3 = 1.0f / f3;
    const float B = f2 * r3, C = f1 * r3, D = f0 * r3;
    const float B3 = B * (1.0f / 3.0f);
    const float p = fmaf(-B, B3, C);
    const float q = fmaf((2.0f / 27.0f) * B * B, B, fmaf(-B3, C, D));
    const float disc = fmaf(0.25f * q, q, (1.0f / 27.0f) * p * p * p);
    if (disc > 0.0f) {
      const float u = -copysignf(cbrtf(0.5f * fabsf(q) + sqrtf(disc)), q);
      ts = (u != 0.0f ? u - p / (3.0f * u) : 0.0f) - B3;
    } else if (p < 0.0f) {
      // roots m cos(phi - 2 pi k / 3) - B/3: k = 0 largest, k = 1 middle, k = 2 smallest
      const float m = 2.0f * sqrtf(-p * (1.0f / 3.0f));
      const float arg = fminf(1.0f, fmaxf(-1.0f, 3.0f * q / (p * m)));
      const float phi = acosf(arg) * (1.0f / 3.0f);
      const float two_pi_3 = 2.09439510239319549f;
      // the hardware cosine is accurate enough for a start
      const float rk[3] = {m * __cosf(phi) - B3, m * __cosf(phi - two_pi_3) - B3,
                           m * __cosf(phi - 2.0f * two_pi_3) - B3};
      // the smallest positive one that G' crosses from + to - (as far as FP32 tells)
      for (int k = 0; k < 3; ++k) {
        const float tk = rk[k];
        if (tk > 0.0f && fmaf(fmaf(3.0f * f3, tk, 2.0f * f2), tk, f1) < 0.0f && (ts < 0.0f || tk < ts))
          ts = tk;
      }
    }
  }
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const float ff = fmaf(fmaf(fmaf(f3, ts, f2), ts, f1), ts, f0);
    const float fd = fmaf(fmaf(3.0f * f3, ts, 2.0f * f2), ts, f1);
    const float tn = ts - ff / fd;
    if (fd < 0.0f && tn > 0.0f && isfinite(tn)) ts = tn;
  }
  const double t32 = f32_to_f64(ts);
  // fast path: one FP64 Newton step from that start on the unscaled
  // coefficients (the roots do not depend on a common scale), accepted when it
  // moves t by at most 2^-20 t (the step squares the start's error) and
  // G'' < 0 on [0, t] (then G' falls from c0 > 0 over [0, t], so t is its
  // first root and a + -> - crossing). G''(0) = c1 < 0 is read from the sign
  // bit; G''(t) < 0 and the vertex test of a concave G'' are evaluated in FP32
  // on the scaled coefficients with a 1e-4 relative margin (their rounding is
  // below 1e-6), and anything within the margin goes to the bracketed search.
  if (e_max >= 2 && ts > 0.0f && isfinite(ts) && __double2hiint(c1) < 0) {
    const double f = fma(fma(fma(c3, t32, c2), t32, c1), t32, c0);
    const double fp = fma(fma(3.0 * c3, t32, mul_pow2(c2, 1)), t32, c1);
    const int hfp = __double2hiint(fp), efp = (hfp >> 20) & 0x7ff;
    if (hfp < 0 && efp > 1023 - 120 && efp < 1023 + 120) {
      // 1/fp from FP32 and one FP64 Newton step
      double r = f32_to_f64(1.0f / f64_to_f32(fp));
      r = r * fma(-fp, r, 2.0);
      const double dt = -f * r;
      const double t = t32 + dt;
      const int ht = __double2hiint(t), hd = __double2hiint(dt);
      const int et = (ht >> 20) & 0x7ff, ed = (hd >> 20) & 0x7ff;
      const bool settled = ed <= et - 21;   // |dt| < 2^-20 t (dt = 0 has ed = 0)
      const float g2 = fmaf(fmaf(3.0f * f3, ts, 2.0f * f2), ts, f1);
      const float gmag = fabsf(f1) + fabsf(2.0f * f2 * ts) + fabsf(3.0f * f3 * ts * ts);
      const bool inside = f3 < 0.0f && f2 > 0.0f && f2 < -3.0f * f3 * ts * (1.0f + 1e-4f);
      const bool vertex_ok = !inside || 3.0f * f1 * f3 > f2 * f2 * (1.0f + 1e-4f);
      if (ht > 0 && et < 0x7ff && settled && g2 < -1e-4f * gmag && vertex_ok) {
        *t_out = t;
        return true;
      }
    }
  }
  // the bracketed search, on the coefficients scaled by a power of two
  double sc;
  if (e_max >= 2 && e_max <= 2044) {
    // 2^(1022 - e_max): the largest magnitude lands in [0.5, 1)
    sc = __hiloint2double((2045 - e_max) << 20, 0);
  } else {
    const double s = fmax(fmax(fabs(c0), fabs(c1)), fmax(fabs(c2), fabs(c3)));
    if (!(s > 0.0)) return false;
    // 2^-e with s = m 2^e, m in [0.5, 1) (subnormal s are scaled twice)
    sc = 1.0;
    double ss = s;
    if (ss < 0x1p-1000) {
      sc = 0x1p+1000;
      ss *= sc;
    }
    const int ex = min(1000, ((__double2hiint(ss) >> 20) & 0x7ff) - 1022);
    sc *= __hiloint2double((1023 - ex) << 20, 0);
  }
  c0 *= sc;
  c1 *= sc;
  c2 *= sc;
  c3 *= sc;
  if (fabs(c3) < 1e-30) c3 = 0.0;
  if (fabs(c2) < 1e-30) c2 = 0.0;
  // positive critical points of G', ascending
  double e0 = -1.0, e1 = -1.0;
  if (c3 != 0.0) {
    const double dd = fma(c2, c2, -3.0 * c1 * c3);   // discriminant of G'' over 4
    if (dd > 0.0) {
      const double qq = -(c2 + copysign(sqrt64(dd), c2));   // G'' roots: qq / (3 c3), c1 / qq
      double ra = qq * rcp64(3.0 * c3);
      double rb = qq != 0.0 ? c1 * rcp64(qq) : ra;
      if (ra > rb) {
        const double tmp = ra;
        ra = rb;
        rb = tmp;
      }
      if (ra > 0.0) {
        e0 = ra;
        if (rb > ra) e1 = rb;
      } else if (rb > 0.0) {
        e0 = rb;
      }
    }
  } else if (c2 != 0.0) {
    const double r = -c1 * rcp64(2.0 * c2);
    if (r > 0.0) e0 = r;
  }
  // the first monotone piece (lo, hi) on which G' falls below zero
  const double lead = c3 != 0.0 ? c3 : c2 != 0.0 ? c2 : c1;
  double lo = 0.0, hi = -1.0;   // hi < 0: unbounded
  bool found = false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (found) break;
    const double b = k == 0 ? e0 : k == 1 ? e1 : -1.0;
    if (k < 2 && !(b > lo)) continue;   // no such critical point
    const double fb = b > 0.0 ? fma(fma(fma(c3, b, c2), b, c1), b, c0) : lead;
    if (fb < 0.0) {
      hi = b;
      found = true;
    } else if (b > 0.0) {
      lo = b;   // G' >= 0 at the end of this piece: no crossing in it
    } else {
      break;    // the last piece stays positive: no maximiser
    }
  }
  if (!found) return false;
  // Newton on G' inside [lo, hi] (G' > 0 at lo, < 0 at hi), bisection or
  // doubling when a step leaves the bracket; bounded. Start: the closed-form
  // root if it lies in the bracket, else the smallest point where a falling
  // term balances c0, (c0 / |c_k|)^(1/k), else the bracket's middle.
  const auto inside = [&](double x) { return isfinite(x) && x > lo && (hi < 0.0 || x < hi); };
  double t = t32;
  if (!inside(t)) {
    double tb = -1.0;
    if (c1 < 0.0) tb = c0 / -c1;
    if (c2 < 0.0) {
      const double r = (double)sqrtf((float)(c0 / -c2));
      if (r > 0.0 && (tb < 0.0 || r < tb)) tb = r;
    }
    if (c3 < 0.0) {
      const double r = (double)cbrtf((float)(c0 / -c3));
      if (r > 0.0 && (tb < 0.0 || r < tb)) tb = r;
    }
    t = inside(tb) ? tb : hi > 0.0 ? 0.5 * (lo + hi) : (lo > 0.0 ? 2.0 * lo : 1.0);
  }
  for (int it = 0; it < 64; ++it) {
    const double f = fma(fma(fma(c3, t, c2), t, c1), t, c0);
    if (f > 0.0) lo = t;
    else if (f < 0.0) hi = t;
    else break;
    const double fp = fma(fma(3.0 * c3, t, 2.0 * c2), t, c1);
    double tn = (fp < 0.0 && isfinite(fp)) ? fma(-f, rcp64(fp), t) : -1.0;
    if (tn > 0.0 && isfinite(tn) && fabs(tn - t) <= 1e-13 * tn) {
      t = tn;   // converged (the step is below the resolution of t)
      break;
    }
    if (!inside(tn)) {
      if (hi < 0.0) tn = 2.0 * fmax(t, lo);
      else if (lo > 0.0 && hi > 4.0 * lo) tn = sqrt64(lo * hi);
      else if (lo == 0.0) tn = 0.25 * hi;
      else tn = 0.5 * (lo + hi);
    }
    t = tn;
  }
  if (t > 0.0 && isfinite(t)) {
    *t_out = t;   // scaling all coefficients by one factor leaves the roots alone
    return true;
  }
  return false;
}

// Exp-map series (Eq. step): sin(th)/th, (1 - cos th)/th^2 and (th - sin th)/th^3
// as polynomials in x = th^2 (truncation error < 1e-16 for x < 0.25), one per
// lane 0..2.
__constant__ double kExpSeries[3][7] = {
    {1.0, -1.0 / 6, 1.0 / 120, -1.0 / 5040, 1.0 / 362880, -1.0 / 39916800, 1.0 / 6227020800.0},
    {0.5, -1.0 / 24, 1.0 / 720, -1.0 / 40320, 1.0 / 3628800, -1.0 / 479001600,
     1.0 / 87178291200.0},
    {1.0 / 6, -1.0 / 120, 1.0 / 5040, -1.0 / 362880, 1.0 / 39916800, -1.0 / 6227020800.0,
     1.0 / 1307674368000.0}};

// Gradient tail, first part (warp 0, between the gradient barrier and the
// step pass): the unit step direction in the centred frame, in FP32, which is
// all the step pass needs. Lane a < 6 holds component a of the gradient before
// the metric factors, x0 = omega' + cX x v (rotation) or v (translation), in
// FP64 (the centring back-map may cancel); the common factor sigma^2 / ell^2
// drops out of the direction, so only 1/a^2 and 1/b^2 are applied. The FP64
// gradient itself (gradient_fp64) is formed during the step pass.
__device__ void gradient_direction(BlockCtx& b, const double* sums, int lane) {
  const TailConst& tc = b.tc;
  const int a = lane % 3, a1 = a == 2 ? 0 : a + 1, a2 = a == 0 ? 2 : a - 1;
  const bool rot = lane < 3;
  const double cr = fma(tc.cX[a1], sums[4 + a2], -(tc.cX[a2] * sums[4 + a1]));
  const double x0 = sums[1 + min(lane, 5)] + (rot ? cr : 0.0);
  if (lane < 6) b.x0[lane] = x0;
  const float x = lane < 6 ? __double2float_rn(x0) * (rot ? tc.inv_a2f : tc.inv_b2f) : 0.0f;
  float nrm2 = x * x;
#pragma unroll
  for (int off = 4; off > 0; off >>= 1) nrm2 += __shfl_xor_sync(kFull, nrm2, off);
  nrm2 = __shfl_sync(kFull, nrm2, 0);
  // 1/|x|: rsqrt and one Newton step (relative error about 1e-7)
  float inv = 0.0f;
  if (nrm2 > 0.0f && nrm2 < INFINITY) {
    inv = rsqrtf(nrm2);
    inv = inv * fmaf(-0.5f * nrm2, inv * inv, 1.5f);
  }
  // omega_a = x_a / |x|, v'_a = (v_a + (omega x cX)_a) / |x|
  const float xa1 = __shfl_sync(kFull, x, a1), xa2 = __shfl_sync(kFull, x, a2);
  const float xv = __shfl_sync(kFull, x, 3 + a);
  const float vc = (xv + fmaf(xa1, tc.cXf[a2], -(xa2 * tc.cXf[a1]))) * inv;
  if (lane < 3) {
    b.om[a] = x * inv;
    b.vc[a] = vc;
  }
  if (lane == 0) b.fin = 0;
  __syncwarp();
}

// Gradient tail, second part (one warp, during the step pass; it writes only
// fields the pass does not read): the metric gradient xi (Eq. metric), |xi|,
// xi / |xi| in FP64, F and the gradient pass's counts.
__device__ void gradient_fp64(BlockCtx& b, const double* sums, int lane) {
  const TailConst& tc = b.tc;
  const double x = lane < 6 ? b.x0[lane] * (lane < 3 ? b.kf_rot : b.kf_tr) : 0.0;
  double nrm2 = x * x;
#pragma unroll
  for (int off = 4; off > 0; off >>= 1) nrm2 += __shfl_xor_sync(kFull, nrm2, off);
  nrm2 = __shfl_sync(kFull, nrm2, 0);
  // |xi| and 1/|xi|: FP32 rsqrt refined by an FP64 Newton step
  // y <- y (1.5 - 0.5 x y^2) (relative error 1e-7 -> 1e-14)
  double inv = 0.0, nrm = 0.0;
  const int e2 = (__double2hiint(nrm2) >> 20) & 0x7ff;
  if (__double2hiint(nrm2) >= 0 && e2 > 1023 - 100 && e2 < 1023 + 100) {
    inv = f32_to_f64(rsqrtf(f64_to_f32(nrm2)));
    inv = inv * fma(-0.5 * nrm2, inv * inv, 1.5);
    nrm = nrm2 * inv;
  } else if (nrm2 > 0.0) {
    nrm = sqrt(nrm2);
    inv = 1.0 / nrm;
  }
  if (lane < 6) {
    b.xi[lane] = x;
    b.u64[lane] = x * inv;
  }
  if (lane == 0) {
    b.xi_norm = nrm;
    b.xi_inv = inv;
    b.small_grad = (!(nrm > 0.0) || nrm < tc.eps_grad) ? 1 : 0;
    b.F = tc.sigma2 * sums[0];
    b.nnz_grad = (unsigned long long)__double_as_longlong(sums[7]);
    b.cand_grad = (unsigned long long)__double_as_longlong(sums[8]);
  }
  __syncwarp();
}

// S0..S4 of the last step pass (Eq. fourth along xi): the pass summed along
// xi / |xi|, so S_m = s_m sigma^2 |xi|^m. Formed for the published results
// only. Any thread.
__device__ __forceinline__ void form_step_sums(BlockCtx& b) {
  double pw = b.tc.sigma2;
  for (int m = 0; m < 5; ++m) {
    b.S[m] = b.s_raw[m] * pw;
    pw *= b.xi_norm;
  }
}

// Step tail: step length, pose update P <- exp(t xi) P, stop test. Warp 0.
// The step length is found in tau = |xi| t, the step along xi / |xi|: G'(t) =
// sum_m m S_m t^(m-1) = sigma^2 |xi| sum_m m s_m tau^(m-1), so the quartic of
// the pass's own sums has the same roots in tau (no powers of |xi| needed),
// and the twist is tau (xi / |xi|).
__device__ void finish_step(BlockCtx& b, const double* sums, int lane) {
  const TailConst& tc = b.tc;
  if (lane < 5) b.s_raw[lane] = sums[lane];
  if (lane == 0) {
    b.nnz_total += b.nnz_grad + (unsigned long long)__double_as_longlong(sums[5]);
    b.cand_total += b.cand_grad + (unsigned long long)__double_as_longlong(sums[6]);
  }
  if (tc.mode == kModeEval) {
    __syncwarp();
    if (lane == 0) {
      form_step_sums(b);
      b.done = 1;
    }
    __syncwarp();
    return;
  }
  // the step length (the same scalar work on every lane)
  double tau;
  int no_ascent = 0, fallback = 0;
  // no step along a gradient below the stop test's threshold (at rounding
  // level S1 can still be positive, and the quartic's root is then arbitrary);
  // S1 > 0 exactly when s1 > 0
  if (b.small_grad || !is_pos(sums[1])) {
    tau = 0.0;
    no_ascent = 1;
  } else {
    bool ok;
    if (tc.step_order == 2) {
      ok = sums[2] < 0.0;
      tau = ok ? -sums[1] / mul_pow2(sums[2], 1) : 0.0;
    } else {
      ok = first_maximiser(sums[1], mul_pow2(sums[2], 1), 3.0 * sums[3], mul_pow2(sums[4], 2),
                           &tau);
    }
    if (!ok) {
      fallback = 1;
      // half the previous step, or 1e-3 / |xi| on the first one (tau = 1e-3)
      tau = b.have_t_prev ? 0.5 * b.t_prev * b.xi_norm : 1e-3;
    }
  }
  // twist tau xi / |xi|: rotation phi (lanes 0..2), translation rho (lanes 3..5)
  const double tw = tau * b.u64[min(lane, 5)];
  const double p0 = __shfl_sync(kFull, tw, 0), p1 = __shfl_sync(kFull, tw, 1);
  const double p2 = __shfl_sync(kFull, tw, 2);
  const double r0 = __shfl_sync(kFull, tw, 3), r1 = __shfl_sync(kFull, tw, 4);
  const double r2 = __shfl_sync(kFull, tw, 5);
  const double x = fma(p0, p0, fma(p1, p1, p2 * p2));
  // A = sin(th)/th, B = (1 - cos th)/th^2, C = (th - sin th)/th^3 on lanes 0, 1, 2.
  // The series alternate with falling terms, so the first term left out
  // bounds the error: 1 term below x = 1e-16, 2 below 1e-8, 3 below 1e-5, 4
  // below 1e-3 (errors below 1e-17 relative), all 7 below 0.25.
  double coef;
  if (x < 0.25) {
    const double* k = kExpSeries[min(lane, 2)];
    const int n = x < 1e-16 ? 0 : x < 1e-8 ? 1 : x < 1e-5 ? 2 : x < 1e-3 ? 3 : 6;
    coef = k[n];
    for (int i = n - 1; i >= 0; --i) coef = fma(coef, x, k[i]);
  } else {
    const double th = sqrt(x);
    const double sn = sin(th), hs = sin(0.5 * th);
    coef = lane == 0 ? sn / th : lane == 1 ? 2.0 * hs * hs / x : (th - sn) / (x * th);
  }
  const double A = __shfl_sync(kFull, coef, 0), B = __shfl_sync(kFull, coef, 1);
  const double C = __shfl_sync(kFull, coef, 2);
  // M = I + c1 W + c2 W^2 (W = hat(phi), W^2 = phi phi^T - |phi|^2 I): lanes 0..8
  // give dR = I + A W + B W^2, lanes 9..17 V = I + B W + C W^2 (Eq. step)
  const int q = lane % 9, i = q / 3, j = q % 3;
  const double pi = i == 0 ? p0 : i == 1 ? p1 : p2;
  const double pj = j == 0 ? p0 : j == 1 ? p1 : p2;
  const int kk = 3 - i - j;   // the third index when i != j
  const double pk = kk == 0 ? p0 : kk == 1 ? p1 : p2;
  const double w = i == j ? 0.0 : flip_sign(pk, (j - i + 3) % 3 == 1);
  const double w2 = fma(pi, pj, i == j ? -x : 0.0);
  const bool first = lane < 9;
  const double mv = fma(first ? A : B, w, fma(first ? B : C, w2, i == j ? 1.0 : 0.0));
  if (lane < 9) b.dR[q] = mv;
  else if (lane < 18) b.V[q] = mv;
  __syncwarp();
  // dT = V rho on lanes 0..2
  const int rr = lane % 3;
  const double dt = fma(b.V[3 * rr], r0, fma(b.V[3 * rr + 1], r1, b.V[3 * rr + 2] * r2));
  // P <- [dR dT] P on lanes 0..11, element (r, c) = (l / 4, l % 4)
  const int l = min(lane, 11), r = l >> 2, c = l & 3;
  const double dtr = __shfl_sync(kFull, dt, r);
  const double pn = fma(b.dR[3 * r], b.P[c],
                        fma(b.dR[3 * r + 1], b.P[4 + c],
                            fma(b.dR[3 * r + 2], b.P[8 + c], c == 3 ? dtr : 0.0)));
  __syncwarp();   // every lane has read the old pose
  if (lane < 12) b.P[lane] = pn;
  if (lane == 0) {
    b.no_ascent += no_ascent;
    b.fallback += fallback;
    const double t = tau * b.xi_inv;
    b.t = t;
    b.t_prev = t;
    b.have_t_prev = 1;
    // Table 1: |t xi| = |tau| below eps_pose, or |xi| below eps_grad, at the floor
    const bool conv = b.at_floor && (fabs(tau) < tc.eps_pose || b.small_grad);
    b.k += 1;
    if (conv || b.k >= tc.max_iters) {
      b.done = 1;
      b.converged = conv ? 1 : 0;
    }
  }
  __syncwarp();
}


// The team barrier counts arrivals on one counter that is never reset during
// a launch: generation g is complete when (g + 1) * nblk blocks have arrived.
// Thread 0 of each block adds its arrival with an acquire-release atomic after
// the block's __syncthreads (so every write the block made before the barrier
// is ordered before it) that returns the count before it: the block whose
// arrival completes the generation goes on at once, the others poll the
// counter with acquire loads. No block has to release the others.
__device__ __forceinline__ unsigned barrier_arrive_count(SolveState* st) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;"
               : "=r"(old)
               : "l"(&st->bar_count)
               : "memory");
  return old;
}

// Wait until `target` arrivals (thread 0). A block that polls `limit` times
// raises kStatusTimeout and returns false; its team then leaves the solve loop
// when the other blocks' own waits run out at the next barrier, which the
// timed-out block never reaches (an error path, bounded).
__device__ __forceinline__ bool barrier_wait(SolveState* st, unsigned target, unsigned limit) {
  unsigned spins = 0;
  while (ld_acquire(&st->bar_count) < target) {
    if (++spins > limit) {
      atomicOr(&st->status, (int)kStatusTimeout);
      return false;
    }
    __nanosleep(32);
  }
  return true;
}

// Bounded barrier of the team's nblk blocks. Every block calls it the same
// number of times; all blocks are resident (cooperative launch).
__device__ bool grid_sync(SolveState* st, unsigned& gen, int* s_flag, int nblk, unsigned limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned target = (gen + 1) * (unsigned)nblk;
    const bool last = barrier_arrive_count(st) + 1 == target;
    *s_flag = (last || barrier_wait(st, target, limit)) ? 1 : 0;
  }
  gen += 1;
  __syncthreads();
  return *s_flag != 0;
}

// Fixed-order FP64 sum of the nblk block partials (nvals <= 10 values each,
// value-major; the last two are counts, held as 64-bit integers in the
// doubles' bits), by one block. Warp w < nvals - 2 sums value w, one
// contiguous run of nblk doubles: lane l adds the value of blocks l, l + 32,
// l + 64, ... in sequence (its loads issued first), then the 32 lane
// sums are added along a fixed shuffle tree, so every FP64 instruction has all
// its lanes busy (on GB300 an FP64 instruction costs the same with one lane or
// 32). The last warp adds the two counts as integers. Results land in out[] (shared).
// Every thread of the block calls it.
template <class Smem>
__device__ void reduce_partials(const double* partials, int nvals, double* out, int nblk,
                                Smem& sm) {
  static_assert(kWarps >= 8, "seven FP values and the counts need eight warps");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kMaxPer = 16;   // nblk <= 512 blocks: 16 per lane
  const int nf = nvals - 2;     // FP64 values; nf <= 7
  if (warp < nf) {
    const int i = warp;
    const bool f32 = sm.b.tc.reduce_fp32 != 0;
    double v[kMaxPer];
#pragma unroll
    for (int k = 0; k < kMaxPer; ++k) {
      const int blk = lane + 32 * k;
      v[k] = blk < nblk ? __ldcg(&partials[(size_t)i * nblk + blk]) : 0.0;
    }
    double acc = 0.0;
    float accf = 0.f;
#pragma unroll
    for (int k = 0; k < kMaxPer; ++k) {
      if (32 * k >= nblk) break;
      if (f32) accf += (float)v[k];
      else acc += v[k];
    }
    if (f32) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) accf += __shfl_xor_sync(kFull, accf, off);
      acc = (double)accf;
    } else {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(kFull, acc, off);
    }
    if (lane == 0) out[i] = acc;
  } else if (warp == kWarps - 1) {
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      unsigned long long n = 0;
      for (int blk = lane; blk < nblk; blk += 32)
        n += (unsigned long long)__double_as_longlong(
            __ldcg(&partials[(size_t)(nf + c) * nblk + blk]));
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) n += __shfl_xor_sync(kFull, n, off);
      if (lane == 0) out[nf + c] = __longlong_as_double((long long)n);
    }
  }
  __syncthreads();
}

// Barrier that also reduces the pass: every block adds its arrival (a release
// reduction after the block's partials are written), waits for the
// generation's last arrival with acquire loads, and then sums all block
// partials itself in the same fixed FP64 order, so that no block has to
// publish totals and release the others. A block reads the partials of
// generation g only before it arrives at generation g + 1, and the next
// writes to the same partial buffer (two generations later) come after that
// arrival, so one buffer per pass kind is enough. Every thread of every block
// gets the totals in sums[]. Bounded like grid_sync.
template <class Smem>
__device__ bool grid_sync_reduce(SolveState* st, unsigned& gen, Smem& sm, const double* partials,
                                 int nvals, int nblk) {
  const unsigned g = gen;
  gen += 1;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned target = (g + 1) * (unsigned)nblk;
    const bool last = barrier_arrive_count(st) + 1 == target;
    sm.flag = (last || barrier_wait(st, target, sm.b.tc.wait_polls)) ? 1 : 0;
  }
  __syncthreads();
  if (!sm.flag) return false;
  reduce_partials(partials, nvals, sm.sums, nblk, sm);
  return true;
}

// Start of a queued solve: wait until every block of the team has claimed its
// slot. Blocks of a team come free at different times (each finishes the pair
// it held), so this wait can last as long as one pair's solve; it is bounded
// by join_limit_ns of the global timer (SolveCfg), after which the pair fails
// with kStatusTimeout.
template <class Smem>
__device__ bool team_join(SolveState* st, int team_size, Smem& sm) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(&st->join_count, 1u);
    const unsigned long long t_start = globaltimer();
    unsigned polls = 0;
    while (ld_acquire(&st->join_count) < (unsigned)team_size) {
      if ((++polls & 255u) == 0 && globaltimer() - t_start > sm.b.tc.join_limit_ns) {
        ok = 0;
        atomicOr(&st->status, (int)kStatusTimeout);
        break;
      }
      __nanosleep(256);
    }
    __threadfence();
    if (ld_acquire((const unsigned*)&st->status) & kStatusTimeout) ok = 0;
    sm.flag = ok;
  }
  __syncthreads();
  return sm.flag != 0;
}

// Squared distance from x to the box [lo, hi] (zero inside), the one form the
// plan and every pass evaluate, so that they agree on each candidate.
__device__ __forceinline__ float box_dist2(float4 x, float4 lo, float4 hi) {
  const float dx = fmaxf(fmaxf(lo.x - x.x, x.x - hi.x), 0.f);
  const float dy = fmaxf(fmaxf(lo.y - x.y, x.y - hi.y), 0.f);
  const float dz = fmaxf(fmaxf(lo.z - x.z, x.z - hi.z), 0.f);
  return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
}

// Plan of one cluster (one warp): transform its points, bounding box, cell
// rows within the plan radius -> segments, candidate count; then the
// candidates themselves are read once and those farther than the plan radius
// from the bounding box are filtered out (they cannot come within the cutoff
// of any of the cluster's points while the plan is valid: a point within r_c
// at the current pose lies within r_c + drift < plan radius of its plan-pose
// position, which is inside the box). Per segment, the number of candidates
// that pass gives the filtered offsets the work split and the passes use.
// s_xs, s_pf, s_cnt: the warp's shared arrays (kMaxSeg + 1 entries).
__device__ void plan_cluster(const SolveCfg* cfg, const BlockCtx& b, SolveState* st, int c,
                             int lane, int* s_xs, int* s_pf, int* s_cnt) {
  const GridView& g = cfg->grids[b.level];
  const ClusterView& cv = cfg->clusters[b.level];
  __syncwarp();   // the shared arrays of the warp's previous cluster are free
  const int p0 = cv.cstart[c];
  const int cs = cv.cstart[c + 1] - p0;
  const bool zv = lane < cs;
  float zx = 0.f, zy = 0.f, zz = 0.f;
  if (zv) {
    const float4 p = cfg->src.xyz[p0 + lane];
    zx = fmaf(b.R[0], p.x, fmaf(b.R[1], p.y, fmaf(b.R[2], p.z, b.T[0])));
    zy = fmaf(b.R[3], p.x, fmaf(b.R[4], p.y, fmaf(b.R[5], p.z, b.T[1])));
    zz = fmaf(b.R[6], p.x, fmaf(b.R[7], p.y, fmaf(b.R[8], p.z, b.T[2])));
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
  const float rp = b.rplan_f;
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
      s_xs[idx] = xs;
      s_pf[idx] = total + incl - keep;
    }
    nseg += __popc(m);
    total += __shfl_sync(kFull, incl, 31);
  }
  if (__any_sync(kFull, overflow) && lane == 0) atomicOr(&st->status, (int)kStatusSegOverflow);
  nseg = min(nseg, kMaxSeg);
  if (lane == 0) s_pf[nseg] = total;
  for (int i = lane; i < nseg; i += 32) s_cnt[i] = 0;
  __syncwarp();
  // the filter: every candidate read once, four rounds of 32 loads in flight.
  // Only a plan that will be reused (the next iteration keeps the lengthscale)
  // is filtered, and only its clusters of at most kFilterMax candidates; the
  // others get the whole space as their box (every candidate passes): a plan
  // used for one iteration does not repay the extra read
  const bool filt = b.plan_filter != 0 && total <= kFilterMax;
  const float4 lo4 = filt ? make_float4(blo[0], blo[1], blo[2], 0.f)
                          : make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
  const float4 hi4 = filt ? make_float4(bhi[0], bhi[1], bhi[2], 0.f)
                          : make_float4(INFINITY, INFINITY, INFINITY, 0.f);
  if (!filt) {
    for (int i = lane; i < nseg; i += 32) s_cnt[i] = s_pf[i + 1] - s_pf[i];
  }
  int seg = 0;
  for (int u0 = 0; filt && u0 < total; u0 += 128) {
    float4 xq[4];
    int sq[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int q = u0 + 32 * k + lane;
      sq[k] = -1 - lane;   // distinct for every lane past the end
      xq[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (q < total) {
        while (s_pf[seg + 1] <= q) ++seg;
        sq[k] = seg;
        xq[k] = g.xyz[s_xs[seg] + (q - s_pf[seg])];
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const bool pass = sq[k] >= 0 && box_dist2(xq[k], lo4, hi4) <= rp2;
      const unsigned m = __ballot_sync(kFull, pass);
      const unsigned grp = __match_any_sync(kFull, sq[k]);
      const int n = __popc(grp & m);
      if (sq[k] >= 0 && lane == __ffs(grp) - 1 && n > 0) atomicAdd(&s_cnt[sq[k]], n);
    }
  }
  __syncwarp();
  // filtered offsets of the segments (exclusive prefix over at most 64)
  const int n0 = lane < nseg ? s_cnt[lane] : 0;
  const int n1 = lane + 32 < nseg ? s_cnt[lane + 32] : 0;
  int i0 = n0, i1 = n1;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int v0 = __shfl_up_sync(kFull, i0, off);
    const int v1 = __shfl_up_sync(kFull, i1, off);
    if (lane >= off) {
      i0 += v0;
      i1 += v1;
    }
  }
  const int t0 = __shfl_sync(kFull, i0, 31);
  const int t1 = __shfl_sync(kFull, i1, 31);
  int* sff = cfg->seg_fpref + (size_t)c * kMaxSeg;
  if (lane < nseg) sff[lane] = i0 - n0;
  if (lane + 32 < nseg) sff[lane + 32] = t0 + i1 - n1;
  cfg->ch_act[(size_t)c * kActChunks + lane] = 0u;
  if (lane == 0) {
    cfg->cl_act[c] = 0;
    cfg->cl_nseg[c] = nseg;
    cfg->cl_cand[c] = total;
    cfg->cl_fcand[c] = t0 + t1;
    cfg->cl_kept[c] = 0;
    // the box at the plan pose, whether or not the plan filtered (w = 1: the
    // segment offsets count the candidates within the plan radius of it)
    cfg->cl_box[2 * (size_t)c] = make_float4(blo[0], blo[1], blo[2], filt ? 1.f : 0.f);
    cfg->cl_box[2 * (size_t)c + 1] = make_float4(bhi[0], bhi[1], bhi[2], 0.f);
  }
}

// Work of cluster c under the current plan, in pair-test units: staging the
// cluster costs cost_cluster, each chunk of 32 filtered candidates its cs4
// pair tests per lane (cluster size padded to a multiple of 4) plus
// cost_chunk of per-chunk overhead, plus (use_kept, once the plan's first
// gradient pass has counted them) cost_kept per kept pair of the cluster,
// spread evenly over its chunks. Chunk j starts at offset cost_cluster + j * k,
// k = the per-chunk cost; within a chunk, the overhead and the first group of
// four source points come first, then one group (4 tests) after another.
// With use_act (a reused plan, once its first gradient pass has recorded
// which source groups of which chunks kept a pair), each such group costs
// kCostActive more (its pair bodies); chunks beyond the recorded ones count
// every group as active.
__device__ __forceinline__ long long cluster_work(const SolveCfg* cfg, const ClusterView& cv,
                                                  int c, int* k_out, bool use_kept,
                                                  bool use_act) {
  const int tc = __ldcg(&cfg->cl_fcand[c]);
  const int cs4 = ((cv.cstart[c + 1] - cv.cstart[c]) + 3) & ~3;
  const int nch = (tc + 31) >> 5;
  int k = cs4 + cfg->cost_chunk;
  if (use_kept && nch > 0)
    k += (int)(cfg->cost_kept * (float)__ldcg(&cfg->cl_kept[c]) / (float)nch);
  *k_out = k;
  if (nch <= 0) return 0;
  long long w = (long long)cfg->cost_cluster + (long long)nch * k;
  if (use_act)
    w += (long long)kCostActive * ((long long)__ldcg(&cfg->cl_act[c]) +
                                   (long long)max(0, nch - kActChunks) * (cs4 >> 2));
  return w;
}

// Entries of a warp's pair list (build_lists), per padded feature width: as
// many as fit beside the block's other static shared memory without taking a
// cache slot from the dynamic part at one block per SM (640 at 5 feature
// planes, 448 at 3 and 8, 400 without features).
template <int DPS>
__host__ __device__ constexpr int list_max() {
  return DPS == 5 ? 640 : DPS == 1 ? 400 : 448;
}
constexpr int kListShift = 22;   // cache_cl of a listed cluster slot: cluster | length << 22
static_assert(kMaxPoints <= (1 << kListShift), "cluster index must fit below the list length");

// Per warp: the cell-row segments of the cluster being staged from the plan
// (plan, cache fill, streamed passes), or, for a warp whose share is cached
// from a plan that will be reused, its pair list (the segments are not needed
// once the cache is filled, and a cached warp never streams).
struct WarpSeg {
  int xs[kMaxSeg];
  int pf[kMaxSeg + 1];
  int fpf[kMaxSeg + 1];   // filtered offsets (the plan: per-segment counts)
};
template <int DPS>
union WarpScratch {
  WarpSeg seg;
  unsigned short list[list_max<DPS>()];
};

// Shared memory of the solve kernel.
template <int DPS, int NU>
struct SolveSmem {
  float4 z[kWarps][kClusterMax];    // staged cluster, local: (-2 z_l, |z_l|^2), see stage_cluster
  float4 zo[kWarps];                // origin of each warp's staged cluster (centred frame)
  float zf[kWarps][DPS][kClusterMax];
  float4 u[kWarps][NU][kClusterMax];
  WarpScratch<DPS> ws[kWarps];      // cell-row segments of the staged cluster, or the pair list
  float red[kWarps][10];
  double red_d[kWarps][16];
  long long scan[kThreads];
  long long bnd_base[2 * kWarps];   // work offset of the group holding each warp boundary
  int bnd_group[2 * kWarps];
  double sums[10];
  int flag, last;
  long long q_slot;                 // queue: claimed slot (-1: none left)
  int q_entry;                      //        entry that slot belongs to
  short cache_n[kWarps];            // slots cached per warp (-1: streamed)
  unsigned short cache_hdr[kWarps][32];
  int cache_cl[kWarps][32];         // cluster of each cached cluster slot (a listed one: | list
                                    //   length << kListShift), chunk index of a chunk slot
  BlockCtx b;
};

// (cluster, chunk, group) of the first unit of work that starts at or after
// s, for s inside group-of-clusters `group` whose work starts at `base` (one
// warp). Units of a cluster whose work starts at e0: its staging
// [e0, e0 + cost_cluster), then per chunk j (starting at e = e0 +
// cost_cluster + j k) the unit of source group 0 at e (it carries the chunk's
// overhead oh = k - cs4) and the unit of source group g > 0 at e + oh + 4 g.
// The chunk may equal the cluster's chunk count, which means the next
// cluster's first chunk.
__device__ void locate(const SolveCfg* cfg, const ClusterView& cv, int group, long long base,
                       long long s, int lane, int* c_out, int* j_out, int* g_out,
                       bool use_kept, bool use_act) {
  const int c = group * 32 + lane;
  long long w = 0;
  int kk = 4;
  if (c < cv.ncl) w = cluster_work(cfg, cv, c, &kk, use_kept, use_act);
  long long incl = w;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const long long v = __shfl_up_sync(kFull, incl, off);
    if (lane >= off) incl += v;
  }
  const long long excl = base + incl - w;
  const unsigned m = __ballot_sync(kFull, c < cv.ncl && w > 0 && s >= excl && s < excl + w);
  if (m) {
    const int src = __ffs(m) - 1;
    const int cc = group * 32 + src;
    const long long e = __shfl_sync(kFull, excl, src) + cfg->cost_cluster;
    const int k4 = __shfl_sync(kFull, kk, src);
    const int cs4 = ((cv.cstart[cc + 1] - cv.cstart[cc]) + 3) & ~3;
    const int oh = k4 - cs4;
    const int G = cs4 >> 2;
    const int nch = (__ldcg(&cfg->cl_fcand[cc]) + 31) >> 5;
    int j = 0, gq = 0;
    if (use_act && s > e) {
      // chunk j costs k4 + kCostActive x (its active groups; all of them past
      // the recorded chunks); lane j holds chunk j's mask
      const unsigned gm = (1u << G) - 1u;
      long long cum = 0;   // end of the chunks before this round, relative to e
      for (int j0 = 0;; j0 += 32) {
        const int jj = j0 + lane;
        unsigned mj = gm;
        if (jj < nch && jj < kActChunks) mj = __ldcg(&cfg->ch_act[(size_t)cc * kActChunks + jj]) & gm;
        const long long kj = jj < nch ? (long long)k4 + (long long)kCostActive * __popc(mj) : 0;
        long long in = kj;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const long long v = __shfl_up_sync(kFull, in, off);
          if (lane >= off) in += v;
        }
        // the chunk whose end lies beyond s (s - e < cum + in)
        const unsigned hit = __ballot_sync(kFull, jj < nch && s - e < cum + in);
        if (hit) {
          const int src2 = __ffs(hit) - 1;
          const long long start = e + cum + __shfl_sync(kFull, in - kj, src2);
          const unsigned m = __shfl_sync(kFull, mj, src2);
          j = j0 + src2;
          if (s > start) {
            // units of the chunk: group 0 at start (with the overhead), group
            // g at start + oh + sum over g' < g of (4 + kCostActive a_g')
            long long u = start + oh + 4 + kCostActive * (long long)(m & 1u);
            gq = G;
            for (int g = 1; g < G; ++g) {
              if (u >= s) {
                gq = g;
                break;
              }
              u += 4 + kCostActive * (long long)((m >> g) & 1u);
            }
            if (gq >= G) {
              ++j;
              gq = 0;
            }
          }
          break;
        }
        cum += __shfl_sync(kFull, in, 31);
        if (j0 + 32 >= nch) {   // past the last chunk (cannot happen: s < end)
          j = nch;
          break;
        }
      }
    } else if (s > e) {
      const long long r = s - e;
      j = (int)(r / k4);
      const int rr = (int)(r - (long long)j * k4);
      if (rr > 0) {
        gq = max(1, (rr - oh + 3) >> 2);   // the first g >= 1 with oh + 4 g >= rr
        if (gq >= (cs4 >> 2)) {
          ++j;
          gq = 0;
        }
      }
    }
    *c_out = cc;
    *j_out = j;
    *g_out = gq;
  } else {
    *c_out = min(group * 32 + 32, cv.ncl);
    *j_out = 0;
    *g_out = 0;
  }
}

// Place the block's warps on an even split of the plan's work: warp w owns the
// units (a chunk's source group) whose work starts in [floor(w TW/NW),
// floor((w+1) TW/NW)).
template <int DPS, int NU>
__device__ void split_work(const SolveCfg* cfg, SolveSmem<DPS, NU>& sm, int tid, Team team) {
  const ClusterView& cv = cfg->clusters[sm.b.level];
  const int ng = (cv.ncl + 31) / 32;
  const int per = (ng + kThreads - 1) / kThreads;
  const int g0 = min(ng, tid * per), g1 = min(ng, g0 + per);
  long long local = 0;
  for (int gi = g0; gi < g1; ++gi) local += __ldcg(&cfg->group_agg[gi]);
  sm.scan[tid] = local;
  if (tid < 2 * kWarps) sm.bnd_group[tid] = -1;
  __syncthreads();
  for (int off = 1; off < kThreads; off <<= 1) {
    const long long v = tid >= off ? sm.scan[tid - off] : 0;
    __syncthreads();
    sm.scan[tid] += v;
    __syncthreads();
  }
  const long long TW = sm.scan[kThreads - 1];
  const long long NW = (long long)team.size * kWarps;
  long long run = sm.scan[tid] - local;
  for (int gi = g0; gi < g1; ++gi) {
    const long long gtests = __ldcg(&cfg->group_agg[gi]);
#pragma unroll
    for (int q = 0; q < 2 * kWarps; ++q) {
      const long long w = (long long)team.rank * kWarps + (q >> 1) + (q & 1);
      const long long s = TW > 0 ? (w * TW) / NW : 0;
      if (gtests > 0 && s >= run && s < run + gtests) {
        sm.bnd_group[q] = gi;
        sm.bnd_base[q] = run;
      }
    }
    run += gtests;
  }
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int q = 2 * warp + h;
    const long long w = (long long)team.rank * kWarps + warp + h;
    const long long s = TW > 0 ? (w * TW) / NW : 0;
    int c, jj, gg;
    if (TW == 0 || s >= TW || sm.bnd_group[q] < 0) {
      c = cv.ncl;   // past the end: no chunk
      jj = gg = 0;
    } else {
      locate(cfg, cv, sm.bnd_group[q], sm.bnd_base[q], s, lane, &c, &jj, &gg,
             sm.b.use_kept != 0, sm.b.use_act != 0);
    }
    if (lane == 0) {
      if (h == 0) {
        sm.b.w_c0[warp] = c;
        sm.b.w_j0[warp] = jj;
        sm.b.w_g0[warp] = gg;
      } else {
        sm.b.w_c1[warp] = c;
        sm.b.w_j1[warp] = jj;
        sm.b.w_g1[warp] = gg;
      }
    }
  }
  __syncthreads();
}

// Stage one cluster for a warp: lane j < cs holds the cluster's centred
// source point p and its features. The transformed point z~' = R p + T is
// stored relative to the cluster's origin o (lane 0's transformed point) as
// (-2 z_l, |z_l|^2), z_l = z~' - o, so that a candidate x_l = x' - o tests
// its squared distance as |x_l|^2 + x_l . (-2 z_l) + |z_l|^2: three FMAs
// with x_l and |x_l|^2 formed once per chunk. The cluster is small (an
// octree cell of the plan's level), so |x_l| and |z_l| stay within a few
// cutoff radii and the expansion loses no more than a few bits to
// cancellation. Padding slots hold (0, 0, 0, +inf): beyond every cutoff,
// zero weight. For the step pass the Taylor coefficient vectors of Eq.
// fourth go to the warp's slots as well, their fourth components holding
// the per-point constants that turn x_l . U_k into e . U_k (e = x' - z~').
template <bool STEP, int DP, int DPS, int NU>
__device__ __forceinline__ void stage_cluster(SolveSmem<DPS, NU>& sm, int warp, int lane, bool zv,
                                              float4 p, const float pf[DPS]) {
  const BlockCtx& b = sm.b;
  float zt[3] = {0.f, 0.f, 0.f};
  if (zv) {
    zt[0] = fmaf(b.R[0], p.x, fmaf(b.R[1], p.y, fmaf(b.R[2], p.z, b.T[0])));
    zt[1] = fmaf(b.R[3], p.x, fmaf(b.R[4], p.y, fmaf(b.R[5], p.z, b.T[1])));
    zt[2] = fmaf(b.R[6], p.x, fmaf(b.R[7], p.y, fmaf(b.R[8], p.z, b.T[2])));
  }
  // lane 0 holds a point of every staged cluster (cs >= 1)
  const float ox = __shfl_sync(kFull, zt[0], 0), oy = __shfl_sync(kFull, zt[1], 0),
              oz = __shfl_sync(kFull, zt[2], 0);
  const float lx = zv ? zt[0] - ox : 0.f, ly = zv ? zt[1] - oy : 0.f, lz = zv ? zt[2] - oz : 0.f;
  sm.z[warp][lane] = zv ? make_float4(-2.f * lx, -2.f * ly, -2.f * lz,
                                      fmaf(lx, lx, fmaf(ly, ly, lz * lz)))
                        : make_float4(0.f, 0.f, 0.f, INFINITY);
  if (lane == 0) sm.zo[warp] = make_float4(ox, oy, oz, 0.f);
#pragma unroll
  for (int d = 0; d < DP; ++d) sm.zf[warp][d][lane] = zv ? pf[d] : 0.f;
  if (STEP) {
    const float* om = b.om;
    const float* vc = b.vc;
    const float inv_l2 = b.inv_l2f;
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
    // beta = e.U1; gamma = e.U2 - k2; delta = e.U3 - k3; eps = e.U4 - k4,
    // with e.U = x_l.U - z_l.U: the fourth components hold -z_l.U - k
    const float c1 = inv_l2, c2 = 0.5f * inv_l2, c3 = inv_l2 * (1.0f / 6.0f),
                c4 = inv_l2 * (1.0f / 24.0f);
    const float k2 = 0.5f * u11 * inv_l2, k3 = 0.5f * u12 * inv_l2,
                k4 = (u13 * (1.0f / 6.0f) + u22 * 0.125f) * inv_l2;
    const float4 U1 = make_float4(u1[0] * c1, u1[1] * c1, u1[2] * c1, 0.f);
    const float4 U2 = make_float4(u2[0] * c2, u2[1] * c2, u2[2] * c2, 0.f);
    const float4 U3 = make_float4(u3[0] * c3, u3[1] * c3, u3[2] * c3, 0.f);
    const float4 U4 = make_float4(u4[0] * c4, u4[1] * c4, u4[2] * c4, 0.f);
    const auto zl_dot = [&](const float4& U) { return fmaf(lx, U.x, fmaf(ly, U.y, lz * U.z)); };
    sm.u[warp][0][lane] = make_float4(U1.x, U1.y, U1.z, -zl_dot(U1));
    sm.u[warp][1 % NU][lane] = make_float4(U2.x, U2.y, U2.z, -zl_dot(U2) - k2);
    sm.u[warp][2 % NU][lane] = make_float4(U3.x, U3.y, U3.z, -zl_dot(U3) - k3);
    sm.u[warp][3 % NU][lane] = make_float4(U4.x, U4.y, U4.z, -zl_dot(U4) - k4);
  }
}

// One 32-candidate chunk against the staged cluster: lane = candidate x'
// (xp, features xf; padding points lie beyond every cutoff), inner loop over
// the cluster's points [jlo, jhi) (multiples of 4, at most the cluster size
// rounded up to 4; padding slots lie beyond the cutoff too). FP32 pair
// arithmetic, one ex2.approx per pair. Distances are taken relative to the
// cluster's origin (stage_cluster): t = x_l . (-2 z_l) + |z_l|^2 equals
// d^2 - |x_l|^2, so a pair is kept when t <= r_c^2 - |x_l|^2, and the
// exponent A d^2 is A t + A |x_l|^2.
// Points are taken four at a time: the four distance tests first, then, if
// any lane of the warp keeps any of the four pairs (one vote, so the branch
// is uniform), the four pair bodies without branches, a rejected pair
// contributing exactly nothing (its weight is selected to zero and its step
// terms are not added). The four bodies are independent, so their latencies
// overlap.
template <bool STEP, int DP, int MODE, int DPS, int NU>
__device__ __forceinline__ unsigned chunk_pairs(SolveSmem<DPS, NU>& sm, int warp, float4 xp,
                                                const float xf[DPS], int jlo, int jhi, float rc2,
                                                float A, float acc[7], unsigned& nnz) {
  const float4 o = sm.zo[warp];
  const float xl = xp.x - o.x, yl = xp.y - o.y, zl = xp.z - o.z;
  const float x2 = fmaf(xl, xl, fmaf(yl, yl, zl * zl));
  const float thr = rc2 - x2;   // about -3e36 for a padding candidate: never kept
  const float q0 = A * x2;
  float W = 0.f, Mx = 0.f, My = 0.f, Mz = 0.f;
  unsigned active = 0u;   // bit g: source group g kept a pair (the same in every lane)
  for (int j0 = jlo; j0 < jhi; j0 += 4) {
    float4 m[4];
    float t[4];
    bool keep[4];
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      m[jj] = sm.z[warp][j0 + jj];
      t[jj] = fmaf(xl, m[jj].x, fmaf(yl, m[jj].y, fmaf(zl, m[jj].z, m[jj].w)));
      keep[jj] = t[jj] <= thr;
    }
    if (!__any_sync(kFull, keep[0] | keep[1] | keep[2] | keep[3])) continue;
    active |= 1u << (j0 >> 2);
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int j = j0 + jj;
      float w;
      if (color_of(MODE) == kColorKernel) {
        float qf = q0;
#pragma unroll
        for (int d = 0; d < DP; ++d) {
          const float df = xf[d] - sm.zf[warp][d][j];
          qf = fmaf(df, df, qf);
        }
        w = ex2_approx(-fmaf(A, t[jj], qf));
      } else if (color_of(MODE) == kColorDot) {
        float cdot = 0.f;
#pragma unroll
        for (int d = 0; d < DP; ++d) cdot = fmaf(xf[d], sm.zf[warp][d][j], cdot);
        w = ex2_approx(-fmaf(A, t[jj], q0)) * cdot;
      } else {
        w = ex2_approx(-fmaf(A, t[jj], q0));
      }
      w = keep[jj] ? w : 0.f;
      nnz += keep[jj] ? 1u : 0u;
      if (!STEP) {
        // m = (-2 z_l, .) is finite, so a zero weight adds exactly zero
        W += w;
        Mx = fmaf(w, m[jj].x, Mx);
        My = fmaf(w, m[jj].y, My);
        Mz = fmaf(w, m[jj].z, Mz);
      } else {
        const float4 U1 = sm.u[warp][0][j], U2 = sm.u[warp][1 % NU][j];
        const float4 U3 = sm.u[warp][2 % NU][j], U4 = sm.u[warp][3 % NU][j];
        const float beta = fmaf(xl, U1.x, fmaf(yl, U1.y, fmaf(zl, U1.z, U1.w)));
        const float gam = fmaf(xl, U2.x, fmaf(yl, U2.y, fmaf(zl, U2.z, U2.w)));
        const float del = fmaf(xl, U3.x, fmaf(yl, U3.y, fmaf(zl, U3.z, U3.w)));
        const float eps = fmaf(xl, U4.x, fmaf(yl, U4.y, fmaf(zl, U4.z, U4.w)));
        const float b2 = beta * beta;
        const float g2 = fmaf(0.5f, b2, gam);
        const float g3 = fmaf(beta, fmaf(b2, 1.0f / 6.0f, gam), del);
        const float g4 = fmaf(b2 * b2, 1.0f / 24.0f,
                              fmaf(0.5f * gam, b2 + gam, fmaf(beta, del, eps)));
        // the polynomial of a far padding pair may overflow: select, not scale
        acc[0] += w;
        acc[1] = keep[jj] ? fmaf(w, beta, acc[1]) : acc[1];
        acc[2] = keep[jj] ? fmaf(w, g2, acc[2]) : acc[2];
        acc[3] = keep[jj] ? fmaf(w, g3, acc[3]) : acc[3];
        acc[4] = keep[jj] ? fmaf(w, g4, acc[4]) : acc[4];
      }
    }
  }
  if (!STEP) {
    // E_i = sum_j w e_ij = x_l W - sum_j w z_l = x_l W + M / 2; x' fixed per
    // lane: sum_j w (z~'_j x e_ij) = x' x E_i. A padding lane has W = M = 0
    // and a finite x_l.
    const float Ex = fmaf(xl, W, 0.5f * Mx);
    const float Ey = fmaf(yl, W, 0.5f * My);
    const float Ez = fmaf(zl, W, 0.5f * Mz);
    acc[0] += W;
    acc[1] += xp.y * Ez - xp.z * Ey;
    acc[2] += xp.z * Ex - xp.x * Ez;
    acc[3] += xp.x * Ey - xp.y * Ex;
    acc[4] += Ex;
    acc[5] += Ey;
    acc[6] += Ez;
  }
  return active;
}

// A warp's range of work (BlockCtx::w_*).
struct WarpRange {
  int c0, j0, g0, c1, j1, g1;
};

__device__ __forceinline__ WarpRange warp_range(const BlockCtx& b, int warp) {
  return WarpRange{b.w_c0[warp], b.w_j0[warp], b.w_g0[warp],
                   b.w_c1[warp], b.w_j1[warp], b.w_g1[warp]};
}

// Chunks [jb, je] of cluster c (nch chunks) that hold work of the range.
__device__ __forceinline__ bool range_chunks(const WarpRange& r, int c, int nch, int& jb, int& je) {
  if (c < r.c0 || c > r.c1) return false;
  jb = c == r.c0 ? r.j0 : 0;
  je = nch - 1;
  if (c == r.c1) je = min(je, r.g1 > 0 ? r.j1 : r.j1 - 1);
  return jb <= je;
}

// Source groups [glo, ghi) of chunk j of cluster c (G groups) in the range.
__device__ __forceinline__ void range_groups(const WarpRange& r, int c, int j, int G, int& glo,
                                             int& ghi) {
  glo = (c == r.c0 && j == r.j0) ? r.g0 : 0;
  ghi = (c == r.c1 && j == r.j1) ? min(r.g1, G) : G;
}

// Segments of cluster c into the warp's shared arrays: first target index,
// candidate offset (then tc) and filtered offset (then fc) of each segment.
template <int DPS, int NU>
__device__ __forceinline__ int load_segments(const SolveCfg* cfg, SolveSmem<DPS, NU>& sm, int warp,
                                             int lane, int c, int tc, int fc) {
  const int nseg = __ldcg(&cfg->cl_nseg[c]);
  for (int i = lane; i < nseg; i += 32) {
    sm.ws[warp].seg.xs[i] = __ldcg(&cfg->seg_xs[(size_t)c * kMaxSeg + i]);
    sm.ws[warp].seg.pf[i] = __ldcg(&cfg->seg_pref[(size_t)c * kMaxSeg + i]);
    sm.ws[warp].seg.fpf[i] = __ldcg(&cfg->seg_fpref[(size_t)c * kMaxSeg + i]);
  }
  if (lane == 0) {
    sm.ws[warp].seg.pf[nseg] = tc;
    sm.ws[warp].seg.fpf[nseg] = fc;
  }
  __syncwarp();
  return nseg;
}

// Candidate q of the staged cluster (padding beyond tc), advancing seg.
template <int DP, int DPS, int NU, bool FB>
__device__ __forceinline__ float4 load_candidate(const GridView& g, SolveSmem<DPS, NU>& sm, int warp,
                                                 int q, int tc, int& seg, float xf[DPS]) {
  float4 xp = make_float4(-kFar, -kFar, -kFar, 0.f);
#pragma unroll
  for (int d = 0; d < DPS; ++d) xf[d] = 0.f;
  if (q < tc) {
    while (sm.ws[warp].seg.pf[seg + 1] <= q) ++seg;
    const int xi = sm.ws[warp].seg.xs[seg] + (q - sm.ws[warp].seg.pf[seg]);
    xp = g.xyz[xi];
#pragma unroll
    for (int d = 0; d < DP; ++d) xf[d] = load_feat<FB>(g.feat, (size_t)d * g.n_pad + xi);
  }
  return xp;
}

// Cursor over the filtered candidates of the cluster whose segments are
// staged: the next block of 32 candidates starts at candidate u; `skip`
// filtered candidates are still to be dropped (they precede the range); seg
// is this lane's segment; made counts the filtered candidates produced.
struct FCursor {
  int u, skip, seg, made;
};

// Cursor at filtered candidate f0 (< fc): the last segment whose filtered
// offset is <= f0 (a segment that filters to nothing shares its offset with
// the next one), from its first candidate.
template <int DPS, int NU>
__device__ __forceinline__ FCursor fcursor_at(const SolveSmem<DPS, NU>& sm, int warp, int nseg,
                                              int f0) {
  int lo = 0, hi = nseg;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (sm.ws[warp].seg.fpf[mid] <= f0) lo = mid;
    else hi = mid;
  }
  FCursor cur;
  cur.u = sm.ws[warp].seg.pf[lo];
  cur.skip = f0 - sm.ws[warp].seg.fpf[lo];
  cur.seg = lo;
  cur.made = 0;
  return cur;
}

// The block of candidates at cur.u (this lane's is xp) through the plan's
// filter: the filtered index (counted from the cursor's start) of this lane's
// candidate, or -1; the cursor moves to the next block.
__device__ __forceinline__ int fplace(FCursor& cur, float4 xp, float4 lo, float4 hi, float rp2,
                                      int lane, int tc) {
  const bool pass = cur.u + lane < tc && box_dist2(xp, lo, hi) <= rp2;
  const unsigned m = __ballot_sync(kFull, pass);
  const int r = __popc(m & ((1u << lane) - 1u));
  const int n = __popc(m);
  const int d = min(cur.skip, n);
  cur.skip -= d;
  const int o = (pass && r >= d) ? cur.made + r - d : -1;
  cur.made += n - d;
  cur.u += 32;
  return o;
}

// Kept pairs of cluster c counted by this warp, added to the plan's
// per-cluster totals (one atomic per warp and cluster).
__device__ __forceinline__ void add_kept(const SolveCfg* cfg, int c, unsigned kept, int lane) {
  unsigned k = kept;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) k += __shfl_down_sync(kFull, k, off);
  if (lane == 0 && c >= 0 && k) atomicAdd(&cfg->cl_kept[c], (int)k);
}

// Source groups of chunk j of cluster c that kept a pair, recorded by the
// plan's first gradient pass (lane 0; the mask is warp-uniform).
__device__ __forceinline__ void add_active(const SolveCfg* cfg, int c, int j, unsigned active,
                                           int lane) {
  if (lane == 0 && active && c >= 0 && j < kActChunks) {
    atomicOr(&cfg->ch_act[(size_t)c * kActChunks + j], active);
    atomicAdd(&cfg->cl_act[c], __popc(active));
  }
}

// Stage cluster c for the warp from global memory (raw centred source points
// and features, transformed by stage_cluster).
template <bool STEP, int DP, int MODE, int DPS, int NU>
__device__ __forceinline__ int stage_from_global(const SolveCfg* cfg, SolveSmem<DPS, NU>& sm,
                                                 const ClusterView& cv, int c, int warp,
                                                 int lane) {
  const int p0 = cv.cstart[c];
  const int cs = cv.cstart[c + 1] - p0;
  const bool zv = lane < cs;
  float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
  float pf[DPS];
#pragma unroll
  for (int d = 0; d < DPS; ++d) pf[d] = 0.f;
  if (zv) {
    p = cfg->src.xyz[p0 + lane];
#pragma unroll
    for (int d = 0; d < DP; ++d)
      pf[d] = load_feat<bf16_of(MODE)>(cfg->src.feat, (size_t)d * cfg->src.m_pad + p0 + lane);
  }
  stage_cluster<STEP, DP, DPS, NU>(sm, warp, lane, zv, p, pf);
  return cs;
}

// One warp's share of a pair pass, streamed from global memory (L2): lane
// sums in acc, counts in nnz / cand. The filtered candidates of each chunk
// are gathered through a ring of 64 entries in the warp's (otherwise unused)
// cache region, with the next block of 32 candidates loading while the
// current chunk runs.
template <bool STEP, int DP, int MODE, int DPS, int NU>
__device__ void pass_stream(const SolveCfg* cfg, SolveSmem<DPS, NU>& sm, int warp, int lane,
                            float* ring, float acc[7], unsigned& nnz, unsigned& cand) {
  const BlockCtx& b = sm.b;
  const GridView& g = cfg->grids[b.level];
  const ClusterView& cv = cfg->clusters[b.level];
  const float rc2 = b.rc2, A = b.A;
  const float rp2 = b.rplan_f * b.rplan_f;
  const WarpRange r = warp_range(b, warp);
  const bool collect = !STEP && b.collect_kept;
  float4* rxyz = reinterpret_cast<float4*>(ring);
  float* rfeat = ring + 4 * 64;
  for (int c = r.c0; c <= r.c1 && c < cv.ncl; ++c) {
    const int tc = __ldcg(&cfg->cl_cand[c]);
    const int fc = __ldcg(&cfg->cl_fcand[c]);
    int jb, je;
    if (!range_chunks(r, c, (fc + 31) >> 5, jb, je)) continue;
    __syncwarp();   // every lane is done with the previous cluster
    const int cs = stage_from_global<STEP, DP, MODE, DPS, NU>(cfg, sm, cv, c, warp, lane);
    const int cs4 = (cs + 3) & ~3;
    const int nseg = load_segments<DPS, NU>(cfg, sm, warp, lane, c, tc, fc);
    const float4 lo = __ldcg(&cfg->cl_box[2 * (size_t)c]);
    const float4 hi = __ldcg(&cfg->cl_box[2 * (size_t)c + 1]);
    FCursor cur = fcursor_at<DPS, NU>(sm, warp, nseg, jb * 32);
    const int want = min(fc, 32 * (je + 1)) - 32 * jb;
    const unsigned nnz0 = nnz;
    if (lo.w == 0.f && !collect && b.compact) {
      // a cluster the plan did not filter (a plan used for one iteration):
      // the candidates of the range's chunks go through the box test here
      // and the survivors are compacted through the ring into full chunks
      // of all source groups. A chunk the range shares with the neighbouring
      // warp (it starts or ends at a source group inside it) runs unfiltered
      // with its own groups, as the plan's numbering of chunks assigns it.
      const int G = cs4 >> 2;
      int glo_b, ghi_b, glo_e, ghi_e;
      range_groups(r, c, jb, G, glo_b, ghi_b);
      range_groups(r, c, je, G, glo_e, ghi_e);
      const bool head = glo_b > 0 || ghi_b < G;
      const bool tail = je != jb && ghi_e < G;
      const auto raw_chunk = [&](int j, int glo, int ghi) {
        FCursor cj = fcursor_at<DPS, NU>(sm, warp, nseg, j * 32);
        float xf[DPS];
        const float4 xp =
            load_candidate<DP, DPS, NU, bf16_of(MODE)>(g, sm, warp, j * 32 + lane, tc, cj.seg, xf);
        if (glo < ghi) {
          const int jlo = 4 * glo, jhi = min(cs4, 4 * ghi);
          if (j * 32 + lane < tc) cand += (unsigned)max(0, min(cs, jhi) - jlo);
          chunk_pairs<STEP, DP, MODE, DPS, NU>(sm, warp, xp, xf, jlo, jhi, rc2, A, acc, nnz);
        }
      };
      if (head) raw_chunk(jb, glo_b, ghi_b);
      const int j0 = head ? jb + 1 : jb, j1 = tail ? je - 1 : je;
      if (j0 <= j1) {
        const int uend = min(tc, 32 * (j1 + 1));
        // a cursor at raw candidate 32 j0 (its segment from the offsets, which
        // count every candidate here), nothing to skip
        FCursor cf = fcursor_at<DPS, NU>(sm, warp, nseg, j0 * 32);
        cf.u = j0 * 32;
        cf.skip = 0;
        float xfn[DPS];
        float4 xpn = load_candidate<DP, DPS, NU, bf16_of(MODE)>(g, sm, warp, cf.u + lane, uend,
                                                                cf.seg, xfn);
        int used = 0;
        for (;;) {
          // place blocks of 32 until a chunk is full or the range is done (at
          // most 63 entries are unread, so the ring never overwrites one)
          while (cf.made - used < 32 && cf.u < uend) {
            const int o = fplace(cf, xpn, lo, hi, rp2, lane, uend);
            if (o >= 0) {
              const int e = o & 63;
              rxyz[e] = xpn;
#pragma unroll
              for (int d = 0; d < DP; ++d) rfeat[d * 64 + e] = xfn[d];
            }
            if (cf.u < uend)
              xpn = load_candidate<DP, DPS, NU, bf16_of(MODE)>(g, sm, warp, cf.u + lane, uend,
                                                               cf.seg, xfn);
          }
          const int cnt = min(32, cf.made - used);
          if (cnt <= 0) break;
          __syncwarp();
          float4 xp = make_float4(-kFar, -kFar, -kFar, 0.f);
          float xf[DPS];
#pragma unroll
          for (int d = 0; d < DPS; ++d) xf[d] = 0.f;
          if (lane < cnt) {
            const int e = (used + lane) & 63;
            xp = rxyz[e];
#pragma unroll
            for (int d = 0; d < DP; ++d) xf[d] = rfeat[d * 64 + e];
            cand += (unsigned)cs;
          }
          __syncwarp();   // read before the next placement reuses the entries
          chunk_pairs<STEP, DP, MODE, DPS, NU>(sm, warp, xp, xf, 0, cs4, rc2, A, acc, nnz);
          used += cnt;
        }
      }
      if (tail) raw_chunk(je, glo_e, ghi_e);
      continue;
    }
    if (lo.w == 0.f) {
      // an unfiltered cluster whose first gradient pass records which source
      // groups kept pairs, chunk by chunk: chunk j holds candidates 32 j ..
      // 32 j + 31, loaded straight into registers, the next chunk's while this
      // one runs
      float xfn[DPS];
      float4 xpn = load_candidate<DP, DPS, NU, bf16_of(MODE)>(g, sm, warp, jb * 32 + lane, tc,
                                                              cur.seg, xfn);
      for (int j = jb; j <= je; ++j) {
        const float4 xp = xpn;
        float xf[DPS];
#pragma unroll
        for (int d = 0; d < DPS; ++d) xf[d] = xfn[d];
        if (j < je)
          xpn = load_candidate<DP, DPS, NU, bf16_of(MODE)>(g, sm, warp, (j + 1) * 32 + lane, tc,
                                                           cur.seg, xfn);
        int glo, ghi;
        range_groups(r, c, j, cs4 >> 2, glo, ghi);
        if (glo < ghi) {
          const int jlo = 4 * glo, jhi = min(cs4, 4 * ghi);
          if (j * 32 + lane < tc) cand += (unsigned)max(0, min(cs, jhi) - jlo);
          const unsigned act =
              chunk_pairs<STEP, DP, MODE, DPS, NU>(sm, warp, xp, xf, jlo, jhi, rc2, A, acc, nnz);
          if (collect) add_active(cfg, c, j, act, lane);
        }
      }
      if (collect) add_kept(cfg, c, nnz - nnz0, lane);
      continue;
    }
    float xfn[DPS];
    float4 xpn = load_candidate<DP, DPS, NU, bf16_of(MODE)>(g, sm, warp, cur.u + lane, tc,
                                                            cur.seg, xfn);
    int used = 0;
    for (int j = jb; j <= je; ++j) {
      const int cnt = min(32, want - used);
      // place blocks until the chunk is complete (at most 63 entries are
      // unread, so the ring never overwrites one)
      while (cur.made - used < cnt && cur.u < tc) {
        const int o = fplace(cur, xpn, lo, hi, rp2, lane, tc);
        if (o >= 0) {
          const int e = o & 63;
          rxyz[e] = xpn;
#pragma unroll
          for (int d = 0; d < DP; ++d) rfeat[d * 64 + e] = xfn[d];
        }
        if (cur.u < tc)
          xpn = load_candidate<DP, DPS, NU, bf16_of(MODE)>(g, sm, warp, cur.u + lane, tc, cur.seg,
                                                           xfn);
      }
      __syncwarp();
      float4 xp = make_float4(-kFar, -kFar, -kFar, 0.f);
      float xf[DPS];
#pragma unroll
      for (int d = 0; d < DPS; ++d) xf[d] = 0.f;
      const bool have = lane < cnt && used + lane < cur.made;
      if (have) {
        const int e = (used + lane) & 63;
        xp = rxyz[e];
#pragma unroll
        for (int d = 0; d < DP; ++d) xf[d] = rfeat[d * 64 + e];
      }
      __syncwarp();   // read before the next placement reuses the entries
      int glo, ghi;
      range_groups(r, c, j, cs4 >> 2, glo, ghi);
      if (glo < ghi) {
        const int jlo = 4 * glo, jhi = min(cs4, 4 * ghi);
        if (have) cand += (unsigned)max(0, min(cs, jhi) - jlo);
        const unsigned act =
            chunk_pairs<STEP, DP, MODE, DPS, NU>(sm, warp, xp, xf, jlo, jhi, rc2, A, acc, nnz);
        if (collect) add_active(cfg, c, j, act, lane);
      }
      used += cnt;
    }
    if (collect) add_kept(cfg, c, nnz - nnz0, lane);
  }
}

// Shared-memory cache of a warp's share of the plan. A slot holds 32 points
// (float4 xyz, then DP feature planes of 32 floats): either the raw centred
// source points of a cluster (header kSlotCluster | cluster size) or the
// candidates of a chunk of filtered candidates (header: number of valid
// candidates | first source group << 6 | end source group << 10; the rest are
// padding points beyond every cutoff). Filled once per plan when the warp's
// whole share fits, so that the passes of every iteration that reuses the
// plan (at the lengthscale floor, most of the solve) read no global memory.
constexpr int kCacheSlots = 32;                 // header capacity per warp
constexpr unsigned short kSlotCluster = 0x8000;
constexpr unsigned short kSlotList = 0x4000;      // cluster slot whose pairs are listed

template <int DP>
__device__ __forceinline__ constexpr int slot_floats() {
  return 32 * (4 + DP);
}

// Pair lists of a plan that will be reused (Verlet-style): for each cached
// cluster, the (candidate, source point) pairs of its cached chunks within
// the plan radius at the plan pose, in slot order and, within a chunk, source
// point by source point. While the plan is valid every source point stays
// within the skin of where it was at the plan pose (the drift test of
// begin_iteration), so these pairs are a superset of the pairs within the
// cutoff, and the passes evaluate only them (each with the exact cutoff test)
// instead of every candidate against every source group. An entry is
// candidate lane | slot << 5 | source point << 10; the lists live in the
// warp's shared scratch (list_max entries). A cluster whose list would not
// fit keeps the chunk-by-chunk evaluation.
template <int DP, int DPS, int NU>
__device__ void build_lists(SolveSmem<DPS, NU>& sm, int warp, int lane, const float* base,
                            int n) {
  unsigned short* pl = sm.ws[warp].list;
  constexpr int kCap = list_max<DPS>();
  const BlockCtx& b = sm.b;
  float R[9], T[3];
#pragma unroll
  for (int i = 0; i < 9; ++i) R[i] = __double2float_rn(b.Rp[i]);
#pragma unroll
  for (int i = 0; i < 3; ++i) T[i] = __double2float_rn(b.Tp[i]);
  const float rp2 = b.rplan_f * b.rplan_f;
  const unsigned lt = (1u << lane) - 1u;
  int run = 0;
  for (int s = 0; s < n; ++s) {
    const unsigned h = sm.cache_hdr[warp][s];
    if (!(h & kSlotCluster)) continue;
    const int cs = (int)(h & 0x3f);
    const float4 p = reinterpret_cast<const float4*>(base + (size_t)s * slot_floats<DP>())[lane];
    const float zx = fmaf(R[0], p.x, fmaf(R[1], p.y, fmaf(R[2], p.z, T[0])));
    const float zy = fmaf(R[3], p.x, fmaf(R[4], p.y, fmaf(R[5], p.z, T[1])));
    const float zz = fmaf(R[6], p.x, fmaf(R[7], p.y, fmaf(R[8], p.z, T[2])));
    const int start = run;
    bool fits = true;
    int t = s + 1;
    for (; t < n && !(sm.cache_hdr[warp][t] & kSlotCluster); ++t) {
      const unsigned hc = sm.cache_hdr[warp][t];
      const int cnt = (int)(hc & 0x3f);
      const int jlo = 4 * (int)((hc >> 6) & 0xf), jhi = min(cs, 4 * (int)((hc >> 10) & 0xf));
      const float4 xp =
          reinterpret_cast<const float4*>(base + (size_t)t * slot_floats<DP>())[lane];
      const bool valid = lane < cnt;
      for (int j = jlo; j < jhi && fits; ++j) {
        const float dx = xp.x - __shfl_sync(kFull, zx, j);
        const float dy = xp.y - __shfl_sync(kFull, zy, j);
        const float dz = xp.z - __shfl_sync(kFull, zz, j);
        const bool in = valid && fmaf(dx, dx, fmaf(dy, dy, dz * dz)) <= rp2;
        const unsigned m = __ballot_sync(kFull, in);
        if (run + __popc(m) > kCap) {
          fits = false;   // warp-uniform
        } else {
          if (in) pl[run + __popc(m & lt)] = (unsigned short)(lane | (t << 5) | (j << 10));
          run += __popc(m);
        }
      }
    }
    if (!fits) run = start;
    if (lane == 0 && fits) {
      sm.cache_hdr[warp][s] = (unsigned short)(h | kSlotList);
      sm.cache_cl[warp][s] |= (run - start) << kListShift;
    }
    s = t - 1;
  }
  __syncwarp();
}

template <int DP, int MODE, int DPS, int NU>
__device__ void fill_cache(const SolveCfg* cfg, SolveSmem<DPS, NU>& sm, int warp, int lane,
                           float* cache, int slots) {
  const BlockCtx& b = sm.b;
  const GridView& g = cfg->grids[b.level];
  const ClusterView& cv = cfg->clusters[b.level];
  const WarpRange r = warp_range(b, warp);
  const float rp2 = b.rplan_f * b.rplan_f;
  // count the slots the share needs
  int need = 0;
  for (int c = r.c0; c <= r.c1 && c < cv.ncl; ++c) {
    int jb, je;
    if (range_chunks(r, c, (__ldcg(&cfg->cl_fcand[c]) + 31) >> 5, jb, je)) need += 2 + je - jb;
  }
  if (need > min(slots, kCacheSlots)) {
    if (lane == 0) sm.cache_n[warp] = -1;
    __syncwarp();
    return;
  }
  float* base = cache + (size_t)warp * slots * slot_floats<DP>();
  int n = 0;
  for (int c = r.c0; c <= r.c1 && c < cv.ncl; ++c) {
    const int tc = __ldcg(&cfg->cl_cand[c]);
    const int fc = __ldcg(&cfg->cl_fcand[c]);
    int jb, je;
    if (!range_chunks(r, c, (fc + 31) >> 5, jb, je)) continue;
    const int p0 = cv.cstart[c];
    const int cs = cv.cstart[c + 1] - p0;
    float* sl = base + (size_t)n * slot_floats<DP>();
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lane < cs) p = cfg->src.xyz[p0 + lane];
    reinterpret_cast<float4*>(sl)[lane] = p;
#pragma unroll
    for (int d = 0; d < DP; ++d)
      sl[128 + d * 32 + lane] =
          lane < cs ? load_feat<bf16_of(MODE)>(cfg->src.feat, (size_t)d * cfg->src.m_pad + p0 + lane)
                    : 0.f;
    if (lane == 0) {
      sm.cache_hdr[warp][n] = (unsigned short)(kSlotCluster | cs);
      sm.cache_cl[warp][n] = c;
    }
    ++n;
    const int nseg = load_segments<DPS, NU>(cfg, sm, warp, lane, c, tc, fc);
    float4 lo = __ldcg(&cfg->cl_box[2 * (size_t)c]);
    float4 hi = __ldcg(&cfg->cl_box[2 * (size_t)c + 1]);
    if (lo.w == 0.f) {   // not filtered by the plan: every candidate of the range is cached
      lo = make_float4(-INFINITY, -INFINITY, -INFINITY, 0.f);
      hi = make_float4(INFINITY, INFINITY, INFINITY, 0.f);
    }
    FCursor cur = fcursor_at<DPS, NU>(sm, warp, nseg, jb * 32);
    const int want = min(fc, 32 * (je + 1)) - 32 * jb;
    float* s0 = base + (size_t)n * slot_floats<DP>();
    while (cur.made < want && cur.u < tc) {
      float xf[DPS];
      const float4 xp =
          load_candidate<DP, DPS, NU, bf16_of(MODE)>(g, sm, warp, cur.u + lane, tc, cur.seg, xf);
      const int o = fplace(cur, xp, lo, hi, rp2, lane, tc);
      if (o >= 0 && o < want) {
        float* sk = s0 + (size_t)(o >> 5) * slot_floats<DP>();
        reinterpret_cast<float4*>(sk)[o & 31] = xp;
#pragma unroll
        for (int d = 0; d < DP; ++d) sk[128 + d * 32 + (o & 31)] = xf[d];
      }
    }
    const int nchk = je - jb + 1;
    for (int o = min(cur.made, want) + lane; o < 32 * nchk; o += 32) {   // padding
      float* sk = s0 + (size_t)(o >> 5) * slot_floats<DP>();
      reinterpret_cast<float4*>(sk)[o & 31] = make_float4(-kFar, -kFar, -kFar, 0.f);
#pragma unroll
      for (int d = 0; d < DP; ++d) sk[128 + d * 32 + (o & 31)] = 0.f;
    }
    if (lane <= je - jb) {
      const int j = jb + lane;
      int glo, ghi;
      range_groups(r, c, j, ((cs + 3) & ~3) >> 2, glo, ghi);
      const int cnt = min(32, want - 32 * lane);
      sm.cache_hdr[warp][n + lane] = (unsigned short)(cnt | (glo << 6) | (ghi << 10));
      sm.cache_cl[warp][n + lane] = j;   // a chunk slot keeps its chunk index
    }
    n += nchk;
    __syncwarp();   // the segment arrays are reused by the next cluster
  }
  if (lane == 0) sm.cache_n[warp] = (short)n;
  __syncwarp();
  if (b.plan_filter) build_lists<DP, DPS, NU>(sm, warp, lane, base, n);
}

// One entry of a cluster's pair list (build_lists) against the staged
// cluster: lane = one (candidate, source point) pair, with the same FP32
// arithmetic as chunk_pairs (the same cutoff test on the same values, so the
// same pairs are kept, and the same weight), the gradient sums formed per pair
// (e = x_l - z_l, z~' x e = x' x e). Returns the kept flag.
template <bool STEP, int DP, int MODE, int DPS, int NU>
__device__ __forceinline__ bool list_pair(SolveSmem<DPS, NU>& sm, int warp, const float* base,
                                          float4 o, unsigned e, bool valid, float rc2, float A,
                                          float acc[7], unsigned& nnz) {
  const int k = (int)(e & 31u), t = (int)((e >> 5) & 31u), j = (int)(e >> 10);
  const float* sl = base + (size_t)t * slot_floats<DP>();
  const float4 xp = reinterpret_cast<const float4*>(sl)[k];
  const float4 m = sm.z[warp][j];
  const float xl = xp.x - o.x, yl = xp.y - o.y, zl = xp.z - o.z;
  const float x2 = fmaf(xl, xl, fmaf(yl, yl, zl * zl));
  const float thr = rc2 - x2;
  const float q0 = A * x2;
  const float tt = fmaf(xl, m.x, fmaf(yl, m.y, fmaf(zl, m.z, m.w)));
  const bool keep = valid && tt <= thr;
  float w;
  if (color_of(MODE) == kColorKernel) {
    float qf = q0;
#pragma unroll
    for (int d = 0; d < DP; ++d) {
      const float df = sl[128 + d * 32 + k] - sm.zf[warp][d][j];
      qf = fmaf(df, df, qf);
    }
    w = ex2_approx(-fmaf(A, tt, qf));
  } else if (color_of(MODE) == kColorDot) {
    float cdot = 0.f;
#pragma unroll
    for (int d = 0; d < DP; ++d) cdot = fmaf(sl[128 + d * 32 + k], sm.zf[warp][d][j], cdot);
    w = ex2_approx(-fmaf(A, tt, q0)) * cdot;
  } else {
    w = ex2_approx(-fmaf(A, tt, q0));
  }
  w = keep ? w : 0.f;
  nnz += keep ? 1u : 0u;
  if (!STEP) {
    // e = x_l - z_l = x_l + m / 2; every term is finite, so w = 0 adds zero
    const float ex = fmaf(0.5f, m.x, xl), ey = fmaf(0.5f, m.y, yl), ez = fmaf(0.5f, m.z, zl);
    acc[0] += w;
    acc[1] = fmaf(w, xp.y * ez - xp.z * ey, acc[1]);
    acc[2] = fmaf(w, xp.z * ex - xp.x * ez, acc[2]);
    acc[3] = fmaf(w, xp.x * ey - xp.y * ex, acc[3]);
    acc[4] = fmaf(w, ex, acc[4]);
    acc[5] = fmaf(w, ey, acc[5]);
    acc[6] = fmaf(w, ez, acc[6]);
  } else {
    const float4 U1 = sm.u[warp][0][j], U2 = sm.u[warp][1 % NU][j];
    const float4 U3 = sm.u[warp][2 % NU][j], U4 = sm.u[warp][3 % NU][j];
    const float beta = fmaf(xl, U1.x, fmaf(yl, U1.y, fmaf(zl, U1.z, U1.w)));
    const float gam = fmaf(xl, U2.x, fmaf(yl, U2.y, fmaf(zl, U2.z, U2.w)));
    const float del = fmaf(xl, U3.x, fmaf(yl, U3.y, fmaf(zl, U3.z, U3.w)));
    const float eps = fmaf(xl, U4.x, fmaf(yl, U4.y, fmaf(zl, U4.z, U4.w)));
    const float b2 = beta * beta;
    const float g2 = fmaf(0.5f, b2, gam);
    const float g3 = fmaf(beta, fmaf(b2, 1.0f / 6.0f, gam), del);
    const float g4 = fmaf(b2 * b2, 1.0f / 24.0f, fmaf(0.5f * gam, b2 + gam, fmaf(beta, del, eps)));
    acc[0] += w;
    acc[1] = keep ? fmaf(w, beta, acc[1]) : acc[1];
    acc[2] = keep ? fmaf(w, g2, acc[2]) : acc[2];
    acc[3] = keep ? fmaf(w, g3, acc[3]) : acc[3];
    acc[4] = keep ? fmaf(w, g4, acc[4]) : acc[4];
  }
  return keep;
}

// A listed cluster (staged): its nl pairs, 64 per round (two per lane, whose
// chains overlap), the next round's entries loading while this one runs. In
// the plan's first gradient pass (collect) the source groups of each chunk that
// kept a pair are gathered per slot: lane t holds slot t's mask in act.
template <bool STEP, int DP, int MODE, int DPS, int NU>
__device__ void list_pairs(SolveSmem<DPS, NU>& sm, int warp, int lane, const float* base,
                           const unsigned short* pl, int nl, float rc2, float A, float acc[7],
                           unsigned& nnz, unsigned& cand, bool collect, unsigned& act) {
  const float4 o = sm.zo[warp];
  unsigned e0 = lane < nl ? pl[lane] : 0u, e1 = lane + 32 < nl ? pl[lane + 32] : 0u;
  for (int r = 0; r < nl; r += 64) {
    const bool v0 = r + lane < nl, v1 = r + 32 + lane < nl;
    const unsigned c0 = e0, c1 = e1;
    e0 = r + 64 + lane < nl ? pl[r + 64 + lane] : 0u;
    e1 = r + 96 + lane < nl ? pl[r + 96 + lane] : 0u;
    cand += (v0 ? 1u : 0u) + (v1 ? 1u : 0u);
    const bool k0 = list_pair<STEP, DP, MODE, DPS, NU>(sm, warp, base, o, c0, v0, rc2, A, acc, nnz);
    const bool k1 = list_pair<STEP, DP, MODE, DPS, NU>(sm, warp, base, o, c1, v1, rc2, A, acc, nnz);
    if (collect) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const bool kk = h ? k1 : k0;
        const unsigned ee = h ? c1 : c0;
        const int ts = (int)((ee >> 5) & 31u);
        const unsigned bit = 1u << (ee >> 12);   // source group j / 4
        unsigned pend = __ballot_sync(kFull, kk);
        while (pend) {
          const int sl = __shfl_sync(kFull, ts, __ffs(pend) - 1);
          const bool mine = kk && ts == sl;
          const unsigned bits = __reduce_or_sync(kFull, mine ? bit : 0u);
          if (lane == sl) act |= bits;
          pend &= ~__ballot_sync(kFull, mine);
        }
      }
    }
  }
}

// The same share as pass_stream, from the warp's cache.
template <bool STEP, int DP, int MODE, int DPS, int NU>
__device__ void pass_cached(const SolveCfg* cfg, SolveSmem<DPS, NU>& sm, int warp, int lane,
                            const float* cache, int slots, float acc[7], unsigned& nnz,
                            unsigned& cand) {
  const float rc2 = sm.b.rc2, A = sm.b.A;
  const bool collect = !STEP && sm.b.collect_kept;
  const float* base = cache + (size_t)warp * slots * slot_floats<DP>();
  const unsigned short* pl = sm.ws[warp].list;
  const int n = sm.cache_n[warp];
  int cs = 0, cs4 = 0, cur = -1, loff = 0;
  unsigned nnz0 = nnz;
  for (int s = 0; s < n; ++s) {
    const unsigned h = sm.cache_hdr[warp][s];
    const float* sl = base + (size_t)s * slot_floats<DP>();
    const float4 p = reinterpret_cast<const float4*>(sl)[lane];
    float f[DPS];
#pragma unroll
    for (int d = 0; d < DPS; ++d) f[d] = d < DP ? sl[128 + d * 32 + lane] : 0.f;
    if (h & kSlotCluster) {
      if (collect) {
        add_kept(cfg, cur, nnz - nnz0, lane);
        nnz0 = nnz;
      }
      cur = sm.cache_cl[warp][s] & ((1 << kListShift) - 1);
      __syncwarp();   // every lane is done with the previous cluster
      cs = (int)(h & 0x3f);
      stage_cluster<STEP, DP, DPS, NU>(sm, warp, lane, lane < cs, p, f);
      cs4 = (cs + 3) & ~3;
      __syncwarp();
      if (h & kSlotList) {
        // the cluster's chunks through its pair list, then past its chunk slots
        int t = s + 1;
        while (t < n && !(sm.cache_hdr[warp][t] & kSlotCluster)) ++t;
        const int nl = (int)((unsigned)sm.cache_cl[warp][s] >> kListShift);
        unsigned act = 0u;
        list_pairs<STEP, DP, MODE, DPS, NU>(sm, warp, lane, base, pl + loff, nl, rc2, A, acc, nnz,
                                            cand, collect, act);
        loff += nl;
        if (collect && lane > s && lane < t && act && cur >= 0) {
          const int j = sm.cache_cl[warp][lane];
          if (j < kActChunks) {
            atomicOr(&cfg->ch_act[(size_t)cur * kActChunks + j], act);
            atomicAdd(&cfg->cl_act[cur], __popc(act));
          }
        }
        s = t - 1;
      }
    } else {
      const int cnt = (int)(h & 0x3f);
      const int jlo = 4 * (int)((h >> 6) & 0xf), jhi = min(cs4, 4 * (int)((h >> 10) & 0xf));
      if (lane < cnt) cand += (unsigned)max(0, min(cs, jhi) - jlo);
      const unsigned act =
          chunk_pairs<STEP, DP, MODE, DPS, NU>(sm, warp, p, f, jlo, jhi, rc2, A, acc, nnz);
      if (collect) add_active(cfg, cur, sm.cache_cl[warp][s], act, lane);
    }
  }
  if (collect) add_kept(cfg, cur, nnz - nnz0, lane);
}

template <bool STEP, int DP, int MODE, int DPS, int NU>
__device__ __forceinline__ void pass_warp(const SolveCfg* cfg, SolveSmem<DPS, NU>& sm, int warp,
                                          int lane, float* cache, int slots, float acc[7],
                                          unsigned& nnz, unsigned& cand) {
  if (sm.cache_n[warp] >= 0)
    pass_cached<STEP, DP, MODE, DPS, NU>(cfg, sm, warp, lane, cache, slots, acc, nnz, cand);
  else
    pass_stream<STEP, DP, MODE, DPS, NU>(cfg, sm, warp, lane,
                                         cache + (size_t)warp * slots * slot_floats<DP>(), acc,
                                         nnz, cand);
}

// One pass over the block's warps, then the block partial (fixed order).
template <bool STEP, int DP, int MODE, int DPS, int NU>
__device__ void run_pass(const SolveCfg* cfg, SolveSmem<DPS, NU>& sm, double* partials,
                         float* cache, int slots) {
  constexpr int NACC = STEP ? 5 : 7;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float acc[7];
#pragma unroll
  for (int i = 0; i < 7; ++i) acc[i] = 0.f;
  unsigned nnz = 0, cand = 0;
  pass_warp<STEP, DP, MODE, DPS, NU>(cfg, sm, warp, lane, cache, slots, acc, nnz, cand);
  __syncwarp();
  if (STEP) {
    // the first warp done with its share forms the FP64 gradient (it reads
    // the gradient totals, which stay in place until the step barrier)
    int first = 0;
    if (lane == 0) first = atomicAdd(&sm.b.fin, 1) == 0 ? 1 : 0;
    if (__shfl_sync(kFull, first, 0)) gradient_fp64(sm.b, sm.sums, lane);
  }
#pragma unroll
  for (int i = 0; i < NACC; ++i) {
    const float v = warp_sum_f(acc[i]);
    if (lane == 0) sm.red[warp][i] = v;
  }
  unsigned wn = nnz, wc = cand;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    wn += __shfl_down_sync(kFull, wn, off);
    wc += __shfl_down_sync(kFull, wc, off);
  }
  if (lane == 0) {
    sm.red[warp][NACC] = __uint_as_float(wn);
    sm.red[warp][NACC + 1] = __uint_as_float(wc);
  }
  __syncthreads();
  if (warp == 0 && lane < NACC + 2) {
    double s = 0.0;
    if (lane < NACC) {
      // the block's eight warp sums in FP32 (fixed order); FP64 starts with the
      // cross-block reduction
      float f = 0.f;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) f += sm.red[w][lane];
      s = (double)f;
    } else {
      unsigned long long n = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) n += __float_as_uint(sm.red[w][lane]);
      s = __longlong_as_double((long long)n);   // a count: its bits, summed as an integer
    }
    partials[(size_t)lane * sm.b.team_size + sm.b.team_rank] = s;
  }
}

__device__ void publish(SolveState* st, BlockCtx& b) {
  form_step_sums(b);
  for (int i = 0; i < 16; ++i) st->P[i] = b.P[i];
  for (int i = 0; i < 6; ++i) st->xi[i] = b.xi[i];
  for (int i = 0; i < 5; ++i) st->S[i] = b.S[i];
  st->xi_norm = b.xi_norm;
  st->F = b.F;
  st->t = b.t;
  st->ell = b.ell;
  st->level = b.level;
  st->iter = b.k;
  st->done = b.done;
  st->converged = b.converged;
  st->fallback_steps = b.fallback;
  st->no_ascent_steps = b.no_ascent;
  st->nnz_total = b.nnz_total;
  st->cand_total = b.cand_total;
  st->nnz_eval = b.nnz_grad;
  st->cand_eval = b.cand_grad;
}

// The whole solve of one pair (or one evaluation) by one team of blocks.
template <int DP, int MODE, int DPS, int NU>
__device__ void solve_pair(const SolveCfg* __restrict__ cfg, SolveState* __restrict__ st,
                           double* __restrict__ partials, IterRecord* __restrict__ records,
                           Team team, SolveSmem<DPS, NU>& sm, bool join, float* cache,
                           int slots) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned gen = 0;
  double* part_g = partials;
  double* part_s = partials + (size_t)team.size * kPartialStride;
  const long long NW = (long long)team.size * kWarps;
  const long long gw = (long long)team.rank * kWarps + warp;

  if (tid == 0) {
    BlockCtx& b = sm.b;
    TailConst& tc = b.tc;
    for (int a = 0; a < 3; ++a) {
      tc.cX[a] = cfg->cX[a];
      tc.cZ[a] = cfg->cZ[a];
    }
    tc.sigma2 = cfg->sigma2;
    tc.inv_a2 = 1.0 / cfg->a2;
    tc.inv_b2 = 1.0 / cfg->b2;
    tc.ell_floor = cfg->ell_floor;
    tc.eps_pose = cfg->eps_pose;
    tc.eps_grad = cfg->eps_grad;
    tc.src_radius = cfg->src_radius;
    tc.mode = cfg->mode;
    tc.step_order = cfg->step_order;
    tc.max_iters = cfg->max_iters;
    tc.reduce_fp32 = cfg->reduce_fp32;
    tc.wait_polls = cfg->wait_polls;
    tc.join_limit_ns = cfg->join_limit_ns;
    for (int a = 0; a < 3; ++a) tc.cXf[a] = (float)cfg->cX[a];
    tc.inv_a2f = (float)(1.0 / cfg->a2);
    tc.inv_b2f = (float)(1.0 / cfg->b2);
    tc.src_radius_f = (float)cfg->src_radius * (1.0f + 1e-6f);
    for (int i = 0; i < 16; ++i) b.P[i] = st->P0[i];
    b.k = 0;
    b.team_rank = team.rank;
    b.team_size = team.size;
    b.level = 0;
    b.plan_level = -1;
    b.plan_filter = 0;
    b.need_plan = 1;
    b.done = cfg->max_iters <= 0 ? 1 : 0;
    b.converged = b.fallback = b.no_ascent = b.have_t_prev = 0;
    b.use_kept = b.collect_kept = b.rebalance = b.use_act = 0;
    b.compact = team.size <= kCompactTeamMax ? 1 : 0;
    b.t = b.t_prev = 0.0;
    b.nnz_total = b.cand_total = b.nnz_grad = b.cand_grad = 0;
    b.F = b.xi_norm = 0.0;
    for (int i = 0; i < 6; ++i) b.xi[i] = 0.0;
    for (int i = 0; i < 5; ++i) b.S[i] = 0.0;
    b.r_plan = 0.0;
    b.plan_ell = 0.0;
  }
  __syncthreads();
  if (warp == 0 && !sm.b.done) begin_iteration(cfg->iters[0], sm.b, lane);
  __syncthreads();
  if (join && !team_join(st, team.size, sm)) {
    if (tid == 0) sm.b.done = 1;   // a team that never assembled runs no iteration
    __syncthreads();
  }
  if (team.rank == 0 && tid == 0) st->t_begin_ns = globaltimer();

  while (!sm.b.done) {
    unsigned long long t0 = 0, t1 = 0, t2 = 0, tg1 = 0, tg2 = 0, ts1 = 0, ts2 = 0;
    const bool stamp = records != nullptr && team.rank == 0 && tid == 0;
    if (stamp) t0 = globaltimer();
    const int replan = sm.b.need_plan;
    // a new plan, or the one rebalance of a plan that is being reused: its
    // work split redone with what its first gradient pass recorded (the source
    // groups that kept pairs; with cost_kept > 0 the kept pairs per cluster)
    const int rebalance = !replan && sm.b.rebalance;
    if (replan || rebalance) {
      const ClusterView& cv = cfg->clusters[sm.b.level];
      if (replan) {
        for (long long c = gw; c < cv.ncl; c += NW)
          plan_cluster(cfg, sm.b, st, (int)c, lane, sm.ws[warp].seg.xs, sm.ws[warp].seg.pf, sm.ws[warp].seg.fpf);
        if (!grid_sync(st, gen, &sm.flag, team.size, sm.b.tc.wait_polls)) break;
      }
      if (tid == 0) {
        sm.b.use_kept = rebalance && cfg->cost_kept > 0.f;
        sm.b.use_act = rebalance && sm.b.plan_filter;
      }
      __syncthreads();
      const int ng = (cv.ncl + 31) / 32;
      for (long long gi = gw; gi < ng; gi += NW) {
        const int c = (int)gi * 32 + lane;
        int kk;
        long long w = c < cv.ncl ? cluster_work(cfg, cv, c, &kk, sm.b.use_kept != 0,
                                                sm.b.use_act != 0)
                                 : 0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) w += __shfl_down_sync(kFull, w, off);
        if (lane == 0) cfg->group_agg[gi] = w;
      }
      if (!grid_sync(st, gen, &sm.flag, team.size, sm.b.tc.wait_polls)) break;
      split_work<DPS, NU>(cfg, sm, tid, team);
      fill_cache<DP, MODE, DPS, NU>(cfg, sm, warp, lane, cache, slots);
      if (tid == 0) {
        sm.b.need_plan = 0;
        sm.b.collect_kept = replan && (cfg->cost_kept > 0.f || sm.b.plan_filter);
        sm.b.rebalance = sm.b.collect_kept;
        if (rebalance) sm.b.rebalance = 0;
      }
      __syncthreads();
    }
    if (stamp) t1 = globaltimer();
    // ---- gradient pass ----
    run_pass<false, DP, MODE, DPS, NU>(cfg, sm, part_g, cache, slots);
    if (stamp) tg1 = globaltimer();
    if (!grid_sync_reduce(st, gen, sm, part_g, 9, team.size)) break;
    if (stamp) tg2 = globaltimer();
    if (warp == 0) {
      if (lane == 0) sm.b.collect_kept = 0;
      gradient_direction(sm.b, sm.sums, lane);
    }
    __syncthreads();
    if (stamp) t2 = globaltimer();
    // ---- step pass ----
    run_pass<true, DP, MODE, DPS, NU>(cfg, sm, part_s, cache, slots);
    if (stamp) ts1 = globaltimer();
    if (!grid_sync_reduce(st, gen, sm, part_s, 7, team.size)) break;
    if (stamp) ts2 = globaltimer();
    if (warp == 0) {
      BlockCtx& b = sm.b;
      const int k = b.k;
      // the next iteration's constants, loaded now and used after the tail
      const IterConst ic_next = cfg->iters[min(k + 1, b.tc.max_iters - 1)];
      const unsigned long long pairs_before = b.nnz_total;
      finish_step(b, sm.sums, lane);
      if (stamp && k < b.tc.max_iters) {
        IterRecord& r = records[k];
        r.ell = b.ell;
        r.t_plan_ns = (float)(t1 - t0);
        r.t_grad_ns = (float)(t2 - t1);
        r.t_step_ns = (float)(globaltimer() - t2);
        r.t_grad_pass_ns = (float)(tg1 - t1);
        r.t_grad_sync_ns = (float)(tg2 - t1);
        r.t_step_pass_ns = (float)(ts1 - t2);
        r.t_step_sync_ns = (float)(ts2 - t2);
        r.replanned = replan;
        r.grad_pairs = (long long)b.nnz_grad;
        r.step_pairs = (long long)(b.nnz_total - pairs_before - b.nnz_grad);
        r.grad_candidates = (long long)b.cand_grad;
      }
      __syncwarp();
      if (!b.done) begin_iteration(ic_next, b, lane);
    }
    __syncthreads();
  }
  if (team.rank == 0 && tid == 0) {
    publish(st, sm.b);
    st->t_end_ns = globaltimer();
  }
  __syncthreads();
}

// The whole solve (or one evaluation) in one cooperative launch: the grid is
// one team.
template <int DP, int MODE>
__global__ void __launch_bounds__(kThreads, CVO_SOLVE_MIN_BLOCKS)
solve_kernel(const SolveCfg* __restrict__ cfg, SolveState* __restrict__ st,
             double* __restrict__ partials, IterRecord* __restrict__ records, int cache_slots) {
  constexpr int DPS = DP > 0 ? DP : 1;
  constexpr int NU = 4;
  __shared__ SolveSmem<DPS, NU> sm;
  extern __shared__ float4 dyn_smem[];
  solve_pair<DP, MODE, DPS, NU>(cfg, st, partials, records, Team{(int)blockIdx.x, (int)gridDim.x},
                                sm, false, reinterpret_cast<float*>(dyn_smem), cache_slots);
}

__device__ __forceinline__ unsigned long long ld_acquire_sys_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_sys_u64(const void* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_sys_s32(int* p, int v) {
  asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Entry fields read at system scope: the entries of a served queue live in
// host memory that the host appends to while the kernel runs.
__device__ QueueEntry load_entry(const QueueEntry* e) {
  static_assert(sizeof(QueueEntry) == 40, "QueueEntry layout");
  QueueEntry r;
  unsigned long long w[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) w[i] = ld_relaxed_sys_u64(reinterpret_cast<const unsigned long long*>(e) + i);
  memcpy(&r, w, sizeof(r));
  return r;
}

// Claim the next slot (thread 0): slots are handed out in order, so every
// slot of an entry is claimed before any slot of a later one. A team whose
// first blocks start before the rest have claimed their slots waits at its
// first barrier; the entries ahead of it never wait on later ones, so the
// blocks they hold come free in bounded time and staff it.
__device__ void claim_slot(const QueueEntry* entries, const QueueCtl* ctl,
                           unsigned long long* head, int* kstatus,
                           unsigned long long idle_limit_ns, long long* slot_out,
                           int* entry_out) {
  const unsigned long long t_start = globaltimer();
  unsigned polls = 0;
  for (;;) {
    const unsigned long long tail = ld_acquire_sys_u64(&ctl->tail);
    const unsigned long long h = atomicAdd(head, 0ull);
    if (h < tail) {
      if (atomicCAS(head, h, h + 1) != h) continue;
      // the entry holding slot h: the last one whose first slot is <= h
      const unsigned long long ne = ld_relaxed_sys_u64(&ctl->n_entries);
      long long lo = 0, hi = (long long)ne;   // invariant: entry lo starts at or before h
      while (hi - lo > 1) {
        const long long mid = (lo + hi) >> 1;
        const QueueEntry em = load_entry(entries + mid);
        if ((unsigned long long)em.slot0 <= h) lo = mid;
        else hi = mid;
      }
      *slot_out = (long long)h;
      *entry_out = (int)lo;
      return;
    }
    if (ld_acquire_sys_u64(&ctl->stop) != 0) break;
    if ((++polls & 63u) == 0 && globaltimer() - t_start > idle_limit_ns) {
      atomicOr(kstatus, (int)kStatusIdleTimeout);
      break;
    }
    __nanosleep(1024);
  }
  *slot_out = -1;
  *entry_out = -1;
}

// Solve results for the host, read at L2 (the team's first block published
// them), the done flag last (release at system scope).
__device__ void write_result(const SolveState* st, PairResult* out) {
  for (int i = 0; i < 16; ++i) out->P[i] = __ldcg(&st->P[i]);
  out->F = __ldcg(&st->F);
  out->t = __ldcg(&st->t);
  out->ell = __ldcg(&st->ell);
  out->device_ms = (double)(__ldcg(&st->t_end_ns) - __ldcg(&st->t_begin_ns)) * 1e-6;
  out->pair_evals = (long long)__ldcg(&st->nnz_total);
  out->candidates = (long long)__ldcg(&st->cand_total);
  out->iters = __ldcg(&st->iter);
  out->converged = __ldcg(&st->converged);
  out->fallback_steps = __ldcg(&st->fallback_steps);
  out->no_ascent_steps = __ldcg(&st->no_ascent_steps);
  out->status = __ldcg(&st->status);
  __threadfence_system();
  st_release_sys_s32(&out->done, 1);
}

// Many pairs in one persistent cooperative launch. Blocks claim slots of a
// queue of entries; the blocks holding the slots of one entry form its team.
template <int DP, int MODE>
__global__ void __launch_bounds__(kThreads, CVO_SOLVE_MIN_BLOCKS)
queue_kernel(const QueueEntry* __restrict__ entries, const QueueCtl* __restrict__ ctl,
             unsigned long long* __restrict__ head, int* __restrict__ kstatus,
             unsigned long long idle_limit_ns, int cache_slots) {
  constexpr int DPS = DP > 0 ? DP : 1;
  constexpr int NU = 4;
  __shared__ SolveSmem<DPS, NU> sm;
  extern __shared__ float4 dyn_smem[];
  for (;;) {
    if (threadIdx.x == 0) {
      long long slot;
      int e;
      claim_slot(entries, ctl, head, kstatus, idle_limit_ns, &slot, &e);
      sm.q_slot = slot;
      sm.q_entry = e;
    }
    __syncthreads();
    if (sm.q_slot < 0) break;
    const QueueEntry en = load_entry(entries + sm.q_entry);
    const Team team{(int)(sm.q_slot - en.slot0), en.team};
    solve_pair<DP, MODE, DPS, NU>(en.cfg, en.st, en.partials, nullptr, team, sm, true,
                                  reinterpret_cast<float*>(dyn_smem), cache_slots);
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned left = atomicAdd(&en.st->leave_count, 1u);
      if (left == (unsigned)en.team - 1 && en.out) {
        __threadfence();
        write_result(en.st, en.out);
      }
    }
    __syncthreads();
  }
}

// Dynamic shared memory of the plan cache: what CVO_SOLVE_MIN_BLOCKS blocks
// per SM leave of the SM's shared memory after their static shared memory,
// in whole warp shares of slots (set once per kernel instantiation).
struct CacheCfg {
  int bytes = 0, slots = 0;
  cudaError_t err = cudaSuccess;
};

template <int DP, int MODE>
const CacheCfg& cache_cfg() {
  static const CacheCfg cfg = [] {
    CacheCfg c;
    int dev = 0, smem_sm = 0, reserved = 0;
    cudaFuncAttributes fa{};
    c.err = cudaGetDevice(&dev);
    if (c.err == cudaSuccess)
      c.err = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (c.err == cudaSuccess)
      c.err = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (c.err == cudaSuccess) c.err = cudaFuncGetAttributes(&fa, solve_kernel<DP, MODE>);
    if (c.err != cudaSuccess) return c;
    const int slot_bytes = 4 * 32 * (4 + DP);
    const int avail = smem_sm / CVO_SOLVE_MIN_BLOCKS - reserved - (int)fa.sharedSizeBytes;
    c.slots = std::max(0, std::min(kCacheSlots, avail / (kWarps * slot_bytes)));
    // the streamed passes gather candidates through two slots of each warp
    if (c.slots < 2) {
      c.err = cudaErrorInvalidConfiguration;
      return c;
    }
    c.bytes = c.slots * kWarps * slot_bytes;
    if (c.bytes > 0) {
      c.err = cudaFuncSetAttribute(solve_kernel<DP, MODE>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, c.bytes);
      if (c.err == cudaSuccess)
        c.err = cudaFuncSetAttribute(queue_kernel<DP, MODE>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, c.bytes);
    }
    return c;
  }();
  return cfg;
}

template <int DP, int MODE>
cudaError_t launch_solve_t(int nblocks, const SolveCfg* cfg, SolveState* st, double* partials,
                           IterRecord* records, cudaStream_t s) {
  const CacheCfg& cc = cache_cfg<DP, MODE>();
  if (cc.err != cudaSuccess) return cc.err;
  int slots = cc.slots;
  void* args[] = {(void*)&cfg, (void*)&st, (void*)&partials, (void*)&records, (void*)&slots};
  return cudaLaunchCooperativeKernel((const void*)solve_kernel<DP, MODE>, dim3(nblocks),
                                     dim3(kThreads), args, (size_t)cc.bytes, s);
}

template <int DP, int MODE>
cudaError_t launch_queue_t(int nblocks, const QueueEntry* entries, const QueueCtl* ctl,
                           unsigned long long* head, int* kstatus, unsigned long long idle_ns,
                           cudaStream_t s) {
  const CacheCfg& cc = cache_cfg<DP, MODE>();
  if (cc.err != cudaSuccess) return cc.err;
  int slots = cc.slots;
  void* args[] = {(void*)&entries, (void*)&ctl,     (void*)&head,
                  (void*)&kstatus, (void*)&idle_ns, (void*)&slots};
  return cudaLaunchCooperativeKernel((const void*)queue_kernel<DP, MODE>, dim3(nblocks),
                                     dim3(kThreads), args, (size_t)cc.bytes, s);
}

template <int DP, int MODE>
int blocks_per_sm_t() {
  const CacheCfg& cc = cache_cfg<DP, MODE>();
  if (cc.err != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, solve_kernel<DP, MODE>, kThreads,
                                                    (size_t)cc.bytes) != cudaSuccess)
    return 0;
  return n;
}

// Launchers of one feature layout (explicitly instantiated, one translation
// unit per feature width, so that the variants compile in parallel).
template <int DP>
cudaError_t launch_solve_dp(int color_mode, int nblocks, const SolveCfg* cfg, SolveState* st,
                            double* partials, IterRecord* records, cudaStream_t s) {
  if constexpr (DP == 0) {
    return launch_solve_t<0, kColorNone>(nblocks, cfg, st, partials, records, s);
  } else {
    switch (color_mode) {
      case kColorKernel:
        return launch_solve_t<DP, kColorKernel>(nblocks, cfg, st, partials, records, s);
      case kColorDot:
        return launch_solve_t<DP, kColorDot>(nblocks, cfg, st, partials, records, s);
      case kColorKernel | kFeatBf16:
        return launch_solve_t<DP, kColorKernel | kFeatBf16>(nblocks, cfg, st, partials, records, s);
      case kColorDot | kFeatBf16:
        return launch_solve_t<DP, kColorDot | kFeatBf16>(nblocks, cfg, st, partials, records, s);
      default:
        return cudaErrorInvalidValue;
    }
  }
}

template <int DP>
cudaError_t launch_queue_dp(int color_mode, int nblocks, const QueueEntry* entries,
                            const QueueCtl* ctl, unsigned long long* head, int* kstatus,
                            unsigned long long idle_limit_ns, cudaStream_t s) {
  if constexpr (DP == 0) {
    return launch_queue_t<0, kColorNone>(nblocks, entries, ctl, head, kstatus, idle_limit_ns, s);
  } else {
    switch (color_mode) {
      case kColorKernel:
        return launch_queue_t<DP, kColorKernel>(nblocks, entries, ctl, head, kstatus,
                                                idle_limit_ns, s);
      case kColorDot:
        return launch_queue_t<DP, kColorDot>(nblocks, entries, ctl, head, kstatus, idle_limit_ns,
                                             s);
      case kColorKernel | kFeatBf16:
        return launch_queue_t<DP, kColorKernel | kFeatBf16>(nblocks, entries, ctl, head, kstatus,
                                                            idle_limit_ns, s);
      case kColorDot | kFeatBf16:
        return launch_queue_t<DP, kColorDot | kFeatBf16>(nblocks, entries, ctl, head, kstatus,
                                                         idle_limit_ns, s);
      default:
        return cudaErrorInvalidValue;
    }
  }
}

template <int DP>
int blocks_per_sm_dp(int color_mode) {
  if constexpr (DP == 0) {
    return blocks_per_sm_t<0, kColorNone>();
  } else {
    switch (color_mode) {
      case kColorKernel: return blocks_per_sm_t<DP, kColorKernel>();
      case kColorDot: return blocks_per_sm_t<DP, kColorDot>();
      case kColorKernel | kFeatBf16: return blocks_per_sm_t<DP, kColorKernel | kFeatBf16>();
      case kColorDot | kFeatBf16: return blocks_per_sm_t<DP, kColorDot | kFeatBf16>();
      default: return 0;
    }
  }
}

}  // namespace

}  // namespace cvo
