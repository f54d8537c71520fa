// Gradient pass without any device allocation: the all-pairs form of the
// gradient pass (every target point against every source point, same cutoff
// test and same FP32 pair arithmetic as the solve kernel), whose block
// partials live in a fixed, file-scope device array instead of memory the
// library allocates. For callers that must not allocate device memory during
// a call: code running where cudaMalloc is not allowed or not wanted (inside
// a real-time loop with a frozen memory footprint, or a host that owns all
// device memory through its own pool).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/cvo.h"
#include "cvo_internal.cuh"

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaMaxBlocks = 512;      // partial slots in the static scratch
constexpr int kNaStride = 8;           // F, omega'(3), v(3), kept pairs
constexpr int kNaMaxDevices = 64;

// Scratch shared by every call on a device: kNaMaxBlocks block partials
// (32 KB). Held by every GPU that loads the library until the process exits.
__device__ __align__(256) double g_na_partials[kNaMaxBlocks * kNaStride];

std::mutex g_na_mu;
double* g_na_addr[kNaMaxDevices] = {};  // device address of g_na_partials per device
thread_local std::string g_na_err;

struct NaArgs {
  double R[9], T[3];       // pose P = [R T]
  float A;                 // log2(e) / (2 ell^2)
  float rc2;               // cutoff radius squared
  float fscale;            // feature pre-scale
  int n, m, D;
};

__device__ __forceinline__ float na_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Thread per source point (grid-stride); target points staged through shared
// memory in tiles of kNaThreads. Coordinates are taken relative to the first
// target point x0 (differences formed in FP64, then rounded), so FP32 pair
// arithmetic never subtracts large coordinates.
template <int DP, int MODE>
__global__ void __launch_bounds__(kNaThreads)
na_grad_kernel(const float* __restrict__ x, const float* __restrict__ fx,
               const float* __restrict__ z, const float* __restrict__ fz, NaArgs a,
               double* __restrict__ partials) {
  constexpr int DPS = DP > 0 ? DP : 1;
  __shared__ float4 s_x[kNaThreads];
  __shared__ float s_f[DPS][kNaThreads];
  __shared__ double s_red[kNaThreads / 32][7];
  __shared__ unsigned long long s_cnt[kNaThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double x0[3] = {x[0], x[1], x[2]};
  const double z0[3] = {z[0], z[1], z[2]};
  float R[9], T[3];
  for (int r = 0; r < 3; ++r) {
    double tr = a.T[r] - x0[r];
    for (int c = 0; c < 3; ++c) {
      R[3 * r + c] = (float)a.R[3 * r + c];
      tr += a.R[3 * r + c] * z0[c];
    }
    T[r] = (float)tr;   // z~' = R (z - z0) + T', T' = R z0 + T - x0
  }
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  // kept pairs: up to n x m = 2^44 over a block, so 64-bit
  unsigned long long cnt = 0;
  for (int j0 = blockIdx.x * kNaThreads; j0 < a.m; j0 += gridDim.x * kNaThreads) {
    const int j = j0 + tid;
    const bool zv = j < a.m;
    float zx = 0.f, zy = 0.f, zz = 0.f, zf[DPS];
#pragma unroll
    for (int d = 0; d < DPS; ++d) zf[d] = 0.f;
    if (zv) {
      const float px = (float)((double)z[3 * (size_t)j] - z0[0]);
      const float py = (float)((double)z[3 * (size_t)j + 1] - z0[1]);
      const float pz = (float)((double)z[3 * (size_t)j + 2] - z0[2]);
      zx = fmaf(R[0], px, fmaf(R[1], py, fmaf(R[2], pz, T[0])));
      zy = fmaf(R[3], px, fmaf(R[4], py, fmaf(R[5], pz, T[1])));
      zz = fmaf(R[6], px, fmaf(R[7], py, fmaf(R[8], pz, T[2])));
#pragma unroll
      for (int d = 0; d < DP; ++d) zf[d] = d < a.D ? fz[(size_t)a.D * j + d] * a.fscale : 0.f;
    }
    float W = 0.f, Ex = 0.f, Ey = 0.f, Ez = 0.f;
    for (int i0 = 0; i0 < a.n; i0 += kNaThreads) {
      const int i = i0 + tid;
      __syncthreads();
      if (i < a.n) {
        s_x[tid] = make_float4((float)((double)x[3 * (size_t)i] - x0[0]),
                               (float)((double)x[3 * (size_t)i + 1] - x0[1]),
                               (float)((double)x[3 * (size_t)i + 2] - x0[2]), 0.f);
#pragma unroll
        for (int d = 0; d < DP; ++d) s_f[d][tid] = d < a.D ? fx[(size_t)a.D * i + d] * a.fscale : 0.f;
      }
      __syncthreads();
      const int cnt_tile = min(kNaThreads, a.n - i0);
      if (zv) {
        for (int k = 0; k < cnt_tile; ++k) {
          const float4 xp = s_x[k];
          const float ex = xp.x - zx, ey = xp.y - zy, ez = xp.z - zz;
          const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
          if (d2 <= a.rc2) {
            float w;
            if (MODE == cvo::kColorKernel) {
              float q = 0.f;
#pragma unroll
              for (int d = 0; d < DP; ++d) {
                const float df = s_f[d][k] - zf[d];
                q = fmaf(df, df, q);
              }
              w = na_ex2(-fmaf(a.A, d2, q));
            } else if (MODE == cvo::kColorDot) {
              float c = 0.f;
#pragma unroll
              for (int d = 0; d < DP; ++d) c = fmaf(s_f[d][k], zf[d], c);
              w = na_ex2(-a.A * d2) * c;
            } else {
              w = na_ex2(-a.A * d2);
            }
            W += w;
            Ex = fmaf(w, ex, Ex);
            Ey = fmaf(w, ey, Ey);
            Ez = fmaf(w, ez, Ez);
            ++cnt;
          }
        }
      }
    }
    if (zv) {  // omega' += z~' x E, v += E, F += W
      acc[0] += W;
      acc[1] += (double)(zy * Ez - zz * Ey);
      acc[2] += (double)(zz * Ex - zx * Ez);
      acc[3] += (double)(zx * Ey - zy * Ex);
      acc[4] += Ex;
      acc[5] += Ey;
      acc[6] += Ez;
    }
  }
#pragma unroll
  for (int k = 0; k < 7; ++k) {
    double v = acc[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) s_red[warp][k] = v;
  }
  unsigned long long c = cnt;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
  if (lane == 0) s_cnt[warp] = c;
  __syncthreads();
  if (tid < 8) {
    double s = 0.0;
    for (int w = 0; w < kNaThreads / 32; ++w) s += tid < 7 ? s_red[w][tid] : (double)s_cnt[w];
    partials[(size_t)blockIdx.x * kNaStride + tid] = s;
  }
}

// Fixed-order reduction of the block partials and the metric gradient.
__global__ void na_finish_kernel(const double* __restrict__ partials, int nblocks,
                                 const float* __restrict__ x, double sigma2, double inv_l2,
                                 double a2, double b2, double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double s[kNaStride] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = 0; b < nblocks; ++b)
    for (int k = 0; k < kNaStride; ++k) s[k] += partials[(size_t)b * kNaStride + k];
  const double x0[3] = {x[0], x[1], x[2]};
  const double v[3] = {s[4], s[5], s[6]};
  const double cxv[3] = {x0[1] * v[2] - x0[2] * v[1], x0[2] * v[0] - x0[0] * v[2],
                         x0[0] * v[1] - x0[1] * v[0]};
  out[0] = sigma2 * s[0];
  for (int k = 0; k < 3; ++k) {
    out[1 + k] = sigma2 * (s[1 + k] + cxv[k]) * inv_l2 / a2;
    out[4 + k] = sigma2 * v[k] * inv_l2 / b2;
  }
  out[7] = s[7];
}

template <int DP, int MODE>
cudaError_t na_launch(int nblocks, const float* x, const float* fx, const float* z, const float* fz,
                      const NaArgs& a, double* partials, cudaStream_t s) {
  na_grad_kernel<DP, MODE><<<nblocks, kNaThreads, 0, s>>>(x, fx, z, fz, a, partials);
  return cudaGetLastError();
}

int na_fail(int code, const char* msg) {
  g_na_err = msg;
  return code;
}

}  // namespace

extern "C" int cvo_eval_gradient_static(const float* d_x, const float* d_fx, int64_t n,
                                        const float* d_z, const float* d_fz, int64_t m,
                                        const cvo_params* params, const double P[16], double ell,
                                        double* d_out, void* stream) {
  g_na_err.clear();
  if (!d_x || !d_z || !d_out || !params || !P)
    return na_fail(CVO_ERR_INVALID_ARG, "NULL pointer argument");
  if (n < 1 || m < 1 || n > cvo::kMaxPoints || m > cvo::kMaxPoints)
    return na_fail(CVO_ERR_INVALID_ARG, "point count outside [1, 2^22]");
  const cvo_params& p = *params;
  if (!(ell > 0.0) || !std::isfinite(ell) || !(p.kcut > 0.0 && p.kcut < 1.0) || !(p.sigma > 0.0) ||
      !(p.a2 > 0.0) || !(p.b2 > 0.0) || p.feat_dim < 0 || p.feat_dim > CVO_MAX_FEAT)
    return na_fail(CVO_ERR_INVALID_ARG, "invalid parameters");
  if (p.color_mode != CVO_COLOR_NONE && p.color_mode != CVO_COLOR_KERNEL &&
      p.color_mode != CVO_COLOR_DOT)
    return na_fail(CVO_ERR_INVALID_ARG, "color_mode must be CVO_COLOR_NONE, _KERNEL or _DOT");
  if (p.color_mode == CVO_COLOR_KERNEL && p.feat_dim > 0 &&
      !(p.ell_color > 0.0 && std::isfinite(p.ell_color)))
    return na_fail(CVO_ERR_INVALID_ARG, "ell_color must be finite and > 0");
  if (p.color_mode == CVO_COLOR_DOT && p.feat_dim > 0 &&
      !(p.color_scale > 0.0 && std::isfinite(p.color_scale)))
    return na_fail(CVO_ERR_INVALID_ARG, "color_scale must be finite and > 0");
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(P[i])) return na_fail(CVO_ERR_INVALID_ARG, "pose has a non-finite entry");
  int mode = p.color_mode;
  int D = p.feat_dim;
  if (mode == CVO_COLOR_NONE || D == 0) {
    mode = CVO_COLOR_NONE;
    D = 0;
  } else if (!d_fx || !d_fz) {
    return na_fail(CVO_ERR_INVALID_ARG, "NULL feature pointer");
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices)
    return na_fail(CVO_ERR_CUDA, "no usable current device");
  double* partials = nullptr;
  {
    // one-time set-up per device: the device address of the static scratch
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, g_na_partials);
      if (e != cudaSuccess) return na_fail(CVO_ERR_CUDA, cudaGetErrorString(e));
      g_na_addr[dev] = static_cast<double*>(ptr);
    }
    partials = g_na_addr[dev];
  }
  NaArgs a{};
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) a.R[3 * r + c] = P[4 * r + c];
    a.T[r] = P[4 * r + 3];
  }
  const double ell2 = ell * ell;
  a.A = (float)(1.4426950408889634 / (2.0 * ell2));
  a.rc2 = (float)(2.0 * ell2 * std::log(1.0 / p.kcut));
  a.fscale = mode == CVO_COLOR_KERNEL
                 ? (float)std::sqrt(1.4426950408889634 / (2.0 * p.ell_color * p.ell_color))
                 : mode == CVO_COLOR_DOT ? (float)std::sqrt(p.color_scale) : 1.0f;
  a.n = (int)n;
  a.m = (int)m;
  a.D = D;
  const int nblocks = (int)std::min<int64_t>((m + kNaThreads - 1) / kNaThreads, kNaMaxBlocks);
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  const int dp = D == 0 ? 0 : D <= 3 ? 3 : D <= 5 ? 5 : 8;
  if (mode == CVO_COLOR_NONE) e = na_launch<0, cvo::kColorNone>(nblocks, d_x, d_fx, d_z, d_fz, a, partials, s);
  else if (mode == CVO_COLOR_KERNEL)
    e = dp == 3 ? na_launch<3, cvo::kColorKernel>(nblocks, d_x, d_fx, d_z, d_fz, a, partials, s)
      : dp == 5 ? na_launch<5, cvo::kColorKernel>(nblocks, d_x, d_fx, d_z, d_fz, a, partials, s)
                : na_launch<8, cvo::kColorKernel>(nblocks, d_x, d_fx, d_z, d_fz, a, partials, s);
  else
    e = dp == 3 ? na_launch<3, cvo::kColorDot>(nblocks, d_x, d_fx, d_z, d_fz, a, partials, s)
      : dp == 5 ? na_launch<5, cvo::kColorDot>(nblocks, d_x, d_fx, d_z, d_fz, a, partials, s)
                : na_launch<8, cvo::kColorDot>(nblocks, d_x, d_fx, d_z, d_fz, a, partials, s);
  if (e != cudaSuccess) return na_fail(CVO_ERR_CUDA, cudaGetErrorString(e));
  na_finish_kernel<<<1, 32, 0, s>>>(partials, nblocks, d_x, p.sigma * p.sigma, 1.0 / ell2, p.a2,
                                    p.b2, d_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(CVO_ERR_CUDA, cudaGetErrorString(e));
  return CVO_OK;
}

// Detail message of the last failed context-free call on this host thread.
const char* cvo_static_last_error() { return g_na_err.c_str(); }
