// Measured issue peaks of the two pipes the pair passes use, for the roofline
// of the benchmark: FP32 fused multiply-adds and MUFU ex2.approx, each timed
// alone with CUDA events on a kernel that keeps every SM's pipe full (many
// resident warps, eight independent dependency chains per thread, so that
// neither latency nor occupancy limits the issue rate). The SM clock the
// kernel ran at is measured inside it (clock64 against the global timer), so
// the peak can be stated per clock as well. Built with nvcc into
// _build/libpeaks.so and called by bench.py through ctypes.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kChains = 8;

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// kind 0: per thread, iters x kChains dependent FFMAs (a <- a * b + c, |a|
// stays bounded); kind 1: iters x kChains ex2.approx (a <- 2^-a, which stays
// in [0.5, 1]). The sums go to out[] only if a thread's result is exactly
// -1 (never), which keeps the chains alive without a memory write per thread.
// clk[blockIdx] receives (clock64 ticks, global-timer ns) of thread 0.
__global__ void __launch_bounds__(256) peak_kernel(int kind, int iters, float seed,
                                                   float* __restrict__ out,
                                                   long long* __restrict__ clk) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = seed + 0.001f * (float)(threadIdx.x + 7 * k);
  const float b = 0.999f, c = 0.0001f;
  long long c0 = 0, t0 = 0;
  if (threadIdx.x == 0) {
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    c0 = clock64();
  }
  if (kind == 0) {
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int r = 0; r < 16; ++r) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
      }
    }
  } else {
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int r = 0; r < 16; ++r) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = ex2_approx(-a[k]);
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.0f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) {
    long long t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    clk[2 * blockIdx.x] = clock64() - c0;
    clk[2 * blockIdx.x + 1] = t1 - t0;
  }
}

}  // namespace

extern "C" {

// Runs kind (0: FP32 FFMA, 1: MUFU ex2) on `device` with blocks_per_sm
// blocks of 256 threads per SM, `iters` outer iterations (16 x 8
// instructions each per thread), best of `reps` timed launches after one
// warm-up. Results: *inst_per_s thread instructions per second, *sm_mhz the
// median SM clock the blocks saw, *ms the best launch's time, *sms the SM
// count. Returns 0, or the CUDA error code.
int peaks_measure(int device, int kind, int blocks_per_sm, int iters, int reps,
                  double* inst_per_s, double* sm_mhz, double* ms, int* sms) {
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return (int)e;
  int nsm = 0;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return (int)e;
  const int threads = 256;
  const int blocks = nsm * blocks_per_sm;
  float* out = nullptr;
  long long* clk = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double best = 1e30, mhz = 0.0;
  if ((e = cudaMalloc(&out, sizeof(float) * (size_t)blocks * threads)) != cudaSuccess) goto done;
  if ((e = cudaMalloc(&clk, sizeof(long long) * 2 * (size_t)blocks)) != cudaSuccess) goto done;
  if ((e = cudaEventCreate(&ev0)) != cudaSuccess) goto done;
  if ((e = cudaEventCreate(&ev1)) != cudaSuccess) goto done;
  for (int r = 0; r <= reps; ++r) {
    cudaEventRecord(ev0);
    peak_kernel<<<blocks, threads>>>(kind, iters, 0.5f, out, clk);
    cudaEventRecord(ev1);
    if ((e = cudaEventSynchronize(ev1)) != cudaSuccess) goto done;
    if ((e = cudaGetLastError()) != cudaSuccess) goto done;
    float t = 0.f;
    cudaEventElapsedTime(&t, ev0, ev1);
    if (r > 0 && t < best) {
      best = t;
      // median over blocks of clock ticks per global-timer nanosecond
      long long* h = new long long[2 * (size_t)blocks];
      e = cudaMemcpy(h, clk, sizeof(long long) * 2 * (size_t)blocks, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        delete[] h;
        goto done;
      }
      double* f = new double[blocks];
      int nf = 0;
      for (int b = 0; b < blocks; ++b)
        if (h[2 * b + 1] > 0) f[nf++] = 1e3 * (double)h[2 * b] / (double)h[2 * b + 1];
      // insertion sort is enough for a few thousand values
      for (int i = 1; i < nf; ++i)
        for (int j = i; j > 0 && f[j - 1] > f[j]; --j) {
          const double tmp = f[j];
          f[j] = f[j - 1];
          f[j - 1] = tmp;
        }
      mhz = nf > 0 ? f[nf / 2] : 0.0;
      delete[] f;
      delete[] h;
    }
  }
  *inst_per_s = (double)blocks * threads * (double)iters * 16.0 * kChains / (best * 1e-3);
  *sm_mhz = mhz;
  *ms = best;
  *sms = nsm;
done:
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (out) cudaFree(out);
  if (clk) cudaFree(clk);
  return (int)e;
}

}  // extern "C"
