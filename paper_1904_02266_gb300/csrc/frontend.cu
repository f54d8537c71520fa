// Semi-dense front end on the GPU (Sec. 5: the points are the pixels with a
// high intensity gradient, back-projected from the depth image). From a depth
// image and an HSV image it selects, back-projects and describes the points
// the solver aligns, with every step in these kernels:
//
//   pixels     validity (depth in range), intensity gradient of the V channel
//              (central differences, one-sided at the border) and its
//              magnitude, FP32 with one rounding per operation
//   threshold  the valid magnitudes are compacted, radix-sorted on their bit
//              patterns (non-negative floats sort as integers) and the
//              linear-interpolation percentile taken from the order
//              statistics in FP64
//   keep       valid and magnitude > threshold; a device-wide scan ranks the
//              kept pixels in raster order; above max_points the ranks
//              floor(k m / max_points) are kept
//   points     z = depth, x = ((u - cx) / fx) z, y = ((v - cy) / fy) z and the
//              features H, S, V, clip(gx / s), clip(gy / s), FP32
//
// Pixel selection is index work: the kept set and its order are exact, the
// same on any run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "runtime.h"

namespace cvo {

namespace {

constexpr int kScanBlock = 1024;

__device__ __forceinline__ float intensity(const float* hsv, int W, int x, int y) {
  return hsv[3 * ((size_t)y * W + x) + 2];
}

__global__ void fe_pixels_kernel(const float* __restrict__ depth, const float* __restrict__ hsv,
                                 int W, int H, float dmin, float dmax, float* __restrict__ gxo,
                                 float* __restrict__ gyo, float* __restrict__ mag,
                                 int* __restrict__ valid) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= W * H) return;
  const int y = p / W, x = p - y * W;
  float gx, gy;
  if (x == 0) gx = __fsub_rn(intensity(hsv, W, 1, y), intensity(hsv, W, 0, y));
  else if (x == W - 1) gx = __fsub_rn(intensity(hsv, W, W - 1, y), intensity(hsv, W, W - 2, y));
  else gx = __fmul_rn(0.5f, __fsub_rn(intensity(hsv, W, x + 1, y), intensity(hsv, W, x - 1, y)));
  if (y == 0) gy = __fsub_rn(intensity(hsv, W, x, 1), intensity(hsv, W, x, 0));
  else if (y == H - 1) gy = __fsub_rn(intensity(hsv, W, x, H - 1), intensity(hsv, W, x, H - 2));
  else gy = __fmul_rn(0.5f, __fsub_rn(intensity(hsv, W, x, y + 1), intensity(hsv, W, x, y - 1)));
  gxo[p] = gx;
  gyo[p] = gy;
  mag[p] = __fsqrt_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)));
  const float d = depth[p];
  valid[p] = (isfinite(d) && d >= dmin && d <= dmax) ? 1 : 0;
}

// Exclusive scan of one block of kScanBlock flags; block totals to sums[].
__global__ void fe_scan_block_kernel(const int* __restrict__ in, int n, int* __restrict__ out,
                                     int* __restrict__ sums) {
  __shared__ int s[kScanBlock];
  const int t = threadIdx.x;
  const int i = blockIdx.x * kScanBlock + t;
  const int v = i < n ? in[i] : 0;
  s[t] = v;
  __syncthreads();
  for (int off = 1; off < kScanBlock; off <<= 1) {
    const int a = t >= off ? s[t - off] : 0;
    __syncthreads();
    s[t] += a;
    __syncthreads();
  }
  if (i < n) out[i] = s[t] - v;
  if (t == kScanBlock - 1) sums[blockIdx.x] = s[t];
}

// Exclusive scan of the block totals (one block, nb <= kScanBlock); total[0]
// receives the grand total.
__global__ void fe_scan_sums_kernel(int* __restrict__ sums, int nb, int* __restrict__ total) {
  __shared__ int s[kScanBlock];
  const int t = threadIdx.x;
  const int v = t < nb ? sums[t] : 0;
  s[t] = v;
  __syncthreads();
  for (int off = 1; off < kScanBlock; off <<= 1) {
    const int a = t >= off ? s[t - off] : 0;
    __syncthreads();
    s[t] += a;
    __syncthreads();
  }
  if (t < nb) sums[t] = s[t] - v;
  if (t == kScanBlock - 1) *total = s[t];
}

__global__ void fe_scan_add_kernel(int* __restrict__ out, int n, const int* __restrict__ sums) {
  const int i = blockIdx.x * kScanBlock + threadIdx.x;
  if (i < n) out[i] += sums[blockIdx.x];
}

// Magnitudes of the valid pixels, compacted, as sort keys.
__global__ void fe_compact_kernel(const float* __restrict__ mag, const int* __restrict__ valid,
                                  const int* __restrict__ pos, int n, uint32_t* __restrict__ keys,
                                  uint32_t* __restrict__ vals) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n || !valid[p]) return;
  keys[pos[p]] = __float_as_uint(mag[p]);
  vals[pos[p]] = (uint32_t)p;
}

// The linear-interpolation percentile (numpy's 'linear' method) of the sorted
// valid magnitudes, FP64, one thread.
__global__ void fe_threshold_kernel(const uint32_t* __restrict__ sorted, const int* __restrict__ nv,
                                    double q, double* __restrict__ thr) {
  const int n = *nv;
  if (n <= 0) {
    *thr = 0.0;
    return;
  }
  const double h = (double)(n - 1) * (q / 100.0);
  const int lo = (int)floor(h);
  const int hi = min(lo + 1, n - 1);
  const double t = h - (double)lo;
  const double a = (double)__uint_as_float(sorted[lo]), b = (double)__uint_as_float(sorted[hi]);
  const double d = b - a;
  *thr = t < 0.5 ? a + d * t : b - d * (1.0 - t);
}

__global__ void fe_keep_kernel(const float* __restrict__ mag, const int* __restrict__ valid, int n,
                               const double* __restrict__ thr, int* __restrict__ keep) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  keep[p] = (valid[p] && (double)mag[p] > *thr) ? 1 : 0;
}

// Kept pixel of rank r goes to output slot r, or, when m > cap, to the slot k
// with floor(k m / cap) == r (if any).
__global__ void fe_emit_kernel(const float* __restrict__ depth, const float* __restrict__ hsv,
                               const float* __restrict__ gx, const float* __restrict__ gy,
                               const int* __restrict__ keep, const int* __restrict__ rank,
                               const int* __restrict__ m_total, int W, int H, long long cap,
                               float fx, float fy, float cx, float cy, float gs,
                               float* __restrict__ out_xyz, float* __restrict__ out_feat,
                               int* __restrict__ out_pix) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= W * H || !keep[p]) return;
  const long long m = *m_total;
  const long long r = rank[p];
  long long k = r;
  if (cap > 0 && m > cap) {
    k = (r * cap + m - 1) / m;   // smallest k with k m / cap >= r
    if (k >= cap || (k * m) / cap != r) return;
  }
  const int y = p / W, x = p - y * W;
  const float z = depth[p];
  out_xyz[3 * k + 0] = __fmul_rn(__fdiv_rn(__fsub_rn((float)x, cx), fx), z);
  out_xyz[3 * k + 1] = __fmul_rn(__fdiv_rn(__fsub_rn((float)y, cy), fy), z);
  out_xyz[3 * k + 2] = z;
  if (out_feat) {
    out_feat[5 * k + 0] = hsv[3 * (size_t)p + 0];
    out_feat[5 * k + 1] = hsv[3 * (size_t)p + 1];
    out_feat[5 * k + 2] = hsv[3 * (size_t)p + 2];
    out_feat[5 * k + 3] = fminf(fmaxf(__fdiv_rn(gx[p], gs), -1.0f), 1.0f);
    out_feat[5 * k + 4] = fminf(fmaxf(__fdiv_rn(gy[p], gs), -1.0f), 1.0f);
  }
  if (out_pix) out_pix[k] = p;
}

inline int nblocks(long long n, int t) { return (int)((n + t - 1) / t); }

// Exclusive scan of n flags into out; the total lands in d_total (device).
cudaError_t scan_flags(const int* in, int n, int* out, int* sums, int* d_total, cudaStream_t s) {
  const int nb = nblocks(n, kScanBlock);
  fe_scan_block_kernel<<<nb, kScanBlock, 0, s>>>(in, n, out, sums);
  fe_scan_sums_kernel<<<1, kScanBlock, 0, s>>>(sums, nb, d_total);
  fe_scan_add_kernel<<<nb, kScanBlock, 0, s>>>(out, n, sums);
  return cudaGetLastError();
}

// The selection into caller-visible device buffers (context lock held).
// out_xyz / out_feat / out_pix have room for cap points (cap > 0) or for
// every pixel (cap == 0).
int frontend_run(cvo_ctx* ctx, const float* depth, const float* hsv, int W, int H,
                 const cvo_frontend_params& fp, bool on_dev, cudaStream_t us, long long cap,
                 float* out_xyz, float* out_feat, int* out_pix, int64_t* n_out) {
  const long long npix = (long long)W * H;
  if (W < 2 || H < 2 || npix > (long long)kScanBlock * kScanBlock)
    return fail(ctx, CVO_ERR_INVALID_ARG, "image must be at least 2 x 2 and at most 2^20 pixels");
  if (!(fp.fx > 0) || !(fp.fy > 0) || !std::isfinite(fp.cx) || !std::isfinite(fp.cy) ||
      !(fp.depth_min <= fp.depth_max) || !(fp.percentile >= 0.0 && fp.percentile <= 100.0) ||
      !(fp.grad_scale > 0) || fp.max_points < 0)
    return fail(ctx, CVO_ERR_INVALID_ARG, "bad front-end parameters");
  cudaStream_t s = ctx->stream;
  const int n = (int)npix;
  const int nb = nblocks(n, kScanBlock);
  // one scratch allocation carved into 256-byte aligned pieces, sized with the
  // same rounding the carving uses: thr, totals, block sums, the images (when
  // they come from the host), then the per-pixel arrays
  auto round_up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t pix4 = round_up(sizeof(float) * (size_t)n);
  const size_t bytes = round_up(sizeof(double) * 2) + round_up(sizeof(int) * 4) +
                       round_up(sizeof(int) * (size_t)(nb + 1)) +
                       (on_dev ? 0 : pix4 + round_up(sizeof(float) * 3 * (size_t)n)) + 9 * pix4;
  char* scratch = nullptr;
  if (cudaMallocFromPoolAsync((void**)&scratch, bytes, ctx->pool, s) != cudaSuccess)
    return fail(ctx, CVO_ERR_CUDA, "front-end scratch allocation failed");
  char* cur = scratch;
  auto take = [&](size_t b) {
    char* r = cur;
    cur += round_up(b);
    return r;
  };
  double* thr = (double*)take(sizeof(double) * 2);
  int* totals = (int*)take(sizeof(int) * 4);   // [0] valid count, [1] kept count
  int* sums = (int*)take(sizeof(int) * (size_t)(nb + 1));
  const float* d_depth = depth;
  const float* d_hsv = hsv;
  cudaError_t e = cudaSuccess;
  if (!on_dev) {
    float* dd = (float*)take(sizeof(float) * (size_t)n);
    float* dh = (float*)take(sizeof(float) * (size_t)n * 3);
    e = cudaMemcpyAsync(dd, depth, sizeof(float) * (size_t)n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dh, hsv, sizeof(float) * (size_t)n * 3, cudaMemcpyHostToDevice, s);
    d_depth = dd;
    d_hsv = dh;
  } else if (us && us != s) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, us);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev, 0);
    cudaEventDestroy(ev);
  }
  float* gx = (float*)take(sizeof(float) * (size_t)n);
  float* gy = (float*)take(sizeof(float) * (size_t)n);
  float* mag = (float*)take(sizeof(float) * (size_t)n);
  int* valid = (int*)take(sizeof(int) * (size_t)n);
  int* pos = (int*)take(sizeof(int) * (size_t)n);
  int* keep = (int*)take(sizeof(int) * (size_t)n);
  int* rank = (int*)take(sizeof(int) * (size_t)n);
  uint32_t* keys = (uint32_t*)take(sizeof(uint32_t) * (size_t)n);
  uint32_t* vals = (uint32_t*)take(sizeof(uint32_t) * (size_t)n);
  if ((size_t)(cur - scratch) > bytes) {   // the sizing above must cover the carving
    cudaFreeAsync(scratch, s);
    return fail(ctx, CVO_ERR_INTERNAL, "front-end scratch sizing");
  }
  const int T = 256;
  if (e == cudaSuccess) {
    fe_pixels_kernel<<<nblocks(n, T), T, 0, s>>>(d_depth, d_hsv, W, H, (float)fp.depth_min,
                                                 (float)fp.depth_max, gx, gy, mag, valid);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = scan_flags(valid, n, pos, sums, totals + 0, s);
  if (e == cudaSuccess) {
    fe_compact_kernel<<<nblocks(n, T), T, 0, s>>>(mag, valid, pos, n, keys, vals);
    e = cudaGetLastError();
  }
  // the sort needs the count on the host
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->h_int, totals, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  const int n_valid = e == cudaSuccess ? ctx->h_int[0] : 0;
  if (e == cudaSuccess && n_valid > 1) e = radix_sort_pairs(keys, vals, n_valid, 32, ctx->pool, s);
  if (e == cudaSuccess) {
    fe_threshold_kernel<<<1, 1, 0, s>>>(keys, totals + 0, fp.percentile, thr);
    fe_keep_kernel<<<nblocks(n, T), T, 0, s>>>(mag, valid, n, thr, keep);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = scan_flags(keep, n, rank, sums, totals + 1, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->h_int, totals, sizeof(int) * 2, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  const long long m = e == cudaSuccess ? ctx->h_int[1] : 0;
  long long n_emit = m;
  if (fp.max_points > 0 && m > fp.max_points) n_emit = fp.max_points;
  if (e == cudaSuccess && cap > 0 && n_emit > cap) {
    cudaFreeAsync(scratch, s);
    return fail(ctx, CVO_ERR_INVALID_ARG, "output buffers too small for the selected points");
  }
  if (e == cudaSuccess && n_emit > 0) {
    fe_emit_kernel<<<nblocks(n, T), T, 0, s>>>(
        d_depth, d_hsv, gx, gy, keep, rank, totals + 1, W, H, fp.max_points, (float)fp.fx,
        (float)fp.fy, (float)fp.cx, (float)fp.cy, (float)fp.grad_scale, out_xyz, out_feat, out_pix);
    e = cudaGetLastError();
  }
  cudaFreeAsync(scratch, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(ctx, CVO_ERR_CUDA, std::string("front end: ") + cudaGetErrorString(e));
  if (n_valid == 0) return fail(ctx, CVO_ERR_INVALID_ARG, "no pixel has a depth in range");
  *n_out = n_emit;
  return CVO_OK;
}

}  // namespace

}  // namespace cvo

using namespace cvo;

extern "C" {

void cvo_frontend_params_default(cvo_frontend_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->fx = p->fy = 525.0;
  p->cx = 319.5;
  p->cy = 239.5;
  p->depth_min = 0.5;
  p->depth_max = 5.0;
  p->percentile = 80.0;
  p->grad_scale = 0.05;
  p->max_points = 0;
}

int cvo_frontend_select(cvo_ctx* ctx, const float* depth, const float* hsv, int width, int height,
                        const cvo_frontend_params* params, uint32_t flags, void* stream,
                        float* out_xyz, float* out_feat, int32_t* out_pixel, int64_t capacity,
                        int64_t* n_out) {
  if (!ctx) return CVO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!depth || !hsv || !params || !out_xyz || !n_out || capacity <= 0)
    return fail(ctx, CVO_ERR_INVALID_ARG, "NULL pointer or capacity <= 0");
  if (serve_active(ctx))
    return fail(ctx, CVO_ERR_BUSY, "the request loop is running (cvo_serve_stop ends it)");
  CK(cudaSetDevice(ctx->device));
  return frontend_run(ctx, depth, hsv, width, height, *params, (flags & CVO_DEVICE_PTR) != 0,
                      (cudaStream_t)stream, capacity, out_xyz, out_feat, out_pixel, n_out);
}

int cvo_frontend_cloud(cvo_ctx* ctx, const float* depth, const float* hsv, int width, int height,
                       const cvo_frontend_params* params, uint32_t flags, void* stream,
                       int32_t* handle_out, int64_t* n_out) {
  if (!ctx) return CVO_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (!depth || !hsv || !params || !handle_out)
    return fail(ctx, CVO_ERR_INVALID_ARG, "NULL pointer");
  const int D = ctx->prm.color_mode == CVO_COLOR_NONE ? 0 : ctx->prm.feat_dim;
  if (D != 0 && D != 5)
    return fail(ctx, CVO_ERR_INVALID_ARG, "the front end makes 5 features (feat_dim must be 5)");
  if (serve_active(ctx))
    return fail(ctx, CVO_ERR_BUSY, "the request loop is running (cvo_serve_stop ends it)");
  CK(cudaSetDevice(ctx->device));
  const long long npix = (long long)width * height;
  long long cap = params->max_points > 0 ? std::min<long long>(params->max_points, npix) : npix;
  if (width < 2 || height < 2) return fail(ctx, CVO_ERR_INVALID_ARG, "image must be at least 2 x 2");
  float* buf = nullptr;
  if (cudaMallocFromPoolAsync((void**)&buf, sizeof(float) * 8 * (size_t)cap, ctx->pool,
                              ctx->stream) != cudaSuccess)
    return fail(ctx, CVO_ERR_CUDA, "front-end output allocation failed");
  int64_t n = 0;
  int rc = frontend_run(ctx, depth, hsv, width, height, *params, (flags & CVO_DEVICE_PTR) != 0,
                        (cudaStream_t)stream, cap, buf, buf + 3 * cap, nullptr, &n);
  if (rc == CVO_OK && n == 0) rc = fail(ctx, CVO_ERR_INVALID_ARG, "no pixel passes the threshold");
  Cloud* c = nullptr;
  if (rc == CVO_OK)
    rc = create_cloud(ctx, buf, D > 0 ? buf + 3 * cap : nullptr, n, true, ctx->stream, &c);
  cudaFreeAsync(buf, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  if (rc != CVO_OK) return rc;
  *handle_out = add_cloud(ctx, c);
  if (n_out) *n_out = n;
  return CVO_OK;
}

}  // extern "C"
