// Cloud preparation kernels: statistics, packing, Morton ordering of source
// clouds and the uniform-grid cell list of target clouds.
//
// The cell list is what makes kernel sparsification (Sec. 5: kernel values
// below 1e-3 are set to zero; Fig. 1 shows the resulting sparse kernel
// matrix) pay off: a source point only visits target cells within the cutoff
// radius r_c = ell sqrt(2 ln(1/kcut)), so a pass costs O(M * neighbours)
// instead of O(N M). Every ordering here is produced by a stable sort, so a
// cloud always packs to the same layout and pair sums are reproducible bit
// for bit.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cvo_internal.cuh"

namespace cvo {

namespace {

inline int blocks_for(int n, int t) { return (n + t - 1) / t; }

constexpr int kSortThreads = 256;   // one thread per 8-bit digit in the histogram and scatter
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;

__global__ void radix_hist_kernel(const uint32_t* __restrict__ keys, int n, int shift,
                                  uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[256];
  const int tid = threadIdx.x;
  h[tid] = 0;
  __syncthreads();
  const int base = blockIdx.x * kSortTile;
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int i = base + r * kSortThreads + tid;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[tid * gridDim.x + blockIdx.x] = h[tid];
}

// In-place exclusive scan of len uint32 values by one block of 1024 threads,
// each owning a contiguous chunk.
__global__ void scan_single_block_kernel(uint32_t* __restrict__ data, int len) {
  __shared__ uint32_t sums[1024];
  const int tid = threadIdx.x;
  const int chunk = (len + 1023) / 1024;
  const int start = tid * chunk;
  const int end = min(len, start + chunk);
  uint32_t local = 0;
  for (int i = start; i < end; ++i) local += data[i];
  sums[tid] = local;
  __syncthreads();
  // Hillis-Steele inclusive scan over the 1024 chunk sums
  for (int off = 1; off < 1024; off <<= 1) {
    uint32_t v = tid >= off ? sums[tid - off] : 0u;
    __syncthreads();
    sums[tid] += v;
    __syncthreads();
  }
  uint32_t run = sums[tid] - local;
  for (int i = start; i < end; ++i) {
    uint32_t v = data[i];
    data[i] = run;
    run += v;
  }
}

static_assert(kSortThreads == 256, "the sort kernels give each digit one thread");

// Sorts of at most this many tiles skip the scan launch: every scatter block
// forms its own digit offsets from the raw histogram.
constexpr int kFusedScanTiles = 64;

// Stable scatter: within a block, elements are ranked in index order
// (round-major, then thread), using match_any for ties inside a warp and
// per-warp digit counts across warps. With `scanned` the histogram holds the
// exclusive scan of the digit-major counts; without, the raw counts (at most
// kFusedScanTiles blocks), which the block scans itself: the offset of digit
// d in block b is the count of smaller digits in all blocks plus the count of
// digit d in the blocks before b.
__global__ void radix_scatter_kernel(const uint32_t* __restrict__ keys,
                                     const uint32_t* __restrict__ vals, int n, int shift,
                                     const uint32_t* __restrict__ hist, bool scanned,
                                     uint32_t* __restrict__ okeys, uint32_t* __restrict__ ovals) {
  __shared__ uint32_t run[256];
  __shared__ uint32_t gbase[256];
  __shared__ uint32_t wc[kSortThreads / 32][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  run[tid] = 0;
  if (scanned) {
    gbase[tid] = hist[tid * gridDim.x + blockIdx.x];
  } else {
    uint32_t tot = 0, before = 0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
      const uint32_t h = hist[tid * gridDim.x + b];
      tot += h;
      before += b < (int)blockIdx.x ? h : 0u;
    }
    // inclusive scan of the 256 digit totals (Hillis-Steele, in run[])
    run[tid] = tot;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
      const uint32_t v = tid >= off ? run[tid - off] : 0u;
      __syncthreads();
      run[tid] += v;
      __syncthreads();
    }
    gbase[tid] = run[tid] - tot + before;
    __syncthreads();
    run[tid] = 0;
  }
#pragma unroll
  for (int w = 0; w < kSortThreads / 32; ++w) wc[w][tid] = 0;
  __syncthreads();
  const int base = blockIdx.x * kSortTile;
  const unsigned lanemask_lt = (1u << lane) - 1u;
  for (int r = 0; r < kSortItems; ++r) {
    const int i = base + r * kSortThreads + tid;
    const bool valid = i < n;
    const uint32_t k = valid ? keys[i] : 0u;
    const uint32_t d = valid ? ((k >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t rank = __popc(peers & lanemask_lt);
    const int leader = __ffs(peers) - 1;
    if (valid && lane == leader) wc[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      uint32_t off = run[d] + rank;
      for (int w = 0; w < warp; ++w) off += wc[w][d];
      const uint32_t pos = gbase[d] + off;
      okeys[pos] = k;
      ovals[pos] = vals[i];
    }
    __syncthreads();
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) {
      tot += wc[w][tid];
      wc[w][tid] = 0;
    }
    run[tid] += tot;
    __syncthreads();
  }
}

// ---- statistics ------------------------------------------------------------

constexpr int kStatThreads = 256;

__global__ void stats_partial_kernel(const float* __restrict__ xyz, const float* __restrict__ feat,
                                     int n, int D, double* __restrict__ psum,
                                     float* __restrict__ plo, float* __restrict__ phi,
                                     int* __restrict__ pbad) {
  __shared__ double ssum[3][kStatThreads];
  __shared__ float slo[3][kStatThreads], shi[3][kStatThreads];
  __shared__ int sbad[kStatThreads];
  const int tid = threadIdx.x;
  double s[3] = {0.0, 0.0, 0.0};
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  int bad = 0;
  for (int i = blockIdx.x * kStatThreads + tid; i < n; i += gridDim.x * kStatThreads) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float v = xyz[3 * (int64_t)i + a];
      if (!isfinite(v)) bad = 1;
      s[a] += (double)v;
      lo[a] = fminf(lo[a], v);
      hi[a] = fmaxf(hi[a], v);
    }
    for (int d = 0; d < D; ++d)
      if (!isfinite(feat[(int64_t)D * i + d])) bad = 1;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    ssum[a][tid] = s[a];
    slo[a][tid] = lo[a];
    shi[a][tid] = hi[a];
  }
  sbad[tid] = bad;
  __syncthreads();
  for (int off = kStatThreads / 2; off > 0; off >>= 1) {
    if (tid < off) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        ssum[a][tid] += ssum[a][tid + off];
        slo[a][tid] = fminf(slo[a][tid], slo[a][tid + off]);
        shi[a][tid] = fmaxf(shi[a][tid], shi[a][tid + off]);
      }
      sbad[tid] |= sbad[tid + off];
    }
    __syncthreads();
  }
  if (tid == 0) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      psum[3 * blockIdx.x + a] = ssum[a][0];
      plo[3 * blockIdx.x + a] = slo[a][0];
      phi[3 * blockIdx.x + a] = shi[a][0];
    }
    pbad[blockIdx.x] = sbad[0];
  }
}

__global__ void stats_final_kernel(const double* __restrict__ psum, const float* __restrict__ plo,
                                   const float* __restrict__ phi, const int* __restrict__ pbad,
                                   int nb, CloudStats* __restrict__ out) {
  if (threadIdx.x != 0) return;
  CloudStats r;
  for (int a = 0; a < 3; ++a) {
    r.sum[a] = 0.0;
    r.lo[a] = INFINITY;
    r.hi[a] = -INFINITY;
  }
  r.bad = 0;
  r.pad = 0;
  for (int b = 0; b < nb; ++b) {  // fixed order: deterministic FP64 sum
    for (int a = 0; a < 3; ++a) {
      r.sum[a] += psum[3 * b + a];
      r.lo[a] = fminf(r.lo[a], plo[3 * b + a]);
      r.hi[a] = fmaxf(r.hi[a], phi[3 * b + a]);
    }
    r.bad |= pbad[b];
  }
  *out = r;
}

template <typename T>
__device__ __forceinline__ T to_feat(float v);
template <>
__device__ __forceinline__ float to_feat<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ __nv_bfloat16 to_feat<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}

template <typename T>
__global__ void pack_kernel(const float* __restrict__ xyz, const float* __restrict__ feat, int n,
                            int D, int dp, int n_pad, double cx, double cy, double cz,
                            float feat_scale, float4* __restrict__ out_xyz,
                            T* __restrict__ out_feat) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pad) return;
  if (i < n) {
    const float x = xyz[3 * (int64_t)i], y = xyz[3 * (int64_t)i + 1], z = xyz[3 * (int64_t)i + 2];
    out_xyz[i] = make_float4((float)((double)x - cx), (float)((double)y - cy),
                             (float)((double)z - cz), 0.0f);
    for (int d = 0; d < dp; ++d)
      out_feat[(int64_t)d * n_pad + i] =
          to_feat<T>(d < D ? feat[(int64_t)D * i + d] * feat_scale : 0.0f);
  } else {
    out_xyz[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int d = 0; d < dp; ++d) out_feat[(int64_t)d * n_pad + i] = to_feat<T>(0.0f);
  }
}

__device__ __forceinline__ uint32_t spread10(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

__device__ __forceinline__ uint32_t quant(float v, float lo, float scale, int levels) {
  float q = floorf((v - lo) * scale);
  q = fminf(fmaxf(q, 0.0f), (float)(levels - 1));
  return (uint32_t)q;
}

__device__ __forceinline__ uint32_t morton_code(float4 p, float lox, float loy, float loz,
                                                float scale) {
  const int L = 1 << kMortonBits;
  const uint32_t qx = quant(p.x, lox, scale, L), qy = quant(p.y, loy, scale, L),
                 qz = quant(p.z, loz, scale, L);
  return spread10(qx) | (spread10(qy) << 1) | (spread10(qz) << 2);
}

__global__ void morton_keys_kernel(const float4* __restrict__ xyz, int n, float lox, float loy,
                                   float loz, float scale, uint32_t* __restrict__ keys,
                                   uint32_t* __restrict__ vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = morton_code(xyz[i], lox, loy, loz, scale);
  vals[i] = (uint32_t)i;
}

// One block of 1024 threads walks the Morton-ordered cloud in tiles. A
// cluster starts where the node prefix changes (a new octree node) or every
// kClusterMax points inside one node; tile carries keep the scan exact.
// One block per requested level (octree depth): block l cuts the Morton-
// ordered points into the clusters of level l.
struct ClusterLevels {
  int shift[kMaxLevels];
  int* cstart[kMaxLevels];
  int* ncl_out[kMaxLevels];
};

__global__ void build_clusters_kernel(const float4* __restrict__ xyz, int n, float lox,
                                      float loy, float loz, float scale, ClusterLevels lv) {
  const int shift = lv.shift[blockIdx.x];
  int* __restrict__ cstart = lv.cstart[blockIdx.x];
  int* __restrict__ ncl_out = lv.ncl_out[blockIdx.x];
  __shared__ int s_a[1024];
  __shared__ int s_b[1024];
  const int tid = threadIdx.x;
  int carry_gs = 0;   // start of the node group open at the end of the last tile
  int carry_cl = 0;   // clusters emitted so far
  for (int base = 0; base < n; base += 1024) {
    const int p = base + tid;
    const bool valid = p < n;
    uint32_t pre = 0u, prev = 0u;
    if (valid) {
      pre = morton_code(xyz[p], lox, loy, loz, scale) >> shift;
      if (p > 0) prev = morton_code(xyz[p - 1], lox, loy, loz, scale) >> shift;
    }
    const bool flag = valid && (p == 0 || pre != prev);
    // inclusive max-scan of group starts
    s_a[tid] = flag ? p : -1;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      const int v = tid >= off ? s_a[tid - off] : -1;
      __syncthreads();
      s_a[tid] = max(s_a[tid], v);
      __syncthreads();
    }
    const int gs = max(s_a[tid], carry_gs);
    const bool newc = valid && (flag || ((p - gs) % kClusterMax) == 0);
    // inclusive sum-scan of cluster starts
    s_b[tid] = newc ? 1 : 0;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
      const int v = tid >= off ? s_b[tid - off] : 0;
      __syncthreads();
      s_b[tid] += v;
      __syncthreads();
    }
    if (newc) cstart[carry_cl + s_b[tid] - 1] = p;
    const int last = min(1023, n - 1 - base);
    const int tile_gs = max(s_a[last], carry_gs);
    const int tile_cl = s_b[last];
    __syncthreads();
    carry_gs = tile_gs;
    carry_cl += tile_cl;
  }
  if (tid == 0) {
    cstart[carry_cl] = n;
    *ncl_out = carry_cl;
  }
}

__global__ void cell_keys_kernel(const float4* __restrict__ xyz, int n, int nx, int ny, int nz,
                                 float ox, float oy, float oz, float inv_h,
                                 uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 p = xyz[i];
  const uint32_t cx = quant(p.x, ox, inv_h, nx), cy = quant(p.y, oy, inv_h, ny),
                 cz = quant(p.z, oz, inv_h, nz);
  keys[i] = cx + (uint32_t)nx * (cy + (uint32_t)ny * cz);
  vals[i] = (uint32_t)i;
}

template <typename T>
__global__ void gather_kernel(const float4* __restrict__ xyz, const T* __restrict__ feat,
                              const uint32_t* __restrict__ perm, int n, int dp, int n_pad,
                              float4* __restrict__ out_xyz, T* __restrict__ out_feat) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_pad) return;
  if (p < n) {
    const uint32_t s = perm[p];
    out_xyz[p] = xyz[s];
    for (int d = 0; d < dp; ++d) out_feat[(int64_t)d * n_pad + p] = feat[(int64_t)d * n_pad + s];
  } else {
    out_xyz[p] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int d = 0; d < dp; ++d) out_feat[(int64_t)d * n_pad + p] = T();
  }
}

// Features are moved as raw 16- or 32-bit values.
void launch_gather(const float4* xyz, const void* feat, const uint32_t* perm, int n, int dp,
                   int n_pad, bool bf16, float4* out_xyz, void* out_feat, cudaStream_t s) {
  if (bf16)
    gather_kernel<uint16_t><<<blocks_for(n_pad, 256), 256, 0, s>>>(
        xyz, static_cast<const uint16_t*>(feat), perm, n, dp, n_pad, out_xyz,
        static_cast<uint16_t*>(out_feat));
  else
    gather_kernel<float><<<blocks_for(n_pad, 256), 256, 0, s>>>(
        xyz, static_cast<const float*>(feat), perm, n, dp, n_pad, out_xyz,
        static_cast<float*>(out_feat));
}

// cell_start[c] = first sorted position whose key is >= c (binary search).
__global__ void cell_start_kernel(const uint32_t* __restrict__ sorted_keys, int n, int ncells,
                                  int* __restrict__ cell_start) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c > ncells) return;
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (sorted_keys[mid] < (uint32_t)c) lo = mid + 1;
    else hi = mid;
  }
  cell_start[c] = lo;
}


}  // namespace

cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, int n, int bits, cudaMemPool_t pool,
                             cudaStream_t s) {
  if (n <= 1) return cudaSuccess;
  const int nb = blocks_for(n, kSortTile);
  uint32_t *k2 = nullptr, *v2 = nullptr, *hist = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&k2, sizeof(uint32_t) * n, pool, s);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&v2, sizeof(uint32_t) * n, pool, s);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&hist, sizeof(uint32_t) * 256 * nb, pool, s);
  uint32_t *ka = keys, *va = vals, *kb = k2, *vb = v2;
  const int passes = (bits + 7) / 8;
  for (int p = 0; p < passes && e == cudaSuccess; ++p) {
    const int shift = 8 * p;
    const bool fused = nb <= kFusedScanTiles;
    radix_hist_kernel<<<nb, kSortThreads, 0, s>>>(ka, n, shift, hist);
    if (!fused) scan_single_block_kernel<<<1, 1024, 0, s>>>(hist, 256 * nb);
    radix_scatter_kernel<<<nb, kSortThreads, 0, s>>>(ka, va, n, shift, hist, !fused, kb, vb);
    e = cudaGetLastError();
    uint32_t* t = ka; ka = kb; kb = t;
    t = va; va = vb; vb = t;
  }
  if (e == cudaSuccess && ka != keys) {
    e = cudaMemcpyAsync(keys, ka, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
  }
  if (k2) cudaFreeAsync(k2, s);
  if (v2) cudaFreeAsync(v2, s);
  if (hist) cudaFreeAsync(hist, s);
  return e;
}

cudaError_t cloud_stats(const float* xyz, const float* feat, int n, int D, CloudStats* d_out,
                        cudaMemPool_t pool, cudaStream_t s) {
  const int nb = min(1024, blocks_for(n, kStatThreads));
  double* psum = nullptr;
  float *plo = nullptr, *phi = nullptr;
  int* pbad = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&psum, sizeof(double) * 3 * nb, pool, s);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&plo, sizeof(float) * 3 * nb, pool, s);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&phi, sizeof(float) * 3 * nb, pool, s);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&pbad, sizeof(int) * nb, pool, s);
  if (e == cudaSuccess) {
    stats_partial_kernel<<<nb, kStatThreads, 0, s>>>(xyz, feat, n, D, psum, plo, phi, pbad);
    stats_final_kernel<<<1, 32, 0, s>>>(psum, plo, phi, pbad, nb, d_out);
    e = cudaGetLastError();
  }
  if (psum) cudaFreeAsync(psum, s);
  if (plo) cudaFreeAsync(plo, s);
  if (phi) cudaFreeAsync(phi, s);
  if (pbad) cudaFreeAsync(pbad, s);
  return e;
}

cudaError_t pack_cloud(const float* xyz, const float* feat, int n, int D, int dp, int n_pad,
                       double cx, double cy, double cz, float feat_scale, bool bf16,
                       float4* out_xyz, void* out_feat, cudaStream_t s) {
  if (bf16)
    pack_kernel<__nv_bfloat16><<<blocks_for(n_pad, 256), 256, 0, s>>>(
        xyz, feat, n, D, dp, n_pad, cx, cy, cz, feat_scale, out_xyz,
        static_cast<__nv_bfloat16*>(out_feat));
  else
    pack_kernel<float><<<blocks_for(n_pad, 256), 256, 0, s>>>(
        xyz, feat, n, D, dp, n_pad, cx, cy, cz, feat_scale, out_xyz, static_cast<float*>(out_feat));
  return cudaGetLastError();
}

MortonFrame morton_frame(const float lo[3], const float hi[3]) {
  MortonFrame mf;
  const float ext = fmaxf(fmaxf(hi[0] - lo[0], hi[1] - lo[1]), hi[2] - lo[2]) * 1.0001f;
  for (int a = 0; a < 3; ++a) mf.lo[a] = lo[a];
  mf.scale = ext > 0.f ? (float)(1 << kMortonBits) / ext : 0.0f;
  mf.cell = ext > 0.f ? ext / (float)(1 << kMortonBits) : 0.0f;
  return mf;
}

cudaError_t morton_order(const float4* xyz, const void* feat, int n, int dp, int n_pad,
                         bool bf16, const MortonFrame& mf, float4* out_xyz, void* out_feat,
                         cudaMemPool_t pool, cudaStream_t s) {
  const float* lo = mf.lo;
  const float scale = mf.scale;
  uint32_t *keys = nullptr, *vals = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&keys, sizeof(uint32_t) * n, pool, s);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&vals, sizeof(uint32_t) * n, pool, s);
  if (e == cudaSuccess) {
    morton_keys_kernel<<<blocks_for(n, 256), 256, 0, s>>>(xyz, n, lo[0], lo[1], lo[2], scale,
                                                          keys, vals);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = radix_sort_pairs(keys, vals, n, 30, pool, s);
  if (e == cudaSuccess) {
    launch_gather(xyz, feat, vals, n, dp, n_pad, bf16, out_xyz, out_feat, s);
    e = cudaGetLastError();
  }
  if (keys) cudaFreeAsync(keys, s);
  if (vals) cudaFreeAsync(vals, s);
  return e;
}

cudaError_t build_clusters(const float4* xyz, int n, const MortonFrame& mf, const float* max_edge,
                           int* const* cstart, int* const* d_ncl, int nlev, cudaStream_t s) {
  if (nlev <= 0) return cudaSuccess;
  if (nlev > kMaxLevels) return cudaErrorInvalidValue;
  ClusterLevels lv{};
  for (int l = 0; l < nlev; ++l) {
    // deepest octree level whose node edge still fits max_edge[l]
    int L = 0;
    float edge = mf.cell * (float)(1 << kMortonBits);
    while (L < kMortonBits && edge > max_edge[l]) {
      edge *= 0.5f;
      ++L;
    }
    lv.shift[l] = 3 * (kMortonBits - L);
    lv.cstart[l] = cstart[l];
    lv.ncl_out[l] = d_ncl[l];
  }
  build_clusters_kernel<<<nlev, 1024, 0, s>>>(xyz, n, mf.lo[0], mf.lo[1], mf.lo[2], mf.scale, lv);
  return cudaGetLastError();
}

cudaError_t build_grid(const float4* xyz, const void* feat, int n, int dp, int n_pad, bool bf16,
                       int nx, int ny, int nz, float ox, float oy, float oz, float h,
                       float4* out_xyz, void* out_feat, int* cell_start, cudaMemPool_t pool,
                       cudaStream_t s) {
  const int ncells = nx * ny * nz;
  int bits = 1;
  while (bits < 32 && (1u << bits) < (uint32_t)ncells) ++bits;
  uint32_t *keys = nullptr, *vals = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync(&keys, sizeof(uint32_t) * n, pool, s);
  if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&vals, sizeof(uint32_t) * n, pool, s);
  if (e == cudaSuccess) {
    cell_keys_kernel<<<blocks_for(n, 256), 256, 0, s>>>(xyz, n, nx, ny, nz, ox, oy, oz, 1.0f / h,
                                                        keys, vals);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = radix_sort_pairs(keys, vals, n, bits, pool, s);
  if (e == cudaSuccess) {
    launch_gather(xyz, feat, vals, n, dp, n_pad, bf16, out_xyz, out_feat, s);
    cell_start_kernel<<<blocks_for(ncells + 1, 256), 256, 0, s>>>(keys, n, ncells, cell_start);
    e = cudaGetLastError();
  }
  if (keys) cudaFreeAsync(keys, s);
  if (vals) cudaFreeAsync(vals, s);
  return e;
}

}  // namespace cvo
