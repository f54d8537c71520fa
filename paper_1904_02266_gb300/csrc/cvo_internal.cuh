// Internal types shared by the CUDA translation units of libcvo.
//
// Frames: every cloud is stored centred on its own FP64 centroid (target
// centroid cX, source centroid cZ) so that FP32 pair arithmetic never
// subtracts two large coordinates. A source point z' (centred) is mapped into
// the target's centred frame by z~' = R z' + T' with T' = R cZ + T - cX; the
// gradient is mapped back to the frame P acts in by omega = omega' + cX x v
// (exact, since z~ = z~' + cX).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cvo {

// Warps per block of the pair passes: one block of 16 warps per SM (all 64K
// registers at 128 a thread), so that the team barriers reduce one partial
// per SM rather than two (on GB300 that FP64 reduction runs at about 64 cycles
// per warp instruction) at the same 16 warps per SM.
#ifndef CVO_WARPS
#define CVO_WARPS 16
#endif
constexpr int kWarps = CVO_WARPS;
constexpr int kThreads = kWarps * 32;     // threads per block
constexpr int kMaxLevels = 8;             // target cell lists one solve may use
// a new cell list (and cluster size) starts when the cutoff radius has
// shrunk to this fraction of the one the current list was built for
#ifndef CVO_LEVEL_RATIO
#define CVO_LEVEL_RATIO 0.5
#endif
constexpr int kMaxFeatPad = 8;            // padded feature planes (3, 5 or 8)
constexpr int kMaxPoints = 1 << 22;       // largest cloud (keeps candidate counts in int32)
constexpr int kMaxCells = 1 << 22;        // largest cell list
constexpr int kPartialStride = 10;        // values per block partial (stored value-major)
constexpr int kClusterMax = 32;           // source points per cluster
constexpr int kMaxSeg = 64;               // cell-row segments per cluster
constexpr int kMortonBits = 10;           // Morton quantisation per axis

enum : int { kColorNone = 0, kColorKernel = 1, kColorDot = 2 };
// Kernel mode = label product | kFeatBf16 when feature planes hold BF16 values.
constexpr int kFeatBf16 = 4;
__host__ __device__ constexpr int color_of(int mode) { return mode & 3; }
__host__ __device__ constexpr bool bf16_of(int mode) { return (mode & kFeatBf16) != 0; }
enum : int { kModeAlign = 0, kModeEval = 1 };
enum : int { kStatusSegOverflow = 1, kStatusTimeout = 2 };   // bits of SolveState::status
enum : int { kStatusIdleTimeout = 4 };   // queue kernel: a block gave up waiting for entries

// One uniform-grid cell list over a target cloud (Sec. 5 sparsification:
// only cells within the cutoff radius of a source point are visited).
struct GridView {
  const float4* xyz;       // n points sorted by cell (x fastest), centred; w unused
  const float* feat;       // dp planes of n_pad values (FP32, or BF16 in bf16 mode), same order,
                           // pre-scaled
  const int* cell_start;   // ncells + 1 offsets into xyz
  int n, n_pad;
  int nx, ny, nz;
  float ox, oy, oz;        // origin of cell (0,0,0), centred frame
  float h, inv_h;          // cell edge and its inverse
};

// Source points in Morton order, cut into spatially bounded clusters
// (octree nodes of the source's own frame, at most kClusterMax points).
struct ClusterView {
  const int* cstart;       // ncl + 1 offsets into the Morton-ordered source
  int ncl;
};

struct SourceView {
  const float4* xyz;       // m points, Morton order, centred
  const float* feat;       // dp planes of m_pad values (FP32 or BF16), pre-scaled
  int m, m_pad;
};

// Constants of one iteration, precomputed on the host from the lengthscale.
struct IterConst {
  double ell;              // lengthscale
  double inv_l2;           // 1 / ell^2
  float A;                 // log2(e) / (2 ell^2)
  float rc2;               // cutoff radius squared
  float rprune;            // traversal radius (r_c widened by 1e-3 relative)
  int level;               // grid / cluster level
  int filter;              // 1: a plan built at this iteration filters its candidates (the
                           //   next iteration keeps the lengthscale, so the plan is reused;
                           //   or an evaluation)
  int at_floor;            // 1: ell is the schedule's floor (the stop test may fire)
  double kf_rot, kf_tr;    // sigma^2 / (ell^2 a^2) and sigma^2 / (ell^2 b^2): the factors that
                           //   turn the pair sums into the metric gradient (Eq. metric)
};

// Constant for one solve plan (device memory).
struct SolveCfg {
  GridView grids[kMaxLevels];
  ClusterView clusters[kMaxLevels];
  SourceView src;
  const IterConst* iters;  // one entry per iteration (one in eval mode)
  // per-iteration work buffers, sized for the largest level
  int* seg_xs;             // first target index of each segment, ncl_max * kMaxSeg
  int* seg_pref;           // candidate offset of each segment in its cluster
  int* cl_nseg;            // segments per cluster
  int* cl_cand;            // candidates per cluster (every point of its segments)
  int* seg_fpref;          // offset of each segment among the cluster's filtered candidates
  int* cl_fcand;           // filtered candidates per cluster: those within the plan radius
                           //   of the cluster's bounding box
  float4* cl_box;          // per cluster: bounding box of its transformed points at the
                           //   plan pose (lo, hi)
  int* cl_kept;            // kept pairs per cluster in the first gradient pass of a plan
  unsigned* ch_act;        // per cluster, 32 words: bit g of word j is set when source group g
                           //   of chunk j kept a pair in the plan's first gradient pass
  int* cl_act;             // per cluster: the number of such bits
  long long* group_agg;    // work of each group of 32 consecutive clusters
  double src_radius;       // max |z'| over the centred source (bounds pose drift)
  int cost_chunk;          // work model: a chunk costs cs4 + cost_chunk pair tests,
  int cost_cluster;        //   staging a cluster cost_cluster, and once kept pairs are
  float cost_kept;         //   known cost_kept per kept pair (spread over the chunks)
  double cX[3], cZ[3];     // FP64 centroids
  double sigma2, a2, b2;
  double ell_floor, eps_pose, eps_grad;
  int max_iters, step_order, mode;
  int reduce_fp32;         // precision study: block and cross-block sums in FP32
  unsigned wait_polls;     // team barrier: polls before a block gives up
  unsigned long long join_limit_ns;   // queued team: longest wait for its blocks to start
};

// Mutable state of one solve (device memory). The host writes the input
// block (P0) before a launch and reads the rest after.
struct SolveState {
  // inputs
  double P0[16];
  // pose and last pass results
  double P[16];
  double xi[6];              // metric gradient at P
  double xi_norm;
  double F;                  // F at P (gradient pass)
  double S[5];               // step sums along xi
  double t, t_prev;
  double ell;                // lengthscale of the current iteration
  int level;                 // level of the current iteration
  int iter, done, converged;
  int fallback_steps, no_ascent_steps, have_t_prev, status;
  unsigned long long nnz_total, cand_total;
  unsigned long long nnz_pass[2], cand_pass[2];
  unsigned long long nnz_eval, cand_eval;   // gradient pass of the last iteration
  unsigned int bar_count;                   // grid barrier: arrivals (zeroed before each launch)
  unsigned int join_count, leave_count;     // queued solves: blocks of the team that have started
                                            // and that are done with the entry
  unsigned long long t_begin_ns, t_end_ns;  // global timer at the start and end of the solve
};

// Per-iteration record of a profiled solve (device timestamps).
struct IterRecord {
  double ell;
  float t_plan_ns, t_grad_ns, t_step_ns;     // %globaltimer intervals on block 0
  float t_grad_pass_ns, t_grad_sync_ns;      // sub-phases of the gradient interval:
  float t_step_pass_ns, t_step_sync_ns;      //   block 0's own pass, and pass + barrier
  int replanned;
  long long grad_pairs, step_pairs, grad_candidates;
};

// Result of one queued solve as the host reads it (host-mapped memory for a
// served request): written after the solve is published, `done` last.
struct PairResult {
  double P[16];
  double F, t, ell;
  double device_ms;
  long long pair_evals, candidates;
  int iters, converged, fallback_steps, no_ascent_steps, status;
  int done;
};

// One pair of a queue. Entries are appended in slot order: entry e owns the
// `team` slots starting at slot0 (the sum of the team sizes before it).
struct QueueEntry {
  const SolveCfg* cfg;
  SolveState* st;            // zeroed, with P0 set, before the entry is published
  double* partials;          // 2 * team * kPartialStride doubles (see launch_solve)
  PairResult* out;           // NULL: the host reads st after the launch; else written by the
                             // team's last block to finish, so that no block of the team
                             // touches the entry once out->done is set
  int team, slot0;
};

// Queue control words (device memory for a batch, host-mapped for serving).
// The host writes entries, then n_entries, then tail (release order).
struct QueueCtl {
  unsigned long long tail;       // published slots
  unsigned long long n_entries;  // published entries
  unsigned long long stop;       // nonzero: nothing more comes; blocks leave once all is claimed
};

// ---- grid.cu --------------------------------------------------------------
// Temporaries are drawn from `pool`, stream-ordered on s.
// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of key.
cudaError_t radix_sort_pairs(uint32_t* keys, uint32_t* vals, int n, int bits,
                             cudaMemPool_t pool, cudaStream_t s);

struct CloudStats {
  double sum[3];
  float lo[3], hi[3];
  int bad;
  int pad;
};
// FP64 sum, FP32 bounding box and a non-finite check of a raw cloud.
cudaError_t cloud_stats(const float* xyz, const float* feat, int n, int D,
                        CloudStats* d_out, cudaMemPool_t pool, cudaStream_t s);

// Centre, pack (float4 xyz) and pre-scale features into dp SoA planes of FP32
// values, or of BF16 values (round to nearest even of the scaled FP32 value)
// when bf16.
cudaError_t pack_cloud(const float* xyz, const float* feat, int n, int D, int dp, int n_pad,
                       double cx, double cy, double cz, float feat_scale, bool bf16,
                       float4* out_xyz, void* out_feat, cudaStream_t s);

// Morton quantisation shared by the source ordering and its clusters.
struct MortonFrame {
  float lo[3];
  float scale;             // quantisation cells per metre
  float cell;              // edge of one quantisation cell
};
MortonFrame morton_frame(const float lo[3], const float hi[3]);

// Reorder a packed cloud along a Morton curve of its bounding box.
cudaError_t morton_order(const float4* xyz, const void* feat, int n, int dp, int n_pad,
                         bool bf16, const MortonFrame& mf, float4* out_xyz, void* out_feat,
                         cudaMemPool_t pool, cudaStream_t s);

// Cut a Morton-ordered cloud into clusters, for nlev (<= kMaxLevels) cluster
// sizes in one launch: for level l, runs sharing the Morton prefix of an
// octree node with edge <= max_edge[l], split into runs of <= kClusterMax;
// cstart[l] receives ncl + 1 offsets (capacity n + 1), *d_ncl[l] the count.
cudaError_t build_clusters(const float4* xyz, int n, const MortonFrame& mf, const float* max_edge,
                           int* const* cstart, int* const* d_ncl, int nlev, cudaStream_t s);

// Build a cell list of edge h over a packed cloud.
cudaError_t build_grid(const float4* xyz, const void* feat, int n, int dp, int n_pad, bool bf16,
                       int nx, int ny, int nz, float ox, float oy, float oz, float h,
                       float4* out_xyz, void* out_feat, int* cell_start, cudaMemPool_t pool,
                       cudaStream_t s);

// ---- pair_kernels.cu -------------------------------------------------------
// The whole solve (or one evaluation, cfg->mode == kModeEval) as one
// cooperative launch of nblocks blocks; partials holds 2 * nblocks *
// kPartialStride doubles, the gradient pass's block partials then the step
// pass's, each value-major (value i of block b at i * nblocks + b, so that the
// reduction reads each value's partials as one contiguous run); records (may
// be NULL) one entry per iteration.
cudaError_t launch_solve(int dp, int color_mode, int nblocks, const SolveCfg* cfg, SolveState* st,
                         double* partials, IterRecord* records, cudaStream_t s);
// color_mode below is the kernel mode: the label product | kFeatBf16.
// Many pairs in one cooperative launch of nblocks blocks (queue_kernel):
// blocks claim slots through *head (zeroed before the launch) until the queue
// is drained and ctl->stop is set, or until they have waited idle_limit_ns for
// an entry (then *kstatus gets kStatusIdleTimeout).
cudaError_t launch_queue(int dp, int color_mode, int nblocks, const QueueEntry* entries,
                         const QueueCtl* ctl, unsigned long long* head, int* kstatus,
                         unsigned long long idle_limit_ns, cudaStream_t s);
// Co-resident blocks per SM of the solve kernel for this feature layout.
int solve_blocks_per_sm(int dp, int color_mode);

}  // namespace cvo
