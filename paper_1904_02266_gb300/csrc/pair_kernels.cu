// Dispatch of the solve and queue kernels by feature layout. The kernels are
// in pair_kernels.cuh, instantiated per feature width in pair_kernels_d*.cu.
#include <cuda_runtime.h>

#include "cvo_internal.cuh"

namespace cvo {

#define CVO_DECLARE_DP(D)                                                                    \
  cudaError_t launch_solve_d##D(int color_mode, int nblocks, const SolveCfg* cfg,            \
                                SolveState* st, double* partials, IterRecord* records,       \
                                cudaStream_t s);                                             \
  cudaError_t launch_queue_d##D(int color_mode, int nblocks, const QueueEntry* entries,      \
                                const QueueCtl* ctl, unsigned long long* head, int* kstatus, \
                                unsigned long long idle_limit_ns, cudaStream_t s);           \
  int blocks_per_sm_d##D(int color_mode);
CVO_DECLARE_DP(0)
CVO_DECLARE_DP(3)
CVO_DECLARE_DP(5)
CVO_DECLARE_DP(8)
#undef CVO_DECLARE_DP

cudaError_t launch_solve(int dp, int color_mode, int nblocks, const SolveCfg* cfg, SolveState* st,
                         double* partials, IterRecord* records, cudaStream_t s) {
  if (color_of(color_mode) == kColorNone || dp == 0)
    return launch_solve_d0(kColorNone, nblocks, cfg, st, partials, records, s);
  if (dp == 3) return launch_solve_d3(color_mode, nblocks, cfg, st, partials, records, s);
  if (dp == 5) return launch_solve_d5(color_mode, nblocks, cfg, st, partials, records, s);
  return launch_solve_d8(color_mode, nblocks, cfg, st, partials, records, s);
}

cudaError_t launch_queue(int dp, int color_mode, int nblocks, const QueueEntry* entries,
                         const QueueCtl* ctl, unsigned long long* head, int* kstatus,
                         unsigned long long idle_limit_ns, cudaStream_t s) {
  if (color_of(color_mode) == kColorNone || dp == 0)
    return launch_queue_d0(kColorNone, nblocks, entries, ctl, head, kstatus, idle_limit_ns, s);
  if (dp == 3)
    return launch_queue_d3(color_mode, nblocks, entries, ctl, head, kstatus, idle_limit_ns, s);
  if (dp == 5)
    return launch_queue_d5(color_mode, nblocks, entries, ctl, head, kstatus, idle_limit_ns, s);
  return launch_queue_d8(color_mode, nblocks, entries, ctl, head, kstatus, idle_limit_ns, s);
}

int solve_blocks_per_sm(int dp, int color_mode) {
  if (color_of(color_mode) == kColorNone || dp == 0) return blocks_per_sm_d0(kColorNone);
  if (dp == 3) return blocks_per_sm_d3(color_mode);
  if (dp == 5) return blocks_per_sm_d5(color_mode);
  return blocks_per_sm_d8(color_mode);
}

}  // namespace cvo
