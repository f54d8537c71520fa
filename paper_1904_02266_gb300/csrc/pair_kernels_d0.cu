// Instantiation of the solve and queue kernels for 0 feature planes
// (the kernels themselves are in pair_kernels.cuh).
#include "pair_kernels.cuh"

namespace cvo {

cudaError_t launch_solve_d0(int color_mode, int nblocks, const SolveCfg* cfg, SolveState* st,
                            double* partials, IterRecord* records, cudaStream_t s) {
  return launch_solve_dp<0>(color_mode, nblocks, cfg, st, partials, records, s);
}

cudaError_t launch_queue_d0(int color_mode, int nblocks, const QueueEntry* entries,
                            const QueueCtl* ctl, unsigned long long* head, int* kstatus,
                            unsigned long long idle_limit_ns, cudaStream_t s) {
  return launch_queue_dp<0>(color_mode, nblocks, entries, ctl, head, kstatus, idle_limit_ns, s);
}

int blocks_per_sm_d0(int color_mode) { return blocks_per_sm_dp<0>(color_mode); }

}  // namespace cvo
