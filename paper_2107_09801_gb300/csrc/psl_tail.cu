// psl_tail.cu -- the step after the neighbourhood score for batches of short walks
// (arXiv 2107.09801, Algorithm 1): one block per walk runs selection, exact re-check,
// decision and update back to back.  Its own translation unit, compiled in parallel.
#include <cstdint>

#include "psl_device.cuh"
#include "psl_internal.h"
#include "psl_step.cuh"

namespace psl {

// ------------------------------------------------------------------------------------
// the step after the neighbourhood score for batches of short walks (every walk with one
// update chunk, one re-check chunk and a window selected by one warp): one block per walk
// runs selection, exact re-check, decision and update back to back, instead of four
// launches of latency-bound kernels
// ------------------------------------------------------------------------------------
// Blocks of one warp: each walk's chain of phases is bound by latency, so the more walks an
// SM holds at once the better.  Measured at L = 1023 x 4096: 256 threads, 3 blocks per SM
// 0.230 ms per step; 64 threads at 80 registers, 12 blocks 0.108 ms (then, after the shared
// header copy, 0.074 ms); 64 registers, 16 blocks 0.067 ms; one warp, 32 blocks 0.063 ms.
// (The register bound stays that of 64-thread blocks: bounding for 32-thread blocks makes
// the compiler spill a kilobyte.)  Every phase below is written for any block size.
constexpr int kTailThreads = 32;

__global__ void __launch_bounds__(64, 16) k_step_tail(WalkDev *hdr, const uint32_t *active, Schedule *sched) {
  // The walk's header lives in shared memory for the whole of its step: the phases below
  // read and write its fields one after another (one block owns the walk, nothing else runs
  // on it meanwhile), so a dependent chain of header accesses costs shared-memory latency
  // instead of L2 latency.  Copied in before, written back after.
  __shared__ WalkDev sW;
  static_assert(sizeof(WalkDev) % 8 == 0 && alignof(WalkDev) <= 8, "the header copies in 8-byte words");
  constexpr int kHdrWords = (int)(sizeof(WalkDev) / 8);
  // the neighbourhood kernel of this step has finished: rearm its work counter
  if (blockIdx.x == 0 && threadIdx.x == 0) sched->hot_next = 0;
  const bool exact = sched->alpha2 != 0;  // the closed form kept every neighbour's exact Delta F
  for (uint32_t a = blockIdx.x; a < sched->nactive; a += gridDim.x) {
    WalkDev &G = hdr[active[a]];
    __syncthreads();  // the previous walk's shared buffers and header copy are free
    if (G.status != kRunning) continue;  // one reading for the block: nothing below changes it before it is read
    for (int q = (int)threadIdx.x; q < kHdrWords; q += (int)blockDim.x)
      reinterpret_cast<uint2 *>(&sW)[q] = reinterpret_cast<const uint2 *>(&G)[q];
    __syncthreads();
    WalkDev &W = sW;
    if (threadIdx.x < 32) select_warp(W);
    __syncthreads();  // candidates, bound and window PSL are visible to the block
    const uint32_t nslots = min(W.ncand, (uint32_t)kQcap);
    for (uint32_t qslot = 0; qslot < nslots; qslot++) {
      __syncthreads();
      recheck_one<true, kRcBoth>(W, 0, qslot, exact);
    }
    __syncthreads();  // re-check partials are visible
    decide_one(W);
    __syncthreads();  // the decision (mode, k*, flips, next exponent) is visible
    if (W.mode == kModeMove)
      apply_move_dispatch(W, 0);
    else
      apply_one(W, 0);
    __syncthreads();
    for (int q = (int)threadIdx.x; q < kHdrWords; q += (int)blockDim.x)
      reinterpret_cast<uint2 *>(&G)[q] = reinterpret_cast<const uint2 *>(&sW)[q];
  }
}

static uint32_t g_tail_per_sm = 4;

cudaError_t prepare_tail_kernel() {
  int nb = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step_tail, kTailThreads, 0);
  g_tail_per_sm = (uint32_t)(nb > 0 ? nb : 1);
  return e;
}

cudaError_t launch_step_tail(const LaunchCtx &c) {
  k_step_tail<<<g_tail_per_sm * c.sm_count, kTailThreads, 0, c.stream>>>(c.hdr, c.active, c.sched);
  return cudaGetLastError();
}

}  // namespace psl
