// psl_recheck.cu -- the exact re-check of a step of Algorithm 1 (arXiv 2107.09801): exact
// Delta F of every certified candidate, one CTA per (walk, k-chunk), all candidates of the
// walk in turn.  Two kernels share the walks of a step: the histogram sums for walks whose
// table exponent e is at most kHistLog (nearly all), the term-by-term 384-bit sums for the
// rest.  Its own translation unit: the per-alpha arithmetic it instantiates compiles in
// parallel with the other kernels.
#include <cstdint>

#include "psl_device.cuh"
#include "psl_internal.h"
#include "psl_step.cuh"

namespace psl {

// persistent grid over (walk, chunk) pairs of the schedule; each pair covers every
// candidate of the walk (slots 0..kQcap-1 by chunk, later ones whole in chunk 0)
template <int PATH>
__global__ void __launch_bounds__(256, PATH == kRcHist ? 4 : 2) k_recheck(WalkDev *hdr, const uint32_t *active,
                                                                         const Schedule *sched) {
  const uint32_t nch = sched->max_chunk_rc, V = sched->nactive * nch;
  const bool exact = sched->alpha2 != 0;  // the closed form kept every neighbour's exact Delta F
  for (uint32_t v = blockIdx.x; v < V; v += gridDim.x) {
    WalkDev &W = hdr[active[v / nch]];
    const uint32_t chunk = v % nch;
    if (W.status != kRunning || chunk >= W.nchunk_rc) continue;  // uniform over the block
    if (W.shard_count > 1 && chunk % W.shard_count != W.shard_rank) continue;  // another rank's chunk
    // the other kernel's walk (the exact copies of the closed form all go to the histogram kernel)
    if (exact ? PATH != kRcHist : (((int)W.e <= kHistLog) != (PATH == kRcHist))) continue;
    const uint32_t nslots = min(W.ncand, (uint32_t)kQcap);
    for (uint32_t qslot = 0; qslot < nslots; qslot++) {
      __syncthreads();
      recheck_one<false, PATH>(W, chunk, qslot, exact);
    }
  }
}

static uint32_t g_recheck_hist_per_sm = 4, g_recheck_terms_per_sm = 2;

cudaError_t prepare_recheck_kernel() {
  int nb = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_recheck<kRcHist>, 256, 0);
  if (e != cudaSuccess) return e;
  g_recheck_hist_per_sm = (uint32_t)(nb > 0 ? nb : 1);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_recheck<kRcTerms>, 256, 0);
  g_recheck_terms_per_sm = (uint32_t)(nb > 0 ? nb : 1);
  return e;
}

cudaError_t launch_recheck(const LaunchCtx &c) {
  k_recheck<kRcHist><<<g_recheck_hist_per_sm * c.sm_count, 256, 0, c.stream>>>(c.hdr, c.active, c.sched);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_recheck<kRcTerms><<<g_recheck_terms_per_sm * c.sm_count, 256, 0, c.stream>>>(c.hdr, c.active, c.sched);
  return cudaGetLastError();
}

}  // namespace psl
