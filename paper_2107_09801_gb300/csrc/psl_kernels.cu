// psl_kernels.cu -- CUDA kernels (sm_103a) for the limited-neighbourhood search of
// Boskovic and Brest, "Two-phase Optimization of Binary Sequences with Low Peak
// Sidelobe Level Value" (arXiv 2107.09801).
//
// One walk step (the body of the while loop of Algorithm 1) is five phases:
//   hot     FP32 filter score of every neighbour in the window (Eq. 4 through the
//           one-element flip of Sec. 3) and, when it can matter, its exact PSL (Eq. 3)
//           -- psl_hot.cu (subset-sum tables), psl_alpha2.cu (the closed form at alpha = 2)
//   select  minimum score, the certified candidate set {score <= min + 2B} plus the
//           FP32 top-k, and the first neighbour of minimum PSL
//   recheck exact Delta F of every candidate -- psl_recheck.cu (two kernels)
//   decide  exact argmin (first in scan order), bookkeeping and phase switch of Alg. 1
//   apply   O(L) update of C, PSL, the next step's per-k tables and near-peak list (two
//           kernels: ordinary moves, and initialisation / phase switches)
// For batches of short walks select..apply run as one kernel (psl_tail.cu).  This file
// holds the walk initialisation, select, decide and apply.  Work shared between blocks of
// a walk ends in a "last block to arrive finishes the walk" counter: no block here waits
// on another.
#include <cfloat>
#include <climits>
#include <cstdint>
#include <mutex>

#include "psl_device.cuh"
#include "psl_internal.h"
#include "psl_step.cuh"

namespace psl {
// ------------------------------------------------------------------------------------
// walk initialisation: Rand(L, SEED) of Alg. 1, C by popcount (Eq. 2), then the
// update pass in init mode
// ------------------------------------------------------------------------------------
__global__ void k_init_bits(WalkDev *hdr, const uint32_t *active) {
  WalkDev &W = hdr[active[blockIdx.y]];
  const int nw = (int)W.nw;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x - kGuardWords;
  if (idx >= nw + kGuardWords) return;
  if (idx < 0 || idx >= nw) {
    W.bits[idx] = 0u;
    W.bits_local[idx] = 0u;
    W.bits_best[idx] = 0u;
    if (W.track_fbest) W.bits_fbest[idx] = 0u;
    return;
  }
  if (!W.has_init_seq) {
    const uint64_t d = splitmix64(W.seed, (uint64_t)(idx >> 1));
    uint32_t word = (idx & 1) ? (uint32_t)(d >> 32) : (uint32_t)d;
    const uint32_t rem = W.L - 32u * (uint32_t)idx;
    if (rem < 32u) word &= (1u << rem) - 1u;
    W.bits[idx] = word;
  }
  if (idx == 0) W.psl = 0;
}

// C_k = (L-k) - 2 popc(x[0..L-k) xor x[k..L)) for one k per thread (Eq. 2 on packed bits);
// PSL by atomicMax.  A block covers 256 consecutive k and streams the packed sequence
// through shared memory in tiles of 2048 words: for thread k the partner window of word w
// is funnel(x[w + k/32], x[w + k/32 + 1], k % 32), with a shift that stays fixed, so each
// iteration costs two broadcast shared loads.
constexpr int kAcTileWords = 2048;

__global__ void __launch_bounds__(256) k_autocorr(WalkDev *hdr, const uint32_t *active) {
  __shared__ uint32_t sa[kAcTileWords];
  __shared__ uint32_t sbw[kAcTileWords + 10];
  WalkDev &W = hdr[active[blockIdx.y]];
  const int L = (int)W.L, nw = (int)W.nw;
  const int k0 = (int)blockIdx.x * 256;
  if (k0 >= L) return;
  const uint32_t *bits = W.bits;
  const int k = k0 + (int)threadIdx.x;
  const int n = L - k;                          // products of C_k (<= 0 past the end)
  const int full = n > 0 ? n >> 5 : 0;          // whole words of x[0..n)
  const int c = (k >> 5) - (k0 >> 5);           // 0..7
  const int sh = k & 31;
  const int wend = (L - k0 + 31) >> 5;          // words the block needs at most
  int cnt = 0;
  for (int w0 = 0; w0 < wend; w0 += kAcTileWords) {
    __syncthreads();
    for (int t = threadIdx.x; t < kAcTileWords + 10; t += 256) {
      if (t < kAcTileWords) sa[t] = (w0 + t < nw) ? bits[w0 + t] : 0u;
      const int g = w0 + (k0 >> 5) + t;        // guard words beyond nw read as zero
      sbw[t] = (g < nw) ? bits[g] : 0u;
    }
    __syncthreads();
    const int wlim = min(full - w0, kAcTileWords);
    if (wlim > 0) {
      uint32_t lo = sbw[c];
      for (int w = 0; w < wlim; w++) {
        const uint32_t hi = sbw[w + c + 1];
        cnt += __popc(sa[w] ^ __funnelshift_r(lo, hi, sh));
        lo = hi;
      }
    }
  }
  int a = 0;
  if (k < L) {
    const int rem = n & 31;
    if (rem) {  // the partial last word of x[0..n)
      const uint32_t d = bits[full] ^ window32(bits, 32 * full + k);
      cnt += __popc(d & ((1u << rem) - 1u));
    }
    const int cv = n - 2 * cnt;
    W.C[k] = cv;
    if (k > 0) a = cv < 0 ? -cv : cv;
  }
  a = warp_max(a);
  if ((threadIdx.x & 31) == 0 && a > 0) atomicMax(&W.psl, a);
}


// Sets up the init-mode update pass once PSL(pivot_0) is known.
__global__ void k_start_init(WalkDev *hdr, const uint32_t *active, uint32_t nactive) {
  const uint32_t a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nactive) return;
  WalkDev &W = hdr[active[a]];
  W.mode = kModeInit;
  W.alpha_next = W.alpha1;
  W.e = bitlen((uint32_t)W.psl + 8u);
  W.ktau_thr = W.psl - 8;
  W.nktau = 0;
  W.arrive = 0;
  W.improved = 0;
  W.psl_improved = 0;
}

// persistent grid over (walk, chunk) pairs of the schedule: the walks whose step was an
// ordinary move (every other walk is the work of k_apply)
__global__ void __launch_bounds__(256) k_apply_move(WalkDev *hdr, const uint32_t *active, const Schedule *sched) {
  const uint32_t nch = sched->max_chunk_apply, V = sched->nactive * nch;
  for (uint32_t v = blockIdx.x; v < V; v += gridDim.x) {
    WalkDev &W = hdr[active[v / nch]];
    const uint32_t chunk = v % nch;
    if (W.status != kRunning || chunk >= W.nchunk_apply || W.mode != kModeMove) continue;  // uniform over the block
    __syncthreads();  // shared reduction buffers of the previous pair are free
    apply_move_dispatch(W, chunk);
  }
}

// persistent grid over (walk, chunk) pairs of the schedule
__global__ void __launch_bounds__(256) k_apply(WalkDev *hdr, const uint32_t *active, const Schedule *sched) {
  if (!sched->general) return;  // every walk's step was an ordinary move: k_apply_move did it all
  const uint32_t nch = sched->max_chunk_apply, V = sched->nactive * nch;
  for (uint32_t v = blockIdx.x; v < V; v += gridDim.x) {
    __syncthreads();  // shared reduction buffers of the previous pair are free
    apply_one(hdr[active[v / nch]], v % nch);
  }
}

// Windows above kSelectWarpN neighbours take a block each; the rest a warp each.
__global__ void __launch_bounds__(1024) k_select(WalkDev *hdr, const uint32_t *active, Schedule *sched) {
  const uint32_t nact = sched->nactive;
  if (blockIdx.x == 0 && threadIdx.x == 0) sched->general = 0;  // k_decide sets it again for a phase switch
  for (uint32_t a = blockIdx.x; a < nact; a += gridDim.x) {
    WalkDev &W = hdr[active[a]];
    if ((int)W.N <= kSelectWarpN) continue;  // the same reading in every thread of the block
    __syncthreads();
    select_one(W);
  }
  const uint32_t nwarps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t a = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); a < nact; a += nwarps) {
    WalkDev &W = hdr[active[a]];
    if ((int)W.N <= kSelectWarpN) select_warp(W);
  }
}

__global__ void __launch_bounds__(256) k_decide(WalkDev *hdr, const uint32_t *active, Schedule *sched) {
  // the neighbourhood kernel of this step has finished: rearm its work counter
  if (blockIdx.x == 0 && threadIdx.x == 0) sched->hot_next = 0;
  for (uint32_t a = blockIdx.x; a < sched->nactive; a += gridDim.x) {
    __syncthreads();
    WalkDev &W = hdr[active[a]];
    decide_one(W);
    if (threadIdx.x == 0 && W.mode == kModeSwitch) sched->general = 1;  // the next update pass needs k_apply
  }
}

// ------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------
// resident blocks per SM of the other persistent kernels (one wave each)
static uint32_t g_apply_per_sm = 4, g_apply_move_per_sm = 4, g_select_per_sm = 1, g_decide_per_sm = 4;

cudaError_t launch_init_bits(const LaunchCtx &c) {
  const uint32_t maxw = (c.maxL + 31) / 32 + 2 * kGuardWords;
  dim3 grid((maxw + 255) / 256, c.ninit);
  k_init_bits<<<grid, 256, 0, c.stream>>>(c.hdr, c.active);
  return cudaGetLastError();
}

cudaError_t launch_autocorr(const LaunchCtx &c) {
  dim3 grid((c.maxL + 255) / 256, c.ninit);
  k_autocorr<<<grid, 256, 0, c.stream>>>(c.hdr, c.active);
  return cudaGetLastError();
}

cudaError_t launch_start_init(const LaunchCtx &c) {
  k_start_init<<<(c.ninit + 127) / 128, 128, 0, c.stream>>>(c.hdr, c.active, c.ninit);
  return cudaGetLastError();
}

cudaError_t launch_apply(const LaunchCtx &c) {
  // walks whose step was an ordinary move, then the rest (initialisation, phase switch)
  k_apply_move<<<g_apply_move_per_sm * c.sm_count, 256, 0, c.stream>>>(c.hdr, c.active, c.sched);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_apply<<<g_apply_per_sm * c.sm_count, 256, 0, c.stream>>>(c.hdr, c.active, c.sched);
  return cudaGetLastError();
}

static cudaError_t blocks_per_sm(const void *f, int threads, uint32_t *out) {
  int nb = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, threads, 0);
  *out = (uint32_t)(nb > 0 ? nb : 1);
  return e;
}

static cudaError_t prepare_kernels_once() {
  cudaError_t e0 = blocks_per_sm((const void *)k_apply, 256, &g_apply_per_sm);
  if (e0 == cudaSuccess) e0 = blocks_per_sm((const void *)k_apply_move, 256, &g_apply_move_per_sm);
  if (e0 == cudaSuccess) e0 = blocks_per_sm((const void *)k_select, 1024, &g_select_per_sm);
  if (e0 == cudaSuccess) e0 = blocks_per_sm((const void *)k_decide, 256, &g_decide_per_sm);
  if (e0 != cudaSuccess) return e0;
  e0 = prepare_hot_kernels();
  if (e0 == cudaSuccess) e0 = prepare_alpha2_kernels();
  if (e0 == cudaSuccess) e0 = prepare_recheck_kernel();
  if (e0 == cudaSuccess) e0 = prepare_tail_kernel();
  if (e0 != cudaSuccess) return e0;
  return cudaSuccess;
}

// Kernel attributes are per device and process; contexts created on several host threads
// share one set-up.
cudaError_t prepare_kernels() {
  static std::once_flag once;
  static cudaError_t result = cudaSuccess;
  std::call_once(once, [] { result = prepare_kernels_once(); });
  return result;
}

cudaError_t launch_select(const LaunchCtx &c) {
  k_select<<<g_select_per_sm * c.sm_count, 1024, 0, c.stream>>>(c.hdr, c.active, c.sched);
  return cudaGetLastError();
}

cudaError_t launch_decide(const LaunchCtx &c) {
  k_decide<<<g_decide_per_sm * c.sm_count, 256, 0, c.stream>>>(c.hdr, c.active, c.sched);
  return cudaGetLastError();
}

}  // namespace psl
