// psl_alpha2.cu -- neighbourhood score for alpha = 2 (arXiv 2107.09801, Eq. 4 with alpha = 2:
// F_2 = sum_k C_k^2, the merit-factor objective) by its closed form, for batches of short walks.
//
// The flip of s_j (Sec. 3) changes C_k by delta_k = -2 s_j (s_{j+k} + s_{j-k}) (terms outside
// the sequence absent), and for alpha = 2 the change of F is linear in C:
//   Delta F(j) = sum_k (2 C_k delta_k + delta_k^2) = -4 s_j (X_j + Y_j) + 4 (L - 1) + 8 Z_j,
//   X_j = sum_{k=1}^{L-1-j} C_k s_{j+k},  Y_j = sum_{k=1}^{j} C_k s_{j-k},
//   Z_j = sum_{k=1}^{min(j, L-1-j)} s_{j+k} s_{j-k}.
// With x the sequence's bits (s = 1 - 2x) and C_k in two's complement over P bit planes
// (P = bitlen(PSL) + 1), sum_k C_k x_{j+k} = sum_p w_p popcount(plane_p AND window), 32 shifts
// per instruction: X_j = S(L-1-j) - 2 that sum, with S(K) = sum_{k=1}^K C_k, likewise Y_j from
// the backward windows, and Z_j = min(j, L-1-j) - 2 popcount of the differing partner bits.
// The result is the exact integer Delta F; it is stored as the FP32 score in the tables' scale
// 2^(-2e) (one rounding, and only above 2^24: inside the bound B of the certified filter, which
// is at least 72 2^-24 S_abs >= 72 2^-24 |Delta F|), so selection, re-check and decision run
// unchanged.
//
// A block takes work items (up to NT window positions of one walk) from the schedule, builds the
// walk's planes and prefix sums of C in shared memory, and scores one position per thread.
// Every position covers about (L-1)/32 words whatever its place in the sequence (the forward
// and backward ranges add up to L - 1), so the warps of a block do equal work and no block
// waits on another.
#include <climits>
#include <cstdint>
#include <cstdio>

#include "psl_device.cuh"
#include "psl_internal.h"

namespace psl {

namespace {

constexpr int kA2Words = (int)((kA2MaxL - 1 + 31) / 32);  // words of shifts k = 1 .. L-1

// Bit planes of C_k, k = 1 + 32 w + t in bit t of word w: 16 per word (four 16-byte vectors,
// planes at and above P are zero), prefix sums of C within each word and over words.
struct A2Smem {
  uint4 plane[kA2Words][4];
  int pre[kA2MaxL];      // pre[k]: sum of C over the shifts of k's word up to k
  int woff[kA2Words];    // sum of C over the words before w
  uint32_t next;
  int run;
};

__device__ __forceinline__ int a2_bitlen(uint32_t v) { return v ? 32 - __clz(v) : 0; }

// S(K) = sum_{k=1}^K C_k
__device__ __forceinline__ int a2_prefix(const A2Smem &sm, int K) {
  return K <= 0 ? 0 : sm.pre[K] + sm.woff[(K - 1) >> 5];
}

// sum over the words of one side of sum_p w_p popcount(plane_p[w] AND window_w): the window of
// word w is win[base + dir 32 w] (bit t: x_{j + dir (1 + 32 w + t)}).
template <int PQ>
__device__ __forceinline__ int a2_side(const A2Smem &sm, const uint32_t *__restrict__ win, int base, int dir, int nw,
                                       const int (&wt)[4 * PQ]) {
  int cnt[4 * PQ];
#pragma unroll
  for (int p = 0; p < 4 * PQ; p++) cnt[p] = 0;
  for (int w = 0; w < nw; w++) {
    const uint32_t x = __ldg(win + base + dir * 32 * w);
#pragma unroll
    for (int q = 0; q < PQ; q++) {
      const uint4 pl = sm.plane[w][q];
      cnt[4 * q + 0] += __popc(pl.x & x);
      cnt[4 * q + 1] += __popc(pl.y & x);
      cnt[4 * q + 2] += __popc(pl.z & x);
      cnt[4 * q + 3] += __popc(pl.w & x);
    }
  }
  int s = 0;
#pragma unroll
  for (int p = 0; p < 4 * PQ; p++) s += wt[p] * cnt[p];
  return s;
}

// Exact Delta F of flipping position j (in the sequence) of walk W, alpha = 2.
template <int PQ>
__device__ __forceinline__ int a2_delta(const A2Smem &sm, const WalkDev &W, int j, int L, int P) {
  int wt[4 * PQ];
#pragma unroll
  for (int p = 0; p < 4 * PQ; p++) wt[p] = p < P - 1 ? (1 << p) : (p == P - 1 ? -(1 << p) : 0);
  const int kplus = L - 1 - j, kin = min(j, kplus);
  // forward: words w < ceil(kplus / 32), windows at j + 1 + 32 w <= L - 1; backward: words
  // w < ceil(j / 32), windows at j - 1 - 32 w >= 0.  Bits past either end read 0.
  const int sx = a2_side<PQ>(sm, W.win_f, j + 1, 1, (kplus + 31) >> 5, wt);
  const int sy = a2_side<PQ>(sm, W.win_r, j - 1, -1, (j + 31) >> 5, wt);
  int zd = 0;
  for (int w = 0; w < ((kin + 31) >> 5); w++) {
    const uint32_t d = __ldg(W.win_f + j + 1 + 32 * w) ^ __ldg(W.win_r + j - 1 - 32 * w);
    const int lim = kin - 32 * w;  // shifts 1 + 32 w + t <= kin
    zd += __popc(lim >= 32 ? d : d & ((1u << lim) - 1u));
  }
  const int X = a2_prefix(sm, kplus) - 2 * sx;
  const int Y = a2_prefix(sm, j) - 2 * sy;
  const int Z = kin - 2 * zd;
  const int sj = getbit(W.bits, j) ? -1 : 1;
  return -4 * sj * (X + Y) + 4 * (L - 1) + 8 * Z;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_hot_alpha2(WalkDev *hdr, const HotItem *items, Schedule *sched) {
  constexpr int NW = NT / 32;
  __shared__ A2Smem sm;
  const int lane = (int)(threadIdx.x & 31u), warp = (int)(threadIdx.x >> 5);
  for (;;) {
    __syncthreads();  // the previous item's shared state is no longer read
    if (threadIdx.x == 0) {
      const uint32_t nx = atomicAdd(&sched->hot_next, 1u);
      sm.next = nx;
      sm.run = nx < sched->nitems && hdr[items[nx].slot].status == kRunning;  // one reading for the block
    }
    __syncthreads();
    const uint32_t item = sm.next;
    if (item >= sched->nitems) return;
    if (!sm.run) continue;
    const HotItem it = items[item];
    WalkDev &W = hdr[it.slot];
    const int L = (int)W.L, N = (int)W.N;
    const int P = a2_bitlen((uint32_t)W.psl) + 1;  // |C_k| <= PSL < 2^(P-1) for k >= 1
    const int nw = (L - 1 + 31) >> 5;
    // planes and in-word prefix sums of C_k, one word of 32 shifts per warp at a time
    for (int w = warp; w < nw; w += NW) {
      const int k = 1 + 32 * w + lane;
      const int c = k < L ? W.C[k] : 0;
      uint32_t pl[16];
#pragma unroll
      for (int p = 0; p < 16; p++) pl[p] = p < P ? __ballot_sync(0xffffffffu, (c >> p) & 1) : 0u;
      if (lane == 0) sm.plane[w][0] = make_uint4(pl[0], pl[1], pl[2], pl[3]);
      if (lane == 1) sm.plane[w][1] = make_uint4(pl[4], pl[5], pl[6], pl[7]);
      if (lane == 2) sm.plane[w][2] = make_uint4(pl[8], pl[9], pl[10], pl[11]);
      if (lane == 3) sm.plane[w][3] = make_uint4(pl[12], pl[13], pl[14], pl[15]);
      int v = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
      }
      if (k < L) sm.pre[k] = v;
      if (lane == 31) sm.woff[w] = v;  // the word's total, turned into an offset below
    }
    __syncthreads();
    if (warp == 0) {  // exclusive prefix over the word totals, kA2Words / 32 per lane
      constexpr int PER = (kA2Words + 31) / 32;
      int t[PER], run = 0;
#pragma unroll
      for (int u = 0; u < PER; u++) {
        const int w = lane * PER + u;
        t[u] = w < nw ? sm.woff[w] : 0;
        run += t[u];
      }
      int incl = run;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += n;
      }
      int acc = incl - run;
#pragma unroll
      for (int u = 0; u < PER; u++) {
        const int w = lane * PER + u;
        if (w < nw) sm.woff[w] = acc;
        acc += t[u];
      }
    }
    __syncthreads();
    const int i = (int)it.i0 + (int)threadIdx.x;  // window position, 1-based
    if (i > N) continue;
    const int j = (int)(((uint64_t)W.start + (uint64_t)i) % (uint64_t)L);
    int dF;
    if (P <= 4)
      dF = a2_delta<1>(sm, W, j, L, P);
    else if (P <= 8)
      dF = a2_delta<2>(sm, W, j, L, P);
    else if (P <= 12)
      dF = a2_delta<3>(sm, W, j, L, P);
    else
      dF = a2_delta<4>(sm, W, j, L, P);
    W.score[i - 1] = ldexpf((float)dF, -2 * (int)W.e);  // the tables' scale 2^(-alpha e)
    // exact neighbour PSL, only when some neighbour may beat psl_best
    int pj = INT_MAX;
    if (W.ktau_on) pj = neighbour_psl(W, W.ktau, (int)W.nktau, j, L, getbit(W.bits, j) ? -1 : 1, W.psl - 8, 0);
    W.pslj[i - 1] = pj;
  }
}

using A2Fn = void (*)(WalkDev *, const HotItem *, Schedule *);

A2Fn a2_variant(uint32_t threads) {
  switch (threads) {
    case 128: return k_hot_alpha2<128>;
    case 448: return k_hot_alpha2<448>;
    case 512: return k_hot_alpha2<512>;
    case 896: return k_hot_alpha2<896>;
    default: return k_hot_alpha2<256>;
  }
}

uint32_t g_a2_blocks_per_sm[5];

int a2_index(uint32_t threads) {
  return threads == 128 ? 0 : threads == 448 ? 2 : threads == 512 ? 3 : threads == 896 ? 4 : 1;
}

}  // namespace

cudaError_t prepare_alpha2_kernels() {
  for (uint32_t t : {128u, 256u, 448u, 512u, 896u}) {
    int nb = 0;
    const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, a2_variant(t), (int)t, 0);
    if (e != cudaSuccess) return e;
    g_a2_blocks_per_sm[a2_index(t)] = (uint32_t)(nb > 0 ? nb : 1);
  }
  return cudaSuccess;
}

cudaError_t launch_hot_alpha2(const LaunchCtx &c) {
  const uint32_t t = c.hot_threads;  // one of the thread counts of a2_variant (the supported configurations)
  a2_variant(t)<<<g_a2_blocks_per_sm[a2_index(t)] * c.sm_count, t, 0, c.stream>>>(c.hdr, c.items, c.sched);
  return cudaGetLastError();
}

cudaError_t launch_hot(const LaunchCtx &c) { return c.alpha2 ? launch_hot_alpha2(c) : launch_hot_batched(c); }

int hot_kernel_name(const LaunchCtx &c, char *out, int cap) {
  if (c.alpha2) return snprintf(out, (size_t)cap, "k_hot_alpha2<%u>", c.hot_threads);
  return hot_batched_name(c, out, cap);
}

}  // namespace psl
