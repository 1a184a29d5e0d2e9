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
// A block takes work items (up to kA2PerThread x NT window positions of one walk) from the
// schedule, builds the walk's planes, prefix sums of C, bit arrays and near-peak entries in
// shared memory, and scores kA2PerThread positions per thread, NT apart.  Every position
// covers about (L-1)/32 words whatever its place in the sequence (the forward and backward
// ranges add up to L - 1), so the warps of a block do equal work and no block waits on
// another.
#include <climits>
#include <cstdint>
#include <cstdio>

#include "psl_device.cuh"
#include "psl_internal.h"

namespace psl {

namespace {

constexpr int kA2Words = (int)((kA2MaxL - 1 + 31) / 32);  // words of shifts k = 1 .. L-1
// two's-complement planes of |C_k| <= PSL <= L - 1 < 2^12 for L <= 4095: P = bitlen(PSL) + 1 <= 13
constexpr int kA2MaxPlanes = 13;
static_assert(kA2Words % 4 == 0 && kA2MaxL < 4096u, "plane groups of four words; 13 planes suffice");

// Bit planes of C_k, k = 1 + 32 w + t in bit t of word w, plane-major so that four
// consecutive words of one plane load as one 16-byte vector; prefix sums of C within each
// word and over words.  (Plane words past the walk's last shift may hold an earlier walk's
// values: they are only ever combined with windows that read 0 there.)
// The sequence's bits forward (bit t of word m: x_{32m+t}) and reversed (r_i = x_{L-1-i}),
// with zero words past the end: a position's partner windows are consecutive 32-bit
// stretches of one of them (forward partners of j start at j + 1 in x, backward partners at
// L - j in r), one shared load and one funnel shift per word, reading 0 past either end.
constexpr int kA2BitWords = 2 * kA2Words + 8;
constexpr int kA2PeakCap = 512;  // near-peak entries staged per item (more: read from the walk's list)
struct A2Smem {
  uint4 plane[kA2MaxPlanes][kA2Words / 4];
  int pre[kA2MaxL];      // pre[k]: sum of C over the shifts of k's word up to k
  int woff[kA2Words];    // sum of C over the words before w
  uint32_t xs[kA2BitWords];
  uint32_t rs[kA2BitWords];
  int2 peak[kA2PeakCap];  // the near-peak entries (k, C_k) with |C_k| >= PSL - 8
  uint32_t next;
  int run;
  int npeak;
};

__device__ __forceinline__ int a2_bitlen(uint32_t v) { return v ? 32 - __clz(v) : 0; }

// S(K) = sum_{k=1}^K C_k
__device__ __forceinline__ int a2_prefix(const A2Smem &sm, int K) {
  return K <= 0 ? 0 : sm.pre[K] + sm.woff[(K - 1) >> 5];
}

// full adder over bit slices: s = a + b + c mod 2, returns the carry
__device__ __forceinline__ uint32_t a2_fa(uint32_t &s, uint32_t a, uint32_t b, uint32_t c) {
  s = a ^ b ^ c;
  return (a & b) | (c & (a ^ b));
}

// One side (forward or backward partners) of sum_p w_p popcount(plane_p[w] AND window_w) over
// the words w < nw: window w is bits [start + 32 w, start + 32 w + 32) of the bit array arr
// (bit t: x_{j +- (1 + 32 w + t)}); past the side's last shift it reads the zero words.
// Words are taken four at a time through carry-save adders per plane (ones, twos, and a
// popcount of the fours), so a population count serves four words instead of one: that unit
// issues at an eighth of the logic-op rate.  Planes PLO .. PHI-1 of P (wider sequences of
// planes go in two passes, to bound the registers of the counters).
template <int PLO, int PHI, int P>
__device__ __forceinline__ int a2_side(const A2Smem &sm, const uint32_t *arr, int start, int nw) {
  constexpr int NP = PHI - PLO;
  uint32_t ones[NP], twos[NP];
  int fours[NP];
#pragma unroll
  for (int p = 0; p < NP; p++) ones[p] = twos[p] = 0u, fours[p] = 0;
  const int ng = (nw + 3) >> 2;
  const int q0 = start >> 5, sh = start & 31;
  uint32_t lo = arr[q0];
  for (int g = 0; g < ng; g++) {
    uint32_t x[4];
#pragma unroll
    for (int u = 0; u < 4; u++) {
      const uint32_t hi = arr[q0 + 4 * g + u + 1];
      x[u] = __funnelshift_r(lo, hi, sh);
      lo = hi;
    }
#pragma unroll
    for (int p = 0; p < NP; p++) {
      const uint4 pl = sm.plane[PLO + p][g];
      uint32_t s1, s2, s4;
      const uint32_t c1 = a2_fa(s1, ones[p], pl.x & x[0], pl.y & x[1]);
      const uint32_t c2 = a2_fa(s2, s1, pl.z & x[2], pl.w & x[3]);
      ones[p] = s2;
      const uint32_t c4 = a2_fa(s4, twos[p], c1, c2);
      twos[p] = s4;
      fours[p] += __popc(c4);
    }
  }
  int s = 0;
#pragma unroll
  for (int p = 0; p < NP; p++) {
    const int v = __popc(ones[p]) + 2 * __popc(twos[p]) + 4 * fours[p];
    const int q = PLO + p;
    s += (q == P - 1 ? -(1 << q) : (1 << q)) * v;  // two's complement: the top plane weighs -2^(P-1)
  }
  return s;
}

template <int P>
__device__ __forceinline__ int a2_side_all(const A2Smem &sm, const uint32_t *arr, int start, int nw) {
  if constexpr (P <= 8)
    return a2_side<0, P, P>(sm, arr, start, nw);
  else
    return a2_side<0, 8, P>(sm, arr, start, nw) + a2_side<8, P, P>(sm, arr, start, nw);
}

// Exact Delta F of flipping position j (in the sequence) of walk W, alpha = 2.
template <int P>
__device__ __forceinline__ int a2_delta(const A2Smem &sm, const WalkDev &W, int j, int L) {
  const int kplus = L - 1 - j, kin = min(j, kplus);
  // forward partners x_{j+k}: x from j + 1, words w < ceil(kplus / 32); backward partners
  // x_{j-k} = r_{L-j-1+k}: r from L - j, words w < ceil(j / 32)
  const int sx = a2_side_all<P>(sm, sm.xs, j + 1, (kplus + 31) >> 5);
  const int sy = a2_side_all<P>(sm, sm.rs, L - j, (j + 31) >> 5);
  int zd = 0;
  {
    const int qf = (j + 1) >> 5, sf = (j + 1) & 31, qr = (L - j) >> 5, sr = (L - j) & 31;
    uint32_t fl = sm.xs[qf], rl = sm.rs[qr];
    for (int w = 0; w < ((kin + 31) >> 5); w++) {
      const uint32_t fh = sm.xs[qf + w + 1], rh = sm.rs[qr + w + 1];
      const uint32_t d = __funnelshift_r(fl, fh, sf) ^ __funnelshift_r(rl, rh, sr);
      fl = fh, rl = rh;
      const int lim = kin - 32 * w;  // shifts 1 + 32 w + t <= kin
      zd += __popc(lim >= 32 ? d : d & ((1u << lim) - 1u));
    }
  }
  const int X = a2_prefix(sm, kplus) - 2 * sx;
  const int Y = a2_prefix(sm, j) - 2 * sy;
  const int Z = kin - 2 * zd;
  const int sj = ((sm.xs[j >> 5] >> (j & 31)) & 1u) ? -1 : 1;
  return -4 * sj * (X + Y) + 4 * (L - 1) + 8 * Z;
}

__device__ __forceinline__ int a2_delta_any(const A2Smem &sm, const WalkDev &W, int j, int L, int P) {
  switch (P) {
    case 1: return a2_delta<1>(sm, W, j, L);
    case 2: return a2_delta<2>(sm, W, j, L);
    case 3: return a2_delta<3>(sm, W, j, L);
    case 4: return a2_delta<4>(sm, W, j, L);
    case 5: return a2_delta<5>(sm, W, j, L);
    case 6: return a2_delta<6>(sm, W, j, L);
    case 7: return a2_delta<7>(sm, W, j, L);
    case 8: return a2_delta<8>(sm, W, j, L);
    case 9: return a2_delta<9>(sm, W, j, L);
    case 10: return a2_delta<10>(sm, W, j, L);
    case 11: return a2_delta<11>(sm, W, j, L);
    case 12: return a2_delta<12>(sm, W, j, L);
    default: return a2_delta<13>(sm, W, j, L);
  }
}

template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) k_hot_alpha2(WalkDev *hdr, const HotItem *items, Schedule *sched) {
  constexpr int NW = NT / 32;
  __shared__ A2Smem sm;
  const int lane = (int)(threadIdx.x & 31u), warp = (int)(threadIdx.x >> 5);
  for (;;) {
    __syncthreads();  // the previous item's shared state is no longer read
    if (threadIdx.x == 0) {
      const uint32_t nx = atomicAdd(&sched->hot_next, 1u);
      sm.next = nx;
      sm.run = nx < sched->nitems && hdr[items[nx].slot].status == kRunning;  // one reading for the block
      sm.npeak = 0;
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
    // the bits forward and reversed, zero past the end of the sequence
    const int nb = (L + 31) >> 5;
    for (int m = (int)threadIdx.x; m < kA2BitWords; m += NT) {
      sm.xs[m] = m < nb ? W.bits[m] : 0u;  // the packed sequence keeps its padding bits 0
      // r word m, bit t: x_{L-1-32m-t} = bit 31-t of the 32 bits from L-32-32m
      sm.rs[m] = m < nb ? __brev(window32(W.bits, L - 32 - 32 * m)) : 0u;
    }
    // the entries of the near-peak list that can reach a neighbour's PSL (|C_k| >= PSL - 8:
    // a flip moves C_k by at most 4, and every neighbour's PSL is at least PSL - 4), once per
    // item instead of once per position; their order does not matter to a maximum
    const bool on = W.ktau_on != 0;
    if (on) {
      const int nk = (int)W.nktau, floor_c = W.psl - 8;
      for (int q = (int)threadIdx.x; q < nk; q += NT) {
        const int2 e = W.ktau[q];
        if ((e.y < 0 ? -e.y : e.y) >= floor_c) {
          const int at = atomicAdd(&sm.npeak, 1);
          if (at < kA2PeakCap) sm.peak[at] = e;
        }
      }
    }
    // planes and in-word prefix sums of C_k, one word of 32 shifts per warp at a time
    uint32_t *plane_w = reinterpret_cast<uint32_t *>(sm.plane);  // [plane][word]
    for (int w = warp; w < nw; w += NW) {
      const int k = 1 + 32 * w + lane;
      const int c = k < L ? W.C[k] : 0;
      uint32_t mine = 0u;  // lane p keeps plane p of this word
#pragma unroll
      for (int p = 0; p < kA2MaxPlanes; p++) {
        if (p < P) {  // the same for every lane
          const uint32_t b = __ballot_sync(0xffffffffu, (c >> p) & 1);
          if (lane == p) mine = b;
        }
      }
      if (lane < P) plane_w[lane * kA2Words + w] = mine;
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
    // kA2PerThread window positions per thread, NT apart: an item's planes, sums and bit arrays
    // serve kA2PerThread x NT positions (every position does the same work)
    for (int r = 0; r < (int)kA2PerThread; r++) {
      const int i = (int)it.i0 + (int)threadIdx.x + r * NT;  // window position, 1-based
      if (i > N) break;
      const int j = (int)(((uint64_t)W.start + (uint64_t)i) % (uint64_t)L);
      const int dF = a2_delta_any(sm, W, j, L, P);
      W.score[i - 1] = ldexpf((float)dF, -2 * (int)W.e);  // the tables' scale 2^(-alpha e)
      reinterpret_cast<int *>(W.score_part)[i - 1] = dF;   // exact, for the re-check of the candidates
      // exact neighbour PSL, only when some neighbour may beat psl_best
      int pj = INT_MAX;
      if (on) {
        const int sj = ((sm.xs[j >> 5] >> (j & 31)) & 1u) ? -1 : 1;
        if (sm.npeak <= kA2PeakCap) {
          pj = 0;
          for (int q = 0; q < sm.npeak; q++) {
            const int2 e = sm.peak[q];
            const int k = e.x;
            int part = 0;
            if (j + k < L) part += 1 - 2 * (int)((sm.xs[(j + k) >> 5] >> ((j + k) & 31)) & 1u);
            if (j >= k) part += 1 - 2 * (int)((sm.xs[(j - k) >> 5] >> ((j - k) & 31)) & 1u);
            const int cn = e.y - 2 * sj * part;
            pj = max(pj, cn < 0 ? -cn : cn);
          }
        } else {
          pj = neighbour_psl(W, W.ktau, (int)W.nktau, j, L, sj, W.psl - 8, 0);
        }
      }
      W.pslj[i - 1] = pj;
    }
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
