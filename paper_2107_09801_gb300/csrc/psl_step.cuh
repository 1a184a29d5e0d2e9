// psl_step.cuh -- per-walk device functions of one step of Algorithm 1 after the
// neighbourhood score (arXiv 2107.09801): the update pass and its finalisation, selection
// of the certified candidates, the exact 384-bit re-check, and the decision.  Shared by the
// kernels of psl_kernels.cu (one launch per phase), psl_recheck.cu and psl_tail.cu (all
// phases of a short walk in one block).  GPU side only.
#pragma once
#include <cfloat>
#include <climits>
#include <cstdint>

#include "psl_device.cuh"
#include "psl_internal.h"

namespace psl {

__device__ __forceinline__ int bitlen(uint32_t v) { return v ? 32 - __clz(v) : 0; }

// ------------------------------------------------------------------------------------
// apply: the O(L) update pass (init / move / switch) fused with the next window's
// tables, PSL, sum of |T| and the near-peak list; the last block to arrive finalises.
// ------------------------------------------------------------------------------------
// Block reductions of one (walk, chunk) pair of the update pass, the chunk's partial record,
// and -- in the last block of the walk to arrive -- the walk's finalisation: the new pivot's
// bits and partner windows, PSL, sum of |T|, exact F (NEED_F: init and switch), the lowest-F
// pivot, best-PSL and local-best bookkeeping, the next window's start.
template <bool NEED_F>
__device__ __forceinline__ void apply_finish(WalkDev &W, uint32_t chunk, uint32_t mode, bool keep_local, int kstar,
                                             int nflip, uint32_t alpha, int pmax, float sabs,
                                             uint32_t (&F)[kWideLimbs]) {
  __shared__ int s_max[8];
  __shared__ float s_sum[8];
  __shared__ uint32_t s_F[NEED_F ? 256 / 32 : 1][kWideLimbs];
  __shared__ uint32_t s_last, s_fcopy;
  __shared__ int s_bm;            // the block's own totals, when it covers the whole walk
  __shared__ float s_bs;
  __shared__ uint32_t s_bF[kWideLimbs];
  constexpr bool need_F = NEED_F;
  // one block covers the walk (one update chunk): it is the last to arrive, and hands its
  // totals to the finalisation directly instead of through the partial records
  const bool single = W.nchunk_apply == 1u;
  const int L = (int)W.L;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  pmax = warp_max(pmax);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sabs += __shfl_xor_sync(0xffffffffu, sabs, o);
  if constexpr (NEED_F) {
    for (int o = 16; o > 0; o >>= 1) {
      uint32_t other[kWideLimbs];
#pragma unroll
      for (int i = 0; i < kWideLimbs; i++) other[i] = __shfl_down_sync(0xffffffffu, F[i], o);
      if (lane < o) wide_add(F, other);
    }
  }
  if (lane == 0) {
    s_max[warp] = pmax;
    s_sum[warp] = sabs;
    if constexpr (NEED_F) wide_store(s_F[warp], F);
  }
  __syncthreads();
  uint32_t *part = W.ap_part + (size_t)chunk * kApplyPartStride;
  if (threadIdx.x == 0) {
    int m = 0;
    float s = 0.f;
    uint32_t Fb[kWideLimbs];
    wide_zero(Fb);
    for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
      m = max(m, s_max[w]);
      s += s_sum[w];
      if constexpr (NEED_F) {
        uint32_t t[kWideLimbs];
        wide_load(t, s_F[w]);
        wide_add(Fb, t);
      }
    }
    if (single) {
      s_bm = m;
      s_bs = s;
      wide_store(s_bF, Fb);
      s_last = 1;
    } else {
      part[0] = (uint32_t)m;
      part[1] = __float_as_uint(s);
      wide_store(part + 2, Fb);
      __threadfence();
      const uint32_t prev = atomicAdd(&W.arrive, 1u);
      s_last = (prev == W.nchunk_apply - 1u);
    }
  }
  __syncthreads();
  if (!s_last) return;
  if (!single) __threadfence();

  // ---------------- finalise (last block of this walk) ----------------
  const int nw = (int)W.nw;
  if (mode == kModeSwitch) {
    // pivot <- Rand_flip(local_best, FLIP_lmt)
    for (int w = threadIdx.x; w < nw; w += blockDim.x) W.bits[w] = W.bits_local[w];
    __syncthreads();
    if (threadIdx.x == 0)
      for (int q = 0; q < nflip; q++) W.bits[W.flips[q] >> 5] ^= 1u << (W.flips[q] & 31);
  } else if (mode == kModeMove) {
    // pivot <- Flip(pivot, k)
    if (threadIdx.x == 0) W.bits[kstar >> 5] ^= 1u << (kstar & 31);
  }
  __syncthreads();
  // partner windows of the new pivot: one move changes 32 entries of each, any other pivot
  // (the start, a perturbed local_best) is rebuilt whole
  if (mode == kModeMove) {
    for (int t = (int)threadIdx.x; t < 64; t += (int)blockDim.x) {  // any block size
      if (t < 32)
        W.win_f[kstar - t] ^= 1u << t;  // s_{p+t} with p + t = k*
      else
        W.win_r[kstar + (t - 32)] ^= 1u << (t - 32);  // s_{p-t} with p - t = k*
    }
  } else {
    for (int p = (int)threadIdx.x - kWinGuard; p < L + kWinGuard; p += blockDim.x) {
      W.win_f[p] = window32(W.bits, p);
      W.win_r[p] = __brev(window32(W.bits, p - 31));
    }
  }
  if (keep_local)
    for (int w = threadIdx.x; w < nw; w += blockDim.x) W.bits_local[w] = W.bits[w];
  if (mode == kModeInit)
    for (int w = threadIdx.x; w < nw; w += blockDim.x) W.bits_best[w] = W.bits[w];
  if (threadIdx.x == 0) {
    int m = 0;
    float s = 0.f;
    uint32_t Fs[kWideLimbs];
    wide_zero(Fs);
    if (single) {
      m = s_bm;
      s = s_bs;
      if (need_F) wide_load(Fs, s_bF);
    } else {
      for (uint32_t c = 0; c < W.nchunk_apply; c++) {
        const uint32_t *p = W.ap_part + (size_t)c * kApplyPartStride;
        m = max(m, (int)__ldcg(p));
        s += __uint_as_float(__ldcg(p + 1));
        if (need_F) {
          uint32_t t[kWideLimbs];
          wide_load_cg(t, p + 2);
          wide_add(Fs, t);
        }
      }
    }
    W.psl = m;
    W.S_abs = s;
    W.alpha = alpha;
    if (need_F) {
      wide_store(W.F, Fs);
      wide_store(W.value_local, Fs);
    }
    // lowest-F pivot: the start, or a perturbed pivot of a switch below it
    s_fcopy = 0;
    if (W.track_fbest && need_F) {
      uint32_t fb[kWideLimbs];
      wide_load(fb, W.F_best);
      if (mode == kModeInit || wide_cmp(Fs, fb) < 0) {
        wide_store(W.F_best, Fs);
        s_fcopy = 1;
      }
    }
    if (mode == kModeInit) {
      W.psl_best = m;
      W.psl_local = m;
    } else if (W.improved) {
      W.psl_local = m;
    }
    W.ktau_on = (m < W.psl_best + 4) ? 1u : 0u;
    const uint64_t step = W.moves;  // moves already counts this step (or 0 at init)
    if (mode != kModeInit && W.trace && step >= 1 && step - 1 < W.trace_cap) W.trace[step - 1].psl = m;
    if (mode != kModeInit && W.moves >= W.budget) {
      W.status = kDone;
    } else {
      W.start = (uint32_t)(splitmix64(W.seed, W.rng_ctr++) % (uint64_t)W.L);
    }
    W.arrive = 0;
  }
  if (W.track_fbest && need_F) {  // the same branch for every thread of the block
    __syncthreads();
    if (s_fcopy)
      for (int w = threadIdx.x; w < nw; w += blockDim.x) W.bits_fbest[w] = W.bits[w];
  }
}


__device__ __forceinline__ void apply_one(WalkDev &W, uint32_t chunk) {
  if (W.status != kRunning) return;
  if (chunk >= W.nchunk_apply) return;
  const uint32_t mode = W.mode;
  if (mode == kModeMove) return;  // k_apply_move's work
  const int L = (int)W.L;
  const int k0 = (int)chunk * kApplyChunk, k1 = min(k0 + kApplyChunk, L);
  const uint32_t alpha = W.alpha_next;
  const float inv2e = ldexpf(1.f, -W.e);
  const int thr = W.ktau_thr;
  const bool keep_local = (mode == kModeInit) || W.improved;
  const int nflip = (int)W.nflip;

  int pmax = 0;
  float sabs = 0.f;
  uint32_t F[kWideLimbs];
  wide_zero(F);
  for (int k = k0 + (int)threadIdx.x; k < k1; k += blockDim.x) {
    int c;
    if (k == 0) {
      c = L;
    } else if (mode == kModeInit) {
      c = W.C[k];
    } else {
      // several flips of local_best at once: a product s_i s_{i+k} changes sign exactly
      // when one of its two positions is flipped
      c = W.C_local[k];
      for (int q = 0; q < nflip; q++) {
        const int f = (int)W.flips[q];
        const int sf = sval(W.bits_local, f);
        const int p = f + k, m = f - k;
        if (p < L) {
          bool in = false;
          for (int r = 0; r < nflip; r++) in |= ((int)W.flips[r] == p);
          if (!in) c -= 2 * sf * sval(W.bits_local, p);
        }
        if (m >= 0) {
          bool in = false;
          for (int r = 0; r < nflip; r++) in |= ((int)W.flips[r] == m);
          if (!in) c -= 2 * sf * sval(W.bits_local, m);
        }
      }
    }
    W.C[k] = c;
    if (keep_local) W.C_local[k] = c;
    if (k >= 1) {
      const int a = c < 0 ? -c : c;
      pmax = max(pmax, a);
      const float4 t = tables_for(c, alpha, inv2e);
      W.T[k] = t;
      sabs += absmax4(t);
      if (a >= thr) {
        const uint32_t at = atomicAdd(&W.nktau, 1u);
        W.ktau[at] = make_int2(k, c);
      }
      add_pow_rt(F, (uint32_t)a, alpha);
    }
  }
  apply_finish<true>(W, chunk, mode, keep_local, 0, nflip, alpha, pmax, sabs, F);
}

// The update pass of an ordinary step (one move, Sec. 3: C'_k = C_k - 2 s_j (s_{j+k} +
// s_{j-k}), absent partners count 0) with the next window's tables for exponent A: four
// consecutive shifts per thread and iteration, C read and written as int4, the mover's
// partner bits for those shifts from one entry of each partner window, the table powers
// unrolled for A.
template <int A>
__device__ __forceinline__ void apply_move_one(WalkDev &W, uint32_t chunk) {
  const int L = (int)W.L;
  const int k0 = (int)chunk * kApplyChunk, k1 = min(k0 + kApplyChunk, L);
  const float inv2e = ldexpf(1.f, -W.e);
  const int thr = W.ktau_thr;
  const bool keep_local = W.improved != 0;
  const int kstar = (int)W.kstar;
  const int sk = sval(W.bits, kstar);
  const int kplus = L - 1 - kstar;  // shifts k <= kplus have the partner k* + k, k <= k* the partner k* - k
  int *__restrict__ C = W.C;
  int *__restrict__ Cl = W.C_local;
  float4 *__restrict__ T = W.T;
  int pmax = 0;
  float sabs = 0.f;
  for (int kq = k0 + 4 * (int)threadIdx.x; kq < k1; kq += 4 * (int)blockDim.x) {
    int c[4];
    if (kq + 3 < L) {
      const int4 v = *reinterpret_cast<const int4 *>(C + kq);
      c[0] = v.x, c[1] = v.y, c[2] = v.z, c[3] = v.w;
    } else {
#pragma unroll
      for (int q = 0; q < 4; q++) c[q] = kq + q < L ? C[kq + q] : 0;
    }
    // bit q: s_{k*+kq+q} and s_{k*-kq-q} (past either end the bits read 0; those shifts have no partner)
    const uint32_t up = W.win_f[min(kstar + kq, L)], dn = W.win_r[max(kstar - kq, -1)];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int k = kq + q;
      const int part = (k <= kplus ? 1 - 2 * (int)((up >> q) & 1u) : 0) + (k <= kstar ? 1 - 2 * (int)((dn >> q) & 1u) : 0);
      c[q] = (k == 0) ? L : c[q] - 2 * sk * part;
    }
    if (kq + 3 < L) {
      *reinterpret_cast<int4 *>(C + kq) = make_int4(c[0], c[1], c[2], c[3]);
      if (keep_local) *reinterpret_cast<int4 *>(Cl + kq) = make_int4(c[0], c[1], c[2], c[3]);
    } else {
#pragma unroll
      for (int q = 0; q < 4; q++)
        if (kq + q < L) {
          C[kq + q] = c[q];
          if (keep_local) Cl[kq + q] = c[q];
        }
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int k = kq + q;
      if (k >= 1 && k < L) {
        const int a = c[q] < 0 ? -c[q] : c[q];
        const float4 tv = tables_for(c[q], (uint32_t)A, inv2e);
        T[k] = tv;
        pmax = max(pmax, a);
        sabs += absmax4(tv);
        if (a >= thr) {
          const uint32_t at = atomicAdd(&W.nktau, 1u);
          W.ktau[at] = make_int2(k, c[q]);
        }
      }
    }
  }
  uint32_t F[kWideLimbs];  // unused: an ordinary move takes F from the exact re-check
  apply_finish<false>(W, chunk, kModeMove, keep_local, kstar, 0, (uint32_t)A, pmax, sabs, F);
}

__device__ __forceinline__ void apply_move_dispatch(WalkDev &W, uint32_t chunk) {
  switch (W.alpha_next) {
    case 1: apply_move_one<1>(W, chunk); break;
    case 2: apply_move_one<2>(W, chunk); break;
    case 3: apply_move_one<3>(W, chunk); break;
    case 4: apply_move_one<4>(W, chunk); break;
    case 5: apply_move_one<5>(W, chunk); break;
    case 6: apply_move_one<6>(W, chunk); break;
    case 7: apply_move_one<7>(W, chunk); break;
    case 8: apply_move_one<8>(W, chunk); break;
    case 9: apply_move_one<9>(W, chunk); break;
    case 10: apply_move_one<10>(W, chunk); break;
    case 11: apply_move_one<11>(W, chunk); break;
    case 12: apply_move_one<12>(W, chunk); break;
    case 13: apply_move_one<13>(W, chunk); break;
    case 14: apply_move_one<14>(W, chunk); break;
    case 15: apply_move_one<15>(W, chunk); break;
    default: apply_move_one<16>(W, chunk); break;
  }
}

// ------------------------------------------------------------------------------------
// select: certified candidate set and the window's first minimum PSL
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t float_order(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ void select_one(WalkDev &W) {
  __shared__ float s_f[32];
  __shared__ unsigned long long s_u[32];
  __shared__ uint32_t s_cnt[32];
  __shared__ float s_m;
  __shared__ unsigned long long s_key;
  __shared__ uint32_t s_extra[16];
  __shared__ uint32_t s_total;
  if (W.status != kRunning) return;
  const int N = (int)W.N;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const float *score = W.score;
  const uint32_t ksplit = W.ksplit;
  if (ksplit > 1) {
    // partial scores of the k-chunks, summed in chunk order
    for (int i = tid; i < N; i += blockDim.x) {
      float sc = W.score_part[i];
      for (uint32_t c = 1; c < ksplit; c++) sc += W.score_part[(size_t)c * N + i];
      W.score[i] = sc;
    }
    __syncthreads();
  }

  float m = FLT_MAX;
  for (int i = tid; i < N; i += blockDim.x) m = fminf(m, score[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) s_f[warp] = m;
  __syncthreads();
  if (tid == 0) {
    float mm = FLT_MAX;
    for (int w = 0; w < nwarps; w++) mm = fminf(mm, s_f[w]);
    s_m = mm;
  }
  __syncthreads();
  m = s_m;
  const double B = score_bound(W.S_abs, W.alpha, W.L, ksplit);
  const float thr = __double2float_ru((double)m + 2.0 * B);

  // ordered compaction of {i : score <= thr}: each thread owns a contiguous segment
  const int seg = (N + (int)blockDim.x - 1) / (int)blockDim.x;
  const int i0 = tid * seg, i1 = min(N, i0 + seg);
  uint32_t cnt = 0;
  for (int i = i0; i < i1; i++) cnt += score[i] <= thr;
  uint32_t incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_cnt[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t v = lane < nwarps ? s_cnt[lane] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    s_cnt[lane] = x - v;  // exclusive prefix of warp totals
  }
  __syncthreads();
  uint32_t off = s_cnt[warp] + incl - cnt;
  for (int i = i0; i < i1; i++)
    if (score[i] <= thr) W.cand[off++] = (uint32_t)(i + 1);
  if (tid == (int)blockDim.x - 1) s_total = off;  // end offset of the last segment
  __syncthreads();
  const uint32_t total = s_total;

  // FP32 top-k beyond the certified set
  const uint32_t topk = min(W.topk, 16u);
  uint32_t nextra = 0;
  unsigned long long last = 0;
  while (total + nextra < topk && total + nextra < (uint32_t)N) {
    unsigned long long best = ~0ull;
    for (int i = tid; i < N; i += blockDim.x) {
      const float f = score[i];
      if (f <= thr) continue;
      const unsigned long long key = ((unsigned long long)float_order(f) << 32) | (uint32_t)i;
      if (key > last) best = min(best, key);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
    if (lane == 0) s_u[warp] = best;
    __syncthreads();
    if (tid == 0) {
      unsigned long long b = ~0ull;
      for (int w = 0; w < nwarps; w++) b = min(b, s_u[w]);
      s_key = b;
    }
    __syncthreads();
    last = s_key;
    __syncthreads();
    if (last == ~0ull) break;
    if (tid == 0) s_extra[nextra] = (uint32_t)(last & 0xffffffffu) + 1u;
    nextra++;
  }
  __syncthreads();
  if (tid == 0) {
    // merge the extra positions into the ascending candidate list
    uint32_t n = total;
    for (uint32_t e = 0; e < nextra; e++) {
      const uint32_t v = s_extra[e];
      uint32_t p = n;
      while (p > 0 && W.cand[p - 1] > v) {
        W.cand[p] = W.cand[p - 1];
        p--;
      }
      W.cand[p] = v;
      n++;
    }
    W.ncand = n;
    W.score_min = m;
    W.bound = (float)B;
  }

  // first minimum of psl_j in scan order
  unsigned long long pk = ~0ull;
  if (W.ktau_on) {
    for (int i = tid; i < N; i += blockDim.x) {
      const int p = W.pslj[i];
      pk = min(pk, ((unsigned long long)(uint32_t)p << 32) | (uint32_t)(i + 1));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) pk = min(pk, __shfl_xor_sync(0xffffffffu, pk, o));
  if (lane == 0) s_u[warp] = pk;
  __syncthreads();
  if (tid == 0) {
    unsigned long long b = ~0ull;
    for (int w = 0; w < nwarps; w++) b = min(b, s_u[w]);
    W.win_psl = (b == ~0ull) ? INT_MAX : (int)(b >> 32);
    W.win_psl_i = (uint32_t)(b & 0xffffffffu);
  }
}

// The same selection by one warp, for windows of at most kSelectWarpN neighbours: the
// compaction goes 32 positions at a time (ballot + popcount keeps scan order) and every
// reduction is a shuffle, so many short walks are served at once without block barriers.
constexpr int kSelectWarpN = 2048;
static_assert(kTailMaxN == (uint32_t)kSelectWarpN && kTailMaxL <= (uint32_t)kRecheckChunk,
              "the fused step tail needs one warp selection, one update chunk and one re-check chunk per walk");

__device__ __forceinline__ void select_warp(WalkDev &W) {
  const int lane = threadIdx.x & 31;
  if (W.status != kRunning) return;
  const int N = (int)W.N;
  float *score = W.score;
  const uint32_t ksplit = W.ksplit;
  if (ksplit > 1) {
    // partial scores of the k-chunks, summed in chunk order
    for (int i = lane; i < N; i += 32) {
      float sc = W.score_part[i];
      for (uint32_t c = 1; c < ksplit; c++) sc += W.score_part[(size_t)c * N + i];
      score[i] = sc;
    }
    __syncwarp();
  }
  float m = FLT_MAX;
  for (int i = lane; i < N; i += 32) m = fminf(m, score[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
  const double B = score_bound(W.S_abs, W.alpha, W.L, ksplit);
  const float thr = __double2float_ru((double)m + 2.0 * B);

  // ordered compaction of {i : score <= thr}
  uint32_t total = 0;
  const uint32_t below = (1u << lane) - 1u;
  for (int base = 0; base < N; base += 32) {
    const int i = base + lane;
    const bool in = i < N && score[i] <= thr;
    const uint32_t bal = __ballot_sync(0xffffffffu, in);
    if (in) W.cand[total + __popc(bal & below)] = (uint32_t)(i + 1);
    total += __popc(bal);
  }

  // FP32 top-k beyond the certified set
  const uint32_t topk = min(W.topk, 16u);
  uint32_t extra[16];
  uint32_t nextra = 0;
  unsigned long long last = 0;
  while (total + nextra < topk && total + nextra < (uint32_t)N) {
    unsigned long long best = ~0ull;
    for (int i = lane; i < N; i += 32) {
      const float f = score[i];
      if (f <= thr) continue;
      const unsigned long long key = ((unsigned long long)float_order(f) << 32) | (uint32_t)i;
      if (key > last) best = min(best, key);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
    last = best;
    if (last == ~0ull) break;
    extra[nextra++] = (uint32_t)(last & 0xffffffffu) + 1u;
  }
  __syncwarp();
  if (lane == 0) {
    // merge the extra positions into the ascending candidate list
    uint32_t n = total;
    for (uint32_t e = 0; e < nextra; e++) {
      const uint32_t v = extra[e];
      uint32_t p = n;
      while (p > 0 && W.cand[p - 1] > v) {
        W.cand[p] = W.cand[p - 1];
        p--;
      }
      W.cand[p] = v;
      n++;
    }
    W.ncand = n;
    W.score_min = m;
    W.bound = (float)B;
  }

  // first minimum of psl_j in scan order
  unsigned long long pk = ~0ull;
  if (W.ktau_on) {
    for (int i = lane; i < N; i += 32) {
      const int p = W.pslj[i];
      pk = min(pk, ((unsigned long long)(uint32_t)p << 32) | (uint32_t)(i + 1));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) pk = min(pk, __shfl_xor_sync(0xffffffffu, pk, o));
  if (lane == 0) {
    W.win_psl = (pk == ~0ull) ? INT_MAX : (int)(pk >> 32);
    W.win_psl_i = (uint32_t)(pk & 0xffffffffu);
  }
}

// ------------------------------------------------------------------------------------
// recheck: exact Delta F = sum_{k: delta != 0} |C_k + delta|^alpha - |C_k|^alpha of the
// candidates, one CTA per (chunk of k, candidate); positive and negative parts are
// accumulated separately as unsigned 384-bit integers.
// ------------------------------------------------------------------------------------
// Delta F of neighbour j over shifts kbeg..kend-1, accumulated as two unsigned sums
// (|C_k + delta|^A and |C_k|^A over the shifts with delta != 0) in NL-limb registers: four
// consecutive shifts per thread and iteration, C read as int4, the neighbour's partner bits
// for those shifts from one entry of each partner window.
template <int A, int NL, typename Acc>
__device__ __forceinline__ void recheck_quads(const WalkDev &W, int j, int kbeg, int kend, Acc &P, Acc &Q) {
  const int L = (int)W.L;
  const int sj = sval(W.bits, j);
  const int kplus = L - 1 - j;  // shifts k <= kplus have the partner j + k, k <= j the partner j - k
  const int *__restrict__ C = W.C;
  for (int kq = (kbeg & ~3) + 4 * (int)threadIdx.x; kq < kend; kq += 4 * (int)blockDim.x) {
    int c[4];
    if (kq + 3 < L) {
      const int4 v = *reinterpret_cast<const int4 *>(C + kq);
      c[0] = v.x, c[1] = v.y, c[2] = v.z, c[3] = v.w;
    } else {
#pragma unroll
      for (int q = 0; q < 4; q++) c[q] = kq + q < L ? C[kq + q] : 0;
    }
    // bit q: s_{j+kq+q} and s_{j-kq-q} (past either end the bits read 0; those shifts have no partner)
    const uint32_t up = W.win_f[min(j + kq, L)], dn = W.win_r[max(j - kq, -1)];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const int k = kq + q;
      const int part = (k <= kplus ? 1 - 2 * (int)((up >> q) & 1u) : 0) + (k <= j ? 1 - 2 * (int)((dn >> q) & 1u) : 0);
      if (k < kbeg || k >= kend || part == 0) continue;
      const int cn = c[q] - 2 * sj * part;
      if constexpr (NL == kWideLimbs) {
        add_pow<A>(P, (uint32_t)(cn < 0 ? -cn : cn));
        add_pow<A>(Q, (uint32_t)(c[q] < 0 ? -c[q] : c[q]));
      } else {
        add_pow_n<A, NL>(P, (uint32_t)(cn < 0 ? -cn : cn));
        add_pow_n<A, NL>(Q, (uint32_t)(c[q] < 0 ? -c[q] : c[q]));
      }
    }
  }
}

template <int A, int NL>
__device__ void recheck_body_n(const WalkDev &W, int j, int kbeg, int kend, uint32_t (&pos)[kWideLimbs],
                               uint32_t (&neg)[kWideLimbs]) {
  uint32_t P[NL], Q[NL];
#pragma unroll
  for (int i = 0; i < NL; i++) P[i] = Q[i] = 0;
  recheck_quads<A, NL>(W, j, kbeg, kend, P, Q);
#pragma unroll
  for (int i = 0; i < kWideLimbs; i++) pos[i] = i < NL ? P[i] : 0u, neg[i] = i < NL ? Q[i] : 0u;
}

// acc += d v^A on NL-limb accumulators, for d < 2^21 and v < 2^VB: after t factors v the
// product has at most 21 + VB t bits, so only the limbs that can be nonzero are multiplied.
// The caller guarantees that d v^A and every partial sum fit in 32 NL bits.
template <int A, int NL, int VB>
__device__ __forceinline__ void add_scaled_pow_n(uint32_t (&acc)[NL], uint32_t v, uint32_t d) {
  uint32_t p[NL];
  p[0] = d;
#pragma unroll
  for (int i = 1; i < NL; i++) p[i] = 0;
#pragma unroll
  for (int t = 1; t <= A; t++) {
    uint64_t carry = 0;
#pragma unroll
    for (int i = 0; i < NL; i++) {
      if (i < (21 + VB * t + 31) / 32) {
        const uint64_t x = (uint64_t)p[i] * v + carry;
        p[i] = (uint32_t)x;
        carry = x >> 32;
      }
    }
  }
  wide_add_n<NL>(acc, p);
}

// Exact Delta F of one candidate over the shifts [kbeg, kend) by value counts (Eq. 4 through
// the flip of Sec. 3).  With n_v and n'_v the numbers of changed shifts whose |C_k| and
// |C_k + delta_k| equal v,  sum_k (|C_k + delta_k|^a - |C_k|^a) = sum_v (n'_v - n_v) v^a,
// an identity of integers.  The count differences go into a shared-memory histogram of 2^e
// bins (every such value of this window is below 2^e); each nonzero count is then raised
// to the power once, instead of two wide powers per shift.  e <= HL (the histogram's size).
template <int A, int NL, int HL>
__device__ void recheck_hist_n(WalkDev &W, int *__restrict__ hist, int j, int kbeg, int kend,
                               uint32_t (&pos)[kWideLimbs], uint32_t (&neg)[kWideLimbs]) {
  const int L = (int)W.L;
  const int nbin = 1 << W.e;
  for (int v = (int)threadIdx.x; v < nbin; v += (int)blockDim.x) hist[v] = 0;
  __syncthreads();
  const int sj = sval(W.bits, j);
  const int kplus = L - 1 - j;  // shifts k <= kplus have the partner j + k, k <= j the partner j - k
  const int *__restrict__ C = W.C;
  const uint32_t *__restrict__ win_f = W.win_f;
  const uint32_t *__restrict__ win_r = W.win_r;
  bool bad = false;
  // U quads of four consecutive shifts per thread in flight: the loop is bound by the
  // latency of these loads, not by the few operations per shift
  constexpr int U = 4;
  const int stride = 4 * (int)blockDim.x;
  for (int kq0 = (kbeg & ~3) + 4 * (int)threadIdx.x; kq0 < kend; kq0 += U * stride) {
    int c[U][4];
    uint32_t up[U], dn[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int kq = kq0 + u * stride;
      if (kq + 3 < L) {
        const int4 x = *reinterpret_cast<const int4 *>(C + kq);
        c[u][0] = x.x, c[u][1] = x.y, c[u][2] = x.z, c[u][3] = x.w;
      } else {
#pragma unroll
        for (int q = 0; q < 4; q++) c[u][q] = kq + q < L ? C[kq + q] : 0;
      }
      // bit q: s_{j+kq+q} and s_{j-kq-q} (past either end the bits read 0; those shifts have no partner)
      up[u] = win_f[min(j + kq, L)];
      dn[u] = win_r[max(j - kq, -1)];
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const int k = kq0 + u * stride + q;
        const int part = (k <= kplus ? 1 - 2 * (int)((up[u] >> q) & 1u) : 0) +
                         (k <= j ? 1 - 2 * (int)((dn[u] >> q) & 1u) : 0);
        if (k < kbeg || k >= kend || part == 0) continue;
        const int cn = c[u][q] - 2 * sj * part;
        const int a = cn < 0 ? -cn : cn, b = c[u][q] < 0 ? -c[u][q] : c[u][q];
        if (a == b) continue;  // the two terms cancel
        if (a < nbin && b < nbin) {
          atomicAdd(&hist[a], 1);
          atomicAdd(&hist[b], -1);
        } else {
          bad = true;  // outside the bound the window was scaled to: an internal error
        }
      }
    }
  }
  __syncthreads();
  uint32_t P[NL], Q[NL];
#pragma unroll
  for (int i = 0; i < NL; i++) P[i] = Q[i] = 0;
  for (int v = (int)threadIdx.x; v < nbin; v += (int)blockDim.x) {
    const int d = hist[v];
    if (d > 0) add_scaled_pow_n<A, NL, HL>(P, (uint32_t)v, (uint32_t)d);
    else if (d < 0) add_scaled_pow_n<A, NL, HL>(Q, (uint32_t)v, (uint32_t)-d);
  }
  if (bad) {
    W.error = (uint32_t)-7;  // PSL_ESTATE of the library header
    W.status = kError;
  }
#pragma unroll
  for (int i = 0; i < kWideLimbs; i++) pos[i] = i < NL ? P[i] : 0u, neg[i] = i < NL ? Q[i] : 0u;
}

// log2 of the bins of the re-check histogram: 16 KB of shared memory in the re-check
// kernel, 4 KB in the short-walk step kernel; windows with a larger e take the
// term-by-term sums
constexpr int kHistLog = 12, kHistLogShort = 10;

// Which sums a re-check kernel instantiates: both (the short-walk step kernel), only the
// histogram (walks with e <= kHistLog), only the term-by-term sums (the rest).  The two
// re-check kernels split the walks of a step between them, so that the frequent histogram
// path is not held to the occupancy of the 12-limb sums.
enum RecheckPath : int { kRcBoth = 0, kRcHist = 1, kRcTerms = 2 };

// SHORT: walks of L <= kTailMaxL only.  There PSL + 8 < 2^14, so e <= 14 and A e + 20 <= 244
// for every A <= 16: the 12-limb accumulators are never needed and are not instantiated.
template <int A, bool SHORT, int PATH>
__device__ void recheck_body(WalkDev &W, int *hist, int j, int kbeg, int kend, uint32_t (&pos)[kWideLimbs],
                             uint32_t (&neg)[kWideLimbs]) {
  // every |C_k + delta| of this window is below 2^e, so each power has at most A e bits and
  // a sum of fewer than 2^20 of them at most A e + 20: narrower accumulators where that fits
  const int bits = A * (int)W.e + 20;
  constexpr int HL = SHORT ? kHistLogShort : kHistLog;
  if constexpr (PATH != kRcTerms) {
    if ((int)W.e <= HL) {  // the same reading in every thread of the block
      // HL <= 12 and A <= 16 give A e + 20 <= 212: 4 or 8 limbs
      if (bits <= 128)
        recheck_hist_n<A, 4, HL>(W, hist, j, kbeg, kend, pos, neg);
      else
        recheck_hist_n<A, 8, HL>(W, hist, j, kbeg, kend, pos, neg);
      return;
    }
  }
  if constexpr (PATH != kRcHist) {
    if (bits <= 128) {
      recheck_body_n<A, 4>(W, j, kbeg, kend, pos, neg);
      return;
    }
    if (SHORT || bits <= 256) {
      recheck_body_n<A, 8>(W, j, kbeg, kend, pos, neg);
      return;
    }
    if constexpr (!SHORT) recheck_quads<A, kWideLimbs>(W, j, kbeg, kend, pos, neg);
  }
}

static_assert(kTailMaxL <= 8192u, "the SHORT re-check relies on e <= 14");

// exact: the step was scored by the alpha = 2 closed form, which kept every neighbour's exact
// Delta F (score_part as int32; such walks have one re-check chunk): the first call copies the
// candidates' values into their records, sign-extended, and the other calls have nothing to do.
template <bool SHORT, int PATH>
__device__ __forceinline__ void recheck_one(WalkDev &W, uint32_t chunk, uint32_t qslot, bool exact) {
  __shared__ uint32_t s_w[8][2 * kWideLimbs];
  __shared__ int s_hist[PATH == kRcTerms ? 1 : 1 << (SHORT ? kHistLogShort : kHistLog)];
  if (W.status != kRunning) return;
  if (chunk >= W.nchunk_rc) return;
  if (exact) {
    if (qslot != 0 || chunk != 0) return;
    const int *dF = reinterpret_cast<const int *>(W.score_part);
    for (uint32_t q = threadIdx.x; q < W.ncand; q += blockDim.x) {
      const int v = dF[W.cand[q] - 1];
      uint32_t P[kWideLimbs];
      P[0] = (uint32_t)v;
#pragma unroll
      for (int t = 1; t < kWideLimbs; t++) P[t] = v < 0 ? 0xffffffffu : 0u;
      const bool whole = q >= (uint32_t)kQcap;
      const size_t slot = whole ? ((size_t)kQcap * W.nchunk_rc + (q - kQcap)) : ((size_t)q * W.nchunk_rc);
      wide_store(W.rc_part + slot * kWideLimbs, P);
    }
    return;
  }
  const int L = (int)W.L;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t q = qslot; q < W.ncand; q += kQcap) {
    const int i = (int)W.cand[q];
    const int j = (int)(((uint64_t)W.start + (uint64_t)i) % (uint64_t)L);
    const int kout = max(j, L - 1 - j);
    const bool whole = q >= (uint32_t)kQcap;  // overflow candidates: one CTA covers every chunk
    if (whole && chunk != 0) continue;
    const int kbeg = whole ? 1 : max(1, (int)chunk * kRecheckChunk);
    const int kend = whole ? kout + 1 : min(kout + 1, ((int)chunk + 1) * kRecheckChunk);
    uint32_t pos[kWideLimbs], neg[kWideLimbs];
    wide_zero(pos);
    wide_zero(neg);
    if (kbeg < kend) {
      switch (W.alpha) {
        case 1: recheck_body<1, SHORT, PATH>(W, s_hist, j, kbeg, kend, pos, neg); break;
        case 2: recheck_body<2, SHORT, PATH>(W, s_hist, j, kbeg, kend, pos, neg); break;
        case 3: recheck_body<3, SHORT, PATH>(W, s_hist, j, kbeg, kend, pos, neg); break;
        case 4: recheck_body<4, SHORT, PATH>(W, s_hist, j, kbeg, kend, pos, neg); break;
        case 5: recheck_body<5, SHORT, PATH>(W, s_hist, j, kbeg, kend, pos, neg); break;
        case 6: recheck_body<6, SHORT, PATH>(W, s_hist, j, kbeg, kend, pos, neg); break;
        case 7: recheck_body<7, SHORT, PATH>(W, s_hist, j, kbeg, kend, pos, neg); break;
        case 8: recheck_body<8, SHORT, PATH>(W, s_hist, j, kbeg, kend, pos, neg); break;
        case 9: recheck_body<9, SHORT, PATH>(W, s_hist, j, kbeg, kend, pos, neg); break;
        case 10: recheck_body<10, SHORT, PATH>(W, s_hist, j, kbeg, kend, pos, neg); break;
        case 11: recheck_body<11, SHORT, PATH>(W, s_hist, j, kbeg, kend, pos, neg); break;
        case 12: recheck_body<12, SHORT, PATH>(W, s_hist, j, kbeg, kend, pos, neg); break;
        case 13: recheck_body<13, SHORT, PATH>(W, s_hist, j, kbeg, kend, pos, neg); break;
        case 14: recheck_body<14, SHORT, PATH>(W, s_hist, j, kbeg, kend, pos, neg); break;
        case 15: recheck_body<15, SHORT, PATH>(W, s_hist, j, kbeg, kend, pos, neg); break;
        default: recheck_body<16, SHORT, PATH>(W, s_hist, j, kbeg, kend, pos, neg); break;
      }
    }
    // the sums fill nl limbs (the accumulator width chosen from alpha e + 20 above): only
    // those travel through the shuffles
    const int bits = (int)W.alpha * (int)W.e + 20;
    const int nl = bits <= 128 ? 4 : (bits <= 256 ? 8 : kWideLimbs);
    for (int o = 16; o > 0; o >>= 1) {
      uint32_t a[kWideLimbs], b[kWideLimbs];
#pragma unroll
      for (int t = 0; t < kWideLimbs; t++) {
        a[t] = t < nl ? __shfl_down_sync(0xffffffffu, pos[t], o) : 0u;  // nl is the same in every lane
        b[t] = t < nl ? __shfl_down_sync(0xffffffffu, neg[t], o) : 0u;
      }
      if (lane < o) {
        wide_add(pos, a);
        wide_add(neg, b);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int t = 0; t < kWideLimbs; t++) {
        s_w[warp][t] = pos[t];
        s_w[warp][kWideLimbs + t] = neg[t];
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t P[kWideLimbs], Q[kWideLimbs];
      wide_zero(P);
      wide_zero(Q);
      for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
        uint32_t a[kWideLimbs], b[kWideLimbs];
#pragma unroll
        for (int t = 0; t < kWideLimbs; t++) {
          a[t] = s_w[w][t];
          b[t] = s_w[w][kWideLimbs + t];
        }
        wide_add(P, a);
        wide_add(Q, b);
      }
      wide_sub(P, Q);  // signed Delta F of this chunk
      const size_t slot = whole ? ((size_t)kQcap * W.nchunk_rc + (q - kQcap)) : ((size_t)q * W.nchunk_rc + chunk);
      wide_store(W.rc_part + slot * kWideLimbs, P);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------
// decide: exact argmin over the candidates (strict "<" in scan order), the best-PSL
// update, and the bookkeeping / phase switch of Alg. 1
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void decide_one(WalkDev &W) {
  __shared__ uint32_t s_best[kWideLimbs];
  __shared__ uint32_t s_bi;
  if (W.status != kRunning) return;
  const int L = (int)W.L;
  if (threadIdx.x == 0) {
    uint32_t F[kWideLimbs], best[kWideLimbs];
    wide_load(F, W.F);
    uint32_t bi = 0;
    for (uint32_t q = 0; q < W.ncand; q++) {
      uint32_t v[kWideLimbs];
      wide_load(v, F);
      if (q < (uint32_t)kQcap) {
        for (uint32_t c = 0; c < W.nchunk_rc; c++) {
          uint32_t t[kWideLimbs];
          wide_load(t, W.rc_part + ((size_t)q * W.nchunk_rc + c) * kWideLimbs);
          wide_add(v, t);
        }
      } else {
        uint32_t t[kWideLimbs];
        wide_load(t, W.rc_part + ((size_t)kQcap * W.nchunk_rc + (q - kQcap)) * kWideLimbs);
        wide_add(v, t);
      }
      if (q == 0 || wide_cmp(v, best) < 0) {
        wide_load(best, v);
        bi = q;
      }
    }
    wide_store(s_best, best);
    s_bi = bi;
  }
  __syncthreads();
  const uint32_t kstar_i = W.cand[s_bi];
  const uint32_t kstar = (uint32_t)(((uint64_t)W.start + kstar_i) % (uint64_t)L);
  // psl_best / solution_best: the first neighbour reaching the window minimum
  const bool psl_imp = W.ktau_on && W.win_psl < W.psl_best;
  const uint32_t pj = (uint32_t)(((uint64_t)W.start + W.win_psl_i) % (uint64_t)L);
  // lowest-F pivot (one objective): the move's result when it is below every earlier pivot
  bool f_imp = false;
  if (W.track_fbest) {
    uint32_t v[kWideLimbs], fb[kWideLimbs];
    wide_load(v, s_best);
    wide_load(fb, W.F_best);
    f_imp = wide_cmp(v, fb) < 0;
  }
  if (psl_imp || f_imp) {
    const int nw = (int)W.nw;
    for (int w = threadIdx.x; w < nw; w += blockDim.x) {
      const uint32_t b = W.bits[w];
      if (psl_imp) W.bits_best[w] = b;
      if (f_imp) W.bits_fbest[w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (psl_imp) W.bits_best[pj >> 5] ^= 1u << (pj & 31);
      if (f_imp) W.bits_fbest[kstar >> 5] ^= 1u << (kstar & 31);
    }
  }
  if (threadIdx.x != 0) return;
  if (f_imp) wide_store(W.F_best, s_best);

  const int32_t e_used = W.e;  // scale of this step's tables, before the next one is chosen
  uint32_t vstep[kWideLimbs], vlocal[kWideLimbs];
  wide_load(vstep, s_best);
  wide_load(vlocal, W.value_local);
  const int cmp = wide_cmp(vstep, vlocal);
  const uint32_t alpha_used = W.alpha;
  uint32_t flags = 0;
  if (psl_imp) {
    W.psl_best = W.win_psl;
    flags |= kPslBest;
  }
  W.kstar = kstar;
  W.kstar_i = kstar_i;
  wide_store(W.value_step, vstep);
  wide_store(W.F, vstep);
  W.improved = 0;
  W.mode = kModeMove;
  W.alpha_next = alpha_used;
  uint32_t nfl = 0;
  if (cmp < 0) {
    flags |= kImproved;
    W.unimproved = 0;
    W.improved = 1;
    wide_store(W.value_local, vstep);
  } else if (cmp > 0) {
    flags |= kWorse;
    W.unimproved++;
    if (W.unimproved > W.ls_lmt) {
      // Rand_flip(local_best, FLIP_lmt): distinct positions drawn with rejection
      nfl = W.nflip;
      uint32_t n = 0;
      while (n < nfl) {
        const uint32_t f = (uint32_t)(splitmix64(W.seed, W.rng_ctr++) % (uint64_t)L);
        bool dup = false;
        for (uint32_t r = 0; r < n; r++) dup |= (W.flips[r] == f);
        if (!dup) W.flips[n++] = f;
      }
      W.mode = kModeSwitch;
      W.alpha_next = (alpha_used == W.alpha1) ? W.alpha2 : W.alpha1;
      W.unimproved = 0;
      W.switches++;
      flags |= kSwitch;
    }
  }
  // scale of the next window's tables and threshold of its near-peak list
  if (W.mode == kModeSwitch) {
    const int bound = W.psl_local + 4 * (int)nfl;
    W.e = bitlen((uint32_t)bound + 8u);
    W.ktau_thr = W.psl_local - 4 * (int)nfl - 8;
  } else {
    W.e = bitlen((uint32_t)W.psl + 8u);
    W.ktau_thr = W.psl - 12;
  }
  W.nktau = 0;
  W.psl_improved = psl_imp ? 1u : 0u;
  W.psl_j = pj;
  const uint64_t step = W.moves;
  W.moves++;
  W.flip_evals += W.N;
  W.rechecks += W.ncand;
  if (W.trace && step < W.trace_cap) {
    TraceRec &r = W.trace[step];
    r.step = step;
    r.start = W.start;
    r.kstar = kstar;
    r.alpha = alpha_used;
    r.unimproved = W.unimproved;
    r.psl = 0;  // filled by the update pass
    r.psl_best = W.psl_best;
    r.win_psl = W.ktau_on ? W.win_psl : INT_MAX;
    r.win_psl_j = W.ktau_on ? pj : 0u;
    r.flags = flags;
    r.nflip = nfl;
    r.ncand = W.ncand;
    r.score_kstar = W.score[kstar_i - 1];
    r.score_min = W.score_min;
    r.bound = W.bound;
    r.scale_e = e_used;
    r.value_step = wide_to_double(vstep);
    wide_store(r.value_exact, vstep);
  }
}

}  // namespace psl
