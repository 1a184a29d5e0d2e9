// psl_kernels.cu -- CUDA kernels (sm_103a) for the limited-neighbourhood search of
// Boskovic and Brest, "Two-phase Optimization of Binary Sequences with Low Peak
// Sidelobe Level Value" (arXiv 2107.09801).
//
// One walk step (the body of the while loop of Algorithm 1) is five kernels:
//   hot     FP32 filter score of every neighbour in the window (Eq. 4 through the
//           one-element flip of Sec. 3) and, when it can matter, its exact PSL (Eq. 3)
//   select  minimum score, the certified candidate set {score <= min + 2B} plus the
//           FP32 top-k, and the first neighbour of minimum PSL
//   recheck exact 384-bit Delta F of every candidate
//   decide  exact argmin (first in scan order), bookkeeping and phase switch of Alg. 1
//   apply   O(L) update of C, PSL, the next step's per-k tables and near-peak list
// Every wait between blocks is a "last block to arrive finishes the walk" counter:
// no block ever spins.
#include <cfloat>
#include <climits>
#include <cstdint>
#include <mutex>

#include "psl_internal.h"

namespace psl {

// ------------------------------------------------------------------------------------
// helpers
// ------------------------------------------------------------------------------------
// Rand of Alg. 1: SplitMix64 (Steele, Lea, Flood 2014), draw n of the walk seeded S.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t n) {
  uint64_t z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// 32 sequence bits starting at bit position pos (pos may lie in the guard words).
__device__ __forceinline__ uint32_t window32(const uint32_t *bits, int pos) {
  const int w = pos >> 5;  // floor division
  return __funnelshift_r(bits[w], bits[w + 1], pos & 31);
}

__device__ __forceinline__ int getbit(const uint32_t *bits, int pos) { return (bits[pos >> 5] >> (pos & 31)) & 1; }

// s_pos in {+1,-1}
__device__ __forceinline__ int sval(const uint32_t *bits, int pos) { return 1 - 2 * getbit(bits, pos); }

// ---- 384-bit unsigned arithmetic on 12 x 32-bit limbs (carry chains in PTX) ----
__device__ __forceinline__ void wide_zero(uint32_t (&a)[kWideLimbs]) {
#pragma unroll
  for (int i = 0; i < kWideLimbs; i++) a[i] = 0;
}

__device__ __forceinline__ void wide_add(uint32_t (&a)[kWideLimbs], const uint32_t (&b)[kWideLimbs]) {
  asm("add.cc.u32 %0, %0, %12;\n\t"
      "addc.cc.u32 %1, %1, %13;\n\t"
      "addc.cc.u32 %2, %2, %14;\n\t"
      "addc.cc.u32 %3, %3, %15;\n\t"
      "addc.cc.u32 %4, %4, %16;\n\t"
      "addc.cc.u32 %5, %5, %17;\n\t"
      "addc.cc.u32 %6, %6, %18;\n\t"
      "addc.cc.u32 %7, %7, %19;\n\t"
      "addc.cc.u32 %8, %8, %20;\n\t"
      "addc.cc.u32 %9, %9, %21;\n\t"
      "addc.cc.u32 %10, %10, %22;\n\t"
      "addc.u32 %11, %11, %23;"
      : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]),
        "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11])
      : "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]), "r"(b[8]),
        "r"(b[9]), "r"(b[10]), "r"(b[11]));
}

__device__ __forceinline__ void wide_sub(uint32_t (&a)[kWideLimbs], const uint32_t (&b)[kWideLimbs]) {
  asm("sub.cc.u32 %0, %0, %12;\n\t"
      "subc.cc.u32 %1, %1, %13;\n\t"
      "subc.cc.u32 %2, %2, %14;\n\t"
      "subc.cc.u32 %3, %3, %15;\n\t"
      "subc.cc.u32 %4, %4, %16;\n\t"
      "subc.cc.u32 %5, %5, %17;\n\t"
      "subc.cc.u32 %6, %6, %18;\n\t"
      "subc.cc.u32 %7, %7, %19;\n\t"
      "subc.cc.u32 %8, %8, %20;\n\t"
      "subc.cc.u32 %9, %9, %21;\n\t"
      "subc.cc.u32 %10, %10, %22;\n\t"
      "subc.u32 %11, %11, %23;"
      : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]),
        "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11])
      : "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]), "r"(b[8]),
        "r"(b[9]), "r"(b[10]), "r"(b[11]));
}

// signed compare of two's-complement values whose magnitudes stay below 2^383
__device__ __forceinline__ int wide_cmp(const uint32_t (&a)[kWideLimbs], const uint32_t (&b)[kWideLimbs]) {
  uint32_t d[kWideLimbs];
#pragma unroll
  for (int i = 0; i < kWideLimbs; i++) d[i] = a[i];
  wide_sub(d, b);
  if (d[kWideLimbs - 1] >> 31) return -1;
  uint32_t any = 0;
#pragma unroll
  for (int i = 0; i < kWideLimbs; i++) any |= d[i];
  return any ? 1 : 0;
}

__device__ __forceinline__ void wide_load(uint32_t (&a)[kWideLimbs], const uint32_t *p) {
#pragma unroll
  for (int i = 0; i < kWideLimbs; i++) a[i] = p[i];
}
__device__ __forceinline__ void wide_store(uint32_t *p, const uint32_t (&a)[kWideLimbs]) {
#pragma unroll
  for (int i = 0; i < kWideLimbs; i++) p[i] = a[i];
}
__device__ __forceinline__ void wide_load_cg(uint32_t (&a)[kWideLimbs], const uint32_t *p) {
#pragma unroll
  for (int i = 0; i < kWideLimbs; i++) a[i] = __ldcg(p + i);
}

// acc += c^A for 0 <= c < 2^21 (limb count grows with the power; loops unroll fully)
template <int A>
__device__ __forceinline__ void add_pow(uint32_t (&acc)[kWideLimbs], uint32_t c) {
  uint32_t p[kWideLimbs];
  p[0] = c;
#pragma unroll
  for (int i = 1; i < kWideLimbs; i++) p[i] = 0;
#pragma unroll
  for (int t = 2; t <= A; t++) {
    uint64_t carry = 0;
#pragma unroll
    for (int i = 0; i < kWideLimbs; i++) {
      if (i < (21 * t + 31) / 32) {
        const uint64_t v = (uint64_t)p[i] * c + carry;
        p[i] = (uint32_t)v;
        carry = v >> 32;
      }
    }
  }
  wide_add(acc, p);
}

__device__ __forceinline__ void add_pow_rt(uint32_t (&acc)[kWideLimbs], uint32_t c, uint32_t alpha) {
  switch (alpha) {
    case 1: add_pow<1>(acc, c); break;
    case 2: add_pow<2>(acc, c); break;
    case 3: add_pow<3>(acc, c); break;
    case 4: add_pow<4>(acc, c); break;
    case 5: add_pow<5>(acc, c); break;
    case 6: add_pow<6>(acc, c); break;
    case 7: add_pow<7>(acc, c); break;
    case 8: add_pow<8>(acc, c); break;
    case 9: add_pow<9>(acc, c); break;
    case 10: add_pow<10>(acc, c); break;
    case 11: add_pow<11>(acc, c); break;
    case 12: add_pow<12>(acc, c); break;
    case 13: add_pow<13>(acc, c); break;
    case 14: add_pow<14>(acc, c); break;
    case 15: add_pow<15>(acc, c); break;
    default: add_pow<16>(acc, c); break;
  }
}

// Correctly rounded (nearest, ties to even) FP64 value of a two's-complement 384-bit integer.
__device__ double wide_to_double(const uint32_t (&a)[kWideLimbs]) {
  uint32_t m[kWideLimbs];
  wide_load(m, a);
  const bool neg = m[kWideLimbs - 1] >> 31;
  if (neg) {
    uint32_t z[kWideLimbs];
    wide_zero(z);
    wide_sub(z, m);
    wide_load(m, z);
  }
  int top = -1;
  for (int i = kWideLimbs - 1; i >= 0; i--)
    if (m[i]) {
      top = 32 * i + 31 - __clz(m[i]);
      break;
    }
  if (top < 0) return 0.0;
  auto bit = [&](int i) -> uint32_t { return (m[i >> 5] >> (i & 31)) & 1u; };
  double r;
  if (top <= 52) {
    r = (double)(((uint64_t)m[1] << 32) | m[0]);
  } else {
    const int drop = top - 52;
    uint64_t mant = 0;
    for (int i = top; i >= drop; i--) mant = (mant << 1) | bit(i);
    const uint32_t round = bit(drop - 1);
    uint32_t sticky = 0;
    for (int i = drop - 2; i >= 0; i--) sticky |= bit(i);
    if (round && (sticky || (mant & 1u))) mant++;
    r = scalbn((double)mant, drop);
  }
  return neg ? -r : r;
}

// Per-k FP32 tables for the next window (Eq. 4 through Sec. 3):
//   Tp4 = s(|c+4|^a - |c|^a), Tm4 = s(|c-4|^a - |c|^a), Tp2 = s(|c+2|^a - |c|^a), Tm2 = s(|c-2|^a - |c|^a)
// with s = 2^(-a*e).  Each is (ra - rb) * sum_i ra^i rb^(a-1-i), ra = |c+d|/2^e, rb = |c|/2^e:
// a sum of non-negative terms, so the relative error stays below (2a+1) 2^-24 (plus an
// absolute underflow term below 2^-140).
__device__ __forceinline__ float4 tables_for(int c, uint32_t alpha, float inv2e) {
  const float rb = fabsf((float)c) * inv2e;
  const float r0 = fabsf((float)(c + 4)) * inv2e, r1 = fabsf((float)(c - 4)) * inv2e;
  const float r2 = fabsf((float)(c + 2)) * inv2e, r3 = fabsf((float)(c - 2)) * inv2e;
  float S0 = 1.f, S1 = 1.f, S2 = 1.f, S3 = 1.f, pb = 1.f;
  for (uint32_t n = 1; n < alpha; n++) {
    pb = pb * rb;
    S0 = fmaf(r0, S0, pb);
    S1 = fmaf(r1, S1, pb);
    S2 = fmaf(r2, S2, pb);
    S3 = fmaf(r3, S3, pb);
  }
  return make_float4((r0 - rb) * S0, (r1 - rb) * S1, (r2 - rb) * S2, (r3 - rb) * S3);
}

__device__ __forceinline__ float absmax4(float4 t) {
  return fmaxf(fmaxf(fabsf(t.x), fabsf(t.y)), fmaxf(fabsf(t.z), fabsf(t.w)));
}

// Compensated flush of an FP32 block sum into (hi, lo): hi + lo keeps every flushed value.
__device__ __forceinline__ void flush_block(float &hi, float &lo, float &blk) {
  const float s = hi + blk;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (blk - bp);
  hi = s;
  lo += err;
  blk = 0.f;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

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

// C_k = (L-k) - 2 popc(x[0..L-k) xor x[k..L)) for one k per thread; PSL by atomicMax.
__global__ void k_autocorr(WalkDev *hdr, const uint32_t *active) {
  WalkDev &W = hdr[active[blockIdx.y]];
  const int L = (int)W.L;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  int a = 0;
  if (k < L) {
    const int n = L - k;
    int cnt = 0;
    for (int w = 0; 32 * w < n; w++) {
      uint32_t d = W.bits[w] ^ window32(W.bits, 32 * w + k);
      const int rem = n - 32 * w;
      if (rem < 32) d &= (1u << rem) - 1u;
      cnt += __popc(d);
    }
    const int c = n - 2 * cnt;
    W.C[k] = c;
    if (k > 0) a = c < 0 ? -c : c;
  }
  a = warp_max(a);
  if ((threadIdx.x & 31) == 0 && a > 0) atomicMax(&W.psl, a);
}

__device__ __forceinline__ int bitlen(uint32_t v) { return v ? 32 - __clz(v) : 0; }

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

// ------------------------------------------------------------------------------------
// apply: the O(L) update pass (init / move / switch) fused with the next window's
// tables, PSL, sum of |T| and the near-peak list; the last block to arrive finalises.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void apply_one(WalkDev &W, uint32_t chunk) {
  __shared__ int s_max[8];
  __shared__ float s_sum[8];
  __shared__ uint32_t s_F[256 / 32][kWideLimbs];
  __shared__ uint32_t s_last;
  if (W.status != kRunning) return;
  if (chunk >= W.nchunk_apply) return;
  const int L = (int)W.L;
  const int k0 = (int)chunk * kApplyChunk, k1 = min(k0 + kApplyChunk, L);
  const uint32_t mode = W.mode;
  const uint32_t alpha = W.alpha_next;
  const float inv2e = ldexpf(1.f, -W.e);
  const int thr = W.ktau_thr;
  const bool keep_local = (mode == kModeInit) || W.improved;
  const bool need_F = mode != kModeMove;
  const int kstar = (int)W.kstar;
  const int sk = (mode == kModeMove) ? sval(W.bits, kstar) : 0;
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
    } else if (mode == kModeMove) {
      // Sec. 3: C'_k = C_k - 2 s_j (s_{j+k} + s_{j-k}), absent partners count 0
      int part = 0;
      if (kstar + k < L) part += sval(W.bits, kstar + k);
      if (kstar >= k) part += sval(W.bits, kstar - k);
      c = W.C[k] - 2 * sk * part;
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
      if (need_F) add_pow_rt(F, (uint32_t)a, alpha);
    }
  }
  // block reductions
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  pmax = warp_max(pmax);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sabs += __shfl_xor_sync(0xffffffffu, sabs, o);
  if (need_F) {
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
    if (need_F) wide_store(s_F[warp], F);
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
      if (need_F) {
        uint32_t t[kWideLimbs];
        wide_load(t, s_F[w]);
        wide_add(Fb, t);
      }
    }
    part[0] = (uint32_t)m;
    part[1] = __float_as_uint(s);
    wide_store(part + 2, Fb);
    __threadfence();
    const uint32_t prev = atomicAdd(&W.arrive, 1u);
    s_last = (prev == W.nchunk_apply - 1u);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();

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
  if (keep_local)
    for (int w = threadIdx.x; w < nw; w += blockDim.x) W.bits_local[w] = W.bits[w];
  if (mode == kModeInit)
    for (int w = threadIdx.x; w < nw; w += blockDim.x) W.bits_best[w] = W.bits[w];
  if (threadIdx.x == 0) {
    int m = 0;
    float s = 0.f;
    uint32_t Fs[kWideLimbs];
    wide_zero(Fs);
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
    W.psl = m;
    W.S_abs = s;
    W.alpha = alpha;
    if (need_F) {
      wide_store(W.F, Fs);
      wide_store(W.value_local, Fs);
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
}

// persistent grid over (walk, chunk) pairs of the schedule
__global__ void __launch_bounds__(256) k_apply(WalkDev *hdr, const uint32_t *active, const Schedule *sched) {
  const uint32_t nch = sched->max_chunk_apply, V = sched->nactive * nch;
  for (uint32_t v = blockIdx.x; v < V; v += gridDim.x) {
    __syncthreads();  // shared reduction buffers of the previous pair are free
    apply_one(hdr[active[v / nch]], v % nch);
  }
}

// ------------------------------------------------------------------------------------
// neighbourhood score, batched form
//
// Lanes are window positions.  For neighbour j and shift k, with u = [s_j s_{j+k} = -1]
// and v = [s_j s_{j-k} = -1]:
//   both partners present:  delta = +4 if u=v=1, -4 if u=v=0, else 0
//   one partner present:    delta = +2 if its bit is 1, else -2
// (k <= kin = min(j, L-1-j): both present; kin < k <= kout = max(j, L-1-j): one; beyond: none.)
// k runs in super-blocks of 30 = 6 groups of 5.  For each group the block keeps three
// 32-entry subset-sum tables in shared memory,
//   W1[b] = sum_{q in b} Tp4_q,  W0[b] = sum_{q in b} Tm4_q,  E[b] = sum_q (b_q ? Tp2_q : Tm2_q),
// so one lookup scores five (j, k) terms.  Super-block sb owns 2304 bytes (6 groups x 3
// tables x 32 floats, 128-byte aligned) and entry b of all its tables sits at b ^ (sb & 31):
// the build (one thread per group, consecutive lanes on consecutive super-blocks) is free
// of bank conflicts, and a lookup address is ((W >> s) & 0x7C) ^ (base_sb | swizzle) plus a
// constant: one shift and one three-input logic op.  Regions are decided per warp and per
// super-block, so the common case runs without per-group tests.
// ------------------------------------------------------------------------------------
constexpr int kSbFloats = 576;           // 6 groups x 3 tables x 32 entries
constexpr int kSbBytes = kSbFloats * 4;  // 2304 bytes = 18 x 128

// tables (rounded up to a 128-byte boundary inside the allocation), two TMA staging
// buffers of the tile's per-k values, and two ints
size_t hot_batched_smem(uint32_t tile_sb) { return (size_t)tile_sb * kSbBytes + 2 * (size_t)tile_sb * kSbK * 16 + 256; }

// ---- TMA bulk copies and mbarriers (sm_90 and later) ----
__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16) signalling mbar
__device__ __forceinline__ void tma_load_1d(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n selp.b32 %0, 1, 0, P1;\n}"
      : "=r"(done)
      : "r"(mbar), "r"(parity)
      : "memory");
  return done != 0;
}
// bounded wait: false if the phase did not complete within the iteration limit
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity, int limit = 1 << 20) {
  for (int it = 0; it < limit; it++)
    if (mbar_try_wait(mbar, parity)) return true;
  return false;
}

template <int OFF>
__device__ __forceinline__ float lds_at(uint32_t addr) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(addr), "n"(OFF));
  return v;
}

// 5-bit field Q of w, times 4 (a byte offset in bits 2..6)
template <int Q>
__device__ __forceinline__ uint32_t field4(uint32_t w) {
  if constexpr (Q == 0)
    return (w << 2) & 0x7Cu;
  else
    return (w >> (5 * Q - 2)) & 0x7Cu;
}

__device__ __forceinline__ uint32_t window32_ro(const uint32_t *__restrict__ bits, int pos) {
  const int w = pos >> 5;
  return __funnelshift_r(__ldg(bits + w), __ldg(bits + w + 1), pos & 31);
}

// tables of group q of super-block sb of the tile (first k of the group: kg)
// (the tile's per-k values come from the shared staging buffer Ts, entry kg - kt0)
__device__ __forceinline__ void build_group(float *tab, int sb, int q, const float4 *Ts, int kt0, int kg, int L) {
  float tp4[5], tm4[5], tp2[5], tm2[5];
#pragma unroll
  for (int t = 0; t < 5; t++) {
    const int k = kg + t;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k < L) v = Ts[k - kt0];
    tp4[t] = v.x;
    tm4[t] = v.y;
    tp2[t] = v.z;
    tm2[t] = v.w;
  }
  // low two bits and high three bits summed separately: every entry is a tree of depth <= 3
  float lo1[4], lo0[4], loe[4], hi1[8], hi0[8], hie[8];
  lo1[0] = 0.f, lo1[1] = tp4[0], lo1[2] = tp4[1], lo1[3] = tp4[0] + tp4[1];
  lo0[0] = 0.f, lo0[1] = tm4[0], lo0[2] = tm4[1], lo0[3] = tm4[0] + tm4[1];
#pragma unroll
  for (int b = 0; b < 4; b++) loe[b] = ((b & 1) ? tp2[0] : tm2[0]) + ((b & 2) ? tp2[1] : tm2[1]);
  {
    const float a23 = tp4[2] + tp4[3], b23 = tm4[2] + tm4[3];
    hi1[0] = 0.f, hi1[1] = tp4[2], hi1[2] = tp4[3], hi1[3] = a23;
    hi1[4] = tp4[4], hi1[5] = tp4[2] + tp4[4], hi1[6] = tp4[3] + tp4[4], hi1[7] = a23 + tp4[4];
    hi0[0] = 0.f, hi0[1] = tm4[2], hi0[2] = tm4[3], hi0[3] = b23;
    hi0[4] = tm4[4], hi0[5] = tm4[2] + tm4[4], hi0[6] = tm4[3] + tm4[4], hi0[7] = b23 + tm4[4];
  }
#pragma unroll
  for (int b = 0; b < 4; b++) {
    const float p = ((b & 1) ? tp2[2] : tm2[2]) + ((b & 2) ? tp2[3] : tm2[3]);
    hie[b] = p + tm2[4];
    hie[b + 4] = p + tp2[4];
  }
  float *base = tab + sb * kSbFloats + q * 96;
  const int sw = sb & 31;
#pragma unroll
  for (int b = 0; b < 32; b++) {
    const int lo = b & 3, hi = b >> 2;
    base[b ^ sw] = lo == 0 ? hi1[hi] : (hi == 0 ? lo1[lo] : lo1[lo] + hi1[hi]);
    base[32 + (b ^ sw)] = lo == 0 ? hi0[hi] : (hi == 0 ? lo0[lo] : lo0[lo] + hi0[hi]);
    base[64 + (b ^ sw)] = loe[lo] + hie[hi];
  }
}

// exact per-term contribution used where a group straddles a region boundary
__device__ __forceinline__ float term_slow(const float4 *__restrict__ T, int k, int kin, int kout, uint32_t U,
                                           uint32_t V, bool plus_side, int t) {
  if (k > kout) return 0.f;
  const float4 tv = __ldg(T + k);
  const uint32_t u = (U >> t) & 1u, v = (V >> t) & 1u;
  if (k <= kin) return (u & v) ? tv.x : ((u | v) ? 0.f : tv.y);
  const uint32_t e = plus_side ? u : v;
  return e ? tv.z : tv.w;
}

// one group of a super-block where lanes may sit in different regions
template <int Q>
__device__ __forceinline__ void group_generic(float &a0, float &a1, uint32_t bsw, uint32_t W1, uint32_t W0,
                                              uint32_t E, uint32_t U, uint32_t V, int ka, int kin, int kout,
                                              bool plus_side, const float4 *__restrict__ T) {
  const int kg = ka + 5 * Q;
  if (kg + 4 <= kin) {
    a0 += lds_at<Q * 384>(field4<Q>(W1) ^ bsw);
    a1 += lds_at<Q * 384 + 128>(field4<Q>(W0) ^ bsw);
  } else if (kg > kin && kg + 4 <= kout) {
    a0 += lds_at<Q * 384 + 256>(field4<Q>(E) ^ bsw);
  } else if (kg <= kout) {
#pragma unroll
    for (int t = 0; t < 5; t++) a1 += term_slow(T, kg + t, kin, kout, U, V, plus_side, 5 * Q + t);
  }
}

// Exact neighbour PSL over the near-peak list: max_k |C_k + delta_jk| for |C_k| >= PSL - 8.
__device__ __forceinline__ int neighbour_psl(const WalkDev &W, const int2 *list, int n, int j, int L, int sj,
                                             int floor_c, int cur) {
  for (int q = 0; q < n; q++) {
    const int2 e = list[q];
    const int k = e.x, c = e.y;
    if ((c < 0 ? -c : c) < floor_c) continue;
    int part = 0;
    if (j + k < L) part += sval(W.bits, j + k);
    if (j >= k) part += sval(W.bits, j - k);
    const int cn = c - 2 * sj * part;
    cur = max(cur, cn < 0 ? -cn : cn);
  }
  return cur;
}

// One super-block where every lane has both partners for all 30 shifts.
__device__ __forceinline__ void sb_interior(float &a0, float &a1, const uint32_t *__restrict__ bits, int pos_u,
                                            int pos_v, uint32_t M, uint32_t bsw) {
  const uint32_t U = window32_ro(bits, pos_u);
  const uint32_t V = __brev(window32_ro(bits, pos_v));
  const uint32_t W1 = (U ^ M) & (V ^ M), W0 = ~((U ^ M) | (V ^ M));
  a0 += lds_at<0 * 384>(field4<0>(W1) ^ bsw);
  a1 += lds_at<0 * 384 + 128>(field4<0>(W0) ^ bsw);
  a0 += lds_at<1 * 384>(field4<1>(W1) ^ bsw);
  a1 += lds_at<1 * 384 + 128>(field4<1>(W0) ^ bsw);
  a0 += lds_at<2 * 384>(field4<2>(W1) ^ bsw);
  a1 += lds_at<2 * 384 + 128>(field4<2>(W0) ^ bsw);
  a0 += lds_at<3 * 384>(field4<3>(W1) ^ bsw);
  a1 += lds_at<3 * 384 + 128>(field4<3>(W0) ^ bsw);
  a0 += lds_at<4 * 384>(field4<4>(W1) ^ bsw);
  a1 += lds_at<4 * 384 + 128>(field4<4>(W0) ^ bsw);
  a0 += lds_at<5 * 384>(field4<5>(W1) ^ bsw);
  a1 += lds_at<5 * 384 + 128>(field4<5>(W0) ^ bsw);
}

// One super-block where every lane has exactly one partner for all 30 shifts.
__device__ __forceinline__ void sb_edge(float &a0, float &a1, const uint32_t *__restrict__ bits, int pos,
                                        bool plus_side, uint32_t M, uint32_t bsw) {
  const uint32_t w = window32_ro(bits, pos);
  const uint32_t E = (plus_side ? w : __brev(w)) ^ M;
  a0 += lds_at<0 * 384 + 256>(field4<0>(E) ^ bsw);
  a1 += lds_at<1 * 384 + 256>(field4<1>(E) ^ bsw);
  a0 += lds_at<2 * 384 + 256>(field4<2>(E) ^ bsw);
  a1 += lds_at<3 * 384 + 256>(field4<3>(E) ^ bsw);
  a0 += lds_at<4 * 384 + 256>(field4<4>(E) ^ bsw);
  a1 += lds_at<5 * 384 + 256>(field4<5>(E) ^ bsw);
}

// One super-block where region boundaries fall inside it for some lane.
__device__ __forceinline__ void sb_generic(float &a0, float &a1, const uint32_t *__restrict__ bits,
                                           const float4 *__restrict__ T, int j, int ka, int kin, int kout,
                                           bool plus_side, uint32_t M, uint32_t bsw, int cap_u) {
  if (ka > kout) return;
  const uint32_t U = window32_ro(bits, min(j + ka, cap_u)) ^ M;
  const uint32_t V = __brev(window32_ro(bits, max(j - ka - 31, -64))) ^ M;
  const uint32_t W1 = U & V, W0 = ~(U | V), E = plus_side ? U : V;
  group_generic<0>(a0, a1, bsw, W1, W0, E, U, V, ka, kin, kout, plus_side, T);
  group_generic<1>(a0, a1, bsw, W1, W0, E, U, V, ka, kin, kout, plus_side, T);
  group_generic<2>(a0, a1, bsw, W1, W0, E, U, V, ka, kin, kout, plus_side, T);
  group_generic<3>(a0, a1, bsw, W1, W0, E, U, V, ka, kin, kout, plus_side, T);
  group_generic<4>(a0, a1, bsw, W1, W0, E, U, V, ka, kin, kout, plus_side, T);
  group_generic<5>(a0, a1, bsw, W1, W0, E, U, V, ka, kin, kout, plus_side, T);
}

__device__ __forceinline__ void flush2(float &hi, float &lo, float &a0, float &a1) {
  float blk = a0 + a1;
  a0 = a1 = 0.f;
  flush_block(hi, lo, blk);
}

// number of super-blocks sb >= 0 of a tile starting at kt0 with kt0 + 30 sb + off <= bound
__device__ __forceinline__ int sb_count(int bound, int kt0, int off, int nsb) {
  const int d = bound - kt0 - off;
  return d < 0 ? 0 : min(nsb, d / kSbK + 1);
}

// Scores one work item (a block of window positions, possibly one k-chunk of them).
// Returns false when a staged copy timed out: the block must then stop taking work.
template <int NT, int NSB>
__device__ __forceinline__ bool hot_one(WalkDev *hdr, const HotItem it) {
  static_assert(NSB <= 32, "the per-super-block swizzle assumes at most 32 super-blocks per tile");
  extern __shared__ __align__(128) float smem_raw[];
  __shared__ __align__(8) uint64_t s_mbar[2];
  const uint32_t raw_s = (uint32_t)__cvta_generic_to_shared(smem_raw);
  const uint32_t tab_s = (raw_s + 127u) & ~127u;  // lookups OR a swizzle into the low 7 bits
  float *tab = smem_raw + (tab_s - raw_s) / 4;
  constexpr int kTileK = NSB * kSbK;
  float4 *stage = reinterpret_cast<float4 *>(tab + NSB * kSbFloats);  // 2 x kTileK staged T values
  const uint32_t stage_s = tab_s + NSB * kSbBytes;
  int *s_kmax = reinterpret_cast<int *>(stage + 2 * kTileK);
  int *s_timeout = s_kmax + 1;
  const uint32_t mbar_s = (uint32_t)__cvta_generic_to_shared(s_mbar);
  WalkDev &W = hdr[it.slot];
  if (W.status != kRunning) return true;
  const int L = (int)W.L, N = (int)W.N;
  const uint32_t *__restrict__ bits = W.bits;
  const float4 *__restrict__ T = W.T;
  const int i = (int)it.i0 + (int)threadIdx.x;  // window position, 1-based
  const bool live = i <= N;
  // lanes past the end of the window shadow the last neighbour (their sums are discarded),
  // so every lane of a partly filled warp stays inside the regions of a real neighbour
  const int j = (int)(((uint64_t)W.start + (uint64_t)min(i, N)) % (uint64_t)L);
  const bool warp_live = (int)it.i0 + (int)(threadIdx.x & ~31u) <= N;
  const int kin = min(j, L - 1 - j), kout = max(j, L - 1 - j);
  const bool plus_side = j < L - 1 - j;
  const uint32_t M = getbit(bits, j) ? 0xffffffffu : 0u;
  const int cap_u = 32 * (int)W.nw;
  const int w_kin_lo = __reduce_min_sync(0xffffffffu, kin);
  const int w_kin_hi = __reduce_max_sync(0xffffffffu, kin);
  const int w_kout_lo = __reduce_min_sync(0xffffffffu, kout);
  const int w_kout_hi = warp_live ? __reduce_max_sync(0xffffffffu, kout) : 0;
  if (threadIdx.x == 0) {
    *s_kmax = 0;
    *s_timeout = 0;
    mbar_init(mbar_s, 1);
    mbar_init(mbar_s + 8, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) atomicMax(s_kmax, w_kout_hi);
  __syncthreads();
  const int kmax = *s_kmax;
  // tiles of this block: all of them, or those of its k-chunk when the k range is split
  const int tiles_per_chunk = (int)W.kchunk_sb / NSB;
  const int tile_lo = W.ksplit > 1 ? (int)it.kc * tiles_per_chunk : 0;
  const int tile_hi = W.ksplit > 1 ? min((kmax + kTileK - 1) / kTileK, tile_lo + tiles_per_chunk)
                                   : (kmax + kTileK - 1) / kTileK;
  const int ntiles = max(0, tile_hi - tile_lo);
  // TMA bulk copy of tile t's per-k values T[kt0 .. kt0 + kTileK) (those below L) into buffer t & 1
  auto stage_tile = [&](int t) {
    const int kt0 = 1 + (tile_lo + t) * kTileK;
    const uint32_t bytes = 16u * (uint32_t)min(kTileK, L - kt0);
    const uint32_t mb = mbar_s + 8u * (t & 1);
    fence_proxy_async();
    mbar_expect_tx(mb, bytes);
    tma_load_1d(stage_s + (uint32_t)((t & 1) * kTileK * 16), T + kt0, bytes, mb);
  };
  // test hook: no copy is issued, so every wait below runs out (short limit) and the walk
  // is marked failed; nothing is left in flight
  const bool stall = W.inject_stall != 0;
  const int wait_limit = stall ? 64 : (1 << 20);
  if (threadIdx.x == 0 && ntiles > 0 && !stall) stage_tile(0);

  float hi = 0.f, lo = 0.f, a0 = 0.f, a1 = 0.f;
  for (int tile = 0; tile < ntiles; tile++) {
    const int kt0 = 1 + (tile_lo + tile) * kTileK;
    __syncthreads();  // previous tile fully consumed (tables, and the staging buffer reused below)
    if (threadIdx.x == 0 && tile + 1 < ntiles && !stall) stage_tile(tile + 1);
    if ((int)threadIdx.x < 6 * NSB) {
      if (!mbar_wait_bounded(mbar_s + 8u * (tile & 1), (uint32_t)(tile >> 1) & 1u, wait_limit)) *s_timeout = 1;
      const float4 *Ts = stage + (tile & 1) * kTileK;
      for (int t = threadIdx.x; t < 6 * NSB; t += NT) {
        const int sb = t % NSB, q = t / NSB;
        build_group(tab, sb, q, Ts, kt0, kt0 + sb * kSbK + 5 * q, L);
      }
    }
    __syncthreads();
    // warp-uniform phases of this tile, in increasing k:
    //   [0, n_int)        every lane interior        (ka + 29 <= min kin)
    //   [n_int, e0)       generic                   (around the kin boundaries)
    //   [e0, n_edge)      every lane one partner     (ka > max kin, ka + 29 <= min kout)
    //   [n_edge, n_all)   generic                   (around the kout boundaries)
    const int n_all = sb_count(w_kout_hi, kt0, 0, NSB);
    const int n_int = min(sb_count(w_kin_lo, kt0, kSbK - 1, NSB), n_all);
    const int e0 = max(n_int, min(n_all, sb_count(w_kin_hi, kt0, 0, NSB)));
    const int n_edge = max(e0, min(n_all, sb_count(w_kout_lo, kt0, kSbK - 1, NSB)));
    const uint32_t bsw0 = tab_s;  // super-block sb: base + 2304 sb, swizzle sb << 2
    int sb = 0;
    {
      int pu = j + kt0, pv = j - kt0 - 31;
      uint32_t bsw = bsw0;
      for (; sb + 1 < n_int; sb += 2) {
        sb_interior(a0, a1, bits, pu, pv, M, bsw);
        sb_interior(a0, a1, bits, pu + kSbK, pv - kSbK, M, bsw + (kSbBytes + 4));
        flush2(hi, lo, a0, a1);
        pu += 2 * kSbK, pv -= 2 * kSbK, bsw += 2 * (kSbBytes + 4);
      }
      if (sb < n_int) {
        sb_interior(a0, a1, bits, pu, pv, M, bsw);
        flush2(hi, lo, a0, a1);
        sb++;
      }
    }
    for (; sb < e0; sb++) {
      sb_generic(a0, a1, bits, T, j, kt0 + sb * kSbK, kin, kout, plus_side, M, bsw0 + sb * (kSbBytes + 4), cap_u);
      flush2(hi, lo, a0, a1);
    }
    {
      const int step = plus_side ? kSbK : -kSbK;
      int pe = plus_side ? j + kt0 + sb * kSbK : j - kt0 - sb * kSbK - 31;
      uint32_t bsw = bsw0 + sb * (kSbBytes + 4);
      for (; sb + 1 < n_edge; sb += 2) {
        sb_edge(a0, a1, bits, pe, plus_side, M, bsw);
        sb_edge(a0, a1, bits, pe + step, plus_side, M, bsw + (kSbBytes + 4));
        flush2(hi, lo, a0, a1);
        pe += 2 * step, bsw += 2 * (kSbBytes + 4);
      }
      if (sb < n_edge) {
        sb_edge(a0, a1, bits, pe, plus_side, M, bsw);
        flush2(hi, lo, a0, a1);
        sb++;
      }
    }
    for (; sb < n_all; sb++) {
      sb_generic(a0, a1, bits, T, j, kt0 + sb * kSbK, kin, kout, plus_side, M, bsw0 + sb * (kSbBytes + 4), cap_u);
      flush2(hi, lo, a0, a1);
    }
  }
  if (*s_timeout) {
    // a staged copy never arrived: give every copy of this block one more bounded wait,
    // then mark the walk failed instead of using its scores
    __syncthreads();
    if (threadIdx.x == 0) {
      if (!stall)
        for (int t = max(0, ntiles - 2); t < ntiles; t++) mbar_wait_bounded(mbar_s + 8u * (t & 1), (uint32_t)(t >> 1) & 1u);
      W.error = (uint32_t)-5;  // PSL_ETIMEOUT of the library header
      W.status = kError;
    }
    return stall;  // after a real timeout a copy may still be in flight: stop using this block
  }
  if (!live) return true;
  if (W.ksplit > 1) {
    W.score_part[(size_t)it.kc * N + (i - 1)] = hi + lo;
    if (it.kc != 0) return true;
  } else {
    W.score[i - 1] = hi + lo;
  }

  // exact neighbour PSL, only when some neighbour may beat psl_best
  int pj = INT_MAX;
  if (W.ktau_on) {
    const int sj = M ? -1 : 1;
    pj = neighbour_psl(W, W.ktau, (int)W.nktau, j, L, sj, W.psl - 8, 0);
  }
  W.pslj[i - 1] = pj;
  return true;
}

// Persistent: every block takes work items one by one from the schedule's counter
// (longest walks first in the item list).
template <int NT, int NSB>
__global__ void __launch_bounds__(NT, 1024 / NT) k_hot_batched(WalkDev *hdr, const HotItem *items, Schedule *sched) {
  __shared__ uint32_t s_item;
  for (;;) {
    __syncthreads();  // the previous item's shared memory is free
    if (threadIdx.x == 0) s_item = atomicAdd(&sched->hot_next, 1u);
    __syncthreads();
    const uint32_t item = s_item;
    if (item >= sched->nitems) break;
    if (!hot_one<NT, NSB>(hdr, items[item])) break;
  }
}

// ------------------------------------------------------------------------------------
// neighbourhood score, plain form: one thread per neighbour, every term accumulated
// on its own (the execution model of the paper's GPU solver)
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_hot_plain(WalkDev *hdrp) {
  const WalkDev &W = *hdrp;
  const int L = (int)W.L, N = (int)W.N;
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
  if (i > N) return;
  const uint32_t *bits = W.bits;
  const float4 *T = W.T;
  const int j = (int)(((uint64_t)W.start + (uint64_t)i) % (uint64_t)L);
  const int kin = min(j, L - 1 - j), kout = max(j, L - 1 - j);
  const bool plus_side = j < L - 1 - j;
  const uint32_t M = getbit(bits, j) ? 0xffffffffu : 0u;
  const int cap_u = 32 * (int)W.nw;
  float hi = 0.f, lo = 0.f, blk = 0.f;
  for (int ka = 1; ka <= kout; ka += kSbK) {
    const uint32_t U = window32(bits, min(j + ka, cap_u)) ^ M;
    const uint32_t V = __brev(window32(bits, max(j - ka - 31, -64))) ^ M;
    const int kend = min(ka + kSbK - 1, kout);
    for (int k = ka; k <= kend; k++) {
      const int t = k - ka;
      const float4 tv = T[k];
      const uint32_t u = (U >> t) & 1u, v = (V >> t) & 1u;
      if (k <= kin) {
        if (u & v)
          blk += tv.x;
        else if (!(u | v))
          blk += tv.y;
      } else {
        blk += (plus_side ? u : v) ? tv.z : tv.w;
      }
    }
    flush_block(hi, lo, blk);
  }
  W.score[i - 1] = hi + lo;
  int pj = INT_MAX;
  if (W.ktau_on) pj = neighbour_psl(W, W.ktau, (int)W.nktau, j, L, M ? -1 : 1, W.psl - 8, 0);
  W.pslj[i - 1] = pj;
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

__global__ void __launch_bounds__(1024) k_select(WalkDev *hdr, const uint32_t *active, const Schedule *sched) {
  for (uint32_t a = blockIdx.x; a < sched->nactive; a += gridDim.x) {
    __syncthreads();
    select_one(hdr[active[a]]);
  }
}

// ------------------------------------------------------------------------------------
// recheck: exact Delta F = sum_{k: delta != 0} |C_k + delta|^alpha - |C_k|^alpha of the
// candidates, one CTA per (chunk of k, candidate); positive and negative parts are
// accumulated separately as unsigned 384-bit integers.
// ------------------------------------------------------------------------------------
template <int A>
__device__ void recheck_body(const WalkDev &W, int j, int kbeg, int kend, uint32_t (&pos)[kWideLimbs],
                             uint32_t (&neg)[kWideLimbs]) {
  const int L = (int)W.L;
  const int sj = sval(W.bits, j);
  for (int k = kbeg + (int)threadIdx.x; k < kend; k += blockDim.x) {
    int part = 0;
    if (j + k < L) part += sval(W.bits, j + k);
    if (j >= k) part += sval(W.bits, j - k);
    if (part == 0) continue;
    const int c = W.C[k];
    const int cn = c - 2 * sj * part;
    add_pow<A>(pos, (uint32_t)(cn < 0 ? -cn : cn));
    add_pow<A>(neg, (uint32_t)(c < 0 ? -c : c));
  }
}

__device__ __forceinline__ void recheck_one(WalkDev &W, uint32_t chunk, uint32_t qslot) {
  __shared__ uint32_t s_w[8][2 * kWideLimbs];
  if (W.status != kRunning) return;
  if (chunk >= W.nchunk_rc) return;
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
        case 1: recheck_body<1>(W, j, kbeg, kend, pos, neg); break;
        case 2: recheck_body<2>(W, j, kbeg, kend, pos, neg); break;
        case 3: recheck_body<3>(W, j, kbeg, kend, pos, neg); break;
        case 4: recheck_body<4>(W, j, kbeg, kend, pos, neg); break;
        case 5: recheck_body<5>(W, j, kbeg, kend, pos, neg); break;
        case 6: recheck_body<6>(W, j, kbeg, kend, pos, neg); break;
        case 7: recheck_body<7>(W, j, kbeg, kend, pos, neg); break;
        case 8: recheck_body<8>(W, j, kbeg, kend, pos, neg); break;
        case 9: recheck_body<9>(W, j, kbeg, kend, pos, neg); break;
        case 10: recheck_body<10>(W, j, kbeg, kend, pos, neg); break;
        case 11: recheck_body<11>(W, j, kbeg, kend, pos, neg); break;
        case 12: recheck_body<12>(W, j, kbeg, kend, pos, neg); break;
        case 13: recheck_body<13>(W, j, kbeg, kend, pos, neg); break;
        case 14: recheck_body<14>(W, j, kbeg, kend, pos, neg); break;
        case 15: recheck_body<15>(W, j, kbeg, kend, pos, neg); break;
        default: recheck_body<16>(W, j, kbeg, kend, pos, neg); break;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      uint32_t a[kWideLimbs], b[kWideLimbs];
#pragma unroll
      for (int t = 0; t < kWideLimbs; t++) {
        a[t] = __shfl_down_sync(0xffffffffu, pos[t], o);
        b[t] = __shfl_down_sync(0xffffffffu, neg[t], o);
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

// persistent grid over (walk, chunk) pairs of the schedule; each pair covers every
// candidate of the walk (slots 0..kQcap-1 by chunk, later ones whole in chunk 0)
__global__ void __launch_bounds__(256) k_recheck(WalkDev *hdr, const uint32_t *active, const Schedule *sched) {
  const uint32_t nch = sched->max_chunk_rc, V = sched->nactive * nch;
  for (uint32_t v = blockIdx.x; v < V; v += gridDim.x) {
    WalkDev &W = hdr[active[v / nch]];
    const uint32_t chunk = v % nch;
    if (W.status != kRunning || chunk >= W.nchunk_rc) continue;  // uniform over the block
    const uint32_t nslots = min(W.ncand, (uint32_t)kQcap);
    for (uint32_t qslot = 0; qslot < nslots; qslot++) {
      __syncthreads();
      recheck_one(W, chunk, qslot);
    }
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
  if (psl_imp) {
    const int nw = (int)W.nw;
    for (int w = threadIdx.x; w < nw; w += blockDim.x) W.bits_best[w] = W.bits[w];
    __syncthreads();
    if (threadIdx.x == 0) W.bits_best[pj >> 5] ^= 1u << (pj & 31);
  }
  if (threadIdx.x != 0) return;

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
    r.value_step = wide_to_double(vstep);
    wide_store(r.value_exact, vstep);
  }
}

__global__ void __launch_bounds__(256) k_decide(WalkDev *hdr, const uint32_t *active, Schedule *sched) {
  // the neighbourhood kernel of this step has finished: rearm its work counter
  if (blockIdx.x == 0 && threadIdx.x == 0) sched->hot_next = 0;
  for (uint32_t a = blockIdx.x; a < sched->nactive; a += gridDim.x) {
    __syncthreads();
    decide_one(hdr[active[a]]);
  }
}

// ------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------
static uint32_t g_hot_blocks_per_sm[3][2];  // occupancy of every variant, measured at set-up
// resident blocks per SM of the other persistent kernels (one wave each)
static uint32_t g_apply_per_sm = 4, g_select_per_sm = 1, g_recheck_per_sm = 3, g_decide_per_sm = 4;

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
  k_apply<<<g_apply_per_sm * c.sm_count, 256, 0, c.stream>>>(c.hdr, c.active, c.sched);
  return cudaGetLastError();
}

using HotFn = void (*)(WalkDev *, const HotItem *, Schedule *);

static int variant_index(uint32_t threads) { return threads == 512 ? 2 : (threads == 128 ? 0 : 1); }

static HotFn hot_variant(uint32_t threads, uint32_t tile_sb) {
  if (threads == 512) return tile_sb == 16 ? k_hot_batched<512, 16> : k_hot_batched<512, 32>;
  if (threads == 128) return tile_sb == 16 ? k_hot_batched<128, 16> : k_hot_batched<128, 32>;
  return tile_sb == 16 ? k_hot_batched<256, 16> : k_hot_batched<256, 32>;
}

bool hot_config_supported(uint32_t threads, uint32_t tile_sb) {
  return (threads == 128 || threads == 256 || threads == 512) && (tile_sb == 16 || tile_sb == 32);
}

static cudaError_t blocks_per_sm(const void *f, int threads, uint32_t *out) {
  int nb = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, threads, 0);
  *out = (uint32_t)(nb > 0 ? nb : 1);
  return e;
}

static cudaError_t prepare_kernels_once() {
  cudaError_t e0 = blocks_per_sm((const void *)k_apply, 256, &g_apply_per_sm);
  if (e0 == cudaSuccess) e0 = blocks_per_sm((const void *)k_select, 1024, &g_select_per_sm);
  if (e0 == cudaSuccess) e0 = blocks_per_sm((const void *)k_recheck, 256, &g_recheck_per_sm);
  if (e0 == cudaSuccess) e0 = blocks_per_sm((const void *)k_decide, 256, &g_decide_per_sm);
  if (e0 != cudaSuccess) return e0;
  for (uint32_t t : {128u, 256u, 512u})
    for (uint32_t sb : {16u, 32u}) {
      HotFn f = hot_variant(t, sb);
      cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hot_batched_smem(sb));
      if (e != cudaSuccess) return e;
      int nb = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, (int)t, hot_batched_smem(sb));
      if (e != cudaSuccess) return e;
      g_hot_blocks_per_sm[variant_index(t)][sb == 32 ? 1 : 0] = (uint32_t)(nb > 0 ? nb : 1);
    }
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

cudaError_t launch_hot_batched(const LaunchCtx &c) {
  const uint32_t per_sm = g_hot_blocks_per_sm[variant_index(c.hot_threads)][c.hot_tile_sb == 32 ? 1 : 0];
  hot_variant(c.hot_threads, c.hot_tile_sb)<<<per_sm * c.sm_count, c.hot_threads, hot_batched_smem(c.hot_tile_sb),
                                              c.stream>>>(c.hdr, c.items, c.sched);
  return cudaGetLastError();
}

cudaError_t launch_hot_plain(WalkDev *hdr_one, uint32_t N, cudaStream_t s) {
  k_hot_plain<<<(N + 127) / 128, 128, 0, s>>>(hdr_one);
  return cudaGetLastError();
}

cudaError_t launch_select(const LaunchCtx &c) {
  k_select<<<g_select_per_sm * c.sm_count, 1024, 0, c.stream>>>(c.hdr, c.active, c.sched);
  return cudaGetLastError();
}

cudaError_t launch_recheck(const LaunchCtx &c) {
  k_recheck<<<g_recheck_per_sm * c.sm_count, 256, 0, c.stream>>>(c.hdr, c.active, c.sched);
  return cudaGetLastError();
}

cudaError_t launch_decide(const LaunchCtx &c) {
  k_decide<<<g_decide_per_sm * c.sm_count, 256, 0, c.stream>>>(c.hdr, c.active, c.sched);
  return cudaGetLastError();
}

}  // namespace psl
