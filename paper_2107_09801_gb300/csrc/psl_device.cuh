// psl_device.cuh -- device helpers shared by the CUDA translation units of the library:
// the walk's random draws, windows of the packed sequence, 384-bit exact arithmetic, the
// per-k FP32 tables and the compensated block flush.  GPU side only.
#pragma once
#include <cstdint>

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

// The same on NL-limb accumulators (NL = 4 or 8), for values whose bound is known: the
// caller guarantees c^A and every partial sum fit in 32 NL bits.
template <int NL>
__device__ __forceinline__ void wide_add_n(uint32_t (&a)[NL], const uint32_t (&b)[NL]) {
  static_assert(NL == 4 || NL == 8, "4 or 8 limbs");
  if constexpr (NL == 4) {
    asm("add.cc.u32 %0, %0, %4;\n\t"
        "addc.cc.u32 %1, %1, %5;\n\t"
        "addc.cc.u32 %2, %2, %6;\n\t"
        "addc.u32 %3, %3, %7;"
        : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3])
        : "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]));
  } else {
    asm("add.cc.u32 %0, %0, %8;\n\t"
        "addc.cc.u32 %1, %1, %9;\n\t"
        "addc.cc.u32 %2, %2, %10;\n\t"
        "addc.cc.u32 %3, %3, %11;\n\t"
        "addc.cc.u32 %4, %4, %12;\n\t"
        "addc.cc.u32 %5, %5, %13;\n\t"
        "addc.cc.u32 %6, %6, %14;\n\t"
        "addc.u32 %7, %7, %15;"
        : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7])
        : "r"(b[0]), "r"(b[1]), "r"(b[2]), "r"(b[3]), "r"(b[4]), "r"(b[5]), "r"(b[6]), "r"(b[7]));
  }
}

template <int A, int NL>
__device__ __forceinline__ void add_pow_n(uint32_t (&acc)[NL], uint32_t c) {
  uint32_t p[NL];
  p[0] = c;
#pragma unroll
  for (int i = 1; i < NL; i++) p[i] = 0;
#pragma unroll
  for (int t = 2; t <= A; t++) {
    uint64_t carry = 0;
#pragma unroll
    for (int i = 0; i < NL; i++) {
      if (i < (21 * t + 31) / 32) {
        const uint64_t v = (uint64_t)p[i] * c + carry;
        p[i] = (uint32_t)v;
        carry = v >> 32;
      }
    }
  }
  wide_add_n<NL>(acc, p);
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
inline __device__ double wide_to_double(const uint32_t (&a)[kWideLimbs]) {
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
// (c and c +- 2, c +- 4 are integers below 2^24, exact in FP32: one conversion serves all five.)
__device__ __forceinline__ float4 tables_for(int c, uint32_t alpha, float inv2e) {
  const float fc = (float)c;
  const float rb = fabsf(fc) * inv2e;
  const float r0 = fabsf(fc + 4.f) * inv2e, r1 = fabsf(fc - 4.f) * inv2e;
  const float r2 = fabsf(fc + 2.f) * inv2e, r3 = fabsf(fc - 2.f) * inv2e;
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

}  // namespace psl
