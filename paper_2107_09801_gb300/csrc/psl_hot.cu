// psl_hot.cu -- the neighbourhood-score kernels (sm_103a) of the limited-neighbourhood
// search of Boskovic and Brest (arXiv 2107.09801): the batched, persistent kernel with
// shared-memory subset-sum tables and TMA-staged k-tiles, and the plain
// one-thread-per-neighbour kernel of the paper's execution model.
#include <climits>
#include <cstdint>
#include <cstdio>

#include "psl_device.cuh"
#include "psl_internal.h"

namespace psl {

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
// super-block, so the common case runs without per-group tests.  Block sums of at most 48
// values are flushed into a compensated (hi, lo) pair.
// ------------------------------------------------------------------------------------
// Table layout of one super-block.  The short-walk variants (MB, "masked boundaries") add two
// tables per group, Ep[b] = sum_{q in b} Tp2_q and Em[b] = sum_{q in b} Tm2_q, so that a group
// where lanes of a warp sit in different regions is scored by four lookups of masked
// indices (the two-partner shifts in W1 and W0, the one-partner shifts in Ep and Em)
// instead of term by term: 640 bytes per group, 3840 per super-block (30 x 128).
template <bool MB>
struct TabLayout {
  static constexpr int GS = MB ? 640 : 384;  // bytes per group: W1, W0, E (, Ep, Em)
  static constexpr int SBB = 6 * GS;         // bytes per super-block: 18 or 30 x 128
  static constexpr int SBF = SBB / 4;
};

// tables (rounded up to a 128-byte boundary inside the allocation), two TMA staging
// buffers of the tile's per-k values, and a few ints of block-wide state
size_t hot_batched_smem(uint32_t tile_sb, bool masked) {
  return (size_t)tile_sb * (masked ? TabLayout<true>::SBB : TabLayout<false>::SBB) + 2 * (size_t)tile_sb * kSbK * 16 +
         256;
}

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
// (the tile's per-k values come from the shared staging buffer Ts, entry kg - kt0).
// W1/W0 are built only when some lane of the block scores a two-partner shift in the
// super-block (need_w), E only when some lane scores a one-partner shift there (need_e),
// Ep/Em (MB variants) only where a region boundary of some lane of the block falls (need_m).
template <bool MB>
__device__ __forceinline__ void build_group(float *tab, int sb, int q, const float4 *Ts, int kt0, int kg, int L,
                                            bool need_w, bool need_e, bool need_m) {
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
  float *base = tab + sb * TabLayout<MB>::SBF + q * (TabLayout<MB>::GS / 4);
  const int sw = sb & 31;
  if (need_w) {
#pragma unroll
    for (int b = 0; b < 32; b++) {
      const int lo = b & 3, hi = b >> 2;
      base[b ^ sw] = lo == 0 ? hi1[hi] : (hi == 0 ? lo1[lo] : lo1[lo] + hi1[hi]);
      base[32 + (b ^ sw)] = lo == 0 ? hi0[hi] : (hi == 0 ? lo0[lo] : lo0[lo] + hi0[hi]);
    }
  }
  if (need_e) {
#pragma unroll
    for (int b = 0; b < 32; b++) base[64 + (b ^ sw)] = loe[b & 3] + hie[b >> 2];
  }
  if constexpr (MB) {
    if (need_m) {
      // subset sums of Tp2 and of Tm2, split into the low two and the high three bits as above
      float lop[4], lom[4], hip[8], him[8];
      lop[0] = 0.f, lop[1] = tp2[0], lop[2] = tp2[1], lop[3] = tp2[0] + tp2[1];
      lom[0] = 0.f, lom[1] = tm2[0], lom[2] = tm2[1], lom[3] = tm2[0] + tm2[1];
      const float p23 = tp2[2] + tp2[3], m23 = tm2[2] + tm2[3];
      hip[0] = 0.f, hip[1] = tp2[2], hip[2] = tp2[3], hip[3] = p23;
      hip[4] = tp2[4], hip[5] = tp2[2] + tp2[4], hip[6] = tp2[3] + tp2[4], hip[7] = p23 + tp2[4];
      him[0] = 0.f, him[1] = tm2[2], him[2] = tm2[3], him[3] = m23;
      him[4] = tm2[4], him[5] = tm2[2] + tm2[4], him[6] = tm2[3] + tm2[4], him[7] = m23 + tm2[4];
#pragma unroll
      for (int b = 0; b < 32; b++) {
        const int lo = b & 3, hi = b >> 2;
        base[96 + (b ^ sw)] = lo == 0 ? hip[hi] : (hi == 0 ? lop[lo] : lop[lo] + hip[hi]);
        base[128 + (b ^ sw)] = lo == 0 ? him[hi] : (hi == 0 ? lom[lo] : lom[lo] + him[hi]);
      }
    }
  }
}

// Shift range of one warp's lanes: min/max of kin and kout over its 32 neighbours.
struct WarpRange {
  int kin_lo, kin_hi, kout_lo, kout_hi;
};

// One group of a super-block where lanes may sit in different regions.  The choice is
// warp-uniform: a table lookup when every lane of the warp has both partners (or every
// lane exactly one) for all five shifts; otherwise, in the MB variants, four lookups of
// indices masked to each lane's own regions, else the five terms one by one from the
// tile's staged per-k values, each lane selecting its own case without a branch.
template <int Q, bool MB>
__device__ __forceinline__ void group_generic(float &a0, float &a1, uint32_t bsw, uint32_t W1, uint32_t W0,
                                              uint32_t E, uint32_t U, uint32_t V, int ka, int kin, int kout,
                                              bool plus_side, const float4 *Ts, int kt0, const WarpRange &wr) {
  constexpr int GS = TabLayout<MB>::GS;
  const int kg = ka + 5 * Q;
  if (kg > wr.kout_hi) return;
  if (kg + 4 <= wr.kin_lo) {
    a0 += lds_at<Q * GS>(field4<Q>(W1) ^ bsw);
    a1 += lds_at<Q * GS + 128>(field4<Q>(W0) ^ bsw);
  } else if (kg > wr.kin_hi && kg + 4 <= wr.kout_lo) {
    a0 += lds_at<Q * GS + 256>(field4<Q>(E) ^ bsw);
  } else if constexpr (MB) {
    // shifts kg .. kg+nb-1 have both partners, kg+nb .. kg+nl-1 one (bits 2..6 of the index)
    const int nb = min(5, max(0, kin - kg + 1)), nl = min(5, max(0, kout - kg + 1));
    const uint32_t mb = ((1u << nb) - 1u) << 2;
    const uint32_t me = (((1u << nl) - 1u) << 2) & ~mb;
    a0 += lds_at<Q * GS>((field4<Q>(W1) & mb) ^ bsw);
    a1 += lds_at<Q * GS + 128>((field4<Q>(W0) & mb) ^ bsw);
    a0 += lds_at<Q * GS + 384>((field4<Q>(E) & me) ^ bsw);   // partner bit 1: delta = +2
    a1 += lds_at<Q * GS + 512>((field4<Q>(~E) & me) ^ bsw);  // partner bit 0: delta = -2
  } else {
#pragma unroll
    for (int t = 0; t < 5; t++) {
      const int k = kg + t;
      const float4 tv = Ts[k - kt0];
      const uint32_t u = (U >> (5 * Q + t)) & 1u, v = (V >> (5 * Q + t)) & 1u;
      const float r_in = (u & v) ? tv.x : ((u | v) ? 0.f : tv.y);  // both partners
      const float r_ed = (plus_side ? u : v) ? tv.z : tv.w;        // one partner
      a1 += k <= kin ? r_in : (k <= kout ? r_ed : 0.f);
    }
  }
}

// One super-block where every lane has both partners for all 30 shifts; wu and wv point at
// the lane's forward and backward partner windows of the super-block's first shift.
template <bool MB>
__device__ __forceinline__ void sb_interior(float &a0, float &a1, const uint32_t *__restrict__ wu,
                                            const uint32_t *__restrict__ wv, uint32_t M, uint32_t bsw) {
  constexpr int GS = TabLayout<MB>::GS;
  const uint32_t U = __ldg(wu);
  const uint32_t V = __ldg(wv);
  const uint32_t W1 = (U ^ M) & (V ^ M), W0 = ~((U ^ M) | (V ^ M));
  a0 += lds_at<0 * GS>(field4<0>(W1) ^ bsw);
  a1 += lds_at<0 * GS + 128>(field4<0>(W0) ^ bsw);
  a0 += lds_at<1 * GS>(field4<1>(W1) ^ bsw);
  a1 += lds_at<1 * GS + 128>(field4<1>(W0) ^ bsw);
  a0 += lds_at<2 * GS>(field4<2>(W1) ^ bsw);
  a1 += lds_at<2 * GS + 128>(field4<2>(W0) ^ bsw);
  a0 += lds_at<3 * GS>(field4<3>(W1) ^ bsw);
  a1 += lds_at<3 * GS + 128>(field4<3>(W0) ^ bsw);
  a0 += lds_at<4 * GS>(field4<4>(W1) ^ bsw);
  a1 += lds_at<4 * GS + 128>(field4<4>(W0) ^ bsw);
  a0 += lds_at<5 * GS>(field4<5>(W1) ^ bsw);
  a1 += lds_at<5 * GS + 128>(field4<5>(W0) ^ bsw);
}

// One super-block where every lane has exactly one partner for all 30 shifts; we points at
// the lane's window of that partner (forward or backward) for the super-block's first shift.
template <bool MB>
__device__ __forceinline__ void sb_edge(float &a0, float &a1, const uint32_t *__restrict__ we, uint32_t M,
                                        uint32_t bsw) {
  constexpr int GS = TabLayout<MB>::GS;
  const uint32_t E = __ldg(we) ^ M;
  a0 += lds_at<0 * GS + 256>(field4<0>(E) ^ bsw);
  a1 += lds_at<1 * GS + 256>(field4<1>(E) ^ bsw);
  a0 += lds_at<2 * GS + 256>(field4<2>(E) ^ bsw);
  a1 += lds_at<3 * GS + 256>(field4<3>(E) ^ bsw);
  a0 += lds_at<4 * GS + 256>(field4<4>(E) ^ bsw);
  a1 += lds_at<5 * GS + 256>(field4<5>(E) ^ bsw);
}

// One super-block where region boundaries fall inside it for some lane of the warp.
// Partner bits outside the sequence (clamped windows) are only ever paired with a case
// that ignores them.
template <bool MB>
__device__ __forceinline__ void sb_generic(float &a0, float &a1, const uint32_t *__restrict__ win_f,
                                           const uint32_t *__restrict__ win_r, const float4 *Ts, int kt0, int j,
                                           int ka, int kin, int kout, bool plus_side, uint32_t M, uint32_t bsw,
                                           int L, const WarpRange &wr) {
  if (ka > wr.kout_hi) return;
  // past either end every partner bit is 0 (entries L and -1 of the windows)
  const uint32_t U = __ldg(win_f + min(j + ka, L)) ^ M;
  const uint32_t V = __ldg(win_r + max(j - ka, -1)) ^ M;
  const uint32_t W1 = U & V, W0 = ~(U | V), E = plus_side ? U : V;
  group_generic<0, MB>(a0, a1, bsw, W1, W0, E, U, V, ka, kin, kout, plus_side, Ts, kt0, wr);
  group_generic<1, MB>(a0, a1, bsw, W1, W0, E, U, V, ka, kin, kout, plus_side, Ts, kt0, wr);
  group_generic<2, MB>(a0, a1, bsw, W1, W0, E, U, V, ka, kin, kout, plus_side, Ts, kt0, wr);
  group_generic<3, MB>(a0, a1, bsw, W1, W0, E, U, V, ka, kin, kout, plus_side, Ts, kt0, wr);
  group_generic<4, MB>(a0, a1, bsw, W1, W0, E, U, V, ka, kin, kout, plus_side, Ts, kt0, wr);
  group_generic<5, MB>(a0, a1, bsw, W1, W0, E, U, V, ka, kin, kout, plus_side, Ts, kt0, wr);
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

// TMA bulk copy of the per-k values T[kt0 .. kt0 + kTileK) (those below L) into staging
// buffer q & 1, signalling that buffer's mbarrier; q counts the block's copies.
template <int NSB>
__device__ __forceinline__ void stage_copy(uint32_t stage_s, uint32_t mbar_s, uint32_t q, const float4 *T, int kt0,
                                           int L) {
  constexpr int kTileK = NSB * kSbK;
  const uint32_t bytes = 16u * (uint32_t)min(kTileK, L - kt0);
  const uint32_t mb = mbar_s + 8u * (q & 1u);
  fence_proxy_async();
  mbar_expect_tx(mb, bytes);
  tma_load_1d(stage_s + (q & 1u) * (uint32_t)(kTileK * 16), T + kt0, bytes, mb);
}

// first shift of the k range a work item scores (its k-chunk, or the whole range)
template <int NSB>
__device__ __forceinline__ int item_tile_lo(const WalkDev &W, const HotItem &it) {
  return W.ksplit > 1 ? (int)it.kc * ((int)W.kchunk_sb / NSB) : 0;
}

// Copies a block has staged: copy q goes to buffer q & 1 and completes phase q >> 1 of that
// buffer's mbarrier, so it is awaited with parity (q >> 1) & 1.  `seq` is the next copy the
// block will consume; `pre` says that copy was already issued for the current item's first
// tile while the previous item scored its last one.
struct HotPipe {
  uint32_t seq;
  bool pre;
};

// Scores one work item (a block of window positions, possibly one k-chunk of them).  At the
// start of its last tile thread 0 takes the next item from the schedule and, when that
// item's walk is running, issues the copy of its first tile, so the copy overlaps this
// tile.  FB super-blocks go into one block sum before each compensated flush.  Returns
// false when a staged copy timed out: the block must then stop taking work.
template <int NT, int NSB, int FB>
__device__ __forceinline__ bool hot_one(WalkDev *hdr, const HotItem *items, Schedule *sched, const uint32_t item,
                                        HotPipe &pipe, uint32_t mbar_s, uint32_t *s_next) {
  static_assert(NSB <= 32, "the per-super-block swizzle assumes at most 32 super-blocks per tile");
  constexpr bool MB = FB == 4;  // short walks: boundary groups by masked lookups
  constexpr int SBB = TabLayout<MB>::SBB;
  extern __shared__ __align__(128) float smem_raw[];
  const uint32_t raw_s = (uint32_t)__cvta_generic_to_shared(smem_raw);
  const uint32_t tab_s = (raw_s + 127u) & ~127u;  // lookups OR a swizzle into the low 7 bits
  float *tab = smem_raw + (tab_s - raw_s) / 4;
  constexpr int kTileK = NSB * kSbK;
  float4 *stage = reinterpret_cast<float4 *>(tab + NSB * TabLayout<MB>::SBF);  // 2 x kTileK staged T values
  const uint32_t stage_s = tab_s + NSB * SBB;
  int *s_kmax = reinterpret_cast<int *>(stage + 2 * kTileK);
  int *s_timeout = s_kmax + 1;
  int *s_kin_lo = s_kmax + 2, *s_kin_hi = s_kmax + 3;  // block-wide range of kin
  int *s_run = s_kmax + 4;                              // the walk was running when the item began
  int *s_pre = s_kmax + 5;                              // the next item's first copy is issued
  int *s_kout_lo = s_kmax + 6;                          // block-wide minimum of kout
  const HotItem it = items[item];
  WalkDev &W = hdr[it.slot];
  // thread 0 takes the next item (copy q issued for its first tile when `prefetch`)
  auto take_next = [&](bool prefetch, uint32_t q) {
    const uint32_t nx = atomicAdd(&sched->hot_next, 1u);
    *s_next = nx;
    *s_pre = 0;
    if (prefetch && nx < sched->nitems) {
      const HotItem in = items[nx];
      const WalkDev &Wn = hdr[in.slot];
      const int kt0n = 1 + item_tile_lo<NSB>(Wn, in) * kTileK;
      if (Wn.status == kRunning && !Wn.inject_stall && kt0n < (int)Wn.L) {
        stage_copy<NSB>(stage_s, mbar_s, q, Wn.T, kt0n, (int)Wn.L);
        *s_pre = 1;
      }
    }
  };
  // every thread waits on copy q (bounded)
  auto wait_copy = [&](uint32_t q, int limit) {
    return mbar_wait_bounded(mbar_s + 8u * (q & 1u), (q >> 1) & 1u, limit);
  };
  if (threadIdx.x == 0) {
    *s_kmax = 0;
    *s_timeout = 0;
    *s_kin_lo = INT_MAX;
    *s_kout_lo = INT_MAX;
    *s_kin_hi = 0;
    *s_run = W.status == kRunning ? 1 : 0;  // one reading for the whole block
  }
  __syncthreads();
  if (!*s_run) {
    // a copy issued for this item is consumed before its buffer is used again
    if (pipe.pre) {
      if (!wait_copy(pipe.seq, 1 << 20)) *s_timeout = 1;
      pipe.seq++;
    }
    __syncthreads();
    if (*s_timeout) return false;  // the copy may still be in flight: stop using this block
    if (threadIdx.x == 0) take_next(false, pipe.seq);
    __syncthreads();
    pipe.pre = *s_pre != 0;
    return true;
  }
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
  const uint32_t *__restrict__ win_f = W.win_f;
  const uint32_t *__restrict__ win_r = W.win_r;
  const int w_kin_lo = __reduce_min_sync(0xffffffffu, kin);
  const int w_kin_hi = __reduce_max_sync(0xffffffffu, kin);
  const int w_kout_lo = __reduce_min_sync(0xffffffffu, kout);
  const int w_kout_hi = warp_live ? __reduce_max_sync(0xffffffffu, kout) : 0;
  const WarpRange wr{w_kin_lo, w_kin_hi, w_kout_lo, w_kout_hi};
  if ((threadIdx.x & 31) == 0) {
    atomicMax(s_kmax, w_kout_hi);
    atomicMin(s_kin_lo, w_kin_lo);
    if (warp_live) atomicMin(s_kout_lo, w_kout_lo);
    atomicMax(s_kin_hi, w_kin_hi);
  }
  __syncthreads();
  const int kmax = *s_kmax;
  const int blk_kin_lo = *s_kin_lo, blk_kin_hi = *s_kin_hi, blk_kout_lo = *s_kout_lo;
  // tiles of this block: all of them, or those of its k-chunk when the k range is split
  const int tiles_per_chunk = (int)W.kchunk_sb / NSB;
  const int tile_lo = item_tile_lo<NSB>(W, it);
  const int tile_hi = W.ksplit > 1 ? min((kmax + kTileK - 1) / kTileK, tile_lo + tiles_per_chunk)
                                   : (kmax + kTileK - 1) / kTileK;
  const int ntiles = max(0, tile_hi - tile_lo);
  // test hook: no copy is issued for this walk, so every wait below runs out (short limit)
  // and the walk is marked failed; nothing of it is left in flight
  const bool stall = W.inject_stall != 0;
  const int wait_limit = stall ? 64 : (1 << 20);
  if (pipe.pre && ntiles == 0) {  // staged for nothing: consume it
    if (!wait_copy(pipe.seq, 1 << 20)) *s_timeout = 1;
    pipe.seq++;
    pipe.pre = false;
  }
  if (threadIdx.x == 0 && ntiles > 0 && !stall && !pipe.pre)
    stage_copy<NSB>(stage_s, mbar_s, pipe.seq, T, 1 + tile_lo * kTileK, L);
  if (ntiles == 0) {
    __syncthreads();
    if (threadIdx.x == 0) take_next(true, pipe.seq);
  }

  float hi = 0.f, lo = 0.f, a0 = 0.f, a1 = 0.f;
  for (int tile = 0; tile < ntiles; tile++) {
    const int kt0 = 1 + (tile_lo + tile) * kTileK;
    const uint32_t cq = pipe.seq + (uint32_t)tile;  // this tile's copy
    __syncthreads();  // previous tile fully consumed (tables, and the staging buffer reused below)
    if (threadIdx.x == 0) {
      if (tile + 1 < ntiles) {
        if (!stall) stage_copy<NSB>(stage_s, mbar_s, cq + 1, T, kt0 + kTileK, L);
      } else {
        take_next(!stall, cq + 1);
      }
    }
    // every thread observes the copy's completion: the builders read the staged values, and
    // so does the generic path of any warp while it scores this tile
    if (!wait_copy(cq, wait_limit)) *s_timeout = 1;
    if ((int)threadIdx.x < 6 * NSB) {
      const float4 *Ts = stage + (cq & 1u) * kTileK;
      for (int t = threadIdx.x; t < 6 * NSB; t += NT) {
        const int sb = t % NSB, q = t / NSB;
        const int ka = kt0 + sb * kSbK;  // first shift of the super-block
        // two-partner shifts k <= kin exist here for some lane iff ka <= max kin; one-partner
        // shifts kin < k <= kout iff ka + 29 > min kin and ka <= max kout
        const bool need_w = ka <= blk_kin_hi;
        const bool need_e = ka + kSbK - 1 > blk_kin_lo && ka <= kmax;
        // a group straddles some lane's kin or kout only inside [min kin - 4, max kin] or
        // [min kout - 4, max kout]
        const bool need_m = MB && ((ka <= blk_kin_hi && ka + kSbK - 1 >= blk_kin_lo - 4) ||
                                   (ka <= kmax && ka + kSbK - 1 >= blk_kout_lo - 4));
        if (need_w || need_e) build_group<MB>(tab, sb, q, Ts, kt0, ka + 5 * q, L, need_w, need_e, need_m);
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
    const uint32_t bsw0 = tab_s;  // super-block sb: base + SBB sb, swizzle sb << 2
    int sb = 0;
    {
      const uint32_t *wu = win_f + (j + kt0), *wv = win_r + (j - kt0);
      uint32_t bsw = bsw0;
      // FB super-blocks per flush: at most 6 FB additions into either accumulator
      for (; sb + FB - 1 < n_int; sb += FB) {
#pragma unroll
        for (int u = 0; u < FB; u++) sb_interior<MB>(a0, a1, wu + u * kSbK, wv - u * kSbK, M, bsw + u * (SBB + 4));
        flush2(hi, lo, a0, a1);
        wu += FB * kSbK, wv -= FB * kSbK, bsw += FB * (SBB + 4);
      }
      if (sb < n_int) {
        for (; sb < n_int; sb++) {
          sb_interior<MB>(a0, a1, wu, wv, M, bsw);
          wu += kSbK, wv -= kSbK, bsw += SBB + 4;
        }
        flush2(hi, lo, a0, a1);
      }
    }
    const float4 *Ts = stage + (cq & 1u) * kTileK;  // this tile's per-k values, still staged
    for (; sb < e0; sb++) {
      sb_generic<MB>(a0, a1, win_f, win_r, Ts, kt0, j, kt0 + sb * kSbK, kin, kout, plus_side, M,
                     bsw0 + sb * (SBB + 4), L, wr);
      flush2(hi, lo, a0, a1);
    }
    {
      const int step = plus_side ? kSbK : -kSbK;
      const uint32_t *we = plus_side ? win_f + (j + kt0 + sb * kSbK) : win_r + (j - kt0 - sb * kSbK);
      uint32_t bsw = bsw0 + sb * (SBB + 4);
      // FB super-blocks per flush: at most 3 FB additions into either accumulator
      for (; sb + FB - 1 < n_edge; sb += FB) {
#pragma unroll
        for (int u = 0; u < FB; u++) sb_edge<MB>(a0, a1, we + u * step, M, bsw + u * (SBB + 4));
        flush2(hi, lo, a0, a1);
        we += FB * step, bsw += FB * (SBB + 4);
      }
      if (sb < n_edge) {
        for (; sb < n_edge; sb++) {
          sb_edge<MB>(a0, a1, we, M, bsw);
          we += step, bsw += SBB + 4;
        }
        flush2(hi, lo, a0, a1);
      }
    }
    for (; sb < n_all; sb++) {
      sb_generic<MB>(a0, a1, win_f, win_r, Ts, kt0, j, kt0 + sb * kSbK, kin, kout, plus_side, M,
                     bsw0 + sb * (SBB + 4), L, wr);
      flush2(hi, lo, a0, a1);
    }
  }
  __syncthreads();  // the next item and its copy flag are visible to every thread
  const bool next_pre = *s_pre != 0;
  if (*s_timeout) {
    // a staged copy never arrived: give every copy of this block one more bounded wait,
    // then mark the walk failed instead of using its scores
    if (threadIdx.x == 0) {
      if (!stall) {
        const uint32_t last = pipe.seq + (uint32_t)ntiles + (next_pre ? 1u : 0u);
        for (uint32_t q = last >= 2 ? last - 2 : 0; q < last; q++) wait_copy(q, 1 << 20);
        // the item taken for this block will not be scored: its walk fails too
        if (*s_next < sched->nitems) {
          WalkDev &Wn = hdr[items[*s_next].slot];
          Wn.error = (uint32_t)-5;
          Wn.status = kError;
        }
      }
      W.error = (uint32_t)-5;  // PSL_ETIMEOUT of the library header
      W.status = kError;
    }
    if (!stall) return false;  // a copy may still be in flight: stop using this block
  }
  if (!stall) pipe.seq += (uint32_t)ntiles;
  pipe.pre = next_pre;
  if (*s_timeout) return true;
  if (!live) return true;
  if (W.ksplit > 1) {
    W.score_part[(size_t)it.kc * N + (i - 1)] = hi + lo;
    if (it.kc != W.kc_psl) return true;
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
template <int NT, int NSB, int FB>
__global__ void __launch_bounds__(NT, 1024 / NT) k_hot_batched(WalkDev *hdr, const HotItem *items, Schedule *sched) {
  __shared__ __align__(8) uint64_t s_mbar[2];
  __shared__ uint32_t s_next;
  const uint32_t mbar_s = (uint32_t)__cvta_generic_to_shared(s_mbar);
  if (threadIdx.x == 0) {
    mbar_init(mbar_s, 1);
    mbar_init(mbar_s + 8, 1);
    fence_mbar_init();
    s_next = atomicAdd(&sched->hot_next, 1u);
  }
  if constexpr (FB == 4) {
    // masked lookups with an empty mask read entry 0 (the empty subset) of tables that a
    // super-block may not have built: start from zero tables, and every build writes 0
    // there again, so entry 0 of every table always holds 0
    extern __shared__ __align__(128) float smem_tab[];
    const uint32_t raw_s = (uint32_t)__cvta_generic_to_shared(smem_tab);
    float *tab = smem_tab + (((raw_s + 127u) & ~127u) - raw_s) / 4;
    for (int q = threadIdx.x; q < NSB * TabLayout<true>::SBF; q += NT) tab[q] = 0.f;
  }
  __syncthreads();
  HotPipe pipe{0u, false};
  for (;;) {
    const uint32_t item = s_next;
    if (item >= sched->nitems) break;
    __syncthreads();  // every thread has read the item before it is replaced
    if (!hot_one<NT, NSB, FB>(hdr, items, sched, item, pipe, mbar_s, &s_next)) break;
  }
}

// ------------------------------------------------------------------------------------
// neighbourhood score, plain form: one thread per neighbour, every term accumulated on its
// own (the execution model of the paper's GPU solver: one walk, one neighbour per core).
// Blocks of 64 threads spread the window over the SMs; each block stages the per-k values
// of 1024 shifts at a time into shared memory with a TMA bulk copy (double-buffered), so
// every term reads its (Tp4, Tm4, Tp2, Tm2) by a broadcast shared load; for each run of 32
// shifts a lane forms four disjoint bit masks (both partners +4 / -4, one partner +2 / -2)
// and every term adds the one value its bit selects, without a branch.
// ------------------------------------------------------------------------------------
constexpr int kPlainThreads = 64;
constexpr int kPlainTileK = 1024;

size_t hot_plain_smem() { return 2 * (size_t)kPlainTileK * 16; }

// TMA bulk copy of the per-k values of shifts 1 + 1024 tile .. (those below L) into staging
// buffer tile & 1, signalling that buffer's mbarrier.
__device__ __forceinline__ void plain_stage_copy(uint32_t stage_s, uint32_t mbar_s, int tile, const float4 *T, int L) {
  const int kt0 = 1 + tile * kPlainTileK;
  const uint32_t bytes = 16u * (uint32_t)min(kPlainTileK, L - kt0);
  const uint32_t mb = mbar_s + 8u * (uint32_t)(tile & 1);
  fence_proxy_async();
  mbar_expect_tx(mb, bytes);
  tma_load_1d(stage_s + (uint32_t)(tile & 1) * (kPlainTileK * 16), T + kt0, bytes, mb);
}

__global__ void __launch_bounds__(kPlainThreads, 1) k_hot_plain(WalkDev *hdrp) {
  extern __shared__ __align__(128) float4 pstage[];  // 2 x kPlainTileK staged per-k values
  __shared__ __align__(8) uint64_t s_mbar[2];
  __shared__ int s_kmax, s_timeout;
  WalkDev &W = *hdrp;
  const int L = (int)W.L, N = (int)W.N;
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;  // window position, 1-based
  // lanes past the end of the window shadow the last neighbour (their sums are discarded)
  const int j = (int)(((uint64_t)W.start + (uint64_t)min(i, N)) % (uint64_t)L);
  const uint32_t *__restrict__ bits = W.bits;
  const int kin = min(j, L - 1 - j), kout = max(j, L - 1 - j);
  const bool plus_side = j < L - 1 - j;
  const uint32_t M = getbit(bits, j) ? 0xffffffffu : 0u;
  const int cap_u = 32 * (int)W.nw;
  const uint32_t mbar_s = (uint32_t)__cvta_generic_to_shared(s_mbar);
  const uint32_t stage_s = (uint32_t)__cvta_generic_to_shared(pstage);
  if (threadIdx.x == 0) {
    s_kmax = 0;
    s_timeout = 0;
    mbar_init(mbar_s, 1);
    mbar_init(mbar_s + 8, 1);
    fence_mbar_init();
  }
  __syncthreads();
  atomicMax(&s_kmax, kout);
  __syncthreads();
  const int ntiles = (s_kmax + kPlainTileK - 1) / kPlainTileK;
  if (threadIdx.x == 0 && ntiles > 0) plain_stage_copy(stage_s, mbar_s, 0, W.T, L);
  float hi = 0.f, lo = 0.f;
  int issued = ntiles > 0 ? 1 : 0;  // copies issued so far (tiles 0 .. issued-1)
  for (int tile = 0; tile < ntiles; tile++) {
    const int kt0 = 1 + tile * kPlainTileK;
    __syncthreads();  // the buffer the next copy overwrites is no longer read
    if (s_timeout) break;  // one reading for the whole block
    if (tile + 1 < ntiles) {
      if (threadIdx.x == 0) plain_stage_copy(stage_s, mbar_s, tile + 1, W.T, L);
      issued = tile + 2;
    }
    if (!mbar_wait_bounded(mbar_s + 8u * (tile & 1), (tile >> 1) & 1)) s_timeout = 1;
    const float4 *Ts = pstage + (tile & 1) * kPlainTileK;
    const int kend = min(kout, kt0 + kPlainTileK - 1);
    for (int k0 = kt0; k0 <= kend; k0 += 32) {
      const uint32_t U = window32_ro(bits, min(j + k0, cap_u)) ^ M;          // bit t: s_j s_{j+k0+t} = -1
      const uint32_t V = __brev(window32_ro(bits, max(j - k0 - 31, -64))) ^ M;  // bit t: s_j s_{j-k0-t} = -1
      const int nb = min(32, max(0, kin - k0 + 1)), nl = min(32, kout - k0 + 1);
      const uint32_t both = nb >= 32 ? 0xffffffffu : ((1u << nb) - 1u);
      const uint32_t live = nl >= 32 ? 0xffffffffu : ((1u << nl) - 1u);
      const uint32_t one = live & ~both;
      const uint32_t P = plus_side ? U : V;
      const uint32_t W1 = U & V & both, W0 = ~(U | V) & both, Ep = P & one, Em = ~P & one;
      const float4 *Tk = Ts + (k0 - kt0);
      float a0 = 0.f, a1 = 0.f;
#pragma unroll
      for (int t = 0; t < 32; t += 2) {
        const float4 x = Tk[t], y = Tk[t + 1];  // shifts past the tile's copy are masked out
        a0 += ((W1 >> t) & 1u) ? x.x : (((W0 >> t) & 1u) ? x.y : (((Ep >> t) & 1u) ? x.z : (((Em >> t) & 1u) ? x.w : 0.f)));
        a1 += ((W1 >> (t + 1)) & 1u) ? y.x
                                      : (((W0 >> (t + 1)) & 1u) ? y.y
                                                                : (((Ep >> (t + 1)) & 1u) ? y.z
                                                                                          : (((Em >> (t + 1)) & 1u) ? y.w : 0.f)));
      }
      float blk = a0 + a1;
      flush_block(hi, lo, blk);
    }
  }
  __syncthreads();
  if (s_timeout) {
    // a staged copy never arrived: give the copies still outstanding one more bounded wait,
    // then mark the walk failed instead of using its scores
    if (threadIdx.x == 0) {
      for (int q = max(0, issued - 2); q < issued; q++) mbar_wait_bounded(mbar_s + 8u * (q & 1), (q >> 1) & 1);
      W.error = (uint32_t)-5;  // PSL_ETIMEOUT of the library header
      W.status = kError;
    }
    return;
  }
  if (i > N) return;
  W.score[i - 1] = hi + lo;
  int pj = INT_MAX;
  if (W.ktau_on) pj = neighbour_psl(W, W.ktau, (int)W.nktau, j, L, M ? -1 : 1, W.psl - 8, 0);
  W.pslj[i - 1] = pj;
}

// ------------------------------------------------------------------------------------
// neighbourhood score, producer / consumer form
//
// The same scoring as k_hot_batched, with the per-tile block barriers taken out of the
// scoring loop: two producer warps stage each k-tile's per-k values (TMA bulk copy) and
// build its tables into one of two buffers, while NWS scorer warps score the previous
// tile from the other buffer.  Per buffer, "full" (the producer arrives once the tables are
// built) and "empty" (every scorer warp arrives once it has scored from the buffer)
// mbarriers order the two sides; a scorer warp never waits for another scorer warp, so the
// warps of a block drift up to one tile apart instead of meeting at every tile.  Every wait
// is bounded; a wait that runs out marks the walk failed and the block stops.  The
// producer derives the block's kin/kout range (which tables a tile needs) from the item's
// window positions directly: they are consecutive modulo L, and kin (kout) rises (falls) to
// the middle of the sequence, so the extremes lie at the ends or at the middle.
// ------------------------------------------------------------------------------------
constexpr int kPcProducerWarps = 2;
constexpr uint32_t kPcEnd = 0xffffffffu;
enum PcFlags : uint32_t { kPcFirst = 1, kPcLast = 2, kPcEmpty = 4, kPcSkip = 8 };

struct PcTile {       // the tile a buffer holds, written by the producer before it arrives on "full"
  uint32_t item;      // work item, or kPcEnd
  int32_t kt0;        // first shift of the tile
  uint32_t flags;     // kPcFirst / kPcLast: first / last tile of the item; kPcEmpty: nothing to score;
                      // kPcSkip: the walk is not running (or failed): nothing to write either
  uint32_t pad;
};

template <int NSB, bool MB>
constexpr size_t pc_smem_bytes() {
  return 2 * (size_t)NSB * TabLayout<MB>::SBB + 2 * (size_t)NSB * kSbK * 16 + 128;
}
size_t hot_pc_smem(uint32_t nsb, bool masked) {
  return 2 * (size_t)nsb * (masked ? TabLayout<true>::SBB : TabLayout<false>::SBB) + 2 * (size_t)nsb * kSbK * 16 + 128;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void producer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(32 * kPcProducerWarps) : "memory"); }

__device__ __forceinline__ int pc_kin(int j, int L) { return min(j, L - 1 - j); }
__device__ __forceinline__ int pc_kout(int j, int L) { return max(j, L - 1 - j); }

// kin / kout extremes over positions x..y (x <= y, no wrap)
__device__ __forceinline__ void pc_seg(int x, int y, int L, int &kin_lo, int &kin_hi, int &kout_lo, int &kout_hi) {
  const int c1 = min(max((L - 1) / 2, x), y), c2 = min(max(L / 2, x), y);
  kin_lo = min(kin_lo, min(pc_kin(x, L), pc_kin(y, L)));
  kin_hi = max(kin_hi, max(max(pc_kin(x, L), pc_kin(y, L)), max(pc_kin(c1, L), pc_kin(c2, L))));
  kout_hi = max(kout_hi, max(pc_kout(x, L), pc_kout(y, L)));
  kout_lo = min(kout_lo, min(min(pc_kout(x, L), pc_kout(y, L)), min(pc_kout(c1, L), pc_kout(c2, L))));
}

template <int NWS, int NSB, int FB>
__global__ void __launch_bounds__(32 * (NWS + kPcProducerWarps), NWS <= 14 ? 2 : 1) k_hot_pc(WalkDev *hdr, const HotItem *items,
                                                                              Schedule *sched) {
  static_assert(NSB <= 32, "the per-super-block swizzle assumes at most 32 super-blocks per tile");
  constexpr bool MB = FB == 4;
  constexpr int NT = 32 * NWS;  // window positions per item
  constexpr int SBB = TabLayout<MB>::SBB, SBF = TabLayout<MB>::SBF;
  constexpr int kTileK = NSB * kSbK;
  extern __shared__ __align__(128) float smem_pc[];
  __shared__ __align__(8) uint64_t s_bar[6];  // full[2], empty[2], copy[2]
  __shared__ PcTile s_hdr[2];
  __shared__ uint32_t s_item;
  __shared__ int s_err, s_pflag, s_prun, s_pstall;
  const uint32_t raw_s = (uint32_t)__cvta_generic_to_shared(smem_pc);
  const uint32_t tab_s0 = (raw_s + 127u) & ~127u;
  float *tab0 = smem_pc + (tab_s0 - raw_s) / 4;
  float4 *stage0 = reinterpret_cast<float4 *>(tab0 + 2 * NSB * SBF);
  const uint32_t stage_s0 = tab_s0 + 2 * NSB * SBB;
  const uint32_t bar_s = (uint32_t)__cvta_generic_to_shared(s_bar);
  auto full_b = [&](int b) { return bar_s + 8u * (uint32_t)b; };
  auto empty_b = [&](int b) { return bar_s + 16u + 8u * (uint32_t)b; };
  auto copy_b = [&](int b) { return bar_s + 32u + 8u * (uint32_t)b; };
  const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; b++) {
      mbar_init(full_b(b), 1);
      mbar_init(empty_b(b), NWS);
      mbar_init(copy_b(b), 1);
    }
    fence_mbar_init();
    s_err = 0;
  }
  if constexpr (MB) {  // masked lookups with an empty mask read entry 0: zero tables, builds keep it 0
    for (int q = threadIdx.x; q < 2 * NSB * SBF; q += blockDim.x) tab0[q] = 0.f;
  }
  __syncthreads();

  if (warp >= NWS) {
    // ---------------------------------- producer ----------------------------------
    const int ptid = (int)threadIdx.x - 32 * NWS;
    uint32_t s = 0;                 // tile sequence number (buffer s & 1, use s >> 1)
    uint32_t ncopy0 = 0u, ncopy1 = 0u;  // copies issued into each staging buffer
    bool ok = true;
    // A bounded wait decided by producer thread 0 and shared with the other producer thread(s),
    // so that both producer warps always take the same branch (they meet at named barriers);
    // after a success each thread observes the completed phase itself (at once).
    auto pwait = [&](uint32_t mbar, uint32_t parity, int limit) {
      if (ptid == 0) s_pflag = mbar_wait_bounded(mbar, parity, limit) ? 1 : 0;
      producer_sync();
      const bool r = s_pflag != 0;
      if (r && ptid != 0) mbar_wait_bounded(mbar, parity, 1 << 20);
      producer_sync();  // s_pflag is free for the next wait
      return r;
    };
    // hands tile s over to the scorers: waits until they have released its buffer
    auto publish = [&](uint32_t item, int kt0, uint32_t flags) {
      const int b = (int)(s & 1u);
      if (ptid == 0) {
        s_hdr[b].item = item;
        s_hdr[b].kt0 = kt0;
        s_hdr[b].flags = flags;
        mbar_arrive(full_b(b));  // release: the tables and the header are visible to the scorers
      }
      s++;
    };
    auto claim = [&]() {  // buffer s & 1 is free once every scorer warp released its use before
      const int b = (int)(s & 1u);
      if (s >= 2 && !pwait(empty_b(b), ((s >> 1) - 1u) & 1u, 1 << 20)) return false;
      return true;
    };
    for (;;) {
      // thread 0 takes the next item and reads the walk's state once for both producer warps
      if (ptid == 0) {
        const uint32_t nx = atomicAdd(&sched->hot_next, 1u);
        s_item = nx;
        s_prun = 0, s_pstall = 0;
        if (nx < sched->nitems) {
          const WalkDev &Wn = hdr[items[nx].slot];
          s_prun = Wn.status == kRunning ? 1 : 0;
          s_pstall = Wn.inject_stall ? 1 : 0;
        }
      }
      producer_sync();
      const uint32_t item = s_item;
      const bool run = s_prun != 0, stall = s_pstall != 0;
      producer_sync();  // every producer thread has read them before thread 0 writes the next
      if (item >= sched->nitems) break;
      const HotItem it = items[item];
      WalkDev &W = hdr[it.slot];
      if (!run) {
        if (!(ok = claim())) break;
        publish(item, 0, kPcFirst | kPcLast | kPcEmpty | kPcSkip);
        continue;
      }
      const int L = (int)W.L, N = (int)W.N;
      // the item's positions: start + i0 .. start + min(i0 + NT - 1, N), modulo L
      const int a = (int)(((uint64_t)W.start + (uint64_t)it.i0) % (uint64_t)L);
      const int cnt = min((int)it.i0 + NT - 1, N) - (int)it.i0 + 1;
      int kin_lo = INT_MAX, kin_hi = 0, kout_lo = INT_MAX, kout_hi = 0;
      if (a + cnt - 1 < L) {
        pc_seg(a, a + cnt - 1, L, kin_lo, kin_hi, kout_lo, kout_hi);
      } else {
        pc_seg(a, L - 1, L, kin_lo, kin_hi, kout_lo, kout_hi);
        pc_seg(0, a + cnt - 1 - L, L, kin_lo, kin_hi, kout_lo, kout_hi);
      }
      const int kmax = kout_hi;
      const int tiles_per_chunk = (int)W.kchunk_sb / NSB;
      const int tile_lo = item_tile_lo<NSB>(W, it);
      const int tile_hi = W.ksplit > 1 ? min((kmax + kTileK - 1) / kTileK, tile_lo + tiles_per_chunk)
                                       : (kmax + kTileK - 1) / kTileK;
      const int ntiles = max(0, tile_hi - tile_lo);
      if (ntiles == 0) {
        if (!(ok = claim())) break;
        publish(item, 0, kPcFirst | kPcLast | kPcEmpty);
        continue;
      }
      bool failed = false;
      for (int tile = 0; tile < ntiles; tile++) {
        const int kt0 = 1 + (tile_lo + tile) * kTileK;
        const uint32_t flags = (tile == 0 ? kPcFirst : 0u) | (tile + 1 == ntiles ? kPcLast : 0u);
        if (!(ok = claim())) break;
        const int b = (int)(s & 1u);
        if (failed) {  // the walk failed on an earlier tile of this item: hand the rest over unscored
          publish(item, kt0, flags | kPcEmpty | kPcSkip);
          continue;
        }
        // stage the tile's per-k values (the test hook issues nothing and waits briefly)
        if (ptid == 0 && !stall) {
          const uint32_t bytes = 16u * (uint32_t)min(kTileK, L - kt0);
          fence_proxy_async();
          mbar_expect_tx(copy_b(b), bytes);
          tma_load_1d(stage_s0 + (uint32_t)b * (kTileK * 16), W.T + kt0, bytes, copy_b(b));
        }
        if (!stall) (b ? ncopy1 : ncopy0)++;
        const uint32_t nc = b ? ncopy1 : ncopy0;
        // copy nc of this buffer completes its phase nc - 1; with no copy issued, the phase in
        // progress (parity nc) never completes and the short wait runs out
        const bool got = stall ? pwait(copy_b(b), nc & 1u, 64) : pwait(copy_b(b), (nc - 1u) & 1u, 1 << 20);
        if (!got) {
          if (!stall) {  // a copy that may still be in flight: stop using this block
            ok = false;
            if (ptid == 0) {
              W.error = (uint32_t)-5;  // PSL_ETIMEOUT of the library header
              W.status = kError;
            }
            break;
          }
          // nothing is in flight: the walk fails, the block carries on
          if (ptid == 0) {
            W.error = (uint32_t)-5;
            W.status = kError;
          }
          failed = true;
          publish(item, kt0, flags | kPcEmpty | kPcSkip);
          continue;
        }
        // build the tile's tables (one group per producer thread at a time)
        const float4 *Ts = stage0 + b * kTileK;
        for (int g = ptid; g < 6 * NSB; g += 32 * kPcProducerWarps) {
          const int sb = g % NSB, q = g / NSB;
          const int ka = kt0 + sb * kSbK;
          const bool need_w = ka <= kin_hi;
          const bool need_e = ka + kSbK - 1 > kin_lo && ka <= kmax;
          const bool need_m = MB && ((ka <= kin_hi && ka + kSbK - 1 >= kin_lo - 4) ||
                                     (ka <= kmax && ka + kSbK - 1 >= kout_lo - 4));
          if (need_w || need_e) build_group<MB>(tab0 + b * NSB * SBF, sb, q, Ts, kt0, ka + 5 * q, L, need_w, need_e, need_m);
        }
        producer_sync();  // every table of the tile is written
        publish(item, kt0, flags);
      }
      if (!ok) break;
    }
    // end of work (or a stopped block): the scorers leave at the next header
    if (ok && claim()) {
      publish(kPcEnd, 0, 0);
    } else if (ptid == 0) {
      s_err = 1;
      // release the scorers waiting on either buffer; they read kPcEnd and leave
      for (int b = 0; b < 2; b++) {
        s_hdr[b].item = kPcEnd;
        mbar_arrive(full_b(b));
      }
    }
    return;
  }

  // ---------------------------------- scorers ----------------------------------
  uint32_t s = 0;
  // state of the item in progress (lane = one window position)
  uint32_t cur = kPcEnd;
  WalkDev *Wp = nullptr;
  int i = 0, j = 0, kin = 0, kout = 0, L = 0, N = 0;
  bool live = false, plus_side = false, skip = false;
  uint32_t M = 0;
  WarpRange wr{0, 0, 0, 0};
  float hi = 0.f, lo = 0.f, a0 = 0.f, a1 = 0.f;
  for (;;) {
    const int b = (int)(s & 1u);
    // one decision for the whole warp (a lane whose wait ran out fails every lane)
    const bool got = mbar_wait_bounded(full_b(b), (s >> 1) & 1u);
    if (__any_sync(0xffffffffu, !got)) {
      if (lane == 0) s_err = 1;
      if (cur != kPcEnd && lane == 0 && Wp) {
        Wp->error = (uint32_t)-5;
        Wp->status = kError;
      }
      break;
    }
    const PcTile h = s_hdr[b];
    if (h.item == kPcEnd) break;
    if (h.flags & kPcFirst) {
      cur = h.item;
      const HotItem it = items[cur];
      Wp = hdr + it.slot;
      skip = (h.flags & kPcSkip) != 0;
      hi = lo = a0 = a1 = 0.f;
      if (!skip) {
        const WalkDev &W = *Wp;
        L = (int)W.L, N = (int)W.N;
        i = (int)it.i0 + 32 * warp + lane;
        live = i <= N;
        j = (int)(((uint64_t)W.start + (uint64_t)min(i, N)) % (uint64_t)L);
        const bool warp_live = (int)it.i0 + 32 * warp <= N;
        kin = min(j, L - 1 - j), kout = max(j, L - 1 - j);
        plus_side = j < L - 1 - j;
        M = getbit(W.bits, j) ? 0xffffffffu : 0u;
        wr.kin_lo = __reduce_min_sync(0xffffffffu, kin);
        wr.kin_hi = __reduce_max_sync(0xffffffffu, kin);
        wr.kout_lo = __reduce_min_sync(0xffffffffu, kout);
        wr.kout_hi = warp_live ? __reduce_max_sync(0xffffffffu, kout) : 0;
      }
    }
    if (h.flags & kPcSkip) skip = true;
    if (!(h.flags & kPcEmpty) && !skip) {
      const WalkDev &W = *Wp;
      const uint32_t *__restrict__ win_f = W.win_f;
      const uint32_t *__restrict__ win_r = W.win_r;
      const int kt0 = h.kt0;
      const float4 *Ts = stage0 + b * kTileK;
      const int n_all = sb_count(wr.kout_hi, kt0, 0, NSB);
      const int n_int = min(sb_count(wr.kin_lo, kt0, kSbK - 1, NSB), n_all);
      const int e0 = max(n_int, min(n_all, sb_count(wr.kin_hi, kt0, 0, NSB)));
      const int n_edge = max(e0, min(n_all, sb_count(wr.kout_lo, kt0, kSbK - 1, NSB)));
      const uint32_t bsw0 = tab_s0 + (uint32_t)b * (NSB * SBB);
      int sb = 0;
      {
        const uint32_t *wu = win_f + (j + kt0), *wv = win_r + (j - kt0);
        uint32_t bsw = bsw0;
        for (; sb + FB - 1 < n_int; sb += FB) {
#pragma unroll
          for (int u = 0; u < FB; u++) sb_interior<MB>(a0, a1, wu + u * kSbK, wv - u * kSbK, M, bsw + u * (SBB + 4));
          flush2(hi, lo, a0, a1);
          wu += FB * kSbK, wv -= FB * kSbK, bsw += FB * (SBB + 4);
        }
        if (sb < n_int) {
          for (; sb < n_int; sb++) {
            sb_interior<MB>(a0, a1, wu, wv, M, bsw);
            wu += kSbK, wv -= kSbK, bsw += SBB + 4;
          }
          flush2(hi, lo, a0, a1);
        }
      }
      for (; sb < e0; sb++) {
        sb_generic<MB>(a0, a1, win_f, win_r, Ts, kt0, j, kt0 + sb * kSbK, kin, kout, plus_side, M,
                       bsw0 + sb * (SBB + 4), L, wr);
        flush2(hi, lo, a0, a1);
      }
      {
        const int step = plus_side ? kSbK : -kSbK;
        const uint32_t *we = plus_side ? win_f + (j + kt0 + sb * kSbK) : win_r + (j - kt0 - sb * kSbK);
        uint32_t bsw = bsw0 + sb * (SBB + 4);
        for (; sb + FB - 1 < n_edge; sb += FB) {
#pragma unroll
          for (int u = 0; u < FB; u++) sb_edge<MB>(a0, a1, we + u * step, M, bsw + u * (SBB + 4));
          flush2(hi, lo, a0, a1);
          we += FB * step, bsw += FB * (SBB + 4);
        }
        if (sb < n_edge) {
          for (; sb < n_edge; sb++) {
            sb_edge<MB>(a0, a1, we, M, bsw);
            we += step, bsw += SBB + 4;
          }
          flush2(hi, lo, a0, a1);
        }
      }
      for (; sb < n_all; sb++) {
        sb_generic<MB>(a0, a1, win_f, win_r, Ts, kt0, j, kt0 + sb * kSbK, kin, kout, plus_side, M,
                       bsw0 + sb * (SBB + 4), L, wr);
        flush2(hi, lo, a0, a1);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(empty_b(b));  // this warp is done with the buffer
    if ((h.flags & kPcLast) && !skip && live) {
      WalkDev &W = *Wp;
      const HotItem it = items[cur];
      if (W.ksplit > 1) {
        W.score_part[(size_t)it.kc * N + (i - 1)] = hi + lo;
      } else {
        W.score[i - 1] = hi + lo;
      }
      if (W.ksplit <= 1 || it.kc == W.kc_psl) {
        // exact neighbour PSL, only when some neighbour may beat psl_best
        int pj = INT_MAX;
        if (W.ktau_on) pj = neighbour_psl(W, W.ktau, (int)W.nktau, j, L, M ? -1 : 1, W.psl - 8, 0);
        W.pslj[i - 1] = pj;
      }
    }
    s++;
  }
}

static uint32_t g_hot_blocks_per_sm[3][2][2];  // occupancy of every variant, measured at set-up

using HotFn = void (*)(WalkDev *, const HotItem *, Schedule *);

static int variant_index(uint32_t threads) { return threads == 512 ? 2 : (threads == 128 ? 0 : 1); }

template <int FB>
static HotFn hot_variant_fb(uint32_t threads, uint32_t tile_sb) {
  if (threads == 512) return tile_sb == 16 ? k_hot_batched<512, 16, FB> : k_hot_batched<512, 32, FB>;
  if (threads == 128) return tile_sb == 16 ? k_hot_batched<128, 16, FB> : k_hot_batched<128, 32, FB>;
  return tile_sb == 16 ? k_hot_batched<256, 16, FB> : k_hot_batched<256, 32, FB>;
}

static HotFn hot_variant(uint32_t threads, uint32_t tile_sb, uint32_t flush_sb) {
  return flush_sb == 4 ? hot_variant_fb<4>(threads, tile_sb) : hot_variant_fb<8>(threads, tile_sb);
}

// Producer / consumer configurations: hot_threads is the number of window positions per work
// item (the scorer lanes); 896 = 28 scorer warps, one block per SM, 32-super-block tiles for
// long walks; 448 = 14 scorer warps, two blocks per SM, 16-super-block tiles.  Short-walk
// batches (five tables per group) use 16-super-block tiles in both.
static bool is_pc(uint32_t threads) { return threads == 896 || threads == 448; }

static HotFn pc_variant(uint32_t threads, uint32_t fb) {
  if (threads == 896) return fb == 4 ? k_hot_pc<28, 16, 4> : k_hot_pc<28, 32, 8>;
  return fb == 4 ? k_hot_pc<14, 16, 4> : k_hot_pc<14, 16, 8>;
}

static uint32_t pc_nsb(uint32_t threads, uint32_t fb) { return (threads == 896 && fb == 8) ? 32u : 16u; }

static uint32_t g_pc_blocks_per_sm[2][2];  // [448 / 896][fb 4 / 8]

bool hot_config_supported(uint32_t threads, uint32_t tile_sb) {
  if (is_pc(threads)) return tile_sb == (threads == 896 ? 32u : 16u);
  return (threads == 128 || threads == 256 || threads == 512) && (tile_sb == 16 || tile_sb == 32);
}

uint32_t hot_flush_for(uint32_t maxL) { return maxL >= 4096u ? 8u : 4u; }

int hot_batched_name(const LaunchCtx &c, char *out, int cap) {
  const uint32_t fb = c.hot_flush_sb == 4 ? 4u : 8u;
  if (is_pc(c.hot_threads))
    return snprintf(out, (size_t)cap, "k_hot_pc<%u,%u,%u>", c.hot_threads / 32, pc_nsb(c.hot_threads, fb), fb);
  return snprintf(out, (size_t)cap, "k_hot_batched<%u,%u,%u>", c.hot_threads, c.hot_tile_sb, fb);
}

cudaError_t prepare_hot_kernels() {
  {
    cudaError_t e = cudaFuncSetAttribute(k_hot_plain, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hot_plain_smem());
    if (e != cudaSuccess) return e;
  }
  for (uint32_t t : {128u, 256u, 512u})
    for (uint32_t sb : {16u, 32u})
      for (uint32_t fb : {4u, 8u}) {
        HotFn f = hot_variant(t, sb, fb);
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hot_batched_smem(sb, fb == 4));
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, (int)t, hot_batched_smem(sb, fb == 4));
        if (e != cudaSuccess) return e;
        g_hot_blocks_per_sm[variant_index(t)][sb == 32 ? 1 : 0][fb == 8 ? 1 : 0] = (uint32_t)(nb > 0 ? nb : 1);
      }
  for (uint32_t t : {448u, 896u})
    for (uint32_t fb : {4u, 8u}) {
      HotFn f = pc_variant(t, fb);
      const size_t smem = hot_pc_smem(pc_nsb(t, fb), fb == 4);
      cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      int nb = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, (int)(t + 32 * kPcProducerWarps), smem);
      if (e != cudaSuccess) return e;
      g_pc_blocks_per_sm[t == 896 ? 1 : 0][fb == 8 ? 1 : 0] = (uint32_t)(nb > 0 ? nb : 1);
    }
  return cudaSuccess;
}

cudaError_t launch_hot_batched(const LaunchCtx &c) {
  const uint32_t fb = c.hot_flush_sb == 4 ? 4u : 8u;
  if (is_pc(c.hot_threads)) {
    const uint32_t per_sm = g_pc_blocks_per_sm[c.hot_threads == 896 ? 1 : 0][fb == 8 ? 1 : 0];
    pc_variant(c.hot_threads, fb)<<<per_sm * c.sm_count, c.hot_threads + 32 * kPcProducerWarps,
                                    hot_pc_smem(pc_nsb(c.hot_threads, fb), fb == 4), c.stream>>>(c.hdr, c.items, c.sched);
    return cudaGetLastError();
  }
  const uint32_t per_sm = g_hot_blocks_per_sm[variant_index(c.hot_threads)][c.hot_tile_sb == 32 ? 1 : 0][fb == 8 ? 1 : 0];
  hot_variant(c.hot_threads, c.hot_tile_sb, fb)<<<per_sm * c.sm_count, c.hot_threads,
                                                  hot_batched_smem(c.hot_tile_sb, fb == 4), c.stream>>>(c.hdr, c.items, c.sched);
  return cudaGetLastError();
}

cudaError_t launch_hot_plain(WalkDev *hdr_one, uint32_t N, cudaStream_t s) {
  k_hot_plain<<<(N + kPlainThreads - 1) / kPlainThreads, kPlainThreads, hot_plain_smem(), s>>>(hdr_one);
  return cudaGetLastError();
}

}  // namespace psl
