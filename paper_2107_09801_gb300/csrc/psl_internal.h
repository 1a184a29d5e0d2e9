// psl_internal.h -- device-resident walk state and launch interface shared by the
// kernels (psl_kernels.cu) and the host runtime (psl_runtime.cu).  GPU side only.
//
// Notation (0-based, as in the library header): s_0..s_{L-1} in {+1,-1}, packed
// one bit per element, bit = 1 meaning s = -1.  C_k (Eq. 2), PSL (Eq. 3),
// F = sum_{k>=1} |C_k|^alpha (Eq. 4).  A "window" is the limited neighbourhood of
// Algorithm 1: N = min(N_lmt, L) neighbours j = (start + i) % L, i = 1..N.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace psl {

constexpr int kGuardWords = 2;     // zero words before and after every packed sequence
constexpr int kWideLimbs = 12;     // exact fitness: 384-bit, 12 x 32-bit limbs
constexpr int kMaxFlips = 64;      // upper bound on FLIP_lmt actually applied
constexpr int kQcap = 64;          // exact re-check candidates handled per pass of the grid
constexpr int kApplyChunk = 8192;  // k per CTA in the O(L) update pass
constexpr int kRecheckChunk = 16384;  // k per CTA in the exact re-check
constexpr int kSbK = 30;           // k per super-block (6 groups of 5)
constexpr int kGroupK = 5;         // k per table group (32-entry tables)
constexpr int kApplyPartStride = 32;  // u32 per apply-chunk partial record
constexpr int kFlushBlockAdds = 64;   // FP32 additions per lane before a compensated flush
constexpr int kKsplitMax = 16;        // most k-chunks one neighbour's score may be split into
constexpr int kKchunkSbUnit = 32;     // k-chunks are whole multiples of 32 super-blocks (960 k)
constexpr int kWinGuard = 32;         // entries before index 0 and past index L-1 of the partner windows

enum WalkStatus : uint32_t { kFree = 0, kRunning = 1, kDone = 2, kError = 3 };
enum ApplyMode : uint32_t { kModeInit = 0, kModeMove = 1, kModeSwitch = 2 };
enum TraceFlags : uint32_t { kImproved = 1, kWorse = 2, kSwitch = 4, kPslBest = 8 };

// Per-step record kept on the device when a walk asks for a trace.
struct TraceRec {
  uint64_t step;
  uint32_t start, kstar, alpha, unimproved;
  int32_t psl, psl_best, win_psl;
  uint32_t win_psl_j, flags, nflip, ncand;
  float score_kstar, score_min, bound;
  int32_t scale_e;                // the step's FP32 tables were scaled by 2^(-alpha * scale_e)
  uint32_t pad;                   // explicit: value_step starts at byte 72, no implicit padding
  double value_step;              // exact F of the chosen neighbour, rounded to FP64
  uint32_t value_exact[kWideLimbs];
};
static_assert(sizeof(TraceRec) == 128 && offsetof(TraceRec, value_step) == 72, "trace record layout");

// One walk slot.  Static fields are written by the host at admission; dynamic
// fields are owned by the device while the walk runs.
struct WalkDev {
  // ---- static ----
  uint32_t L, N, nw, nflip;
  uint32_t alpha1, alpha2, ls_lmt, topk;
  uint64_t seed, budget;
  uint32_t nchunk_apply, nchunk_rc, trace_cap, has_init_seq;
  uint32_t track_fbest, pad_static;  // keep the lowest-F pivot (alpha1 == alpha2: one objective)
  uint32_t shard_rank, shard_count;  // k-sharding of one walk over ranks: this rank scores and re-checks the
                                     // k-chunks c with c % shard_count == shard_rank (count <= 1: all of them)
  uint32_t *bits, *bits_local, *bits_best;  // logical word 0 (guards before and after)
  uint32_t *bits_fbest;                     // lowest-F pivot (when track_fbest)
  // partner windows of the pivot for every position p (neighbourhood kernel): bit t of
  // win_f[p] is the bit of s_{p+t}, bit t of win_r[p] that of s_{p-t} (0 outside 0..L-1);
  // indices -kWinGuard .. L-1+kWinGuard
  uint32_t *win_f, *win_r;
  int32_t *C, *C_local;
  float4 *T;          // per k: (Tp4, Tm4, Tp2, Tm2), scaled by 2^(-alpha*e)
  float *score;       // FP32 filter score of window position i at [i-1]
  float *score_part;  // per-k-chunk partial scores [chunk][N] when the k range is split; with the
                      // alpha = 2 closed form (never split) the exact Delta F of each neighbour, as int32
  int32_t *pslj;      // exact neighbour PSL (or INT32_MAX when not needed)
  int2 *ktau;         // near-peak list (k, C_k)
  uint32_t *cand;     // candidate window positions, ascending
  uint32_t *rc_part;  // exact re-check partials [cand][chunk][2*kWideLimbs]
  uint32_t *ap_part;  // update-pass partials [chunk][kApplyPartStride]
  TraceRec *trace;
  // ---- dynamic ----
  uint32_t status, error;
  uint32_t alpha, unimproved;
  int32_t psl, psl_best, psl_local;
  uint32_t start;
  uint64_t rng_ctr, moves, flip_evals, switches, rechecks;
  int32_t e;              // table scale exponent: 2^e >= max|C| + 4 over the next window
  float S_abs;            // sum_k max |T_k| (bounds the FP32 error of every score)
  uint32_t nktau, ktau_on;
  int32_t ktau_thr;       // list threshold on |C_k| for the running update pass
  uint32_t ncand;
  uint32_t kstar, kstar_i;
  uint32_t mode, improved, psl_improved, psl_j;
  int32_t win_psl;
  uint32_t win_psl_i;
  uint32_t arrive;
  uint32_t alpha_next;
  uint32_t ksplit, kchunk_sb;  // k-chunks of the neighbourhood kernel and their size (super-blocks)
  uint32_t kc_psl, pad_kc;     // the k-chunk whose blocks also compute the neighbours' exact PSL
  uint32_t inject_stall;       // test hook: the next neighbourhood pass waits on copies never issued
  float score_min, bound;
  uint32_t flips[kMaxFlips];
  uint32_t F[kWideLimbs], value_local[kWideLimbs], value_step[kWideLimbs];
  uint32_t F_best[kWideLimbs];  // exact F of bits_fbest
};

// One unit of the neighbourhood kernel: a block of consecutive window positions.
struct HotItem {
  uint32_t slot;
  uint32_t i0;  // first window position (1-based) of the block
  uint32_t kc;  // k-chunk of the block (0 when the walk's k range is not split)
  uint32_t pad;
};

// What one step's persistent kernels work on, kept in device memory so that a captured
// CUDA graph of steps serves every batch composition: the host rewrites it between launches.
struct Schedule {
  uint32_t nactive;          // running walks listed in the active array
  uint32_t nitems;           // neighbourhood work items
  uint32_t max_chunk_apply;  // most update-pass chunks of any listed walk
  uint32_t max_chunk_rc;     // most re-check chunks of any listed walk
  uint32_t hot_next;         // next neighbourhood item to hand out (reset by k_decide)
  uint32_t general;          // some listed walk needs the general update pass (initialisation or a phase
                             // switch): set by the host and by k_decide, cleared by k_select
  uint32_t alpha2;           // the batch is scored by the alpha = 2 closed form: every neighbour's exact
                             // Delta F is in its walk's score_part (as int32), so the re-check copies it
  uint32_t pad;
};

struct LaunchCtx {
  WalkDev *hdr;            // device array of walk slots
  const uint32_t *active;  // device list of active slots
  Schedule *sched;         // device schedule of this launch sequence
  const HotItem *items;    // device list of neighbourhood blocks
  uint32_t hot_threads;    // neighbours per block of the batched kernel
  uint32_t hot_tile_sb;    // super-blocks per k-tile
  uint32_t hot_flush_sb;   // super-blocks per block sum of the batched kernel (4 or 8)
  uint32_t sm_count;
  uint32_t alpha2;         // every running walk has alpha = 2 and L <= kA2MaxL: the closed-form score
  uint32_t maxL;           // longest walk of an initialisation launch
  uint32_t ninit;          // walks of an initialisation launch
  cudaStream_t stream;
};

// ---- launchers (psl_kernels.cu) ----
cudaError_t prepare_kernels();      // one-off kernel attributes (call before any capture)
cudaError_t prepare_hot_kernels();  // the neighbourhood kernels' part of it (psl_hot.cu)
cudaError_t prepare_recheck_kernel();  // psl_recheck.cu
cudaError_t prepare_tail_kernel();     // psl_tail.cu
cudaError_t launch_init_bits(const LaunchCtx &c);
cudaError_t launch_autocorr(const LaunchCtx &c);
cudaError_t launch_apply(const LaunchCtx &c);
cudaError_t launch_hot_batched(const LaunchCtx &c);
// neighbourhood score of a batch: the alpha = 2 closed form (psl_alpha2.cu) when c.alpha2,
// else the subset-sum table kernels (psl_hot.cu)
cudaError_t launch_hot(const LaunchCtx &c);
cudaError_t launch_hot_alpha2(const LaunchCtx &c);
cudaError_t prepare_alpha2_kernels();
// name of the neighbourhood kernel that launch_hot runs for c (for profiles and reports),
// snprintf-style: the length of the full name
int hot_kernel_name(const LaunchCtx &c, char *out, int cap);
int hot_batched_name(const LaunchCtx &c, char *out, int cap);
cudaError_t launch_hot_plain(WalkDev *hdr_one, uint32_t N, cudaStream_t s);
cudaError_t launch_select(const LaunchCtx &c);
cudaError_t launch_recheck(const LaunchCtx &c);
cudaError_t launch_decide(const LaunchCtx &c);
cudaError_t launch_step_tail(const LaunchCtx &c);  // select..apply in one kernel, short walks only
constexpr uint32_t kA2MaxL = 4095;  // walks up to this length can take the alpha = 2 closed form
constexpr uint32_t kA2PerThread = 4;  // window positions per thread of the closed-form kernel (per work item:
                                      // this many times the block size)
constexpr uint32_t kTailMaxL = kApplyChunk;      // walks up to this length (one update chunk, one re-check chunk)
constexpr uint32_t kTailMaxN = 2048;             // and windows up to this size (one warp selects)
cudaError_t launch_start_init(const LaunchCtx &c);
size_t hot_batched_smem(uint32_t tile_sb, bool masked);  // masked: the short-walk variants (five tables per group)
bool hot_config_supported(uint32_t threads, uint32_t tile_sb);  // block sizes 128/256/512, tiles 16/32
uint32_t hot_flush_for(uint32_t maxL);  // super-blocks per block sum for a batch whose longest walk is maxL

// Candidate threshold shared bit-for-bit by the device select and the host select
// of the plain form.  Returns the largest FP32 score that may still belong to the
// exact argmin: min + 2B rounded up, with B bounding |FP32 score - exact score|.
// With the k range split into ksplit chunks, each chunk's partial score is rounded once
// more and the partials are summed in chunk order (ksplit - 1 further roundings).
__host__ __device__ inline double score_bound(float S_abs, uint32_t alpha, uint32_t L, uint32_t ksplit) {
  const double u = 5.9604644775390625e-08;  // 2^-24
  const double nflush = (double)(L / kSbK + 2 * ksplit);
  const double rel = (2.0 * alpha + 68.0 + 2.0 * ksplit) * u + (nflush * u) * (nflush * u);
  return rel * (double)S_abs * 1.01 + (double)L * 7.52316384526264e-37;  // + L * 2^-120
}

}  // namespace psl
