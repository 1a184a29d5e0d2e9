/*
 * psl.h -- C ABI of the GB300 library for the limited-neighbourhood search of
 * Boskovic and Brest, "Two-phase Optimization of Binary Sequences with Low Peak
 * Sidelobe Level Value" (arXiv 2107.09801).
 *
 * What the library computes (paper notation, 0-based indices):
 *   a sequence s_0..s_{L-1}, s_i in {+1,-1}                          (Eq. 1)
 *   C_k = sum_{i=0}^{L-1-k} s_i s_{i+k}, k = 0..L-1                   (Eq. 2)
 *   PSL = max_{k=1..L-1} |C_k|                                        (Eq. 3, range read as 1..L-1)
 *   F_alpha = sum_{k=1}^{L-1} |C_k|^alpha                             (Eq. 4)
 * and runs the search of Algorithm 1: every step scores a window of
 * N = min(N_lmt, L) single-flip neighbours j = (start + i) % L, i = 1..N, with
 * start = Rand() % L, through the one-element flip update of Sec. 3
 * (C'_k = C_k - 2 s_j (s_{j+k} + s_{j-k}), absent partners counting 0), moves to
 * the first neighbour of minimum F in scan order (a forced move), keeps the first
 * neighbour of minimum PSL ever evaluated as the best solution, and after more
 * than LS_lmt non-improving steps restarts from local_best with FLIP_lmt random
 * flips while toggling alpha between alpha1 and alpha2.
 *
 * Decisions are exact: F is held as an exact 384-bit integer and every
 * comparison of Algorithm 1 is made on exact values.  The GPU ranks neighbours
 * with an FP32 score whose rounding error is bounded rigorously, and re-scores
 * exactly every neighbour that the bound cannot exclude (plus the FP32 top-k).
 * Results of a walk depend only on its parameters, never on which other walks
 * share the GPU.
 *
 * Readings where the paper is silent: Rand is SplitMix64 seeded per walk (draw
 * order: ceil(L/64) draws for the start sequence, bit b of draw q giving
 * s_{64q+b} with bit 1 meaning -1; one draw per step for start; at a switch,
 * draws % L until min(FLIP_lmt, L) distinct flip positions are found); psl_best,
 * solution_best and local_best start at the start sequence; local_best is kept
 * at a switch; the budget counts steps (each step is one move); alpha is an
 * integer in 1..16.
 *
 * Conventions: functions return PSL_OK (0) or a count >= 0 on success and a
 * negative PSL_E* code on failure.  The library owns all device memory it
 * allocates (or the caller-provided arena) and every device buffer inside it;
 * the caller owns every host buffer passed in.  A context is used by one host
 * thread at a time.
 */
#ifndef PSL_H
#define PSL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define PSL_API __attribute__((visibility("default")))
#else
#define PSL_API
#endif

#define PSL_OK 0
#define PSL_EINVAL (-1)   /* an argument is outside its documented range      */
#define PSL_ENOMEM (-2)   /* the walk can never fit the arena / allocation failed */
#define PSL_ENOENT (-3)   /* unknown walk id                                   */
#define PSL_EBUSY (-4)    /* the walk is still queued or running               */
#define PSL_ETIMEOUT (-5) /* a bounded device wait expired                     */
#define PSL_ECUDA (-6)    /* a CUDA runtime call failed (see psl_last_error)   */
#define PSL_ESTATE (-7)   /* the walk is in an error state                     */

#define PSL_FORM_BATCHED 0 /* all running walks advance together; persistent-style batched kernels */
#define PSL_FORM_PLAIN 1   /* one walk per launch, one thread per neighbour, host-side selection   */

#define PSL_QUEUED 0
#define PSL_RUNNING 1
#define PSL_DONE 2
#define PSL_ERROR 3

typedef struct psl_ctx psl_ctx;

/* Library configuration.  Fill with psl_config_default() and override. */
typedef struct {
  int32_t n_lmt;            /* default N_lmt (Sec. 4.1: 6912)                         */
  int32_t ls_lmt;           /* default LS_lmt (Sec. 4.1: 2000)                        */
  int32_t flip_lmt;         /* default FLIP_lmt (Sec. 4.1: 10)                        */
  int32_t device;           /* CUDA device ordinal                                    */
  uint64_t arena_bytes;     /* device arena size in bytes; 0 = library default       */
  void *arena;              /* optional caller-owned device buffer of arena_bytes    */
  void *stream;             /* cudaStream_t for all work; NULL = library-owned stream */
  int32_t form;             /* PSL_FORM_BATCHED or PSL_FORM_PLAIN                     */
  int32_t max_walks;        /* number of walk slots                                   */
  int32_t hot_tile_sb;      /* k-tile of the batched kernel in super-blocks of 30 k: 16 or 32; 0 = auto */
  int32_t steps_per_graph;  /* steps captured per CUDA graph launch; 0 = plain launches */
  int32_t hot_threads;      /* neighbours per block of the batched kernel: 128, 256 or 512; or 448 / 896
                               for the producer / consumer form (with hot_tile_sb 16 / 32); 0 = auto */
  int32_t max_sms;          /* SMs' worth of resident blocks the persistent kernels launch (0 = all);
                               lets contexts on different streams share the GPU side by side */
  int32_t alpha2_tables;    /* 0: batches whose every walk has alpha1 = alpha2 = 2 and L <= 4095 (the
                               merit-factor case) are scored by the closed form of Eq. 4 at alpha = 2
                               (exact integer changes of F from bit planes of C); 1: by the subset-sum
                               tables like every other batch.  Results are identical. */
} psl_config;

/* Per-walk parameters of psl_submit_ex.  n_lmt, flip_lmt <= 0 and ls_lmt < 0 take
 * the context default; topk <= 0 means 1. */
typedef struct {
  uint32_t L;               /* sequence length, 2 <= L <= 2^20 - 1                     */
  uint64_t seed;            /* walk seed of Rand                                      */
  int32_t alpha1, alpha2;   /* integer exponents of Eq. 4 for the two phases, 1..16   */
  uint64_t budget;          /* number of steps (moves), >= 1                          */
  int32_t n_lmt, ls_lmt, flip_lmt;
  int32_t topk;             /* FP32-ranked neighbours re-scored exactly besides the certified set (1..16) */
  const int8_t *init_seq;   /* optional host array of L values +-1 replacing Rand(L, SEED); copied */
  uint32_t trace_cap;       /* per-step records kept on the device (0 = none)        */
  uint32_t shard_rank;      /* single-walk k-sharding (psl_shard_*): this context's rank ...          */
  uint32_t shard_count;     /* ... of shard_count ranks; 0 or 1 = not sharded                        */
} psl_walk_params;

/* Snapshot of one walk (psl_poll). */
typedef struct {
  int32_t state;            /* PSL_QUEUED / PSL_RUNNING / PSL_DONE / PSL_ERROR        */
  int32_t error;            /* PSL_E* code when state == PSL_ERROR                    */
  uint32_t L;
  uint32_t alpha;           /* exponent of the current phase                          */
  uint64_t moves;           /* steps completed                                        */
  uint64_t flip_evals;      /* neighbours scored (N per step)                         */
  uint64_t switches;        /* phase switches                                         */
  uint64_t rechecks;        /* neighbours re-scored exactly                           */
  int32_t psl;              /* PSL of the current pivot                               */
  int32_t psl_best;         /* best PSL over every evaluated neighbour                */
  uint32_t unimproved;      /* counter of Alg. 1                                      */
  uint32_t pad;
  double F;                 /* F_alpha(pivot), correctly rounded from the exact value */
  double value_local;       /* value_local of Alg. 1, correctly rounded               */
  double t_submit, t_start, t_done; /* host monotonic seconds                         */
} psl_status;

/* Per-step record (psl_trace).  value_exact holds the exact F of the chosen
 * neighbour as 12 little-endian 32-bit limbs of a two's-complement integer. */
typedef struct {
  uint64_t step;
  uint32_t start, kstar, alpha, unimproved;
  int32_t psl, psl_best, win_psl;
  uint32_t win_psl_j, flags, nflip, ncand;
  float score_kstar, score_min, bound;
  int32_t scale_e;          /* score_kstar, score_min and bound are in units of 2^(alpha * scale_e) */
  uint32_t pad;             /* explicit padding: the record has no implicit padding (128 bytes) */
  double value_step;
  uint32_t value_exact[12];
} psl_trace_rec;

/* Full state of one walk for decision replay (psl_export_state). */
typedef struct {
  uint32_t L, N, alpha, unimproved;
  int32_t psl, psl_best, psl_local;
  uint32_t start;           /* window start of the next step                           */
  uint64_t rng_ctr, moves;
  uint32_t F[12], value_local[12];  /* exact, two's complement, little-endian limbs    */
  int32_t state;
  uint32_t pad;
} psl_walk_state;

/* Fills *cfg with defaults: N_lmt 6912, LS_lmt 2000, FLIP_lmt 10 (Sec. 4.1),
 * device 0, library arena, library stream, batched form, 4096 slots. */
PSL_API void psl_config_default(psl_config *cfg);

/* Creates a context on cfg->device.  Errors: PSL_EINVAL (bad field),
 * PSL_ECUDA / PSL_ENOMEM (device or arena unavailable). */
PSL_API int psl_init(const psl_config *cfg, psl_ctx **out);

/* Queues a walk of Algorithm 1 with the context's N_lmt / LS_lmt / FLIP_lmt.
 * alpha1, alpha2 must be integers in 1..16; budget >= 1 steps.  Returns the walk
 * id (>= 0) or PSL_EINVAL / PSL_ENOMEM (the walk can never fit the arena). */
PSL_API int64_t psl_submit(psl_ctx *ctx, uint32_t L, uint64_t seed, double alpha1, double alpha2, uint64_t budget);

/* As psl_submit with every per-walk field of psl_walk_params. */
PSL_API int64_t psl_submit_ex(psl_ctx *ctx, const psl_walk_params *p);

/* Admits queued walks while the arena has room, then advances every running walk
 * by up to max_moves steps (walks stop at their budget).  Blocks until the work
 * is done.  Returns the number of walks still queued or running, or a PSL_E* code. */
PSL_API int psl_step(psl_ctx *ctx, uint32_t max_moves);

/* Status of a walk as of the end of the last psl_step.  PSL_ENOENT if unknown. */
PSL_API int psl_poll(psl_ctx *ctx, int64_t id, psl_status *out);

/* Best sequence found so far (solution_best of Alg. 1): *psl receives its PSL and
 * seq_pm1[0..L-1] its values +-1; cap must be >= L.  PSL_EBUSY while queued. */
PSL_API int psl_best(psl_ctx *ctx, int64_t id, int32_t *psl, int8_t *seq_pm1, size_t cap);

/* psl_best for n walks at once: psl_out[q] receives the PSL of walk ids[q]'s best sequence
 * and seqs[q * cap .. q * cap + L - 1] its values +-1 (cap >= the longest L; either output
 * may be NULL).  The sequences are copied back together with one synchronisation.
 * PSL_ENOENT / PSL_EBUSY / PSL_EINVAL as psl_best, for the first walk that fails. */
PSL_API int psl_best_many(psl_ctx *ctx, const int64_t *ids, size_t n, int32_t *psl_out, int8_t *seqs, size_t cap);

/* Frees the walk's slot and device memory.  Running walks are cancelled. */
PSL_API int psl_release(psl_ctx *ctx, int64_t id);

/* Copies the walk's state (pivot, local_best, solution_best as +-1 arrays of cap >= L
 * values each, any of them may be NULL; C_0..C_{L-1} if C != NULL). */
PSL_API int psl_export_state(psl_ctx *ctx, int64_t id, psl_walk_state *st, int8_t *pivot, int8_t *local_best,
                     int8_t *sol_best, int32_t *C, size_t cap);

/* Copies up to cap per-step records; returns the number copied. */
PSL_API int psl_trace(psl_ctx *ctx, int64_t id, psl_trace_rec *out, size_t cap);

/* Aperiodic autocorrelation (Eq. 2) of nseq sequences given as +-1 host arrays
 * (row-major nseq x L) into host C (nseq x L), computed on the device by the same
 * bit-packed popcount kernel that initialises walks.  PSL_EINVAL on bad sizes. */
PSL_API int psl_autocorr(psl_ctx *ctx, const int8_t *seq_pm1, uint32_t nseq, uint32_t L, int32_t *C);

/* Device bytes a walk of length L with window n_lmt and trace_cap records needs. */
PSL_API uint64_t psl_walk_bytes(uint32_t L, int32_t n_lmt, uint32_t trace_cap);

/* Device time of the library's kernels, accumulated while profiling is enabled. */
typedef struct {
  char name[24];            /* kernel family: hot, select, recheck, decide, apply, hot_plain, init */
  uint64_t launches;
  double total_ms;          /* sum of CUDA-event durations measured on the context's stream */
} psl_kernel_time;

/* Enables CUDA-event timing of the kernel launches of psl_step: 1 every kernel, 2 the
 * neighbourhood-score kernel only (and whole graph launches), 0 off.  Steps run from a CUDA
 * graph are timed by event-record nodes inside the graph (the graph is captured again when
 * the mode changes), and the stream is synchronised after each graph launch to read them;
 * every graph launch is also timed as one unit under "graph".  Enabling resets the totals;
 * PSL_EINVAL for other values. */
PSL_API int psl_profile(psl_ctx *ctx, int enable);

/* Copies up to cap per-kernel totals; returns the number of kernel families. */
PSL_API int psl_profile_read(psl_ctx *ctx, psl_kernel_time *out, size_t cap);

/* Bytes the context has copied from host to device (*h2d) and from device to host (*d2h)
 * since psl_init: walk headers, schedules, start sequences, status readback, best
 * sequences, traces, exported state.  Either pointer may be NULL.  Counted at each copy,
 * not estimated.  PSL_EINVAL for a null ctx. */
PSL_API int psl_transfer_bytes(psl_ctx *ctx, uint64_t *h2d, uint64_t *d2h);

/* Sets how many steps of the batched form one CUDA graph launch runs (0 = plain launches)
 * and, when walks are running, captures that graph now, so that a later psl_step only
 * launches it (the capture reads the device schedule, so it serves any later batch
 * composition).  A graph captured while profiling is enabled carries event-record nodes
 * around the kernels the profile mode times.  PSL_EINVAL for the plain form or steps < 0;
 * PSL_ECUDA if the capture fails. */
PSL_API int psl_set_steps_per_graph(psl_ctx *ctx, int32_t steps);

/* Measured issue rates of the CUDA-core pipes that bound the neighbourhood kernel (no
 * counterpart in the paper: the denominator of its roofline).  Five kernels fill every SM
 * of the device for a few tens of milliseconds each, timed with CUDA events on stream.
 * Rates are per second over the whole device, at whatever SM clock the device ran. */
typedef struct {
  int32_t sm_count;         /* cudaDevAttrMultiProcessorCount                              */
  int32_t max_clock_mhz;    /* cudaDevAttrClockRate                                        */
  int32_t blocks_per_sm;    /* resident blocks of the microbenchmark kernels                */
  int32_t threads_per_block;
  double fadd;              /* FP32 adds per second (independent chains)                    */
  double alu;               /* integer adds and three-input logic ops per second, 1:1     */
  double mix;               /* FP32 add, integer add and logic op 1:1:1, lane-ops per second */
  double lookup;            /* the neighbourhood kernel's inner pattern (shift, logic op forming a
                               table address, shared-memory load, FP32 add): lookups per second */
  double popc;              /* the bit-plane step of the alpha = 2 closed form (three-input logic op,
                               population count, integer add): plane steps per second        */
  double ms[5];             /* duration of the timed launch of each (fadd, alu, mix, lookup, popc) */
} psl_alu_peak_t;

/* Runs the microbenchmarks on device (stream: a cudaStream_t of that device, or NULL) and
 * fills *out.  Makes device current.  PSL_EINVAL for a null out or device < 0; PSL_ECUDA
 * if a launch fails. */
PSL_API int psl_alu_peak(int32_t device, void *stream, psl_alu_peak_t *out);

/* Autotuner of the batched form: admits queued walks, then times every supported
 * configuration of the neighbourhood kernel (neighbours per block 128/256/512 x k-tile
 * of 16/32 super-blocks, which sets the shared-memory footprint, and the producer /
 * consumer form: 448 x 16, 896 x 32, where two producer warps stage and build each tile's
 * tables into one of two buffers while the other warps score) on the walks now
 * running, reps launches each, and keeps the fastest for this context.  The timed
 * launches only recompute window scores that the next step recomputes, so no result
 * changes.  Returns threads | (tile_sb << 16) of the choice, PSL_ESTATE when no walk
 * is running, PSL_EINVAL for the plain form or reps < 1. */
PSL_API int psl_autotune(psl_ctx *ctx, int reps);

/* Writes into name (cap bytes, NUL-terminated, truncated if short) the name of the
 * neighbourhood kernel the next step of ctx launches, after admitting queued walks: e.g.
 * "k_hot_pc<28,32,8>", "k_hot_batched<512,16,4>", "k_hot_alpha2<256>", "k_hot_plain".
 * Returns the length of the full name, PSL_EINVAL for a null argument or cap < 1. */
PSL_API int psl_hot_variant(psl_ctx *ctx, char *name, int32_t cap);

/* Sets the neighbourhood-kernel configuration of the batched form directly (for a
 * choice cached from an earlier psl_autotune).  PSL_EINVAL for unsupported values. */
PSL_API int psl_set_hot_config(psl_ctx *ctx, int32_t threads, int32_t tile_sb);

/* The lowest fitness F over every pivot the walk has visited (its start, each move, each
 * perturbed pivot of a phase switch; the first one on ties) and that pivot.  It is kept
 * when both phases use the same exponent (alpha1 == alpha2), so the objective never
 * changes; with alpha = 2 it is the energy E = sum_{k>=1} C_k^2, and L^2 / (2E) is the
 * merit factor defined in Sec. 2.  value_limbs receives 12 little-endian 32-bit limbs of
 * the exact non-negative integer, value its correctly rounded double, seq_pm1 the
 * sequence as +1/-1 bytes (cap >= L); each may be NULL.  PSL_ESTATE when alpha1 !=
 * alpha2, PSL_EBUSY while the walk is queued, PSL_ENOENT for an unknown id. */
PSL_API int psl_best_fitness(psl_ctx *ctx, int64_t id, uint32_t *value_limbs, double *value, int8_t *seq_pm1,
                             size_t cap);

/* Resizes the persistent kernels of the context for max_sms SMs (0 = all SMs of the
 * device; larger values are clamped to the device).  Takes effect at the next psl_step;
 * results do not change, only which SMs share the work.  Several contexts on one device
 * whose shares add up to at most the SM count run their steps side by side.  Returns the
 * SM count now in use, or PSL_EINVAL for a null ctx or max_sms < 0. */
PSL_API int psl_set_max_sms(psl_ctx *ctx, int32_t max_sms);

/* No counterpart in the paper.  For callers that must not allocate device memory
 * themselves -- code running under another framework's allocator, where a raw cudaFree
 * would synchronise the whole device, or services that reserve every buffer at start-up
 * so that no later request can block or fail on an allocation: the autocorrelation of
 * Eq. 2 for one sequence already in device memory, computed with a scratch area built
 * into the library (128 KiB per device, held until the process exits) instead of
 * allocating.  seq_dev: device array of L int8 values (negative means -1, anything else
 * +1); C_dev: device array of L int32 receiving C_0..C_{L-1}; stream: a cudaStream_t of
 * the current device (cudaGetDevice; the scratch used is that device's), or NULL.
 * Requires 1 <= L <= 2^20 - 1 (PSL_EINVAL otherwise, and for NULL pointers); PSL_ECUDA if
 * the scratch lookup or a launch fails, and, without launching anything, if a CUDA error is
 * already pending when the call starts (that error is left for its owner to read).  Calls
 * no allocator.  Work is queued
 * on the stream and the caller synchronises.  The first call on each device looks up the
 * scratch address, so make that first call before any stream capture.  Every call on a
 * device uses the same scratch, which keeps the previous call's contents (each call
 * rewrites all of it that it reads): calls that can overlap on the GPU, such as calls on
 * different streams with no ordering between them, race and give wrong results. */
PSL_API int psl_autocorr_static(const int8_t *seq_dev, uint32_t L, int32_t *C_dev, void *stream);

/* Test hook for the failure path (no counterpart in the paper): the walk's next
 * neighbourhood pass waits for staged copies that are never issued, with a short limit,
 * so its bounded waits run out; the walk then ends in PSL_ERROR with error PSL_ETIMEOUT
 * while every other walk and the context carry on.  Nothing faults and nothing is left in
 * flight.  PSL_ENOENT / PSL_EBUSY if the walk is unknown or not yet admitted. */
PSL_API int psl_inject_stall(psl_ctx *ctx, int64_t id);

/* Single-walk k-sharding over several ranks (one context per rank, typically one GPU each):
 * the parallel evaluation of Sec. 3 split over k, the sum of Eq. 4 being a sum over k.  A walk
 * submitted with shard_count = R > 1 (2 <= R <= min(16, ceil((L-1)/960)); the context must
 * hold no other walk) keeps its whole state on every rank, but each rank scores and
 * re-checks only the k-chunks c with c % R == shard_rank.  One step of Algorithm 1 is:
 *   n = psl_shard_score(ctx, id, parts, cap)      this rank's partial FP32 scores, [ksplit][N],
 *                                                  other ranks' chunks zero
 *   parts <- sum over ranks of parts              (exact: every entry has one non-zero term)
 *   m = psl_shard_select(ctx, id, parts, rc, cap)  selection on the full scores (identical on
 *                                                  every rank), then this rank's exact re-check
 *                                                  partials of the candidates, m uint32 words
 *                                                  (other ranks' chunks zero)
 *   rc <- sum over ranks of rc, word by word      (exact for the same reason: no carries)
 *   psl_shard_decide(ctx, id, rc, m)              the exact decision and the O(L) update, the
 *                                                  same on every rank; returns PSL_RUNNING or
 *                                                  PSL_DONE
 * The walk's trajectory equals that of the same walk run unsharded.  psl_step refuses a
 * context that holds a sharded walk (PSL_ESTATE).  psl_shard_layout gives the sizes: ksplit
 * (k-chunks), N (window) and the most re-check words a step can produce.  Errors:
 * PSL_ENOENT (unknown id), PSL_EINVAL (not sharded, cap too small), PSL_ESTATE (the walk is
 * done or failed), PSL_ETIMEOUT (a bounded device wait ran out; the walk failed). */
PSL_API int psl_shard_layout(psl_ctx *ctx, int64_t id, uint32_t *ksplit, uint32_t *N, uint32_t *rc_words_max);
PSL_API int psl_shard_score(psl_ctx *ctx, int64_t id, float *parts, size_t cap);
PSL_API int psl_shard_select(psl_ctx *ctx, int64_t id, const float *parts, uint32_t *rc_parts, size_t cap);
PSL_API int psl_shard_decide(psl_ctx *ctx, int64_t id, const uint32_t *rc_parts, size_t words);

/* Destroys the context and frees its device memory.  NULL is ignored. */
PSL_API void psl_shutdown(psl_ctx *ctx);

/* Message of the last error of this context (or of the last failed psl_init). */
PSL_API const char *psl_last_error(psl_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* PSL_H */
