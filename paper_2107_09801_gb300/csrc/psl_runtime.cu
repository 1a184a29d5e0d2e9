// psl_runtime.cu -- host runtime behind the C ABI of include/psl.h: device arena,
// walk slots, admission of queued walks by device memory, the batched and plain
// step loops (Algorithm 1 of arXiv 2107.09801) and state export.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "psl.h"
#include "psl_internal.h"

using namespace psl;

namespace {

thread_local std::string g_init_error;

enum ProfKind { kPHot = 0, kPSelect, kPRecheck, kPDecide, kPApply, kPHotPlain, kPInit, kPGraph, kPTail, kProfKinds };
const char *kProfNames[kProfKinds] = {"hot", "select", "recheck", "decide", "apply", "hot_plain", "init", "graph",
                                      "tail"};

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Layout {
  size_t bits, bits_local, bits_best, bits_fbest, win_f, win_r, C, C_local, T, score, score_part, pslj, ktau, cand,
      rc_part, ap_part, trace, total;
};

Layout layout_for(uint32_t L, uint32_t N, uint32_t trace_cap) {
  Layout o{};
  const size_t nw = (L + 31) / 32;
  const size_t words = nw + 2 * kGuardWords;
  const size_t nchunk_rc = (L + kRecheckChunk - 1) / kRecheckChunk;
  const size_t nchunk_ap = (L + kApplyChunk - 1) / kApplyChunk;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes, 256);
    return at;
  };
  o.bits = take(words * 4);
  o.bits_local = take(words * 4);
  o.bits_best = take(words * 4);
  o.bits_fbest = take(words * 4);
  o.win_f = take(((size_t)L + 2 * kWinGuard) * 4);
  o.win_r = take(((size_t)L + 2 * kWinGuard) * 4);
  o.C = take((size_t)L * 4);
  o.C_local = take((size_t)L * 4);
  o.T = take((size_t)L * 16);
  o.score = take((size_t)N * 4);
  o.score_part = take((size_t)kKsplitMax * N * 4);
  o.pslj = take((size_t)N * 4);
  o.ktau = take((size_t)L * 8);
  o.cand = take((size_t)N * 4);
  o.rc_part = take(((size_t)kQcap * nchunk_rc + N) * kWideLimbs * 4);
  o.ap_part = take(nchunk_ap * kApplyPartStride * 4);
  o.trace = take((size_t)trace_cap * sizeof(TraceRec));
  o.total = off;
  return o;
}

// First-fit allocator over the arena with coalescing free list.
struct Arena {
  size_t size = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  void reset(size_t n) {
    size = n;
    free_.clear();
    if (n) free_[0] = n;
  }
  bool alloc(size_t n, size_t *off) {
    n = align_up(n, 256);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n, at = it->first + n;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = align_up(n, 256);
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

struct HostWalk {
  int64_t id = -1;
  psl_walk_params p{};
  std::vector<int8_t> init_seq;
  int32_t state = PSL_QUEUED;
  int32_t error = 0;
  int32_t slot = -1;
  size_t off = 0, bytes = 0;
  Layout lay{};
  double t_submit = 0, t_start = 0, t_done = 0;
};

}  // namespace

struct psl_ctx {
  psl_config cfg{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  char *arena = nullptr;
  bool own_arena = false;
  Arena alloc;
  WalkDev *d_hdr = nullptr;
  std::vector<WalkDev> h_hdr;
  uint32_t *d_active = nullptr;
  uint32_t *d_list_aux = nullptr;  // slot lists of initialisation and plain-form launches
  Schedule *d_sched = nullptr;     // [0] batched steps, [1] initialisation, [2] plain form
  HotItem *d_items = nullptr;
  uint32_t items_cap = 0;
  uint32_t *h_pinned = nullptr;
  std::vector<int32_t> free_slots;
  std::map<int64_t, HostWalk> walks;
  std::deque<int64_t> queue;
  std::vector<uint32_t> active;  // running slots
  bool active_dirty = true;
  uint32_t nitems = 0, max_chunk_apply = 1, max_chunk_rc = 1;
  int64_t next_id = 0;
  uint32_t hot_flush_sb = 8;  // super-blocks per block sum of the neighbourhood kernel
  bool tail_fused = false;    // every running walk is short: select..apply run as one kernel
  bool alpha2 = false;        // every running walk has alpha1 = alpha2 = 2, L <= kA2MaxL: closed-form score
  uint32_t sm_count = 152;   // SMs the persistent kernels are sized for
  uint32_t dev_sms = 152;    // SMs of the device
  std::string err;
  // CUDA graph of steps_per_graph steps over the current active set
  cudaGraphExec_t graph = nullptr;
  uint32_t graph_steps = 0;
  int graph_prof = 0;  // profile mode the graph was captured with (its event nodes)
  // CUDA-event profile of kernel launches: 0 off, 1 every kernel, 2 the neighbourhood kernel only
  int prof = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
  std::vector<int> ev_kind;
  size_t ev_used = 0;
  // event pairs recorded by the nodes of the captured graph (read after each graph launch)
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> gev;
  std::vector<int> gev_kind;
  double prof_ms[kProfKinds] = {};
  uint64_t prof_n[kProfKinds] = {};
  // bytes the library copied between host and device memory since creation
  uint64_t h2d_bytes = 0, d2h_bytes = 0;
};

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e__ = (call);                                                             \
    if (e__ != cudaSuccess) return fail(ctx, PSL_ECUDA, "%s: %s", #call, cudaGetErrorString(e__)); \
  } while (0)

static int fail(psl_ctx *ctx, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx)
    ctx->err = buf;
  else
    g_init_error = buf;
  return code;
}

// Every host<->device copy of the library goes through here (on the context's stream), so
// that the bytes moved are counted, not estimated.
static cudaError_t xfer(psl_ctx *ctx, void *dst, const void *src, size_t bytes, cudaMemcpyKind kind) {
  if (kind == cudaMemcpyHostToDevice) ctx->h2d_bytes += bytes;
  if (kind == cudaMemcpyDeviceToHost) ctx->d2h_bytes += bytes;
  return cudaMemcpyAsync(dst, src, bytes, kind, ctx->stream);
}

extern "C" int psl_transfer_bytes(psl_ctx *ctx, uint64_t *h2d, uint64_t *d2h) {
  if (!ctx) return PSL_EINVAL;
  if (h2d) *h2d = ctx->h2d_bytes;
  if (d2h) *d2h = ctx->d2h_bytes;
  return PSL_OK;
}

// Whether launches of this kind are bracketed by events in the current profile mode.
static bool prof_wants(const psl_ctx *ctx, int kind) {
  return ctx->prof == 1 || (ctx->prof == 2 && (kind == kPHot || kind == kPHotPlain || kind == kPGraph));
}

// Records an event pair around one launch when profiling is on.
static cudaError_t prof_begin(psl_ctx *ctx, int kind) {
  if (!prof_wants(ctx, kind)) return cudaSuccess;
  if (ctx->ev_used == ctx->ev.size()) {
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e != cudaSuccess) return e;
    ctx->ev.push_back({a, b});
    ctx->ev_kind.push_back(kind);
  }
  ctx->ev_kind[ctx->ev_used] = kind;
  return cudaEventRecord(ctx->ev[ctx->ev_used].first, ctx->stream);
}

static cudaError_t prof_end(psl_ctx *ctx, int kind) {
  if (!prof_wants(ctx, kind)) return cudaSuccess;
  return cudaEventRecord(ctx->ev[ctx->ev_used++].second, ctx->stream);
}

// Event pairs for the graph's event-record nodes, created before the capture begins.
static cudaError_t gprof_reserve(psl_ctx *ctx, size_t pairs) {
  while (ctx->gev.size() < pairs) {
    cudaEvent_t a, b;
    cudaError_t e = cudaEventCreate(&a);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
      cudaEventDestroy(a);
      return e;
    }
    ctx->gev.push_back({a, b});
  }
  ctx->gev_kind.clear();
  return cudaSuccess;
}

// Inside a stream capture: an event pair recorded by graph nodes around one kernel
// (external records, so that each launch of the graph timestamps them).
static cudaError_t gprof_begin(psl_ctx *ctx, int kind) {
  if (!prof_wants(ctx, kind)) return cudaSuccess;
  const size_t q = ctx->gev_kind.size();
  if (q >= ctx->gev.size()) return cudaErrorInvalidValue;  // reserved too few (not reached)
  ctx->gev_kind.push_back(kind);
  return cudaEventRecordWithFlags(ctx->gev[q].first, ctx->stream, cudaEventRecordExternal);
}

static cudaError_t gprof_end(psl_ctx *ctx, int kind) {
  if (!prof_wants(ctx, kind)) return cudaSuccess;
  return cudaEventRecordWithFlags(ctx->gev[ctx->gev_kind.size() - 1].second, ctx->stream, cudaEventRecordExternal);
}

static void gprof_clear(psl_ctx *ctx) {
  for (auto &pr : ctx->gev) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  ctx->gev.clear();
  ctx->gev_kind.clear();
}

static void drop_graph(psl_ctx *ctx) {
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  ctx->graph = nullptr;
  gprof_clear(ctx);
}

// Folds the times of the last graph launch into the totals (the stream must be synchronised).
static void gprof_collect(psl_ctx *ctx) {
  for (size_t i = 0; i < ctx->gev_kind.size(); i++) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->gev[i].first, ctx->gev[i].second) == cudaSuccess) {
      ctx->prof_ms[ctx->gev_kind[i]] += ms;
      ctx->prof_n[ctx->gev_kind[i]] += 1;
    }
  }
}

// Folds the recorded pairs into the totals (the stream must be synchronised).
static void prof_collect(psl_ctx *ctx) {
  for (size_t i = 0; i < ctx->ev_used; i++) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->ev[i].first, ctx->ev[i].second) == cudaSuccess) {
      ctx->prof_ms[ctx->ev_kind[i]] += ms;
      ctx->prof_n[ctx->ev_kind[i]] += 1;
    }
  }
  ctx->ev_used = 0;
}

extern "C" int psl_profile(psl_ctx *ctx, int enable) {
  if (!ctx || enable < 0 || enable > 2) return PSL_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream));
  prof_collect(ctx);
  ctx->prof = enable;
  if (ctx->prof)
    for (int k = 0; k < kProfKinds; k++) ctx->prof_ms[k] = 0.0, ctx->prof_n[k] = 0;
  return PSL_OK;
}

extern "C" int psl_profile_read(psl_ctx *ctx, psl_kernel_time *out, size_t cap) {
  if (!ctx || (!out && cap)) return PSL_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream));
  prof_collect(ctx);
  for (size_t k = 0; k < cap && k < (size_t)kProfKinds; k++) {
    std::memset(&out[k], 0, sizeof out[k]);
    std::snprintf(out[k].name, sizeof out[k].name, "%s", kProfNames[k]);
    out[k].launches = ctx->prof_n[k];
    out[k].total_ms = ctx->prof_ms[k];
  }
  return kProfKinds;
}

extern "C" void psl_config_default(psl_config *cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof *cfg);
  cfg->n_lmt = 6912;
  cfg->ls_lmt = 2000;
  cfg->flip_lmt = 10;
  cfg->device = 0;
  cfg->form = PSL_FORM_BATCHED;
  cfg->max_walks = 4096;
  cfg->hot_tile_sb = 0;
  cfg->steps_per_graph = 0;
  cfg->hot_threads = 0;
}

extern "C" uint64_t psl_walk_bytes(uint32_t L, int32_t n_lmt, uint32_t trace_cap) {
  if (L < 2) return 0;
  const uint32_t N = (n_lmt <= 0) ? L : std::min<uint32_t>((uint32_t)n_lmt, L);
  return layout_for(L, N, trace_cap).total;
}

extern "C" const char *psl_last_error(psl_ctx *ctx) { return ctx ? ctx->err.c_str() : g_init_error.c_str(); }

extern "C" int psl_init(const psl_config *cfg_in, psl_ctx **out) {
  if (!out) return fail(nullptr, PSL_EINVAL, "out is NULL");
  *out = nullptr;
  psl_config cfg;
  if (cfg_in)
    cfg = *cfg_in;
  else
    psl_config_default(&cfg);
  if (cfg.n_lmt < 1 || cfg.ls_lmt < 0 || cfg.flip_lmt < 0 || cfg.flip_lmt > kMaxFlips || cfg.max_walks < 1 ||
      (cfg.form != PSL_FORM_BATCHED && cfg.form != PSL_FORM_PLAIN) || cfg.steps_per_graph < 0 || cfg.max_sms < 0 ||
      !hot_config_supported(cfg.hot_threads ? (uint32_t)cfg.hot_threads : 256u,
                            cfg.hot_tile_sb ? (uint32_t)cfg.hot_tile_sb : 32u))
    return fail(nullptr, PSL_EINVAL, "invalid psl_config field");
  if (cfg.arena && cfg.arena_bytes == 0) return fail(nullptr, PSL_EINVAL, "arena given without arena_bytes");
  psl_ctx *ctx = new psl_ctx();
  ctx->cfg = cfg;
  if (ctx->cfg.hot_tile_sb == 0) ctx->cfg.hot_tile_sb = 32;
  if (ctx->cfg.hot_threads == 0) ctx->cfg.hot_threads = 256;
  auto bail = [&](int code) {
    psl_shutdown(ctx);
    return code;
  };
  cudaError_t e = cudaSetDevice(cfg.device);
  if (e != cudaSuccess) {
    fail(nullptr, PSL_ECUDA, "cudaSetDevice(%d): %s", cfg.device, cudaGetErrorString(e));
    delete ctx;
    return PSL_ECUDA;
  }
  if (cfg.stream) {
    ctx->stream = (cudaStream_t)cfg.stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      fail(nullptr, PSL_ECUDA, "cudaStreamCreate failed");
      delete ctx;
      return PSL_ECUDA;
    }
    ctx->own_stream = true;
  }
  size_t bytes = cfg.arena_bytes;
  if (cfg.arena) {
    ctx->arena = (char *)cfg.arena;
  } else {
    if (bytes == 0) {
      size_t fr = 0, tot = 0;
      if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        fail(nullptr, PSL_ECUDA, "cudaMemGetInfo failed");
        return bail(PSL_ECUDA);
      }
      bytes = std::min<size_t>(fr / 2, (size_t)64 << 30);
    }
    if (cudaMalloc(&ctx->arena, bytes) != cudaSuccess) {
      cudaGetLastError();
      fail(nullptr, PSL_ENOMEM, "cudaMalloc(arena %zu bytes) failed", bytes);
      return bail(PSL_ENOMEM);
    }
    ctx->own_arena = true;
  }
  {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, cfg.device) == cudaSuccess && sms > 0)
      ctx->sm_count = ctx->dev_sms = (uint32_t)sms;
    if (cfg.max_sms > 0) ctx->sm_count = std::min<uint32_t>(ctx->sm_count, (uint32_t)cfg.max_sms);
  }
  if (prepare_kernels() != cudaSuccess) {
    cudaGetLastError();
    fail(nullptr, PSL_ECUDA, "kernel attribute setup failed");
    return bail(PSL_ECUDA);
  }
  ctx->alloc.reset(bytes);
  ctx->h_hdr.assign(cfg.max_walks, WalkDev{});
  if (cudaMalloc(&ctx->d_hdr, sizeof(WalkDev) * cfg.max_walks) != cudaSuccess ||
      cudaMalloc(&ctx->d_active, sizeof(uint32_t) * cfg.max_walks) != cudaSuccess ||
      cudaMalloc(&ctx->d_list_aux, sizeof(uint32_t) * cfg.max_walks) != cudaSuccess ||
      cudaMalloc(&ctx->d_sched, sizeof(Schedule) * 3) != cudaSuccess ||
      cudaMallocHost(&ctx->h_pinned, sizeof(uint32_t) * cfg.max_walks) != cudaSuccess) {
    cudaGetLastError();
    fail(nullptr, PSL_ENOMEM, "slot table allocation failed");
    return bail(PSL_ENOMEM);
  }
  cudaMemset(ctx->d_hdr, 0, sizeof(WalkDev) * cfg.max_walks);
  cudaMemset(ctx->d_sched, 0, sizeof(Schedule) * 3);
  for (int s = cfg.max_walks - 1; s >= 0; s--) ctx->free_slots.push_back(s);
  *out = ctx;
  return PSL_OK;
}

extern "C" void psl_shutdown(psl_ctx *ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  drop_graph(ctx);
  for (auto &pr : ctx->ev) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  if (ctx->own_arena && ctx->arena) cudaFree(ctx->arena);
  if (ctx->d_hdr) cudaFree(ctx->d_hdr);
  if (ctx->d_active) cudaFree(ctx->d_active);
  if (ctx->d_list_aux) cudaFree(ctx->d_list_aux);
  if (ctx->d_sched) cudaFree(ctx->d_sched);
  if (ctx->d_items) cudaFree(ctx->d_items);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

static int check_params(psl_ctx *ctx, psl_walk_params &p) {
  if (p.L < 2 || p.L > (1u << 20) - 1u) return fail(ctx, PSL_EINVAL, "L=%u outside 2..2^20-1", p.L);
  if (p.alpha1 < 1 || p.alpha1 > 16 || p.alpha2 < 1 || p.alpha2 > 16)
    return fail(ctx, PSL_EINVAL, "alpha must be an integer in 1..16");
  if (p.budget < 1) return fail(ctx, PSL_EINVAL, "budget must be >= 1");
  if (p.n_lmt <= 0) p.n_lmt = ctx->cfg.n_lmt;
  if (p.ls_lmt < 0) p.ls_lmt = ctx->cfg.ls_lmt;  // 0 is a valid LS_lmt
  if (p.flip_lmt <= 0) p.flip_lmt = ctx->cfg.flip_lmt;
  if (p.flip_lmt > kMaxFlips) return fail(ctx, PSL_EINVAL, "flip_lmt > %d", kMaxFlips);
  if (p.topk <= 0) p.topk = 1;
  if (p.topk > 16) return fail(ctx, PSL_EINVAL, "topk > 16");
  if (p.shard_count > 1) {
    const uint32_t unitK = kKchunkSbUnit * kSbK;
    const uint32_t max_split = std::max<uint32_t>(1u, (p.L - 1 + unitK - 1) / unitK);
    if (p.shard_rank >= p.shard_count || p.shard_count > std::min<uint32_t>(kKsplitMax, max_split))
      return fail(ctx, PSL_EINVAL, "shard_rank %u / shard_count %u: need rank < count <= min(16, ceil((L-1)/960))",
                  p.shard_rank, p.shard_count);
    if (ctx->cfg.form != PSL_FORM_BATCHED) return fail(ctx, PSL_EINVAL, "a sharded walk needs the batched form");
    if (!ctx->walks.empty()) return fail(ctx, PSL_EINVAL, "a sharded walk needs a context of its own");
  } else if (!ctx->walks.empty() && ctx->walks.begin()->second.p.shard_count > 1) {
    return fail(ctx, PSL_EINVAL, "the context holds a sharded walk");
  }
  return PSL_OK;
}

extern "C" int64_t psl_submit_ex(psl_ctx *ctx, const psl_walk_params *pin) {
  if (!ctx || !pin) return PSL_EINVAL;
  psl_walk_params p = *pin;
  int rc = check_params(ctx, p);
  if (rc) return rc;
  HostWalk w;
  w.id = ctx->next_id++;
  w.p = p;
  if (p.init_seq) {
    w.init_seq.assign(p.init_seq, p.init_seq + p.L);
    for (int8_t v : w.init_seq)
      if (v != 1 && v != -1) return fail(ctx, PSL_EINVAL, "init_seq values must be +1 or -1");
  }
  w.p.init_seq = nullptr;
  const uint32_t N = std::min<uint32_t>((uint32_t)p.n_lmt, p.L);
  w.lay = layout_for(p.L, N, p.trace_cap);
  w.bytes = w.lay.total;
  if (w.bytes > ctx->alloc.size) return fail(ctx, PSL_ENOMEM, "walk needs %zu bytes, arena holds %zu", w.bytes,
                                             ctx->alloc.size);
  w.t_submit = now_s();
  const int64_t id = w.id;
  ctx->walks.emplace(id, std::move(w));
  ctx->queue.push_back(id);
  return id;
}

extern "C" int64_t psl_submit(psl_ctx *ctx, uint32_t L, uint64_t seed, double alpha1, double alpha2,
                              uint64_t budget) {
  if (!ctx) return PSL_EINVAL;
  if (alpha1 != std::floor(alpha1) || alpha2 != std::floor(alpha2))
    return fail(ctx, PSL_EINVAL, "alpha must be an integer");
  psl_walk_params p{};
  p.L = L;
  p.seed = seed;
  p.alpha1 = (int32_t)std::max(-1.0, std::min(alpha1, 1e6));
  p.alpha2 = (int32_t)std::max(-1.0, std::min(alpha2, 1e6));
  p.budget = budget;
  p.ls_lmt = -1;
  return psl_submit_ex(ctx, &p);
}

// ---------------------------------------------------------------------------------
// admission and launch plumbing
// ---------------------------------------------------------------------------------
static void fill_header(psl_ctx *ctx, HostWalk &w, WalkDev &h) {
  std::memset(&h, 0, sizeof h);
  const psl_walk_params &p = w.p;
  char *base = ctx->arena + w.off;
  h.L = p.L;
  h.N = std::min<uint32_t>((uint32_t)p.n_lmt, p.L);
  h.nw = (p.L + 31) / 32;
  h.nflip = std::min<uint32_t>((uint32_t)p.flip_lmt, p.L);
  h.alpha1 = (uint32_t)p.alpha1;
  h.alpha2 = (uint32_t)p.alpha2;
  h.ls_lmt = (uint32_t)p.ls_lmt;
  h.topk = (uint32_t)p.topk;
  h.seed = p.seed;
  h.budget = p.budget;
  h.nchunk_apply = (p.L + kApplyChunk - 1) / kApplyChunk;
  h.nchunk_rc = (p.L + kRecheckChunk - 1) / kRecheckChunk;
  h.trace_cap = p.trace_cap;
  h.has_init_seq = w.init_seq.empty() ? 0u : 1u;
  h.bits = (uint32_t *)(base + w.lay.bits) + kGuardWords;
  h.bits_local = (uint32_t *)(base + w.lay.bits_local) + kGuardWords;
  h.bits_best = (uint32_t *)(base + w.lay.bits_best) + kGuardWords;
  h.bits_fbest = (uint32_t *)(base + w.lay.bits_fbest) + kGuardWords;
  h.track_fbest = p.alpha1 == p.alpha2 ? 1u : 0u;
  h.win_f = (uint32_t *)(base + w.lay.win_f) + kWinGuard;
  h.win_r = (uint32_t *)(base + w.lay.win_r) + kWinGuard;
  h.C = (int32_t *)(base + w.lay.C);
  h.C_local = (int32_t *)(base + w.lay.C_local);
  h.T = (float4 *)(base + w.lay.T);
  h.score = (float *)(base + w.lay.score);
  h.score_part = (float *)(base + w.lay.score_part);
  h.ksplit = 1;
  h.kchunk_sb = kKchunkSbUnit;
  h.kc_psl = 0;
  h.shard_rank = p.shard_count > 1 ? p.shard_rank : 0u;
  h.shard_count = p.shard_count > 1 ? p.shard_count : 1u;
  h.pslj = (int32_t *)(base + w.lay.pslj);
  h.ktau = (int2 *)(base + w.lay.ktau);
  h.cand = (uint32_t *)(base + w.lay.cand);
  h.rc_part = (uint32_t *)(base + w.lay.rc_part);
  h.ap_part = (uint32_t *)(base + w.lay.ap_part);
  h.trace = p.trace_cap ? (TraceRec *)(base + w.lay.trace) : nullptr;
  h.status = kRunning;
  h.alpha = h.alpha1;
  h.alpha_next = h.alpha1;
  h.rng_ctr = (p.L + 63) / 64;
}

static int rebuild_active(psl_ctx *ctx) {
  ctx->active.clear();
  for (auto &kv : ctx->walks)
    if (kv.second.state == PSL_RUNNING) ctx->active.push_back((uint32_t)kv.second.slot);
  // long walks first: their blocks are the longest-running units
  std::sort(ctx->active.begin(), ctx->active.end(),
            [&](uint32_t a, uint32_t b) { return ctx->h_hdr[a].L > ctx->h_hdr[b].L; });
  std::vector<HotItem> items;
  ctx->max_chunk_apply = 1;
  ctx->max_chunk_rc = 1;
  // short walks run their few super-blocks with shorter block sums (less unrolled code)
  uint32_t maxL = 0;
  for (uint32_t s : ctx->active) maxL = std::max(maxL, ctx->h_hdr[s].L);
  const uint32_t fb = hot_flush_for(maxL);
  if (fb != ctx->hot_flush_sb) {
    ctx->hot_flush_sb = fb;
    drop_graph(ctx);  // captured with the other kernel variant
  }
  bool short_only = !ctx->active.empty();
  for (uint32_t s : ctx->active)
    short_only = short_only && ctx->h_hdr[s].L <= kTailMaxL && ctx->h_hdr[s].N <= kTailMaxN &&
                 ctx->h_hdr[s].shard_count <= 1;
  if (short_only != ctx->tail_fused) {
    ctx->tail_fused = short_only;
    drop_graph(ctx);  // captured with the other kernel sequence
  }
  // alpha = 2 batches of short walks take the closed-form score (unless the configuration
  // asks for the tables); it scores every neighbour whole, so their k range is never split
  bool a2 = !ctx->active.empty() && ctx->cfg.alpha2_tables == 0 && ctx->cfg.form == PSL_FORM_BATCHED;
  for (uint32_t s : ctx->active) {
    const WalkDev &h = ctx->h_hdr[s];
    a2 = a2 && h.alpha1 == 2 && h.alpha2 == 2 && h.L <= kA2MaxL && h.shard_count <= 1;
  }
  if (a2 != ctx->alpha2) {
    ctx->alpha2 = a2;
    drop_graph(ctx);  // captured with the other kernel
  }
  // Split every walk's k range into chunks when the neighbour blocks alone would leave
  // SMs idle (few walks, or a long walk on its own): aim for about four blocks per SM.
  const uint32_t T_ = (uint32_t)ctx->cfg.hot_threads * (a2 ? kA2PerThread : 1u);  // window positions per item
  uint64_t nblocks = 0;
  for (uint32_t s : ctx->active) nblocks += (ctx->h_hdr[s].N + T_ - 1) / T_;
  const uint64_t target = 4ull * (uint64_t)ctx->sm_count;
  uint32_t want = nblocks == 0 ? 1u : (uint32_t)std::min<uint64_t>(kKsplitMax, (target + nblocks - 1) / nblocks);
  if (ctx->cfg.form == PSL_FORM_PLAIN || a2) want = 1;  // these kernels score each neighbour whole
  for (uint32_t s : ctx->active) {
    WalkDev &h = ctx->h_hdr[s];
    const uint32_t unitK = kKchunkSbUnit * kSbK;
    const uint32_t max_split = std::max<uint32_t>(1u, (h.L - 1 + unitK - 1) / unitK);
    uint32_t ks = std::min(want, max_split);
    const uint32_t R = h.shard_count;
    if (R > 1)  // a sharded walk: the same chunks on every rank whatever its SM count, the same number per rank
      ks = std::min<uint32_t>(kKsplitMax, max_split) / R * R;
    const uint32_t units = ((h.L - 1 + unitK - 1) / unitK + ks - 1) / ks;  // chunk size in 960-k units
    h.ksplit = ks;
    h.kchunk_sb = units * kKchunkSbUnit;
    h.kc_psl = R > 1 ? h.shard_rank : 0u;  // the rank's first chunk also computes the neighbours' PSL
    static_assert(offsetof(WalkDev, kc_psl) == offsetof(WalkDev, ksplit) + 8, "ksplit, kchunk_sb, kc_psl adjacent");
    CK(xfer(ctx, (char *)(ctx->d_hdr + s) + offsetof(WalkDev, ksplit), &h.ksplit, 16, cudaMemcpyHostToDevice));
    for (uint32_t i0 = 1; i0 <= h.N; i0 += T_)
      for (uint32_t c = 0; c < ks; c++)
        if (R <= 1 || c % R == h.shard_rank) items.push_back(HotItem{s, i0, c, 0});
    ctx->max_chunk_apply = std::max(ctx->max_chunk_apply, h.nchunk_apply);
    ctx->max_chunk_rc = std::max(ctx->max_chunk_rc, h.nchunk_rc);
  }
  if (items.size() > ctx->items_cap) {
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->d_items) cudaFree(ctx->d_items);
    ctx->items_cap = (uint32_t)std::max<size_t>(2 * items.size(), 4096);
    CK(cudaMalloc(&ctx->d_items, sizeof(HotItem) * ctx->items_cap));
    drop_graph(ctx);  // the captured steps point at the old buffer
  }
  ctx->nitems = (uint32_t)items.size();
  if (!items.empty())
    CK(xfer(ctx, ctx->d_items, items.data(), sizeof(HotItem) * items.size(), cudaMemcpyHostToDevice));
  if (!ctx->active.empty()) {
    std::copy(ctx->active.begin(), ctx->active.end(), ctx->h_pinned);
    CK(xfer(ctx, ctx->d_active, ctx->h_pinned, sizeof(uint32_t) * ctx->active.size(), cudaMemcpyHostToDevice));
  }
  Schedule sc{};
  sc.nactive = (uint32_t)ctx->active.size();
  sc.nitems = ctx->nitems;
  sc.max_chunk_apply = ctx->max_chunk_apply;
  sc.max_chunk_rc = ctx->max_chunk_rc;
  sc.hot_next = 0;
  sc.general = 1;
  sc.alpha2 = ctx->alpha2 ? 1u : 0u;
  CK(xfer(ctx, ctx->d_sched, &sc, sizeof sc, cudaMemcpyHostToDevice));
  CK(cudaStreamSynchronize(ctx->stream));  // h_pinned and sc are reused / temporaries
  ctx->active_dirty = false;
  return PSL_OK;
}

static LaunchCtx launch_ctx(psl_ctx *ctx, const uint32_t *d_list, Schedule *d_sched) {
  LaunchCtx c{};
  c.hdr = ctx->d_hdr;
  c.active = d_list;
  c.sched = d_sched;
  c.items = ctx->d_items;
  c.hot_threads = (uint32_t)ctx->cfg.hot_threads;
  c.hot_tile_sb = (uint32_t)ctx->cfg.hot_tile_sb;
  c.hot_flush_sb = ctx->hot_flush_sb;
  c.alpha2 = ctx->alpha2 ? 1u : 0u;
  c.sm_count = ctx->sm_count;
  c.stream = ctx->stream;
  return c;
}

static int upload_schedule(psl_ctx *ctx, Schedule *d, uint32_t nactive, uint32_t apply_chunks, uint32_t rc_chunks) {
  Schedule sc{};
  sc.nactive = nactive;
  sc.max_chunk_apply = apply_chunks;
  sc.max_chunk_rc = rc_chunks;
  sc.general = 1;  // initialisation and the plain form run the general update pass every time
  CK(xfer(ctx, d, &sc, sizeof sc, cudaMemcpyHostToDevice));
  CK(cudaStreamSynchronize(ctx->stream));
  return PSL_OK;
}

static void pack_pm1(const int8_t *s, uint32_t L, std::vector<uint32_t> &words) {
  words.assign((L + 31) / 32, 0u);
  for (uint32_t i = 0; i < L; i++)
    if (s[i] < 0) words[i >> 5] |= 1u << (i & 31);
}

// Admits queued walks (FIFO, skipping those that do not fit yet) and initialises them.
static int admit(psl_ctx *ctx) {
  std::vector<uint32_t> fresh;
  uint32_t maxL = 0, maxchunk = 1;
  for (auto it = ctx->queue.begin(); it != ctx->queue.end();) {
    HostWalk &w = ctx->walks.at(*it);
    if (ctx->free_slots.empty()) break;
    size_t off;
    if (!ctx->alloc.alloc(w.bytes, &off)) {
      ++it;
      continue;
    }
    w.off = off;
    w.slot = ctx->free_slots.back();
    ctx->free_slots.pop_back();
    w.state = PSL_RUNNING;
    w.t_start = now_s();
    WalkDev &h = ctx->h_hdr[w.slot];
    fill_header(ctx, w, h);
    CK(xfer(ctx, ctx->d_hdr + w.slot, &h, sizeof(WalkDev), cudaMemcpyHostToDevice));
    if (!w.init_seq.empty()) {
      std::vector<uint32_t> words;
      pack_pm1(w.init_seq.data(), w.p.L, words);
      CK(xfer(ctx, h.bits, words.data(), words.size() * 4, cudaMemcpyHostToDevice));
      CK(cudaStreamSynchronize(ctx->stream));  // words is a temporary
    }
    fresh.push_back((uint32_t)w.slot);
    maxL = std::max(maxL, w.p.L);
    maxchunk = std::max(maxchunk, h.nchunk_apply);
    it = ctx->queue.erase(it);
  }
  if (fresh.empty()) return PSL_OK;
  CK(xfer(ctx, ctx->d_list_aux, fresh.data(), sizeof(uint32_t) * fresh.size(), cudaMemcpyHostToDevice));
  int rc = upload_schedule(ctx, ctx->d_sched + 1, (uint32_t)fresh.size(), maxchunk, 1);
  if (rc) return rc;
  LaunchCtx c = launch_ctx(ctx, ctx->d_list_aux, ctx->d_sched + 1);
  c.maxL = maxL;
  c.ninit = (uint32_t)fresh.size();
  cudaError_t e = prof_begin(ctx, kPInit);
  if (e == cudaSuccess) e = launch_init_bits(c);
  if (e == cudaSuccess) e = launch_autocorr(c);
  if (e == cudaSuccess) e = launch_start_init(c);
  if (e == cudaSuccess) e = launch_apply(c);
  if (e == cudaSuccess) e = prof_end(ctx, kPInit);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) prof_collect(ctx);
  if (e != cudaSuccess) return fail(ctx, PSL_ECUDA, "walk initialisation: %s", cudaGetErrorString(e));
  ctx->active_dirty = true;
  return PSL_OK;
}

static int refresh_headers(psl_ctx *ctx) {
  // copy back the slot headers (one contiguous copy up to the highest running slot)
  uint32_t top = 0;
  for (uint32_t s : ctx->active) top = std::max(top, s + 1);
  std::vector<WalkDev> tmp(top);
  if (top) {
    CK(xfer(ctx, tmp.data(), ctx->d_hdr, sizeof(WalkDev) * top, cudaMemcpyDeviceToHost));
    CK(cudaStreamSynchronize(ctx->stream));
    for (uint32_t s : ctx->active) ctx->h_hdr[s] = tmp[s];
  }
  prof_collect(ctx);
  const double t = now_s();
  for (auto &kv : ctx->walks) {
    HostWalk &w = kv.second;
    if (w.state != PSL_RUNNING) continue;
    const WalkDev &h = ctx->h_hdr[w.slot];
    if (h.status == kDone) {
      w.state = PSL_DONE;
      w.t_done = t;
      ctx->active_dirty = true;
    } else if (h.status == kError) {
      w.state = PSL_ERROR;
      w.error = (int32_t)h.error;
      w.t_done = t;
      ctx->active_dirty = true;
    }
  }
  return PSL_OK;
}

// One step of the batched form.  Outside a capture each kernel may be bracketed by events
// on the stream; inside a capture (captured = true) by event-record nodes of the graph.
static cudaError_t enqueue_batched_step(psl_ctx *ctx, const LaunchCtx &c, bool captured) {
  cudaError_t (*fns[5])(const LaunchCtx &) = {launch_hot, launch_select, launch_recheck, launch_decide, launch_apply};
  int kinds[5] = {kPHot, kPSelect, kPRecheck, kPDecide, kPApply};
  int n = 5;
  if (ctx->tail_fused) {  // short walks only: selection, re-check, decision and update in one kernel
    fns[1] = launch_step_tail;
    kinds[1] = kPTail;
    n = 2;
  }
  for (int q = 0; q < n; q++) {
    cudaError_t e = captured ? gprof_begin(ctx, kinds[q]) : prof_begin(ctx, kinds[q]);
    if (e == cudaSuccess) e = fns[q](c);
    if (e == cudaSuccess) e = captured ? gprof_end(ctx, kinds[q]) : prof_end(ctx, kinds[q]);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Captures steps_per_graph steps over the context's device schedule into one CUDA graph,
// with event-record nodes around the kernels that the current profile mode times.
static int capture_graph(psl_ctx *ctx) {
  drop_graph(ctx);
  const uint32_t G = (uint32_t)ctx->cfg.steps_per_graph;
  LaunchCtx c = launch_ctx(ctx, ctx->d_active, ctx->d_sched);
  if (ctx->prof) CK(gprof_reserve(ctx, (size_t)G * 5));  // at most five profiled phases a step
  cudaGraph_t g;
  CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (uint32_t t = 0; t < G && e == cudaSuccess; t++) e = enqueue_batched_step(ctx, c, true);
  cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    gprof_clear(ctx);
    return fail(ctx, PSL_ECUDA, "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&ctx->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    ctx->graph = nullptr;
    gprof_clear(ctx);
    return fail(ctx, PSL_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  ctx->graph_steps = G;
  ctx->graph_prof = ctx->prof;
  return PSL_OK;
}

static int run_batched(psl_ctx *ctx, uint32_t steps) {
  if (ctx->active.empty() || steps == 0) return PSL_OK;
  LaunchCtx c = launch_ctx(ctx, ctx->d_active, ctx->d_sched);
  const uint32_t G = (uint32_t)ctx->cfg.steps_per_graph;
  uint32_t done = 0;
  if (G > 0 && steps >= G) {
    if (!ctx->graph || ctx->graph_steps != G || ctx->graph_prof != ctx->prof) {
      int rc = capture_graph(ctx);
      if (rc) return rc;
    }
    while (steps - done >= G) {
      CK(prof_begin(ctx, kPGraph));
      CK(cudaGraphLaunch(ctx->graph, ctx->stream));
      CK(prof_end(ctx, kPGraph));
      if (!ctx->gev_kind.empty()) {  // the next launch re-records the graph's events: read them now
        CK(cudaStreamSynchronize(ctx->stream));
        gprof_collect(ctx);
      }
      done += G;
    }
  }
  for (; done < steps; done++) {
    cudaError_t e = enqueue_batched_step(ctx, c, false);
    if (e != cudaSuccess) return fail(ctx, PSL_ECUDA, "step launch: %s", cudaGetErrorString(e));
  }
  return PSL_OK;
}

extern "C" int psl_set_steps_per_graph(psl_ctx *ctx, int32_t steps) {
  if (!ctx || steps < 0 || ctx->cfg.form != PSL_FORM_BATCHED) return PSL_EINVAL;
  CK(cudaSetDevice(ctx->cfg.device));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->cfg.steps_per_graph = steps;
  drop_graph(ctx);
  if (steps == 0) return PSL_OK;
  int rc = admit(ctx);
  if (rc) return rc;
  if (ctx->active_dirty && (rc = rebuild_active(ctx))) return rc;
  if (ctx->active.empty()) return PSL_OK;  // captured at the first step that runs walks
  return capture_graph(ctx);
}

// Host-side selection of the plain form: the same rule as k_select.
static void host_select(const WalkDev &h, const std::vector<float> &score, const std::vector<int32_t> &pslj,
                        std::vector<uint32_t> &cand, float *m_out, double *B_out, int32_t *win_psl,
                        uint32_t *win_i) {
  const uint32_t N = h.N;
  float m = 3.4028234663852886e38f;
  for (uint32_t i = 0; i < N; i++) m = std::min(m, score[i]);
  const double B = score_bound(h.S_abs, h.alpha, h.L, 1u);
  const double td = (double)m + 2.0 * B;
  float thr = (float)td;
  if ((double)thr < td) thr = std::nextafter(thr, 3.4e38f);  // round up
  cand.clear();
  for (uint32_t i = 0; i < N; i++)
    if (score[i] <= thr) cand.push_back(i + 1);
  const uint32_t topk = std::min<uint32_t>(h.topk, 16u);
  if (cand.size() < topk) {
    std::vector<std::pair<float, uint32_t>> rest;
    for (uint32_t i = 0; i < N; i++)
      if (!(score[i] <= thr)) rest.push_back({score[i], i + 1});
    std::sort(rest.begin(), rest.end());
    for (size_t r = 0; r < rest.size() && cand.size() < topk; r++) cand.push_back(rest[r].second);
    std::sort(cand.begin(), cand.end());
  }
  *m_out = m;
  *B_out = B;
  *win_psl = INT32_MAX;
  *win_i = 0;
  if (h.ktau_on) {
    for (uint32_t i = 0; i < N; i++)
      if (pslj[i] < *win_psl) {
        *win_psl = pslj[i];
        *win_i = i + 1;
      }
  }
}

static int run_plain(psl_ctx *ctx, uint32_t steps) {
  std::vector<float> score;
  std::vector<int32_t> pslj;
  std::vector<uint32_t> cand;
  for (uint32_t s : ctx->active) {
    WalkDev *dh = ctx->d_hdr + s;
    uint32_t list_host = s;
    CK(xfer(ctx, ctx->d_list_aux, &list_host, sizeof(uint32_t), cudaMemcpyHostToDevice));
    int rc = upload_schedule(ctx, ctx->d_sched + 2, 1, ctx->h_hdr[s].nchunk_apply, ctx->h_hdr[s].nchunk_rc);
    if (rc) return rc;
    LaunchCtx c = launch_ctx(ctx, ctx->d_list_aux, ctx->d_sched + 2);
    for (uint32_t t = 0; t < steps; t++) {
      WalkDev h;
      CK(xfer(ctx, &h, dh, sizeof h, cudaMemcpyDeviceToHost));
      CK(cudaStreamSynchronize(ctx->stream));
      if (h.status != kRunning) break;
      CK(prof_begin(ctx, kPHotPlain));
      cudaError_t e = launch_hot_plain(dh, h.N, ctx->stream);
      if (e != cudaSuccess) return fail(ctx, PSL_ECUDA, "plain kernel: %s", cudaGetErrorString(e));
      CK(prof_end(ctx, kPHotPlain));
      score.resize(h.N);
      pslj.resize(h.N);
      uint32_t status_after = kRunning;
      CK(xfer(ctx, score.data(), h.score, 4 * h.N, cudaMemcpyDeviceToHost));
      CK(xfer(ctx, pslj.data(), h.pslj, 4 * h.N, cudaMemcpyDeviceToHost));
      CK(xfer(ctx, &status_after, (char *)dh + offsetof(WalkDev, status), 4, cudaMemcpyDeviceToHost));
      CK(cudaStreamSynchronize(ctx->stream));
      if (status_after != kRunning) break;  // a bounded wait of the kernel ran out: the walk failed
      float m;
      double B;
      int32_t wp;
      uint32_t wi;
      host_select(h, score, pslj, cand, &m, &B, &wp, &wi);
      const uint32_t n = (uint32_t)cand.size();
      const float bf = (float)B;
      CK(xfer(ctx, h.cand, cand.data(), 4 * n, cudaMemcpyHostToDevice));
      CK(xfer(ctx, (char *)dh + offsetof(WalkDev, ncand), &n, 4, cudaMemcpyHostToDevice));
      CK(xfer(ctx, (char *)dh + offsetof(WalkDev, score_min), &m, 4, cudaMemcpyHostToDevice));
      CK(xfer(ctx, (char *)dh + offsetof(WalkDev, bound), &bf, 4, cudaMemcpyHostToDevice));
      CK(xfer(ctx, (char *)dh + offsetof(WalkDev, win_psl), &wp, 4, cudaMemcpyHostToDevice));
      CK(xfer(ctx, (char *)dh + offsetof(WalkDev, win_psl_i), &wi, 4, cudaMemcpyHostToDevice));
      CK(prof_begin(ctx, kPRecheck));
      e = launch_recheck(c);
      if (e == cudaSuccess) e = prof_end(ctx, kPRecheck);
      if (e == cudaSuccess) e = prof_begin(ctx, kPDecide);
      if (e == cudaSuccess) e = launch_decide(c);
      if (e == cudaSuccess) e = prof_end(ctx, kPDecide);
      if (e == cudaSuccess) e = prof_begin(ctx, kPApply);
      if (e == cudaSuccess) e = launch_apply(c);
      if (e == cudaSuccess) e = prof_end(ctx, kPApply);
      if (e != cudaSuccess) return fail(ctx, PSL_ECUDA, "plain step: %s", cudaGetErrorString(e));
      CK(cudaStreamSynchronize(ctx->stream));  // host buffers above are reused next step
      prof_collect(ctx);
    }
  }
  return PSL_OK;
}

// NVTX range for the duration of a scope (visible in Nsight timelines)
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

static bool holds_sharded_walk(const psl_ctx *ctx) {
  return !ctx->walks.empty() && ctx->walks.begin()->second.p.shard_count > 1;
}

extern "C" int psl_step(psl_ctx *ctx, uint32_t max_moves) {
  if (!ctx) return PSL_EINVAL;
  if (holds_sharded_walk(ctx))
    return fail(ctx, PSL_ESTATE, "a sharded walk steps through psl_shard_score / _select / _decide");
  NvtxRange r_step("psl_step");
  CK(cudaSetDevice(ctx->cfg.device));
  int rc;
  {
    NvtxRange r("psl_step/admit");
    rc = admit(ctx);
    if (rc) return rc;
    if (ctx->active_dirty) {
      rc = rebuild_active(ctx);
      if (rc) return rc;
    }
  }
  // never run past the largest remaining budget
  uint64_t remaining = 0;
  for (uint32_t s : ctx->active) {
    const WalkDev &h = ctx->h_hdr[s];
    uint64_t done = h.moves;
    remaining = std::max<uint64_t>(remaining, h.budget > done ? h.budget - done : 0);
  }
  const uint32_t steps = (uint32_t)std::min<uint64_t>(max_moves, remaining);
  {
    NvtxRange r("psl_step/steps");
    rc = ctx->cfg.form == PSL_FORM_PLAIN ? run_plain(ctx, steps) : run_batched(ctx, steps);
    if (rc) return rc;
  }
  {
    NvtxRange r("psl_step/status");
    rc = refresh_headers(ctx);
    if (rc) return rc;
  }
  int n = (int)ctx->queue.size();
  for (auto &kv : ctx->walks) n += kv.second.state == PSL_RUNNING;
  return n;
}

static HostWalk *find(psl_ctx *ctx, int64_t id) {
  auto it = ctx->walks.find(id);
  return it == ctx->walks.end() ? nullptr : &it->second;
}

static double limbs_to_double(const uint32_t *a) {
  // correctly rounded conversion of a two's-complement 384-bit value
  uint32_t m[kWideLimbs];
  std::memcpy(m, a, sizeof m);
  const bool neg = m[kWideLimbs - 1] >> 31;
  if (neg) {
    uint64_t carry = 1;
    for (int i = 0; i < kWideLimbs; i++) {
      const uint64_t v = (uint64_t)(uint32_t)~m[i] + carry;
      m[i] = (uint32_t)v;
      carry = v >> 32;
    }
  }
  int top = -1;
  for (int i = 32 * kWideLimbs - 1; i >= 0; i--)
    if ((m[i >> 5] >> (i & 31)) & 1u) {
      top = i;
      break;
    }
  if (top < 0) return 0.0;
  auto bit = [&](int i) -> uint64_t { return (m[i >> 5] >> (i & 31)) & 1u; };
  double r;
  if (top <= 52) {
    r = (double)(((uint64_t)m[1] << 32) | m[0]);
  } else {
    const int drop = top - 52;
    uint64_t mant = 0;
    for (int i = top; i >= drop; i--) mant = (mant << 1) | bit(i);
    const uint64_t rnd = bit(drop - 1);
    uint64_t sticky = 0;
    for (int i = drop - 2; i >= 0; i--) sticky |= bit(i);
    if (rnd && (sticky || (mant & 1u))) mant++;
    r = std::ldexp((double)mant, drop);
  }
  return neg ? -r : r;
}

extern "C" int psl_poll(psl_ctx *ctx, int64_t id, psl_status *out) {
  if (!ctx || !out) return PSL_EINVAL;
  HostWalk *w = find(ctx, id);
  if (!w) return PSL_ENOENT;
  std::memset(out, 0, sizeof *out);
  out->state = w->state;
  out->error = w->error;
  out->L = w->p.L;
  out->t_submit = w->t_submit;
  out->t_start = w->t_start;
  out->t_done = w->t_done;
  if (w->slot >= 0) {
    const WalkDev &h = ctx->h_hdr[w->slot];
    out->alpha = h.alpha;
    out->moves = h.moves;
    out->flip_evals = h.flip_evals;
    out->switches = h.switches;
    out->rechecks = h.rechecks;
    out->psl = h.psl;
    out->psl_best = h.psl_best;
    out->unimproved = h.unimproved;
    out->F = limbs_to_double(h.F);
    out->value_local = limbs_to_double(h.value_local);
  } else {
    out->alpha = (uint32_t)w->p.alpha1;
  }
  return PSL_OK;
}

static int download_pm1(psl_ctx *ctx, const uint32_t *dbits, uint32_t L, int8_t *out) {
  std::vector<uint32_t> words((L + 31) / 32);
  CK(xfer(ctx, words.data(), dbits, words.size() * 4, cudaMemcpyDeviceToHost));
  CK(cudaStreamSynchronize(ctx->stream));
  for (uint32_t i = 0; i < L; i++) out[i] = ((words[i >> 5] >> (i & 31)) & 1u) ? -1 : 1;
  return PSL_OK;
}

extern "C" int psl_best(psl_ctx *ctx, int64_t id, int32_t *psl_out, int8_t *seq, size_t cap) {
  if (!ctx) return PSL_EINVAL;
  HostWalk *w = find(ctx, id);
  if (!w) return PSL_ENOENT;
  if (w->slot < 0) return PSL_EBUSY;
  if (seq && cap < w->p.L) return fail(ctx, PSL_EINVAL, "cap %zu < L %u", cap, w->p.L);
  const WalkDev &h = ctx->h_hdr[w->slot];
  if (psl_out) *psl_out = h.psl_best;
  if (seq) return download_pm1(ctx, h.bits_best, w->p.L, seq);
  return PSL_OK;
}

extern "C" int psl_best_many(psl_ctx *ctx, const int64_t *ids, size_t n, int32_t *psl_out, int8_t *seqs,
                             size_t cap) {
  if (!ctx || (n && !ids)) return PSL_EINVAL;
  std::vector<const HostWalk *> ws(n);
  size_t words_total = 0;
  for (size_t q = 0; q < n; q++) {
    const HostWalk *w = find(ctx, ids[q]);
    if (!w) return fail(ctx, PSL_ENOENT, "unknown walk %lld", (long long)ids[q]);
    if (w->slot < 0) return fail(ctx, PSL_EBUSY, "walk %lld is queued", (long long)ids[q]);
    if (seqs && cap < w->p.L) return fail(ctx, PSL_EINVAL, "cap %zu < L %u", cap, w->p.L);
    ws[q] = w;
    words_total += (w->p.L + 31) / 32;
  }
  if (psl_out)
    for (size_t q = 0; q < n; q++) psl_out[q] = ctx->h_hdr[ws[q]->slot].psl_best;
  if (!seqs || n == 0) return PSL_OK;
  // every walk's packed best sequence copied back in one go, then unpacked on the host
  std::vector<uint32_t> words(words_total);
  size_t at = 0;
  for (size_t q = 0; q < n; q++) {
    const size_t nw = (ws[q]->p.L + 31) / 32;
    CK(xfer(ctx, words.data() + at, ctx->h_hdr[ws[q]->slot].bits_best, nw * 4, cudaMemcpyDeviceToHost));
    at += nw;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  at = 0;
  for (size_t q = 0; q < n; q++) {
    const uint32_t L = ws[q]->p.L;
    int8_t *out = seqs + q * cap;
    for (uint32_t i = 0; i < L; i++) out[i] = ((words[at + (i >> 5)] >> (i & 31)) & 1u) ? -1 : 1;
    at += (L + 31) / 32;
  }
  return PSL_OK;
}

extern "C" int psl_best_fitness(psl_ctx *ctx, int64_t id, uint32_t *value_limbs, double *value, int8_t *seq,
                                size_t cap) {
  if (!ctx) return PSL_EINVAL;
  HostWalk *w = find(ctx, id);
  if (!w) return PSL_ENOENT;
  if (w->slot < 0) return PSL_EBUSY;
  if (w->p.alpha1 != w->p.alpha2) return fail(ctx, PSL_ESTATE, "alpha1 != alpha2: F of the two phases differ");
  if (seq && cap < w->p.L) return fail(ctx, PSL_EINVAL, "cap %zu < L %u", cap, w->p.L);
  const WalkDev &h = ctx->h_hdr[w->slot];
  if (value_limbs) std::memcpy(value_limbs, h.F_best, sizeof h.F_best);
  if (value) *value = limbs_to_double(h.F_best);
  if (seq) return download_pm1(ctx, h.bits_fbest, w->p.L, seq);
  return PSL_OK;
}

extern "C" int psl_release(psl_ctx *ctx, int64_t id) {
  if (!ctx) return PSL_EINVAL;
  HostWalk *w = find(ctx, id);
  if (!w) return PSL_ENOENT;
  if (w->state == PSL_QUEUED) {
    ctx->queue.erase(std::remove(ctx->queue.begin(), ctx->queue.end(), id), ctx->queue.end());
  } else if (w->slot >= 0) {
    CK(cudaStreamSynchronize(ctx->stream));
    WalkDev z{};
    z.status = kFree;
    CK(cudaMemcpy(ctx->d_hdr + w->slot, &z, sizeof z, cudaMemcpyHostToDevice));
    ctx->h_hdr[w->slot] = z;
    ctx->alloc.release(w->off, w->bytes);
    ctx->free_slots.push_back(w->slot);
    if (w->state == PSL_RUNNING) ctx->active_dirty = true;
  }
  ctx->walks.erase(id);
  return PSL_OK;
}

extern "C" int psl_export_state(psl_ctx *ctx, int64_t id, psl_walk_state *st, int8_t *pivot, int8_t *local_best,
                                int8_t *sol_best, int32_t *C, size_t cap) {
  if (!ctx) return PSL_EINVAL;
  HostWalk *w = find(ctx, id);
  if (!w) return PSL_ENOENT;
  if (w->slot < 0) return PSL_EBUSY;
  const uint32_t L = w->p.L;
  if ((pivot || local_best || sol_best || C) && cap < L) return fail(ctx, PSL_EINVAL, "cap < L");
  WalkDev h;
  CK(xfer(ctx, &h, ctx->d_hdr + w->slot, sizeof h, cudaMemcpyDeviceToHost));
  CK(cudaStreamSynchronize(ctx->stream));
  if (st) {
    std::memset(st, 0, sizeof *st);
    st->L = h.L;
    st->N = h.N;
    st->alpha = h.alpha;
    st->unimproved = h.unimproved;
    st->psl = h.psl;
    st->psl_best = h.psl_best;
    st->psl_local = h.psl_local;
    st->start = h.start;
    st->rng_ctr = h.rng_ctr;
    st->moves = h.moves;
    std::memcpy(st->F, h.F, sizeof st->F);
    std::memcpy(st->value_local, h.value_local, sizeof st->value_local);
    st->state = w->state;
  }
  int rc = PSL_OK;
  if (pivot && (rc = download_pm1(ctx, h.bits, L, pivot))) return rc;
  if (local_best && (rc = download_pm1(ctx, h.bits_local, L, local_best))) return rc;
  if (sol_best && (rc = download_pm1(ctx, h.bits_best, L, sol_best))) return rc;
  if (C) {
    CK(xfer(ctx, C, h.C, (size_t)L * 4, cudaMemcpyDeviceToHost));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return PSL_OK;
}

extern "C" int psl_trace(psl_ctx *ctx, int64_t id, psl_trace_rec *out, size_t cap) {
  if (!ctx || (!out && cap)) return PSL_EINVAL;
  HostWalk *w = find(ctx, id);
  if (!w) return PSL_ENOENT;
  if (w->slot < 0) return PSL_EBUSY;
  static_assert(sizeof(psl_trace_rec) == sizeof(TraceRec), "trace record layout");
  const WalkDev &h = ctx->h_hdr[w->slot];
  const uint64_t n = std::min<uint64_t>(std::min<uint64_t>(h.moves, h.trace_cap), cap);
  if (n) {
    CK(xfer(ctx, out, h.trace, n * sizeof(TraceRec), cudaMemcpyDeviceToHost));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return (int)n;
}

extern "C" int psl_autocorr(psl_ctx *ctx, const int8_t *seq, uint32_t nseq, uint32_t L, int32_t *C) {
  if (!ctx || !seq || !C || nseq == 0 || L < 1 || L > (1u << 20) - 1u) return PSL_EINVAL;
  // runs as init-only walks in temporary slots of a private header array
  const uint32_t nw = (L + 31) / 32;
  const size_t words = nw + 2 * kGuardWords;
  const size_t per = align_up(words * 4, 256) * 3 + align_up((size_t)L * 4, 256);
  char *buf = nullptr;
  WalkDev *dh = nullptr;
  uint32_t *dl = nullptr;
  CK(cudaMalloc(&buf, per * nseq));
  std::vector<WalkDev> hh(nseq);
  std::vector<uint32_t> list(nseq);
  std::vector<uint32_t> packed;
  int rc = PSL_OK;
  cudaError_t e = cudaSuccess;
  for (uint32_t q = 0; q < nseq && e == cudaSuccess; q++) {
    WalkDev &h = hh[q];
    std::memset(&h, 0, sizeof h);
    char *b = buf + per * q;
    h.L = L;
    h.nw = nw;
    h.has_init_seq = 1;
    h.bits = (uint32_t *)b + kGuardWords;
    h.bits_local = (uint32_t *)(b + align_up(words * 4, 256)) + kGuardWords;
    h.bits_best = (uint32_t *)(b + 2 * align_up(words * 4, 256)) + kGuardWords;
    h.C = (int32_t *)(b + 3 * align_up(words * 4, 256));
    h.status = kRunning;
    list[q] = q;
    pack_pm1(seq + (size_t)q * L, L, packed);
    e = cudaMemcpy(h.bits, packed.data(), packed.size() * 4, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMalloc(&dh, sizeof(WalkDev) * nseq);
  if (e == cudaSuccess) e = cudaMalloc(&dl, sizeof(uint32_t) * nseq);
  if (e == cudaSuccess) e = cudaMemcpy(dh, hh.data(), sizeof(WalkDev) * nseq, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dl, list.data(), sizeof(uint32_t) * nseq, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    LaunchCtx c{};
    c.hdr = dh;
    c.active = dl;
    c.maxL = L;
    c.ninit = nseq;
    c.sm_count = ctx->sm_count;
    c.stream = ctx->stream;
    e = launch_init_bits(c);
    if (e == cudaSuccess) e = launch_autocorr(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  }
  for (uint32_t q = 0; q < nseq && e == cudaSuccess; q++)
    e = cudaMemcpy(C + (size_t)q * L, hh[q].C, (size_t)L * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) rc = fail(ctx, PSL_ECUDA, "psl_autocorr: %s", cudaGetErrorString(e));
  cudaFree(buf);
  if (dh) cudaFree(dh);
  if (dl) cudaFree(dl);
  return rc;
}

extern "C" int psl_autotune(psl_ctx *ctx, int reps) {
  if (!ctx || reps < 1 || ctx->cfg.form != PSL_FORM_BATCHED) return PSL_EINVAL;
  CK(cudaSetDevice(ctx->cfg.device));
  int rc = admit(ctx);
  if (rc) return rc;
  if (ctx->active_dirty && (rc = rebuild_active(ctx))) return rc;
  if (ctx->active.empty()) return fail(ctx, PSL_ESTATE, "no running walk to tune on");
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  float best_ms = 3.4e38f;
  int32_t best_t = ctx->cfg.hot_threads, best_sb = ctx->cfg.hot_tile_sb;
  const int32_t configs[8][2] = {{128, 16}, {128, 32}, {256, 16}, {256, 32}, {512, 16}, {512, 32},
                                 {448, 16}, {896, 32}};  // the last two: producer / consumer form
  for (const auto &cf : configs) {
    {
      const int32_t t = cf[0], sb = cf[1];
      ctx->cfg.hot_threads = t;
      ctx->cfg.hot_tile_sb = sb;
      if ((rc = rebuild_active(ctx))) return rc;
      LaunchCtx c = launch_ctx(ctx, ctx->d_active, ctx->d_sched);
      uint32_t *next = &ctx->d_sched->hot_next;
      CK(launch_hot(c));  // warm-up
      CK(cudaMemsetAsync(next, 0, 4, ctx->stream));
      CK(cudaEventRecord(a, ctx->stream));
      for (int r = 0; r < reps; r++) {
        CK(launch_hot(c));
        CK(cudaMemsetAsync(next, 0, 4, ctx->stream));  // the persistent kernel consumed its work counter
      }
      CK(cudaEventRecord(b, ctx->stream));
      CK(cudaEventSynchronize(b));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, a, b));
      if (ms < best_ms) best_ms = ms, best_t = t, best_sb = sb;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  ctx->cfg.hot_threads = best_t;
  ctx->cfg.hot_tile_sb = best_sb;
  drop_graph(ctx);  // captured with another kernel variant
  if ((rc = rebuild_active(ctx))) return rc;
  return best_t | (best_sb << 16);
}

extern "C" int psl_hot_variant(psl_ctx *ctx, char *name, int32_t cap) {
  if (!ctx || !name || cap < 1) return PSL_EINVAL;
  int rc = admit(ctx);
  if (rc) return rc;
  if (ctx->active_dirty && (rc = rebuild_active(ctx))) return rc;
  if (ctx->cfg.form == PSL_FORM_PLAIN) return snprintf(name, (size_t)cap, "k_hot_plain");
  return hot_kernel_name(launch_ctx(ctx, ctx->d_active, ctx->d_sched), name, cap);
}

extern "C" int psl_set_hot_config(psl_ctx *ctx, int32_t threads, int32_t tile_sb) {
  if (!ctx || threads < 0 || tile_sb < 0 || !hot_config_supported((uint32_t)threads, (uint32_t)tile_sb))
    return PSL_EINVAL;
  ctx->cfg.hot_threads = threads;
  ctx->cfg.hot_tile_sb = tile_sb;
  ctx->active_dirty = true;  // the block list depends on the block size
  drop_graph(ctx);  // captured with another kernel variant
  return PSL_OK;
}

extern "C" int psl_set_max_sms(psl_ctx *ctx, int32_t max_sms) {
  if (!ctx || max_sms < 0) return PSL_EINVAL;
  const uint32_t n = max_sms == 0 ? ctx->dev_sms : std::min<uint32_t>(ctx->dev_sms, (uint32_t)max_sms);
  if (n == ctx->sm_count) return (int)n;
  ctx->sm_count = n;
  ctx->cfg.max_sms = max_sms;
  ctx->active_dirty = true;  // the k split of each walk depends on the SM count
  drop_graph(ctx);  // captured with the old grid sizes
  return (int)n;
}

extern "C" int psl_inject_stall(psl_ctx *ctx, int64_t id) {
  if (!ctx) return PSL_EINVAL;
  HostWalk *w = find(ctx, id);
  if (!w) return PSL_ENOENT;
  if (w->slot < 0) return PSL_EBUSY;
  const uint32_t one = 1;
  CK(xfer(ctx, (char *)(ctx->d_hdr + w->slot) + offsetof(WalkDev, inject_stall), &one, 4, cudaMemcpyHostToDevice));
  CK(cudaStreamSynchronize(ctx->stream));
  return PSL_OK;
}

// ---------------------------------------------------------------------------------
// single-walk k-sharding: one step split into the rank's share of the work and two
// exchanges that the caller performs (sums over ranks of zero-filled arrays)
// ---------------------------------------------------------------------------------
// The sharded walk of the context, admitted and listed; nullptr after fail().
static HostWalk *shard_walk(psl_ctx *ctx, int64_t id, int *rc) {
  *rc = PSL_OK;
  HostWalk *w = find(ctx, id);
  if (!w) {
    *rc = PSL_ENOENT;
    return nullptr;
  }
  if (w->p.shard_count < 2) {
    *rc = fail(ctx, PSL_EINVAL, "walk %lld is not sharded", (long long)id);
    return nullptr;
  }
  if (cudaSetDevice(ctx->cfg.device) != cudaSuccess) {
    *rc = fail(ctx, PSL_ECUDA, "cudaSetDevice failed");
    return nullptr;
  }
  if ((*rc = admit(ctx))) return nullptr;
  if (ctx->active_dirty && (*rc = rebuild_active(ctx))) return nullptr;
  if (w->state != PSL_RUNNING) {
    *rc = fail(ctx, w->state == PSL_QUEUED ? PSL_ENOMEM : PSL_ESTATE, "walk %lld is not running", (long long)id);
    return nullptr;
  }
  return w;
}

extern "C" int psl_shard_layout(psl_ctx *ctx, int64_t id, uint32_t *ksplit, uint32_t *N, uint32_t *rc_words_max) {
  if (!ctx) return PSL_EINVAL;
  HostWalk *w = find(ctx, id);
  if (!w) return PSL_ENOENT;
  if (w->p.shard_count < 2) return fail(ctx, PSL_EINVAL, "walk %lld is not sharded", (long long)id);
  if (w->slot < 0) {  // queued: admit it, so that its chunks are known
    int rc;
    if (!shard_walk(ctx, id, &rc)) return rc;
  }
  const WalkDev &h = ctx->h_hdr[w->slot];
  if (ksplit) *ksplit = h.ksplit;
  if (N) *N = h.N;
  if (rc_words_max) *rc_words_max = ((uint32_t)kQcap * h.nchunk_rc + h.N) * kWideLimbs;
  return PSL_OK;
}

extern "C" int psl_shard_score(psl_ctx *ctx, int64_t id, float *parts, size_t cap) {
  if (!ctx || !parts) return PSL_EINVAL;
  int rc;
  HostWalk *w = shard_walk(ctx, id, &rc);
  if (!w) return rc;
  const WalkDev &h = ctx->h_hdr[w->slot];
  const size_t n = (size_t)h.ksplit * h.N;
  if (cap < n) return fail(ctx, PSL_EINVAL, "cap %zu < ksplit x N = %zu", cap, n);
  LaunchCtx c = launch_ctx(ctx, ctx->d_active, ctx->d_sched);
  // other ranks' chunks stay zero, so that the sum over ranks of every rank's array is exact
  CK(cudaMemsetAsync(h.score_part, 0, n * 4, ctx->stream));
  CK(cudaMemsetAsync(&ctx->d_sched->hot_next, 0, 4, ctx->stream));
  CK(prof_begin(ctx, kPHot));
  CK(launch_hot_batched(c));
  CK(prof_end(ctx, kPHot));
  CK(xfer(ctx, parts, h.score_part, n * 4, cudaMemcpyDeviceToHost));
  uint32_t status = kRunning;
  CK(xfer(ctx, &status, (char *)(ctx->d_hdr + w->slot) + offsetof(WalkDev, status), 4, cudaMemcpyDeviceToHost));
  CK(cudaStreamSynchronize(ctx->stream));
  prof_collect(ctx);
  if (status != kRunning) {
    refresh_headers(ctx);
    return fail(ctx, PSL_ETIMEOUT, "a bounded wait of the neighbourhood kernel ran out");
  }
  return (int)n;
}

extern "C" int psl_shard_select(psl_ctx *ctx, int64_t id, const float *parts, uint32_t *rc_parts, size_t cap) {
  if (!ctx || !parts || !rc_parts) return PSL_EINVAL;
  int rc;
  HostWalk *w = shard_walk(ctx, id, &rc);
  if (!w) return rc;
  const WalkDev &h = ctx->h_hdr[w->slot];
  const size_t n = (size_t)h.ksplit * h.N;
  LaunchCtx c = launch_ctx(ctx, ctx->d_active, ctx->d_sched);
  CK(xfer(ctx, h.score_part, parts, n * 4, cudaMemcpyHostToDevice));
  CK(prof_begin(ctx, kPSelect));
  CK(launch_select(c));
  CK(prof_end(ctx, kPSelect));
  uint32_t ncand = 0;
  CK(xfer(ctx, &ncand, (char *)(ctx->d_hdr + w->slot) + offsetof(WalkDev, ncand), 4, cudaMemcpyDeviceToHost));
  CK(cudaStreamSynchronize(ctx->stream));
  const size_t slots = ncand <= (uint32_t)kQcap ? (size_t)ncand * h.nchunk_rc
                                                 : (size_t)kQcap * h.nchunk_rc + (ncand - kQcap);
  const size_t words = slots * kWideLimbs;
  if (cap < words) return fail(ctx, PSL_EINVAL, "cap %zu < %zu re-check words", cap, words);
  // other ranks' chunks stay zero: the limbs of each slot come from one rank only
  CK(cudaMemsetAsync(h.rc_part, 0, words * 4, ctx->stream));
  CK(prof_begin(ctx, kPRecheck));
  CK(launch_recheck(c));
  CK(prof_end(ctx, kPRecheck));
  CK(xfer(ctx, rc_parts, h.rc_part, words * 4, cudaMemcpyDeviceToHost));
  CK(cudaStreamSynchronize(ctx->stream));
  prof_collect(ctx);
  return (int)words;
}

extern "C" int psl_shard_decide(psl_ctx *ctx, int64_t id, const uint32_t *rc_parts, size_t words) {
  if (!ctx || (!rc_parts && words)) return PSL_EINVAL;
  int rc;
  HostWalk *w = shard_walk(ctx, id, &rc);
  if (!w) return rc;
  const WalkDev &h = ctx->h_hdr[w->slot];
  if (words > ((size_t)kQcap * h.nchunk_rc + h.N) * kWideLimbs) return fail(ctx, PSL_EINVAL, "too many words");
  LaunchCtx c = launch_ctx(ctx, ctx->d_active, ctx->d_sched);
  if (words) CK(xfer(ctx, h.rc_part, rc_parts, words * 4, cudaMemcpyHostToDevice));
  CK(prof_begin(ctx, kPDecide));
  CK(launch_decide(c));
  CK(prof_end(ctx, kPDecide));
  CK(prof_begin(ctx, kPApply));
  CK(launch_apply(c));
  CK(prof_end(ctx, kPApply));
  if ((rc = refresh_headers(ctx))) return rc;
  return w->state;
}
