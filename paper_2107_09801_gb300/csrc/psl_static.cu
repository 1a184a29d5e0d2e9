// psl_static.cu -- aperiodic autocorrelation of one device-resident sequence that uses a
// fixed scratch area compiled into the library instead of allocating device memory.
//
// Who needs this: code that must not call cudaMalloc / cudaFree itself.  Typical cases
// are a host framework that owns all device memory through its own allocator (a raw
// cudaFree synchronises the whole device and would stall the framework's other
// streams), and long-running services that reserve every buffer at start-up so that no
// request can fail or block on an allocation later.  Such callers hand in input and
// output buffers they already own; the only extra memory this path needs is the packed
// copy of the sequence, and that lives in the static array below.
#include <cstdint>
#include <mutex>

#include "psl.h"

namespace {

constexpr uint32_t kStaticMaxL = (1u << 20) - 1u;          // longest sequence accepted
constexpr uint32_t kStaticGuard = 2;                       // zero words on each side
constexpr uint32_t kStaticWords = (kStaticMaxL + 31) / 32 + 2 * kStaticGuard;  // 32772 words, 128 KiB

// Packed sequence (bit = 1 means -1) with zero guard words.  Every device that loads the
// library holds one copy until the process exits.  All calls share it.
static __device__ __align__(256) uint32_t psl_static_scratch[kStaticWords];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices];  // address of psl_static_scratch on each device, once known
std::mutex g_scratch_mu;

// Packs s (int8, negative = -1) into the scratch words and zeroes every other word the
// autocorrelation may read, so nothing left by an earlier call can leak in.
__global__ void k_static_pack(uint32_t *scratch, const int8_t *__restrict__ s, uint32_t L) {
  const uint32_t nw = (L + 31) / 32;
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nw + 2 * kStaticGuard; w += gridDim.x * blockDim.x) {
    uint32_t word = 0;
    if (w >= kStaticGuard && w < nw + kStaticGuard) {
      const uint32_t i0 = 32 * (w - kStaticGuard);
      for (uint32_t b = 0; b < 32 && i0 + b < L; b++) word |= (s[i0 + b] < 0 ? 1u : 0u) << b;
    }
    scratch[w] = word;
  }
}

// C_k = (L - k) - 2 popc(x[0..L-k) xor x[k..L)) for one k per thread (Eq. 2 on packed bits).
__global__ void k_static_autocorr(const uint32_t *scratch, uint32_t L, int32_t *C) {
  const uint32_t *bits = scratch + kStaticGuard;
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= L) return;
  const uint32_t n = L - k;
  uint32_t cnt = 0;
  for (uint32_t w = 0; 32 * w < n; w++) {
    const uint32_t pos = 32 * w + k;
    const uint32_t shifted = __funnelshift_r(bits[pos >> 5], bits[(pos >> 5) + 1], pos & 31);
    uint32_t d = bits[w] ^ shifted;
    const uint32_t rem = n - 32 * w;
    if (rem < 32) d &= (1u << rem) - 1u;
    cnt += __popc(d);
  }
  C[k] = (int32_t)n - 2 * (int32_t)cnt;
}

}  // namespace

extern "C" int psl_autocorr_static(const int8_t *seq_dev, uint32_t L, int32_t *C_dev, void *stream) {
  if (!seq_dev || !C_dev || L < 1 || L > kStaticMaxL) return PSL_EINVAL;
  // an error left pending by the caller's own earlier work is not this call's to report
  // or to clear: refuse to launch and leave it in place
  if (cudaPeekAtLastError() != cudaSuccess) return PSL_ECUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PSL_ECUDA;
  void *scratch = nullptr;
  {
    // first call on this device: look up the device address of the static array (host
    // code cannot use the symbol itself); later calls reuse it
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, psl_static_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return PSL_ECUDA;
      }
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t words = (L + 31) / 32 + 2 * kStaticGuard;
  k_static_pack<<<(words + 255) / 256, 256, 0, s>>>((uint32_t *)scratch, seq_dev, L);
  if (cudaGetLastError() != cudaSuccess) return PSL_ECUDA;
  k_static_autocorr<<<(L + 255) / 256, 256, 0, s>>>((const uint32_t *)scratch, L, C_dev);
  return cudaGetLastError() == cudaSuccess ? PSL_OK : PSL_ECUDA;
}
