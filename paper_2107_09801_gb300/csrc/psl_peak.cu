// psl_peak.cu -- measured issue rates of the CUDA-core pipes that bound the neighbourhood
// kernel (the denominator of its roofline; no counterpart in the paper).
//
// The neighbourhood score is not a contraction and one pass over C serves N neighbours, so
// it is bound by instruction issue on the FP32 and integer/logic pipes, not by tensor cores
// or memory.  Four kernels measure what those pipes deliver on the device at hand:
//   fadd    independent FP32 add chains                      (FP32 adds per second)
//   alu     an integer add and a three-input logic op in turn (integer/logic ops per second)
//   mix     FP32 add, integer add and logic op, one of each   (lane-ops per second)
//   lookup  the neighbourhood kernel's inner pattern: a shift, a logic op forming a table
//           address, a shared-memory load and an FP32 add    (lookups per second)
//   popc    the bit-plane step of the alpha = 2 closed form: a logic op, a population count
//           and an integer add                                (plane steps per second)
// Each op is written as inline PTX on a dependency chain the compiler cannot fold (adds
// and logic ops alternate; FP32 adds do not reassociate), and every chain ends in a value
// that is stored conditionally, so no work is removed.
#include <cstdint>

#include "psl.h"

namespace {

constexpr int kPeakThreads = 256;
constexpr int kChains = 8;

__device__ __forceinline__ float fadd_ptx(float a, float b) {
  float r;
  asm volatile("add.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ uint32_t iadd_ptx(uint32_t a, uint32_t b) {
  uint32_t r;
  asm volatile("add.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t lop3_ptx(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(a), "r"(b), "r"(c));  // a ^ b ^ c
  return r;
}

// 4 x kChains FP32 adds per iteration
__global__ void __launch_bounds__(kPeakThreads) k_peak_fadd(float *sink, int iters, float b0) {
  float a[kChains], b[kChains];
#pragma unroll
  for (int i = 0; i < kChains; i++) a[i] = (float)threadIdx.x * 1e-3f + (float)i, b[i] = b0 * (float)(i + 1);
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
      for (int i = 0; i < kChains; i++) a[i] = fadd_ptx(a[i], b[i]);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; i++) s += a[i];
  if (s == -1.2345f) sink[0] = s;
}

// 2 x 2 x kChains integer/logic ops per iteration (add, logic, add, logic)
__global__ void __launch_bounds__(kPeakThreads) k_peak_alu(uint32_t *sink, int iters, uint32_t y, uint32_t z) {
  uint32_t x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; i++) x[i] = threadIdx.x * 0x9E3779B9u + (uint32_t)i;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int u = 0; u < 2; u++)
#pragma unroll
      for (int i = 0; i < kChains; i++) x[i] = lop3_ptx(iadd_ptx(x[i], y), z, (uint32_t)i);
  }
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kChains; i++) s ^= x[i];
  if (s == 0x12345u) sink[0] = s;
}

// 3 x 2 x kChains ops per iteration: FP32 add, integer add, logic op on interleaved chains
__global__ void __launch_bounds__(kPeakThreads) k_peak_mix(uint32_t *sink, int iters, uint32_t y, uint32_t z, float b0) {
  uint32_t x[kChains];
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; i++) x[i] = threadIdx.x * 0x9E3779B9u + (uint32_t)i, a[i] = (float)x[i] * 1e-9f;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int u = 0; u < 2; u++)
#pragma unroll
      for (int i = 0; i < kChains; i++) {
        a[i] = fadd_ptx(a[i], b0);
        x[i] = lop3_ptx(iadd_ptx(x[i], y), z, (uint32_t)i);
      }
  }
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kChains; i++) s ^= x[i] ^ __float_as_uint(a[i]);
  if (s == 0x12345u) sink[0] = s;
}

// 6 x 4 lookups per iteration, each: a shift, a logic op (mask the 5-bit field and XOR the
// table base into it: a byte address), a shared-memory load and an FP32 add -- the inner
// loop of the neighbourhood kernel.  The 32-bit word the fields come from changes every
// iteration (one multiply-add per word).
template <int Q>
__device__ __forceinline__ float lookup_ptx(uint32_t w, uint32_t mask, uint32_t base) {
  uint32_t f, addr;
  if constexpr (Q == 0)
    asm volatile("shl.b32 %0, %1, 2;" : "=r"(f) : "r"(w));
  else
    asm volatile("shr.b32 %0, %1, %2;" : "=r"(f) : "r"(w), "n"(5 * Q - 2));
  asm volatile("lop3.b32 %0, %1, %2, %3, 0x6A;" : "=r"(addr) : "r"(f), "r"(mask), "r"(base));  // (f & mask) ^ base
  float v;
  asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(addr), "n"(128 * Q));
  return v;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_lookup(float *sink, int iters, uint32_t seed) {
  __shared__ __align__(128) float tab[6 * 32];
  for (int t = threadIdx.x; t < 6 * 32; t += blockDim.x) tab[t] = (float)t * 0.25f;
  __syncthreads();
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(tab);
  const uint32_t mask = 0x7Cu;
  uint32_t w[4];
  float acc[4];
#pragma unroll
  for (int c = 0; c < 4; c++) w[c] = (threadIdx.x + 977u * c) * seed, acc[c] = 0.f;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int c = 0; c < 4; c++) {
      acc[c] = fadd_ptx(acc[c], lookup_ptx<0>(w[c], mask, base));
      acc[c] = fadd_ptx(acc[c], lookup_ptx<1>(w[c], mask, base));
      acc[c] = fadd_ptx(acc[c], lookup_ptx<2>(w[c], mask, base));
      acc[c] = fadd_ptx(acc[c], lookup_ptx<3>(w[c], mask, base));
      acc[c] = fadd_ptx(acc[c], lookup_ptx<4>(w[c], mask, base));
      acc[c] = fadd_ptx(acc[c], lookup_ptx<5>(w[c], mask, base));
      w[c] = w[c] * 0x9E3779B1u + (uint32_t)it;
    }
  }
  float s = acc[0] + acc[1] + acc[2] + acc[3];
  if (s == -1.2345f) sink[0] = s;
}

// 4 x kChains bit-plane steps per iteration, each: a three-input logic op (an AND of the
// running value with two words), a population count, and an integer add into the running value
__global__ void __launch_bounds__(kPeakThreads) k_peak_popc(uint32_t *sink, int iters, uint32_t y) {
  uint32_t x[kChains], w[kChains];
#pragma unroll
  for (int i = 0; i < kChains; i++) x[i] = threadIdx.x * 0x9E3779B9u + (uint32_t)i, w[i] = ~(y * (uint32_t)(i + 3));
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
      for (int i = 0; i < kChains; i++) {
        uint32_t a, c;
        asm volatile("lop3.b32 %0, %1, %2, %3, 0x80;" : "=r"(a) : "r"(x[i]), "r"(w[i]), "r"(y));  // x & w & y
        asm volatile("popc.b32 %0, %1;" : "=r"(c) : "r"(a));
        x[i] = iadd_ptx(x[i], c);
      }
  }
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kChains; i++) s ^= x[i];
  if (s == 0x12345u) sink[0] = s;
}

}  // namespace

extern "C" int psl_alu_peak(int32_t device, void *stream, psl_alu_peak_t *out) {
  if (!out || device < 0) return PSL_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return PSL_ECUDA;
  int sms = 0, clk = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms <= 0)
    return PSL_ECUDA;
  cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, device);  // kHz
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_peak_mix, kPeakThreads, 0) != cudaSuccess || nb < 1) nb = 1;
  const int blocks = sms * nb;
  const double threads = (double)blocks * kPeakThreads;
  cudaStream_t s = (cudaStream_t)stream;
  void *sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = PSL_OK;
  if (cudaMalloc(&sink, 64) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = PSL_ECUDA;
  } else {
    // iterations sized for launches of a few tens of milliseconds
    const int it_fadd = 40000, it_alu = 20000, it_mix = 15000, it_lookup = 15000, it_popc = 10000;
    const double ops[5] = {threads * it_fadd * 4 * kChains, threads * it_alu * 4 * kChains,
                           threads * it_mix * 6 * kChains, threads * it_lookup * 24, threads * it_popc * 4 * kChains};
    for (int kind = 0; kind < 5 && rc == PSL_OK; kind++) {
      float ms = 0.f;
      for (int rep = 0; rep < 2 && rc == PSL_OK; rep++) {  // the first launch warms up
        if (rep == 1 && cudaEventRecord(e0, s) != cudaSuccess) rc = PSL_ECUDA;
        switch (kind) {
          case 0: k_peak_fadd<<<blocks, kPeakThreads, 0, s>>>((float *)sink, it_fadd, 1e-7f); break;
          case 1: k_peak_alu<<<blocks, kPeakThreads, 0, s>>>((uint32_t *)sink, it_alu, 0x9E3779B9u, 0x7F4A7C15u); break;
          case 2: k_peak_mix<<<blocks, kPeakThreads, 0, s>>>((uint32_t *)sink, it_mix, 0x9E3779B9u, 0x7F4A7C15u, 1e-7f);
            break;
          case 3: k_peak_lookup<<<blocks, kPeakThreads, 0, s>>>((float *)sink, it_lookup, 0x2545F491u); break;
          default: k_peak_popc<<<blocks, kPeakThreads, 0, s>>>((uint32_t *)sink, it_popc, 0xF0F0F0F7u); break;
        }
        if (cudaGetLastError() != cudaSuccess) rc = PSL_ECUDA;
      }
      if (rc == PSL_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                           cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = PSL_ECUDA;
      if (rc == PSL_OK) {
        out->ms[kind] = ms;
        const double rate = ops[kind] / (ms * 1e-3);
        if (kind == 0) out->fadd = rate;
        if (kind == 1) out->alu = rate;
        if (kind == 2) out->mix = rate;
        if (kind == 3) out->lookup = rate;
        if (kind == 4) out->popc = rate;
      }
    }
  }
  out->sm_count = sms;
  out->max_clock_mhz = clk / 1000;
  out->blocks_per_sm = nb;
  out->threads_per_block = kPeakThreads;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  return rc;
}
