// vit_probe.cu -- instruction-rate microbenchmark (include/vit_probe.h): the
// measured peak that the decoder's roofline fraction is taken against.
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/vit.h"
#include "../../include/vit_probe.h"
#include "vit_internal.h"

namespace {

constexpr int kPairs = 8;   // independent register pairs per thread
constexpr int kSteps = 16;  // unrolled steps per round

// One step of pair c: both registers updated, each from the other and from a
// neighbouring pair, with the instruction under test.
template <int KIND>
__device__ __forceinline__ void step(uint32_t (&x)[kPairs], uint32_t (&y)[kPairs], int c) {
  const int n1 = (c + 1) % kPairs, n3 = (c + 3) % kPairs;
  if constexpr (KIND == VIT_PROBE_IADD) {
    asm("add.u32 %0, %0, %1;" : "+r"(x[c]) : "r"(y[n1]));
    asm("add.u32 %0, %0, %1;" : "+r"(y[c]) : "r"(x[c]));
  } else if constexpr (KIND == VIT_PROBE_VMAX16) {
    asm("max.u16x2 %0, %0, %1;" : "+r"(x[c]) : "r"(y[n1]));
    asm("max.u16x2 %0, %0, %1;" : "+r"(y[c]) : "r"(x[n3]));
  } else if constexpr (KIND == VIT_PROBE_IMAD) {
    asm("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(y[n1]), "r"(x[n3]));
    asm("mad.lo.u32 %0, %0, %1, %2;" : "+r"(y[c]) : "r"(x[c]), "r"(y[n3]));
  } else if constexpr (KIND == VIT_PROBE_PRMT) {
    asm("prmt.b32 %0, %0, %1, 0x5140;" : "+r"(x[c]) : "r"(y[n1]));
    asm("prmt.b32 %0, %0, %1, 0x6273;" : "+r"(y[c]) : "r"(x[c]));
  } else if constexpr (KIND == VIT_PROBE_LOP3) {
    asm("lop3.b32 %0, %0, %1, %2, 0xEA;" : "+r"(x[c]) : "r"(y[n1]), "r"(x[n3]));
    asm("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(y[c]) : "r"(x[c]), "r"(y[n3]));
  } else if constexpr (KIND == VIT_PROBE_FADD) {
    asm("add.f32 %0, %0, %1;" : "+r"(x[c]) : "r"(y[n1]));
    asm("add.f32 %0, %0, %1;" : "+r"(y[c]) : "r"(x[c]));
  } else if constexpr (KIND == VIT_PROBE_FMAX) {
    asm("max.f32 %0, %0, %1;" : "+r"(x[c]) : "r"(y[n1]));
    asm("max.f32 %0, %0, %1;" : "+r"(y[c]) : "r"(x[n3]));
  } else if constexpr (KIND == VIT_PROBE_EX2) {
    asm("ex2.approx.ftz.f32 %0, %1;" : "=r"(x[c]) : "r"(y[n1]));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=r"(y[c]) : "r"(x[c]));
  } else {
    asm("lg2.approx.ftz.f32 %0, %1;" : "=r"(x[c]) : "r"(y[n1]));
    asm("lg2.approx.ftz.f32 %0, %1;" : "=r"(y[c]) : "r"(x[c]));
  }
}

template <int KIND>
__global__ void probe_kernel(int iters, uint32_t seed, long long* cycles, uint32_t* sink) {
  uint32_t x[kPairs], y[kPairs];
#pragma unroll
  for (int c = 0; c < kPairs; c++) {
    x[c] = seed * (2u * c + 1u) + threadIdx.x;
    y[c] = seed ^ (0x9e3779b9u * (c + 1)) ^ blockIdx.x;
  }
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int u = 0; u < kSteps; u++)
#pragma unroll
      for (int c = 0; c < kPairs; c++) step<KIND>(x, y, c);
  }
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) {
    uint32_t smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    cycles[3 * blockIdx.x] = t0;
    cycles[3 * blockIdx.x + 1] = t1;
    cycles[3 * blockIdx.x + 2] = smid;
  }
  uint32_t acc = 0;
#pragma unroll
  for (int c = 0; c < kPairs; c++) acc ^= x[c] ^ y[c];
  if (acc == seed) sink[0] = acc;  // keeps the chains live; almost never stored
}

template <int KIND>
cudaError_t launch_probe(int grid, int threads, int iters, long long* cyc, uint32_t* sink, cudaStream_t s,
                         int* per_sm) {
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, probe_kernel<KIND>, threads, 0);
  if (e != cudaSuccess) return e;
  probe_kernel<KIND><<<grid, threads, 0, s>>>(iters, 0x1234567u, cyc, sink);
  return cudaGetLastError();
}

}  // namespace

extern "C" int vit_probe_rate(int kind, int ctas_per_sm, int warps, int iters, void* stream,
                              double* warp_instr_per_clk_sm, double* ms, int* sms) {
  if (kind < 0 || kind >= VIT_PROBE_KINDS) return vit::set_error(VIT_EINVAL, "unknown probe kind %d", kind);
  if (ctas_per_sm < 1 || ctas_per_sm > 32 || warps < 1 || warps > 32 || iters < 1 || iters > (1 << 20))
    return vit::set_error(VIT_EINVAL, "probe shape out of range");
  if (!warp_instr_per_clk_sm || !ms || !sms) return vit::set_error(VIT_EINVAL, "null output pointer");
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return vit::set_error(VIT_ECUDA, "device query: %s", cudaGetErrorString(e));
  const int grid = nsm * ctas_per_sm, threads = 32 * warps;
  cudaStream_t s = (cudaStream_t)stream;
  long long* d_cyc = nullptr;
  uint32_t* d_sink = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  e = cudaMalloc(&d_cyc, sizeof(long long) * 3 * grid);
  if (e == cudaSuccess) e = cudaMalloc(&d_sink, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  int per_sm = 0;
  if (e == cudaSuccess) e = cudaEventRecord(a, s);
  if (e == cudaSuccess) {
    switch (kind) {
      case VIT_PROBE_IADD: e = launch_probe<VIT_PROBE_IADD>(grid, threads, iters, d_cyc, d_sink, s, &per_sm); break;
      case VIT_PROBE_VMAX16: e = launch_probe<VIT_PROBE_VMAX16>(grid, threads, iters, d_cyc, d_sink, s, &per_sm); break;
      case VIT_PROBE_IMAD: e = launch_probe<VIT_PROBE_IMAD>(grid, threads, iters, d_cyc, d_sink, s, &per_sm); break;
      case VIT_PROBE_PRMT: e = launch_probe<VIT_PROBE_PRMT>(grid, threads, iters, d_cyc, d_sink, s, &per_sm); break;
      case VIT_PROBE_LOP3: e = launch_probe<VIT_PROBE_LOP3>(grid, threads, iters, d_cyc, d_sink, s, &per_sm); break;
      case VIT_PROBE_FADD: e = launch_probe<VIT_PROBE_FADD>(grid, threads, iters, d_cyc, d_sink, s, &per_sm); break;
      case VIT_PROBE_FMAX: e = launch_probe<VIT_PROBE_FMAX>(grid, threads, iters, d_cyc, d_sink, s, &per_sm); break;
      case VIT_PROBE_EX2: e = launch_probe<VIT_PROBE_EX2>(grid, threads, iters, d_cyc, d_sink, s, &per_sm); break;
      default: e = launch_probe<VIT_PROBE_LG2>(grid, threads, iters, d_cyc, d_sink, s, &per_sm); break;
    }
  }
  int rc = VIT_OK;
  if (e == cudaSuccess && per_sm < ctas_per_sm)
    rc = vit::set_error(VIT_EINVAL, "%d CTAs of %d warps per SM are not co-resident (at most %d)", ctas_per_sm, warps,
                        per_sm);
  if (e == cudaSuccess) e = cudaEventRecord(b, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  long long* h = nullptr;
  if (e == cudaSuccess && rc == VIT_OK) {
    h = new long long[3 * (size_t)grid];
    e = cudaMemcpy(h, d_cyc, sizeof(long long) * 3 * grid, cudaMemcpyDeviceToHost);
  }
  if (e != cudaSuccess && rc == VIT_OK) rc = vit::set_error(VIT_ECUDA, "probe: %s", cudaGetErrorString(e));
  if (rc == VIT_OK) {
    // per SM: the span from its first CTA's start to its last CTA's end (the
    // block scheduler need not give every SM the same number of CTAs), and
    // the instructions of its CTAs; every thread retires
    // iters * kSteps * kPairs * 2 instructions
    std::vector<long long> lo(1024, LLONG_MAX), hi(1024, LLONG_MIN);
    std::vector<int> cnt(1024, 0);
    for (int i = 0; i < grid; i++) {
      const int sm = (int)(h[3 * i + 2] & 1023);
      lo[sm] = std::min(lo[sm], h[3 * i]);
      hi[sm] = std::max(hi[sm], h[3 * i + 1]);
      cnt[sm]++;
    }
    const double per_cta = (double)warps * iters * kSteps * kPairs * 2.0;
    double instr = 0.0, span = 0.0;
    for (int sm = 0; sm < 1024; sm++)
      if (cnt[sm] > 0) {
        instr += cnt[sm] * per_cta;
        span += (double)(hi[sm] - lo[sm]);
      }
    *warp_instr_per_clk_sm = instr / span;
    *ms = t;
    *sms = nsm;
  }
  delete[] h;
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(d_cyc);
  cudaFree(d_sink);
  return rc;
}
