// vit_internal.h -- kernel arguments, the table of compiled codes and the
// launcher template shared by the per-code translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "vit_acs.cuh"

namespace vit {

constexpr int kWarpsPerCta = 4;   // default CTA size (warps)
constexpr int kMaxRegs = 168;     // registers per thread of the tile decoders

// Arguments of the tile decoder.  A "task" is one warp: 32 lanes x 2 tiles.
struct KArgs {
  Frame f0;              // single frame (frames == nullptr)
  const Frame* frames;   // batch frames (device), or nullptr
  const int64_t* tile0;  // batch: first global tile of each frame, ascending
  int nframes;
  int64_t ntiles;        // tiles in this launch
  Tiling tl;
  uint32_t M;            // finite "-infinity" of a known start
  int64_t ntasks;        // warps with work
  uint32_t* slab;        // survivor words, task_words per task
  int64_t task_words;
  int64_t task_base;     // first task index of this launch (for chunked launches)
};

VIT_HD int64_t find_frame(const int64_t* tile0, int nframes, int64_t gt) {
  int lo = 0, hi = nframes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tile0[mid] <= gt)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

#if defined(__CUDACC__)
// Decodes warp task `task` of one code: 64 / G tiles, lanes grouped G per
// tile pair.
template <class C, bool kWords = true>
__device__ __forceinline__ void run_task(const KArgs& a, int64_t task, int lane) {
  constexpr int TPT = 64 / C::G;  // tiles per task
  const int pair = lane / C::G;
  Half hw[2];
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int64_t gt = task * TPT + 2 * pair + h;
    if (gt >= a.ntiles) {
      hw[h] = idle_half();
    } else if (a.frames == nullptr) {
      hw[h] = make_half(a.f0, gt, a.tl);
    } else {
      const int64_t fi = find_frame(a.tile0, a.nframes, gt);
      hw[h] = make_half(a.frames[fi], gt - a.tile0[fi], a.tl);
    }
  }
  int L = 1;
#pragma unroll
  for (int h = 0; h < 2; h++)
    if (hw[h].active) L = max(L, (int)(hw[h].t1 - hw[h].t0));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) L = max(L, __shfl_xor_sync(0xffffffffu, L, o));
  const int Lw = ((L + C::U - 1) / C::U) * C::U;
  int mu = 0;
#pragma unroll
  for (int h = 0; h < 2; h++)
    if (hw[h].active) {
      hw[h].start = Lw - (int)(hw[h].t1 - hw[h].t0);
      mu = max(mu, hw[h].start + 1);
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mu = max(mu, __shfl_xor_sync(0xffffffffu, mu, o));
  Slab sl{a.slab + task * a.task_words + lane * C::WORDS, 32 * C::WORDS};
  // word loads need every active tile's groups to start on 4-byte boundaries
  bool aligned = true;
#pragma unroll
  for (int h = 0; h < 2; h++)
    if (hw[h].active)
      aligned = aligned && ((reinterpret_cast<uintptr_t>(hw[h].llr) +
                             (uintptr_t)((hw[h].t0 - hw[h].start) * C::BETA)) % 4u == 0u);
  const bool words_ok = kWords && __all_sync(0xffffffffu, aligned);
  if constexpr (C::G == 1)
    decode_pair<C>(hw, Lw, mu, a.M, sl, words_ok);
  else
    decode_pair_rot<C>(hw, Lw, mu, a.M, sl, lane, words_ok);
}

// One warp per task, tasks in launch order.
template <class C>
__global__ void __maxnreg__(kMaxRegs) decode_tiles_kernel(const KArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t task = a.task_base + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (task >= a.ntasks) return;  // warp-uniform
  run_task<C, (C::G == 1)>(a, task, lane);
}

// Persistent kernel over the tasks of two codes: each warp takes the next
// entry of a cost-ordered queue (one atomic per task) until it is empty.
struct MixTask {
  int32_t code;  // 0 or 1
  int32_t pad;
  int64_t task;  // task index within that code's launch arguments
};
struct MixArgs {
  KArgs g[2];
  const MixTask* queue;
  int64_t nqueue;
  unsigned long long* counter;  // zeroed before every launch
};

// Out-of-line task bodies keep the two codes' register allocations apart.
template <class C>
__device__ __noinline__ void run_task_call(const KArgs a, int64_t task, int lane) {
  run_task<C, (C::G == 1)>(a, task, lane);
}

template <class C0, class C1>
__global__ void __maxnreg__(kMaxRegs) decode_mixed_kernel(const MixArgs a) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long q = 0;
    if (lane == 0) q = atomicAdd(a.counter, 1ull);
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q >= (unsigned long long)a.nqueue) break;
    const MixTask t = a.queue[q];
    if (t.code == 0)
      run_task_call<C0>(a.g[0], t.task, lane);
    else
      run_task_call<C1>(a.g[1], t.task, lane);
  }
}
#endif

// One compiled code.
struct CodeEntry {
  int K, beta;
  uint32_t polys[4];
  int words;  // survivor words per lane per stage
  int unroll; // stages per unrolled group
  int tiles_per_task;
  cudaError_t (*launch)(const KArgs&, int warps, cudaStream_t);
};

// A compiled persistent kernel for a pair of codes.
struct MixEntry {
  const CodeEntry* code[2];
  cudaError_t (*launch)(const MixArgs&, int warps, cudaStream_t);
};

#if defined(__CUDACC__)
template <class C>
cudaError_t launch_decode(const KArgs& a, int warps, cudaStream_t s) {
  if (warps < 1 || warps > 8) warps = kWarpsPerCta;
  // grid.x is limited to 2^31-1 CTAs; split very large launches
  const int64_t maxc = (int64_t)1 << 30;
  for (int64_t t0 = 0; t0 < a.ntasks; t0 += maxc * warps) {
    KArgs b = a;
    b.task_base = t0;
    const int64_t tasks = (a.ntasks - t0 < maxc * warps) ? a.ntasks - t0 : maxc * warps;
    const unsigned grid = (unsigned)((tasks + warps - 1) / warps);
    decode_tiles_kernel<C><<<grid, warps * 32, 0, s>>>(b);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <class C0, class C1>
cudaError_t launch_mixed(const MixArgs& a, int warps, cudaStream_t s) {
  if (warps < 1 || warps > 8) warps = kWarpsPerCta;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, decode_mixed_kernel<C0, C1>, warps * 32, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)sms * per_sm;
  const int64_t need = (a.nqueue + warps - 1) / warps;
  if (grid > need) grid = need > 0 ? need : 1;
  decode_mixed_kernel<C0, C1><<<(unsigned)grid, warps * 32, 0, s>>>(a);
  return cudaGetLastError();
}

template <class C>
constexpr CodeEntry make_entry() {
  return CodeEntry{C::K, C::BETA, {C::poly(0), C::poly(1), C::poly(2), C::poly(3)}, C::WORDS, C::U,
                   64 / C::G, &launch_decode<C>};
}
#endif

// Registry filled by the per-code translation units.
const CodeEntry* find_code(int K, int beta, const uint32_t* polys);
void register_codes(const CodeEntry* e, int n);
// Persistent two-code kernels, registered by their translation units with
// the codes' (K, beta, polys); looked up by code entry.
struct MixKey {
  int K, beta;
  uint32_t polys[4];
};
void register_mixed(const MixKey& a, const MixKey& b, cudaError_t (*launch)(const MixArgs&, int, cudaStream_t));
const MixEntry* find_mixed(const CodeEntry* a, const CodeEntry* b, bool* swapped);

}  // namespace vit

// The opaque handle of include/vit.h.
struct vit_code {
  int K, beta;
  uint32_t polys[4];
  int64_t f, v1, v2;
  int mode;
  int period;  // puncturing period (0 = none)
  uint8_t mask[4 * 64];
  const vit::CodeEntry* entry;
};

namespace vit {
// Sets the thread-local message returned by vit_last_error and returns code.
int set_error(int code, const char* fmt, ...);
// Decodes one frame with the given device scratch (no argument checks).
int decode_into(const vit_code* c, const int8_t* llr, int64_t n, uint8_t* bits_out, void* ws, size_t ws_bytes,
                cudaStream_t s);
}  // namespace vit
