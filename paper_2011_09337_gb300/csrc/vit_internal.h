// vit_internal.h -- kernel arguments, the table of compiled codes and the
// launcher template shared by the per-code translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "vit_acs.cuh"

namespace vit {

constexpr int kWarpsPerCta = 4;   // default CTA size (warps)
constexpr int kMaxCtaWarps = 32;  // largest CTA a launcher accepts (1024 threads)
constexpr int kMaxRegs = 168;     // registers per thread of the tile decoders
// Rotating-slot (K = 8, 9) decoders with word loads: 128 registers let 4
// CTAs of 4 warps share an SM, so a 2^26-bit K=9 stream (2048 warp tasks)
// runs in one wave (2.90 ms against 3.31 ms at 168 registers and 3 CTAs).
constexpr int kMaxRegsRotWords = 128;
// Single frames of at most kWarpTileLimit tiles whose windows fit
// kWarpSmemStages stages (48 KB of 64-bit decision words per warp) are
// decoded one warp per tile (lower latency than 64 tiles per warp).
constexpr int kWarpSmemStages = 6144;
constexpr int64_t kWarpTileLimit = 1024;

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
  uint32_t* slab;        // survivor words, task_words per slot
  int64_t task_words;
  // slab slots: 0 = one per task (task t uses slot t); otherwise the launch
  // has at most `slots` warps, warp w decodes tasks w, w + W, ... (W = the
  // launch's warps) and uses slot w, so the slab is bounded whatever n is
  int64_t slots;
  int64_t task_base;     // first task index of this launch (for chunked launches)
  // parallel traceback (pt_f0 > 0): subframe length, start rule, SplitMix64
  // key, and one byte per subframe of every tile (pt_nsub per tile)
  int64_t pt_f0;
  int pt_rule;
  uint64_t pt_seed;
  uint8_t* pt_states;
  int64_t pt_nsub;
  // the generators (read by the decoders of codes known only at run time)
  uint32_t polys[4];
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
// The lane's two tiles of warp task `task` (64 / G tiles per task, lanes
// grouped G per tile pair), their end-aligned windows over Lw iterations,
// the first iteration at which every window of the warp has started, and the
// lane's survivor slab.  e1f: each tile's emitted end before clipping to the
// frame's output count (global tile indices in gt).
template <class C>
__device__ __forceinline__ void task_setup(const KArgs& a, int64_t task, int64_t slot, int lane, Half (&hw)[2],
                                           int64_t (&gt)[2], int64_t (&e1f)[2], int& Lw, int& mu, Slab& sl) {
  constexpr int TPT = 64 / C::G;  // tiles per task
  const int pair = lane / C::G;
#pragma unroll
  for (int h = 0; h < 2; h++) {
    gt[h] = task * TPT + 2 * pair + h;
    e1f[h] = 0;
    if (gt[h] >= a.ntiles) {
      hw[h] = idle_half();
    } else {
      const int64_t fi = (a.frames == nullptr) ? -1 : find_frame(a.tile0, a.nframes, gt[h]);
      const Frame& fr = (fi < 0) ? a.f0 : a.frames[fi];
      const int64_t b = (fi < 0) ? gt[h] : gt[h] - a.tile0[fi];
      hw[h] = make_half(fr, b, a.tl);
      const int64_t fb = tile_len(fr.n, a.tl.f);
      e1f[h] = (b * fb + fb < fr.n) ? b * fb + fb : fr.n;
    }
  }
  int L = 1;
#pragma unroll
  for (int h = 0; h < 2; h++)
    if (hw[h].active) L = max(L, (int)(hw[h].t1 - hw[h].t0));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) L = max(L, __shfl_xor_sync(0xffffffffu, L, o));
  Lw = ((L + C::U - 1) / C::U) * C::U;
  mu = 0;
#pragma unroll
  for (int h = 0; h < 2; h++)
    if (hw[h].active) {
      hw[h].start = Lw - (int)(hw[h].t1 - hw[h].t0);
      mu = max(mu, hw[h].start + 1);
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mu = max(mu, __shfl_xor_sync(0xffffffffu, mu, o));
  sl = Slab{a.slab + slot * a.task_words + lane * C::WORDS, 32 * C::WORDS};
}

// Decodes warp task `task` of one code.
template <class C, bool kWords = true>
__device__ __forceinline__ void run_task(const KArgs& a, int64_t task, int64_t slot, int lane) {
  Half hw[2];
  int64_t gt[2], e1f[2];
  int Lw, mu;
  Slab sl;
  task_setup<C>(a, task, slot, lane, hw, gt, e1f, Lw, mu, sl);
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
    decode_pair_rot<C, kWords>(hw, Lw, mu, a.M, sl, lane, words_ok);
}

// Calls body(task, slot) for the warp tasks of this warp: one task per warp
// in launch order (a.slots == 0), or tasks w, w + W, ... on slot w.
template <class F>
__device__ __forceinline__ void for_each_task(const KArgs& a, F&& body) {
  const int64_t wid = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (a.slots == 0) {
    const int64_t task = a.task_base + wid;
    if (task < a.ntasks) body(task, task);  // warp-uniform
    return;
  }
  if (wid >= a.slots) return;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t task = a.task_base + wid; task < a.ntasks; task += nw) body(task, wid);
}

// One warp per task, tasks in launch order.  kWords = false compiles the
// byte-load path only (used for batches of short frames, where most groups
// of a warp are loaded with masking anyway and the kernel with both paths
// needs more registers).
template <class C, bool kWords = true>
__global__ void __maxnreg__((C::G > 1 && kWords) ? kMaxRegsRotWords : kMaxRegs) decode_tiles_kernel(const KArgs a) {
  const int lane = threadIdx.x & 31;
  for_each_task(a, [&](int64_t task, int64_t slot) { run_task<C, kWords>(a, task, slot, lane); });
}

// Persistent kernel over the tasks of two codes: each warp takes the next
// entry of a cost-ordered queue (one atomic per task) until it is empty.
// Both task bodies are inlined, so the kernel runs with the larger register
// allocation of the two (out-of-line bodies kept them apart but paid for the
// calls in spills: 0.98 against 0.90 ms on the mixed benchmark batch; the
// same plan as two concurrent launches takes 0.54 ms and is the default).
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
      run_task<C0, (C0::G == 1)>(a.g[0], t.task, t.task, lane);
    else
      run_task<C1, (C1::G == 1)>(a.g[1], t.task, t.task, lane);
  }
}
#endif

// One compiled code (or, with generic set, every code of its K and beta).
struct CodeEntry {
  int K, beta;
  uint32_t polys[4];
  int words;  // survivor words per lane per stage
  int unroll; // stages per unrolled group
  int tiles_per_task;
  int slab_lanes;  // lanes whose survivor words one task stores per stage (32; 1 for one warp per tile)
  int generic;     // 1: patterns from the code's generators at run time
  int64_t (*resident)(int warps);  // resident warps of `launch` on the current device
  cudaError_t (*launch)(const KArgs&, int warps, cudaStream_t);
  cudaError_t (*launch_bytes)(const KArgs&, int warps, cudaStream_t);  // byte loads only
};
typedef cudaError_t (*LaunchFn)(const KArgs&, int warps, cudaStream_t);

// A compiled persistent kernel for a pair of codes.
struct MixEntry {
  const CodeEntry* code[2];
  cudaError_t (*launch)(const MixArgs&, int warps, cudaStream_t);
};

#if defined(__CUDACC__)
// Launches `kernel` over the tasks [a.task_base, a.ntasks) of `a`, one warp
// per task (grid.x is limited to 2^31-1 CTAs, so very large launches are
// split).
template <void (*kernel)(const KArgs)>
cudaError_t launch_tasks(const KArgs& a, int warps, cudaStream_t s) {
  if (warps < 1 || warps > kMaxCtaWarps) warps = kWarpsPerCta;
  if (a.slots > 0) {  // at most `slots` warps stride over the tasks
    const int64_t need = a.ntasks - a.task_base < a.slots ? a.ntasks - a.task_base : a.slots;
    kernel<<<(unsigned)((need + warps - 1) / warps), warps * 32, 0, s>>>(a);
    return cudaGetLastError();
  }
  const int64_t maxc = (int64_t)1 << 30;
  for (int64_t t0 = a.task_base; t0 < a.ntasks; t0 += maxc * warps) {
    KArgs b = a;
    b.task_base = t0;
    const int64_t tasks = (a.ntasks - t0 < maxc * warps) ? a.ntasks - t0 : maxc * warps;
    const unsigned grid = (unsigned)((tasks + warps - 1) / warps);
    kernel<<<grid, warps * 32, 0, s>>>(b);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Warps of `kernel` (CTAs of `warps` warps) resident at once on the current
// device, or 0 when the device cannot be queried.
template <void (*kernel)(const KArgs)>
int64_t resident_warps(int warps) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, warps * 32, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (int64_t)sms * per_sm * warps;
}

template <class C>
cudaError_t launch_decode(const KArgs& a, int warps, cudaStream_t s) {
  return launch_tasks<decode_tiles_kernel<C, true>>(a, warps, s);
}


template <class C>
cudaError_t launch_decode_bytes(const KArgs& a, int warps, cudaStream_t s) {
  return launch_tasks<decode_tiles_kernel<C, false>>(a, warps, s);
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
constexpr LaunchFn bytes_launcher() {
  if constexpr (C::G > 1 && kWordLoads<C>)
    return &launch_decode_bytes<C>;
  else
    return &launch_decode<C>;
}

template <class C>
constexpr CodeEntry make_entry() {
  return CodeEntry{C::K,       C::BETA, {C::poly(0), C::poly(1), C::poly(2), C::poly(3)}, C::WORDS, C::U, 64 / C::G,
                   32,         0,       &resident_warps<decode_tiles_kernel<C, true>>,    &launch_decode<C>,
                   bytes_launcher<C>()};
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
// Tile decoders with the parallel traceback, registered by (K, beta, polys).
void register_pt(const MixKey& k, LaunchFn launch);
LaunchFn find_pt(const CodeEntry* e);
// Warp-per-tile decoders for frames with few tiles, by (K, beta, polys).
void register_warp(const MixKey& k, LaunchFn launch);
LaunchFn find_warp(const CodeEntry* e);
// Decoders for codes known only at run time, by (K, beta): the tile decoder
// entry (one warp per tile, decisions in the slab, any window) and the
// single-frame warp-per-tile decoder with decisions in shared memory (K <= 7).
void register_generic(const CodeEntry* e);
const CodeEntry* find_generic(int K, int beta);
void register_warp_generic(int K, int beta, LaunchFn launch);
LaunchFn find_warp_generic(int K, int beta);
// Tile decoders that spread each tile pair over several lanes (fewer tiles
// per warp task), for frames with too few tiles to fill the GPU, by
// (K, beta, polys).
void register_spread(const MixKey& k, const CodeEntry* e);
const CodeEntry* find_spread(const CodeEntry* e);

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
  int64_t pt_f0;      // parallel traceback subframe length (0: serial traceback)
  int pt_rule;        // VIT_PT_STORED or VIT_PT_RANDOM
  uint64_t pt_seed;
  vit::LaunchFn pt_launch;
  vit::LaunchFn warp_launch;  // warp-per-tile decoder, or nullptr
  const vit::CodeEntry* spread;  // tile decoder with several lanes per tile pair, or nullptr
  int decoder;                // VIT_DECODER_AUTO, _TILES, _SHARED or _SPREAD
};

namespace vit {
// Sets the thread-local message returned by vit_last_error and returns code.
int set_error(int code, const char* fmt, ...);
// Decodes one frame with the given device scratch (no argument checks).
int decode_into(const vit_code* c, const int8_t* llr, int64_t n, uint8_t* bits_out, void* ws, size_t ws_bytes,
                cudaStream_t s);
}  // namespace vit
