// vit_kernels.cuh -- kernel templates and launchers shared by the per-code
// translation units: the warp-per-tile decoders (vit_warp.cuh) and the tile
// decoder with the parallel traceback (vit_pt.cuh), each for codes fixed at
// compile time (Code) and codes known only at run time (GCode).
#pragma once
#include "vit_internal.h"
#include "vit_pt.cuh"
#include "vit_warp.cuh"

namespace vit {

// One warp (CTA) per tile of a single frame; the tile's decision words live
// in the CTA's shared memory (windows of at most kWarpSmemStages stages).
template <class C>
__global__ void __launch_bounds__(32) decode_warp_kernel(const KArgs a) {
  extern __shared__ uint64_t warp_dec[];
  const int64_t gt = (int64_t)blockIdx.x + a.task_base;
  if (gt >= a.ntiles) return;
  decode_tile_warp<C>(make_half(a.f0, gt, a.tl), a.M, warp_dec, threadIdx.x & 31, a.polys);
}

template <class C>
cudaError_t launch_warp(const KArgs& a, int, cudaStream_t s) {
  int64_t Lmax = tile_len(a.f0.n, a.tl.f) + a.tl.v1 + a.tl.v2;
  if (Lmax > a.f0.n) Lmax = a.f0.n;
  if (Lmax > kWarpSmemStages) return cudaErrorInvalidValue;  // the caller checks the window first
  const size_t smem = (size_t)Lmax * sizeof(uint64_t);
  const int64_t maxc = (int64_t)1 << 30;
  for (int64_t t0 = 0; t0 < a.ntiles; t0 += maxc) {
    KArgs b = a;
    b.task_base = t0;
    const int64_t n = a.ntiles - t0 < maxc ? a.ntiles - t0 : maxc;
    decode_warp_kernel<C><<<(unsigned)n, 32, smem, s>>>(b);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One warp per tile of a code known only at run time (any window length;
// decisions in the task's slab area, a.task_words words per tile).  A task
// is one tile; frames of a batch are found from the tile index.
template <class C>
__global__ void __launch_bounds__(256) decode_warp_gen_kernel(const KArgs a) {
  const int lane = threadIdx.x & 31;
  for_each_task(a, [&](int64_t t, int64_t slot) {
    const int64_t fi = (a.frames == nullptr) ? -1 : find_frame(a.tile0, a.nframes, t);
    const Frame& fr = (fi < 0) ? a.f0 : a.frames[fi];
    const int64_t b = (fi < 0) ? t : t - a.tile0[fi];
    decode_tile_warp_gen<C>(make_half(fr, b, a.tl), a.M, a.slab + slot * a.task_words, lane, a.polys);
  });
}

template <class C>
cudaError_t launch_warp_gen(const KArgs& a, int warps, cudaStream_t s) {
  return launch_tasks<decode_warp_gen_kernel<C>>(a, warps, s);
}

// Codes known only at run time: one warp per tile, max(S/32, 1) words of
// decisions per stage in the slab, windows rounded up to blocks of 32.
template <class C>
constexpr CodeEntry make_gen_entry() {
  return CodeEntry{C::K, C::BETA, {0, 0, 0, 0}, C::S >= 32 ? C::S / 32 : 1, 32, 1, 1, 1,
                   &resident_warps<decode_warp_gen_kernel<C>>, &launch_warp_gen<C>, &launch_warp_gen<C>};
}

// Warp task of the tile decoder with the parallel traceback.
template <class C>
__device__ __forceinline__ void pt_task(const KArgs& a, int64_t task, int64_t slot, int lane) {
  Half hw[2];
  int64_t gt[2], e1f[2];
  int Lw, mu;
  Slab sl;
  task_setup<C>(a, task, slot, lane, hw, gt, e1f, Lw, mu, sl);
  uint8_t* const st[2] = {hw[0].active ? a.pt_states + gt[0] * a.pt_nsub : nullptr,
                          hw[1].active ? a.pt_states + gt[1] * a.pt_nsub : nullptr};
  const PtParams pt{a.pt_f0, a.pt_rule, a.pt_seed};
  // word loads need every active tile's groups to start on 4-byte boundaries
  bool aligned = true;
#pragma unroll
  for (int h = 0; h < 2; h++)
    if (hw[h].active)
      aligned = aligned && ((reinterpret_cast<uintptr_t>(hw[h].llr) +
                             (uintptr_t)((hw[h].t0 - hw[h].start) * C::BETA)) % 4u == 0u);
  decode_pair_pt<C>(hw, e1f, Lw, mu, a.M, sl, a.tl.v2, pt, st, __all_sync(0xffffffffu, aligned));
}

template <class C>
__global__ void __maxnreg__(kMaxRegs) decode_tiles_pt_kernel(const KArgs a) {
  const int lane = threadIdx.x & 31;
  for_each_task(a, [&](int64_t task, int64_t slot) { pt_task<C>(a, task, slot, lane); });
}

template <class C>
cudaError_t launch_pt(const KArgs& a, int warps, cudaStream_t s) {
  return launch_tasks<decode_tiles_pt_kernel<C>>(a, warps, s);
}


template <class C>
MixKey key_of() {
  return MixKey{C::K, C::BETA, {C::poly(0), C::poly(1), C::poly(2), C::poly(3)}};
}

// Registers the decoders of every code of (K, beta) known only at run time:
// one warp per tile with decisions in the slab, and for K <= 7 the
// single-frame decoder with decisions in shared memory.
template <int K, int B>
void register_gen() {
  using C = GCode<K, B>;
  static const CodeEntry e = make_gen_entry<C>();
  register_generic(&e);
  if constexpr (K <= 7) register_warp_generic(K, B, &launch_warp<C>);
}

}  // namespace vit
