// Compiled tile decoders with the parallel traceback (Sec. "Parallel
// Traceback Algorithm") for the codes whose states fit one lane.
#include "vit_internal.h"
#include "vit_pt.cuh"

namespace vit {
namespace {

template <class C>
__global__ void __maxnreg__(kMaxRegs) decode_tiles_pt_kernel(const KArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t task = a.task_base + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (task >= a.ntasks) return;  // warp-uniform
  Half hw[2];
  int64_t gt[2], e1f[2];
  int Lw, mu;
  Slab sl;
  task_setup<C>(a, task, lane, hw, gt, e1f, Lw, mu, sl);
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
cudaError_t launch_pt(const KArgs& a, int warps, cudaStream_t s) {
  return launch_tasks<decode_tiles_pt_kernel<C>>(a, warps, s);
}

template <class C>
MixKey key() {
  return MixKey{C::K, C::BETA, {C::poly(0), C::poly(1), C::poly(2), C::poly(3)}};
}

struct Reg {
  Reg() {
    register_pt(key<Code<7, 2, 0171, 0133>>(), &launch_pt<Code<7, 2, 0171, 0133>>);
    register_pt(key<Code<7, 2, 0133, 0171>>(), &launch_pt<Code<7, 2, 0133, 0171>>);
    register_pt(key<Code<7, 3, 0133, 0171, 0165>>(), &launch_pt<Code<7, 3, 0133, 0171, 0165>>);
    register_pt(key<Code<5, 2, 023, 035>>(), &launch_pt<Code<5, 2, 023, 035>>);
    register_pt(key<Code<3, 2, 07, 05>>(), &launch_pt<Code<3, 2, 07, 05>>);
  }
} reg_;

}  // namespace
}  // namespace vit
