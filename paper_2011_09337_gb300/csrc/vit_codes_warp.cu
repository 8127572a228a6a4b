// Compiled warp-per-tile decoders (vit_warp.cuh) for the codes whose states
// fit one warp with at most two per lane (K <= 7).
#include "vit_internal.h"
#include "vit_warp.cuh"

namespace vit {
namespace {

// One warp (CTA) per tile of a single frame; the tile's decision words live
// in the CTA's shared memory (windows of at most kWarpSmemStages stages).
template <class C>
__global__ void __launch_bounds__(32) decode_warp_kernel(const KArgs a) {
  extern __shared__ uint64_t warp_dec[];
  const int64_t gt = (int64_t)blockIdx.x + a.task_base;
  if (gt >= a.ntiles) return;
  decode_tile_warp<C>(make_half(a.f0, gt, a.tl), a.M, warp_dec, threadIdx.x & 31);
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

template <class C>
MixKey key() {
  return MixKey{C::K, C::BETA, {C::poly(0), C::poly(1), C::poly(2), C::poly(3)}};
}

template <class C>
void reg() {
  register_warp(key<C>(), &launch_warp<C>);
}

struct Reg {
  Reg() {
    reg<Code<7, 2, 0171, 0133>>();
    reg<Code<7, 2, 0133, 0171>>();
    reg<Code<7, 3, 0133, 0171, 0165>>();
    reg<Code<3, 2, 07, 05>>();
    reg<Code<5, 2, 023, 035>>();
    reg<Code<4, 4, 013, 015, 017, 011>>();
    reg<Code<6, 2, 053, 046>>();
    reg<Code<5, 3, 025, 033, 037>>();
  }
} reg_;

}  // namespace
}  // namespace vit
