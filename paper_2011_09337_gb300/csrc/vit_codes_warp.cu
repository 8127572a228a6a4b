// Compiled warp-per-tile decoders (vit_warp.cuh) for the codes whose states
// fit one warp with at most two per lane (K <= 7).
#include "vit_kernels.cuh"

namespace vit {
namespace {

template <class C>
void reg() {
  register_warp(key_of<C>(), &launch_warp<C>);
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
