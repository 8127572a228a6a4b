// Decoders for codes known only at run time: every K in [3, 9] and rate
// 1/2, 1/3, 1/4 with any generators, one warp per tile with the branch
// patterns formed from the generators (decode_tile_warp_gen, and for K <= 7
// the single-frame decode_tile_warp).  Codes with a compiled kernel use that
// kernel instead.
#include "vit_kernels.cuh"

namespace vit {
namespace {
struct Reg {
  Reg() {
    register_gen<3, 2>();
    register_gen<3, 3>();
    register_gen<3, 4>();
    register_gen<4, 2>();
    register_gen<4, 3>();
    register_gen<4, 4>();
    register_gen<5, 2>();
    register_gen<5, 3>();
    register_gen<5, 4>();
    register_gen<6, 2>();
    register_gen<6, 3>();
    register_gen<6, 4>();
    register_gen<7, 2>();
    register_gen<7, 3>();
    register_gen<7, 4>();
    register_gen<8, 2>();
    register_gen<8, 3>();
    register_gen<8, 4>();
    register_gen<9, 2>();
    register_gen<9, 3>();
    register_gen<9, 4>();
  }
} reg_;
}  // namespace
}  // namespace vit
