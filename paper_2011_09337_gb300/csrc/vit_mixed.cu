// Compiled persistent two-code decoder: K=7 rate-1/3 (133,171,165) with
// K=9 rate-1/2 (561,753) tasks in one launch.
#include "vit_internal.h"
namespace vit {
namespace {
using A = Code<7, 3, 0133, 0171, 0165>;
using B = Code<9, 2, 0561, 0753>;
struct Reg {
  Reg() {
    register_mixed(MixKey{A::K, A::BETA, {A::poly(0), A::poly(1), A::poly(2), A::poly(3)}},
                   MixKey{B::K, B::BETA, {B::poly(0), B::poly(1), B::poly(2), B::poly(3)}}, &launch_mixed<A, B>);
  }
} reg_;
}  // namespace
}  // namespace vit
