// Compiled decoders: short codes (K = 3..6), including a beta = 4 code and a
// code whose generators lack the first and last taps (no butterfly symmetry).
#include "vit_internal.h"
namespace vit {
namespace {
using C1 = Code<3, 2, 07, 05>;
using C2 = Code<5, 2, 023, 035>;
using C3 = Code<4, 4, 013, 015, 017, 011>;
using C4 = Code<6, 2, 053, 046>;
using C5 = Code<5, 3, 025, 033, 037>;
struct Reg {
  Reg() {
    static const CodeEntry e[] = {make_entry<C1>(), make_entry<C2>(), make_entry<C3>(), make_entry<C4>(),
                                  make_entry<C5>()};
    register_codes(e, 5);
  }
} reg_;
}  // namespace
}  // namespace vit
