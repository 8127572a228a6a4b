// Compiled decoders: K=7 rate-1/2 codes (171,133 is the code of Fig. 1).
#include "vit_internal.h"
namespace vit {
namespace {
using C1 = Code<7, 2, 0171, 0133>;
using C2 = Code<7, 2, 0133, 0171>;
struct Reg {
  Reg() {
    static const CodeEntry e[] = {make_entry<C1>(), make_entry<C2>()};
    register_codes(e, 2);
  }
} reg_;
}  // namespace
}  // namespace vit
