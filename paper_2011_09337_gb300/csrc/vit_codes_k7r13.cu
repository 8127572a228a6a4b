// Compiled decoders: K=7 rate-1/3 code (133,171,165).
#include "vit_internal.h"
namespace vit {
namespace {
using C1 = Code<7, 3, 0133, 0171, 0165>;
struct Reg {
  Reg() {
    static const CodeEntry e[] = {make_entry<C1>()};
    register_codes(e, 1);
  }
} reg_;
}  // namespace
}  // namespace vit
