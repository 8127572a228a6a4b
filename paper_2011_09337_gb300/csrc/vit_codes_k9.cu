// Compiled decoders: K=9 rate-1/2 code (561,753), four lanes per tile pair.
#include "vit_internal.h"
namespace vit {
namespace {
using C1 = Code<9, 2, 0561, 0753>;
struct Reg {
  Reg() {
    static const CodeEntry e[] = {make_entry<C1>()};
    register_codes(e, 1);
  }
} reg_;
}  // namespace
}  // namespace vit
