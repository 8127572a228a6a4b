// Spread tile decoders of the K=7 rate-1/2 codes (171,133) and (133,171):
// four lanes per tile pair, 16 of the 64 states per lane in the rotating
// slot map of the K=8, 9 decoders, so a warp task holds 16 tiles instead of
// 64.  Single frames with too few tiles to fill the GPU with 64-tile tasks
// (a 2^24-bit stream at f = 1024, or a 2^26-bit stream at f = 2048) get four
// times as many warps.
#include "vit_internal.h"
namespace vit {
namespace {
using S1 = Code<7, 2, 0171, 0133, 0, 0, 16>;
using S2 = Code<7, 2, 0133, 0171, 0, 0, 16>;
template <class C>
MixKey key() {
  return MixKey{C::K, C::BETA, {C::poly(0), C::poly(1), C::poly(2), C::poly(3)}};
}
// single frames only (batches use the codes' own tile decoders): the
// word-load kernel serves both launch slots
template <class C>
constexpr CodeEntry spread_entry() {
  return CodeEntry{C::K, C::BETA, {C::poly(0), C::poly(1), C::poly(2), C::poly(3)}, C::WORDS, C::U, 64 / C::G, 32, 0,
                   &resident_warps<decode_tiles_kernel<C, true>>, &launch_decode<C>, &launch_decode<C>};
}
struct Reg {
  Reg() {
    static const CodeEntry e1 = spread_entry<S1>(), e2 = spread_entry<S2>();
    register_spread(key<S1>(), &e1);
    register_spread(key<S2>(), &e2);
  }
} reg_;
}  // namespace
}  // namespace vit
