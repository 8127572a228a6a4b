// Compiled decoders: K=9 rate-1/2 code (561,753), four lanes per tile pair.
// The word-load kernel is compiled here and the byte-load kernel in
// vit_codes_k9_bytes.cu, so that the two large kernels build in parallel.
#include "vit_internal.h"
namespace vit {
cudaError_t launch_k9_561_753_bytes(const KArgs& a, int warps, cudaStream_t s);
namespace {
using C1 = Code<9, 2, 0561, 0753>;
struct Reg {
  Reg() {
    static const CodeEntry e[] = {CodeEntry{C1::K, C1::BETA, {C1::poly(0), C1::poly(1), C1::poly(2), C1::poly(3)},
                                            C1::WORDS, C1::U, 64 / C1::G, 32, 0,
                                            &resident_warps<decode_tiles_kernel<C1, true>>, &launch_decode<C1>,
                                            &launch_k9_561_753_bytes}};
    register_codes(e, 1);
  }
} reg_;
}  // namespace
}  // namespace vit
