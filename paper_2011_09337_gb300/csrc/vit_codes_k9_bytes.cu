// Byte-load tile decoder of the K=9 rate-1/2 code (561,753), registered by
// vit_codes_k9.cu (batches of short frames use it).
#include "vit_internal.h"
namespace vit {
cudaError_t launch_k9_561_753_bytes(const KArgs& a, int warps, cudaStream_t s) {
  return launch_decode_bytes<Code<9, 2, 0561, 0753>>(a, warps, s);
}
}  // namespace vit
