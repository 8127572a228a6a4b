// Compiled tile decoders with the parallel traceback (Sec. "Parallel
// Traceback Algorithm") for the codes whose states fit one lane.
#include "vit_kernels.cuh"

namespace vit {
namespace {

struct Reg {
  Reg() {
    register_pt(key_of<Code<7, 2, 0171, 0133>>(), &launch_pt<Code<7, 2, 0171, 0133>>);
    register_pt(key_of<Code<7, 2, 0133, 0171>>(), &launch_pt<Code<7, 2, 0133, 0171>>);
    register_pt(key_of<Code<7, 3, 0133, 0171, 0165>>(), &launch_pt<Code<7, 3, 0133, 0171, 0165>>);
    register_pt(key_of<Code<5, 2, 023, 035>>(), &launch_pt<Code<5, 2, 023, 035>>);
    register_pt(key_of<Code<3, 2, 07, 05>>(), &launch_pt<Code<3, 2, 07, 05>>);
  }
} reg_;

}  // namespace
}  // namespace vit
