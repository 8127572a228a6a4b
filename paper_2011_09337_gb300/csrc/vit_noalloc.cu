// vit_noalloc.cu -- an allocation-free variant of vit_decode_ws.
//
// Some callers cannot allocate device memory at decode time: a real-time
// receive loop that must never call cudaMalloc (it can synchronise the device
// and its latency is unbounded), a plugin that is handed only its input and
// output buffers by a host framework that owns every allocation, or a process
// whose memory budget is fixed after start-up.  vit_decode_noalloc serves
// them: its survivor scratch is a fixed device array compiled into this
// library, so the caller passes only inputs and outputs.
//
// The array is kVitNoallocScratchBytes (16 MiB) per GPU, held by every device
// that loads the library until the process exits.  Its device address is
// looked up once per device (cudaGetSymbolAddress, on the first call made
// with that device current) and cached; a cudaDeviceReset of that device
// rebuilds the module and invalidates the cached address, so the entry point
// must not be used on a device after it has been reset.  The caller's stream
// must belong to the current device (checked: the scratch address is the
// current device's).  Every call on a device shares the array; the decoder
// writes each scratch word before reading it in the same launch (survivor
// words of a stage before the traceback reads them, de-punctured LLRs before
// the decode launch reads them), so nothing needs clearing, but calls whose
// kernels overlap on the GPU (for example on two streams) race on it.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/vit.h"
#include "vit_internal.h"

namespace {

constexpr size_t kVitNoallocScratchBytes = (size_t)16 << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) uint8_t g_noalloc_scratch[kVitNoallocScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices];

// Device address of the scratch array for the current device.
int scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return vit::set_error(VIT_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return vit::set_error(VIT_EUNSUPPORTED, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return vit::set_error(VIT_ECUDA, "cudaGetSymbolAddress of the scratch array: %s", cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return VIT_OK;
}

}  // namespace

extern "C" {

int vit_decode_noalloc(const vit_code* c, const int8_t* llr, int64_t n, uint8_t* bits_out, vit_stream_t stream) {
  if (c == nullptr) return vit::set_error(VIT_EINVAL, "null code handle");
  if (n <= 0) return vit::set_error(VIT_EINVAL, "n must be >= 1");
  if (llr == nullptr || bits_out == nullptr) return vit::set_error(VIT_EINVAL, "null device pointer");
  if (c->mode == VIT_TERMINATED && n <= c->K - 1)
    return vit::set_error(VIT_EINVAL, "terminated frame shorter than its tail");
  const size_t need = vit_decode_workspace(c, n);
  if (need > kVitNoallocScratchBytes)
    return vit::set_error(VIT_EINVAL,
                          "frame needs %zu bytes of decoder scratch; the allocation-free entry point has %zu "
                          "(use vit_decode_ws or shorter frames)",
                          need, kVitNoallocScratchBytes);
  int cur = -1, sdev = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e == cudaSuccess) e = cudaStreamGetDevice((cudaStream_t)stream, &sdev);
  if (e != cudaSuccess) return vit::set_error(VIT_ECUDA, "stream device query: %s", cudaGetErrorString(e));
  if (sdev != cur)
    return vit::set_error(VIT_EINVAL, "stream belongs to device %d but device %d is current", sdev, cur);
  void* ws = nullptr;
  if (int r = scratch_address(&ws)) return r;
  return vit::decode_into(c, llr, n, bits_out, ws, kVitNoallocScratchBytes, (cudaStream_t)stream);
}

}  // extern "C"
