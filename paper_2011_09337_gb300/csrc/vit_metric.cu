// vit_metric.cu -- best-path metric of zero-terminated frames over float32
// LLRs and its gradient (not defined by the paper; the definitions follow the
// oracle):
//   hard (tau == 0):  M = max over 0-rooted, 0-terminated paths of sum_t delta_t
//                     (Eq. 2 / Eq. 3 in max-plus form); dM/dllr_t[b] = the +-1
//                     symbol (-1)^{c_t[b]} of the traced best path (Alg. 2).
//   soft (tau > 0):   M_tau = tau log sum_paths exp(sum_t delta_t / tau); the
//                     gradient is the posterior expectation of the +-1 symbols,
//                     from forward (alpha) and backward (beta) recursions.
// One warp per frame; states j = lane + 32 k (k < S/32) live in registers and
// are exchanged through shared memory each stage.  Metrics are renormalised
// by their per-stage maximum (offsets summed in fp64), and posteriors are
// normalised per stage, so fp32 keeps relative precision over long frames.
// The soft backward checkpoints alpha every C stages in the workspace and
// recomputes it inside each segment.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "../../include/vit.h"
#include "vit_internal.h"

namespace {

constexpr int kWarps = 4;
constexpr int kMaxS = 256;

struct MArgs {
  int K, beta, S, spl;  // spl = states per lane = S / 32 (>= 1; K >= 6) or 1 with lanes >= S idle
  uint32_t polys[4];
  const float* llr;     // [F][n][beta]
  int F;
  int64_t n;
  float tau;
  int C;
  float* metric;        // [F]
  const float* gmet;    // [F]
  float* grad;          // [F][n][beta]
  uint8_t* ws;
  int64_t ws_frame;     // bytes of workspace per frame
  int64_t nck;          // checkpoints per frame (soft)
};

__device__ __forceinline__ float lse2(float a, float b, float tau) {
  const float m = fmaxf(a, b);
  if (m == -INFINITY) return -INFINITY;
  return m + tau * log1pf(__expf(-fabsf(a - b) / tau));
}

__device__ __forceinline__ float warp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// delta for register word R (Eq. 2) from the stage's LLRs
__device__ __forceinline__ float bm(const uint8_t* aout, int R, const float* l, int beta) {
  const uint32_t o = aout[R];
  float d = 0.f;
  #pragma unroll
  for (int b = 0; b < 4; b++)
    if (b < beta) d += ((o >> b) & 1u) ? -l[b] : l[b];
  return d;
}

struct Smem {
  uint8_t aout[2 * kMaxS];
  float buf[kWarps][2][kMaxS];
  float lw[kWarps][4];
  uint16_t path[kWarps][64];
};

__device__ void setup_aout(Smem& sm, const MArgs& a) {
  for (int R = threadIdx.x; R < (1 << a.K); R += blockDim.x) {
    uint32_t o = 0;
    #pragma unroll
    for (int b = 0; b < 4; b++)
      if (b < a.beta) o |= (uint32_t)(__popc(a.polys[b] & (uint32_t)R) & 1) << b;
    sm.aout[R] = (uint8_t)o;
  }
  __syncthreads();
}

// One forward stage over the SPL states of this lane (SPL = a.spl, a
// template parameter so the per-lane arrays stay in registers): reads cur,
// writes nxt (normalised), returns the normaliser.  hard: also the decision
// ballots.
template <int SPL>
__device__ float fwd_stage(const MArgs& a, const Smem& sm, const float* cur, float* nxt, const float* l, int lane,
                           uint32_t* dec) {
  const int S = a.S;
  float v[SPL];
  float mx = -INFINITY;
#pragma unroll
  for (int k = 0; k < SPL; k++) {
    const int j = lane + 32 * k;
    float r = -INFINITY;
    bool d = false;
    if (j < S) {
      const int i0 = (2 * j) & (S - 1), i1 = i0 | 1;
      const float x0 = cur[i0] + bm(sm.aout, 2 * j, l, a.beta);
      const float x1 = cur[i1] + bm(sm.aout, 2 * j + 1, l, a.beta);
      if (a.tau > 0.f) {
        r = lse2(x0, x1, a.tau);
      } else {
        d = x1 > x0;  // ties keep the lower predecessor
        r = d ? x1 : x0;
      }
    }
    if (dec) dec[k] = __ballot_sync(0xffffffffu, d);
    v[k] = r;
    mx = fmaxf(mx, r);
  }
  mx = warp_max(mx);
  if (mx == -INFINITY) mx = 0.f;
#pragma unroll
  for (int k = 0; k < SPL; k++) {
    const int j = lane + 32 * k;
    if (j < S) nxt[j] = v[k] - mx;
  }
  __syncwarp();
  return mx;
}

template <int SPL>
__global__ void __launch_bounds__(kWarps * 32) metric_fwd_kernel(const MArgs a) {
  __shared__ Smem sm;
  setup_aout(sm, a);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int f = blockIdx.x * kWarps + w;
  if (f >= a.F) return;
  const int S = a.S;
  float* b0 = sm.buf[w][0];
  float* b1 = sm.buf[w][1];
  for (int j = lane; j < S; j += 32) b0[j] = (j == 0) ? 0.f : -INFINITY;
  __syncwarp();
  const float* llr = a.llr + (int64_t)f * a.n * a.beta;
  uint8_t* ws = a.ws + (int64_t)f * a.ws_frame;
  double off = 0.0;
  for (int64_t t = 0; t < a.n; t++) {
    float l[4];
    #pragma unroll
    for (int b = 0; b < 4; b++)
      if (b < a.beta) l[b] = llr[t * a.beta + b];
    const float* cur = (t & 1) ? b1 : b0;
    float* nxt = (t & 1) ? b0 : b1;
    if (a.tau > 0.f) {
      if (t % a.C == 0) {  // checkpoint of the metrics entering stage t
        float* ck = (float*)ws + (t / a.C) * S;
        for (int j = lane; j < S; j += 32) ck[j] = cur[j];
      }
      off += (double)fwd_stage<SPL>(a, sm, cur, nxt, l, lane, nullptr);
    } else {
      uint32_t dec[SPL];
      off += (double)fwd_stage<SPL>(a, sm, cur, nxt, l, lane, dec);
      uint32_t* dw = (uint32_t*)ws + t * ((S + 31) / 32);
      if (lane < (S + 31) / 32) {
        uint32_t x = 0;
#pragma unroll
        for (int k = 0; k < SPL; k++)
          if (k == lane) x = dec[k];
        dw[lane] = (S < 32) ? (x & ((1u << S) - 1u)) : x;
      }
    }
    __syncwarp();
  }
  const float* fin = (a.n & 1) ? b1 : b0;
  if (lane == 0) a.metric[f] = (float)(off + (double)fin[0]);
}

// hard backward: traceback from state 0 through the stored decisions, then the
// +-1 branch symbols times the upstream gradient
__global__ void __launch_bounds__(kWarps * 32) metric_bwd_hard_kernel(const MArgs a) {
  __shared__ Smem sm;
  setup_aout(sm, a);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int f = blockIdx.x * kWarps + w;
  if (f >= a.F) return;
  const int S = a.S;
  const int nw = (S + 31) / 32;
  const uint32_t* dw = (const uint32_t*)(a.ws + (int64_t)f * a.ws_frame);
  const float g = a.gmet[f];
  float* grad = a.grad + (int64_t)f * a.n * a.beta;
  int j = 0;
  // chunks of 64 stages: lane 0 walks them, then all lanes write the gradient
  for (int64_t hi = a.n; hi > 0; hi -= 64) {
    const int64_t lo = hi - 64 > 0 ? hi - 64 : 0;
    if (lane == 0) {
      for (int64_t t = hi - 1; t >= lo; t--) {
        const uint32_t word = dw[t * nw + (j >> 5)];
        const int d = (int)((word >> (j & 31)) & 1u);
        const int R = 2 * j + d;
        sm.path[w][t - lo] = (uint16_t)R;
        j = R & (S - 1);
      }
    }
    __syncwarp();
    for (int64_t t = lo + lane; t < hi; t += 32) {
      const uint32_t o = sm.aout[sm.path[w][t - lo]];
      #pragma unroll
      for (int b = 0; b < 4; b++)
        if (b < a.beta) grad[t * a.beta + b] = ((o >> b) & 1u) ? -g : g;
    }
    __syncwarp();
  }
}

// soft backward: beta recursion from the end; alpha recomputed per segment
template <int SPL>
__global__ void __launch_bounds__(kWarps * 32) metric_bwd_soft_kernel(const MArgs a) {
  __shared__ Smem sm;
  setup_aout(sm, a);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int f = blockIdx.x * kWarps + w;
  if (f >= a.F) return;
  const int S = a.S, K = a.K;
  const float tau = a.tau;
  const float g = a.gmet[f];
  const float* llr = a.llr + (int64_t)f * a.n * a.beta;
  float* grad = a.grad + (int64_t)f * a.n * a.beta;
  float* ck = (float*)(a.ws + (int64_t)f * a.ws_frame);
  float* seg = ck + a.nck * S;  // C + 1 rows of alpha for the current segment
  float* bb0 = sm.buf[w][0];
  float* bb1 = sm.buf[w][1];
  for (int j = lane; j < S; j += 32) bb0[j] = (j == 0) ? 0.f : -INFINITY;  // beta after the last stage
  __syncwarp();
  int cur = 0;
  for (int64_t s = a.nck - 1; s >= 0; s--) {
    const int64_t t0 = s * a.C;
    const int64_t t1 = (t0 + a.C < a.n) ? t0 + a.C : a.n;
    // recompute alpha rows t0..t1-1 (row r = metrics entering stage t0 + r)
    for (int j = lane; j < S; j += 32) seg[j] = ck[s * S + j];
    __syncwarp();
    for (int64_t t = t0; t < t1 - 1; t++) {
      float l[4];
      #pragma unroll
      for (int b = 0; b < 4; b++)
        if (b < a.beta) l[b] = llr[t * a.beta + b];
      fwd_stage<SPL>(a, sm, seg + (t - t0) * S, seg + (t - t0 + 1) * S, l, lane, nullptr);
    }
    __syncwarp();
    for (int64_t t = t1 - 1; t >= t0; t--) {
      float l[4];
      #pragma unroll
      for (int b = 0; b < 4; b++)
        if (b < a.beta) l[b] = llr[t * a.beta + b];
      const float* al = seg + (t - t0) * S;   // alpha entering stage t
      const float* be = cur ? bb1 : bb0;       // beta leaving stage t
      float* bn = cur ? bb0 : bb1;
      float u[SPL][2], p[SPL][2];
      float mx = -INFINITY, bmx = -INFINITY;
#pragma unroll
      for (int k = 0; k < SPL; k++) {
        const int i = lane + 32 * k;
        for (int in = 0; in < 2; in++) {
          u[k][in] = -INFINITY;
          p[k][in] = -INFINITY;
        }
        if (i >= S) continue;
        for (int in = 0; in < 2; in++) {
          const int R = (in << (K - 1)) | i;
          const int j = R >> 1;
          u[k][in] = bm(sm.aout, R, l, a.beta) + be[j];
          p[k][in] = al[i] + u[k][in];
          mx = fmaxf(mx, p[k][in]);
        }
        bmx = fmaxf(bmx, lse2(u[k][0], u[k][1], tau));
      }
      mx = warp_max(mx);
      bmx = warp_max(bmx);
      if (bmx == -INFINITY) bmx = 0.f;
      float z = 0.f, gb[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int k = 0; k < SPL; k++) {
        const int i = lane + 32 * k;
        if (i >= S) continue;
        for (int in = 0; in < 2; in++) {
          const float q = (p[k][in] == -INFINITY) ? 0.f : __expf((p[k][in] - mx) / tau);
          z += q;
          const uint32_t o = sm.aout[(in << (K - 1)) | i];
          #pragma unroll
          for (int b = 0; b < 4; b++)
            if (b < a.beta) gb[b] += ((o >> b) & 1u) ? -q : q;
        }
        bn[i] = lse2(u[k][0], u[k][1], tau) - bmx;
      }
      z = warp_sum(z);
      #pragma unroll
      for (int b = 0; b < 4; b++)
        if (b < a.beta) gb[b] = warp_sum(gb[b]);
      if (lane < a.beta) {
        float gv = 0.f;
        for (int b = 0; b < a.beta; b++)
          if (b == lane) gv = gb[b];
        grad[t * a.beta + lane] = g * gv / z;
      }
      __syncwarp();
      cur ^= 1;
    }
  }
}

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

size_t frame_bytes(const vit_code* c, int64_t n, float tau, int C) {
  const int S = 1 << (c->K - 1);
  if (tau > 0.f) {
    const int64_t nck = (n + C - 1) / C;
    return align_up((size_t)(nck + C) * S * sizeof(float));
  }
  return align_up((size_t)n * ((S + 31) / 32) * sizeof(uint32_t));
}

int fill(MArgs& a, const vit_code* c, int F, int64_t n, float tau, int C) {
  if (c == nullptr) return vit::set_error(VIT_EINVAL, "null code handle");
  if (F <= 0 || n < c->K) return vit::set_error(VIT_EINVAL, "need F >= 1 and n >= K stages");
  if (!(tau >= 0.f) || !isfinite(tau)) return vit::set_error(VIT_EINVAL, "tau must be finite and >= 0");
  if (tau > 0.f && (C < 2 || C > 4096)) return vit::set_error(VIT_EINVAL, "checkpoint interval C in [2, 4096]");
  if (c->period) return vit::set_error(VIT_EUNSUPPORTED, "path metrics take de-punctured LLRs");
  memset(&a, 0, sizeof a);
  a.K = c->K;
  a.beta = c->beta;
  a.S = 1 << (c->K - 1);
  a.spl = a.S >= 32 ? a.S / 32 : 1;
  for (int b = 0; b < 4; b++) a.polys[b] = c->polys[b];
  a.F = F;
  a.n = n;
  a.tau = tau;
  a.C = tau > 0.f ? C : 1;
  a.nck = tau > 0.f ? (n + C - 1) / C : 0;
  a.ws_frame = (int64_t)frame_bytes(c, n, tau, C);
  return VIT_OK;
}

}  // namespace

extern "C" {

size_t vit_metric_workspace(const vit_code* c, int nframes, int64_t n, float tau, int C) {
  MArgs a;
  if (fill(a, c, nframes, n, tau, C) != VIT_OK) return 0;
  return (size_t)nframes * (size_t)a.ws_frame;
}

int vit_metric_fwd(const vit_code* c, const float* llr, int nframes, int64_t n, float tau, int C, float* metric_out,
                   void* ws, size_t ws_bytes, vit_stream_t stream) {
  MArgs a;
  if (int r = fill(a, c, nframes, n, tau, C)) return r;
  if (llr == nullptr || metric_out == nullptr || ws == nullptr) return vit::set_error(VIT_EINVAL, "null pointer");
  if (((uintptr_t)ws % kAlign) != 0) return vit::set_error(VIT_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < (size_t)nframes * (size_t)a.ws_frame) return vit::set_error(VIT_EINVAL, "workspace too small");
  a.llr = llr;
  a.metric = metric_out;
  a.ws = (uint8_t*)ws;
  const unsigned grid = (unsigned)((nframes + kWarps - 1) / kWarps);
  cudaStream_t s = (cudaStream_t)stream;
  switch (a.spl) {
    case 1: metric_fwd_kernel<1><<<grid, kWarps * 32, 0, s>>>(a); break;
    case 2: metric_fwd_kernel<2><<<grid, kWarps * 32, 0, s>>>(a); break;
    case 4: metric_fwd_kernel<4><<<grid, kWarps * 32, 0, s>>>(a); break;
    default: metric_fwd_kernel<8><<<grid, kWarps * 32, 0, s>>>(a); break;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return vit::set_error(VIT_ECUDA, "metric forward launch: %s", cudaGetErrorString(e));
  return VIT_OK;
}

int vit_metric_bwd(const vit_code* c, const float* llr, const float* grad_metric, int nframes, int64_t n, float tau,
                   int C, const void* ws, size_t ws_bytes, float* grad_llr, vit_stream_t stream) {
  MArgs a;
  if (int r = fill(a, c, nframes, n, tau, C)) return r;
  if (llr == nullptr || grad_metric == nullptr || ws == nullptr || grad_llr == nullptr)
    return vit::set_error(VIT_EINVAL, "null pointer");
  if (((uintptr_t)ws % kAlign) != 0) return vit::set_error(VIT_EINVAL, "workspace must be 256-byte aligned");
  if (ws_bytes < (size_t)nframes * (size_t)a.ws_frame) return vit::set_error(VIT_EINVAL, "workspace too small");
  a.llr = llr;
  a.gmet = grad_metric;
  a.grad = grad_llr;
  a.ws = (uint8_t*)const_cast<void*>(ws);
  const unsigned grid = (unsigned)((nframes + kWarps - 1) / kWarps);
  cudaStream_t s = (cudaStream_t)stream;
  if (tau > 0.f) {
    switch (a.spl) {
      case 1: metric_bwd_soft_kernel<1><<<grid, kWarps * 32, 0, s>>>(a); break;
      case 2: metric_bwd_soft_kernel<2><<<grid, kWarps * 32, 0, s>>>(a); break;
      case 4: metric_bwd_soft_kernel<4><<<grid, kWarps * 32, 0, s>>>(a); break;
      default: metric_bwd_soft_kernel<8><<<grid, kWarps * 32, 0, s>>>(a); break;
    }
  } else
    metric_bwd_hard_kernel<<<grid, kWarps * 32, 0, (cudaStream_t)stream>>>(a);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return vit::set_error(VIT_ECUDA, "metric backward launch: %s", cudaGetErrorString(e));
  return VIT_OK;
}

}  // extern "C"
