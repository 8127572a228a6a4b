// vit_metric.cu -- best-path metric of zero-terminated frames over float32
// LLRs and its gradient (not defined by the paper; the definitions follow the
// oracle):
//   hard (tau == 0):  M = max over 0-rooted, 0-terminated paths of sum_t delta_t
//                     (Eq. 2 / Eq. 3 in max-plus form); dM/dllr_t[b] = the +-1
//                     symbol (-1)^{c_t[b]} of the traced best path (Alg. 2).
//   soft (tau > 0):   M_tau = tau log sum_paths exp(sum_t delta_t / tau); the
//                     gradient is the posterior expectation of the +-1 symbols,
//                     from forward (alpha) and backward (beta) recursions.
// One warp per frame, laid out like the warp-per-tile decoders: lane l holds
// the metrics of states R l + r (R = S / 32 for S >= 32, else one state per
// lane l < S), the two predecessors of a state come from lanes 2l and 2l + 1
// (mod 32) by shuffle, and each lane forms its branch patterns (Eq. 1) once.
// The LLRs of 32 stages arrive with one coalesced load (lane k holds stage
// i0 + k) and reach each stage by shuffle.  Every 32 stages the metrics are
// re-referenced to state 0's (the offsets summed in fp64), so fp32 keeps
// its precision over long frames.  Hard decisions are ballots (bit l of word
// r = state R l + r), stored per block of 32 stages.  The soft backward
// checkpoints alpha every C stages, recomputes a segment's alphas from its
// checkpoint, and runs the beta recursion with lanes holding predecessor
// states; the per-stage gradient sums go through shared memory, one stage per
// lane, 32 stages at a time.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "../../include/vit.h"
#include "vit_internal.h"

namespace {

constexpr int kWarps = 4;      // frames per CTA (forward, hard backward)
constexpr int kWarpsSoft = 2;  // frames per CTA of the soft backward (its shared reduction buffer)

struct MArgs {
  int K, beta, S, spl;  // spl: states per lane (R)
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

// output pattern of register word Rw (Eq. 1)
__device__ __forceinline__ uint32_t aout_m(const MArgs& a, uint32_t Rw) {
  uint32_t o = 0;
#pragma unroll
  for (int b = 0; b < 4; b++)
    if (b < a.beta) o |= (uint32_t)(__popc(a.polys[b] & Rw) & 1) << b;
  return o;
}

// signed branch metric sum_b (-1)^{c_b} l_b
__device__ __forceinline__ float bm4(const float (&s)[4], const float (&l)[4]) {
  return s[0] * l[0] + s[1] * l[1] + s[2] * l[2] + s[3] * l[3];
}

__device__ __forceinline__ void signs(const MArgs& a, uint32_t c, float (&s)[4]) {
#pragma unroll
  for (int b = 0; b < 4; b++) s[b] = (b < a.beta) ? (((c >> b) & 1u) ? -1.f : 1.f) : 0.f;
}

// tau log(exp(x/tau) + exp(y/tau)) = max + tau log(1 + e), e = exp(-|x-y|/tau)
// in (0, 1]: both transcendentals are the hardware approximations (1 + e
// lies in [1, 2], where the logarithm's absolute error is ~1e-7)
__device__ __forceinline__ float lse2(float x, float y, float tau, float inv_tau) {
  const float mx = fmaxf(x, y);
  if (mx == -INFINITY) return -INFINITY;
  return mx + tau * __logf(1.f + __expf(-fabsf(x - y) * inv_tau));
}

// Lane-side constants of the forward layout (lane l holds successor states
// j = R l + r; predecessors 2j, 2j + 1 mod S).
template <int R>
struct FwdLane {
  float sA[R][4], sB[R][4];  // branch signs from 2j (A) and 2j + 1 (B)
  int la, lb;                // source lanes of the predecessors
  bool live;
  __device__ void init(const MArgs& a, int lane) {
    live = R * lane < a.S;
#pragma unroll
    for (int r = 0; r < R; r++) {
      const uint32_t j = (uint32_t)(R * lane + r);
      signs(a, aout_m(a, 2u * j), sA[r]);
      signs(a, aout_m(a, 2u * j + 1u), sB[r]);
    }
    if (R == 1) {
      la = (2 * lane) & (a.S - 1);
      lb = (2 * lane + 1) & (a.S - 1);
    } else {
      la = (2 * lane) & 31;
      lb = (2 * lane + 1) & 31;
    }
  }
};

// One forward stage (Eq. 3 in max-plus or log-sum-exp form) on the lane's
// metrics m; hard: returns the ballots of the decisions in bal.
template <int R, bool SOFT>
__device__ __forceinline__ void fwd_step(float (&m)[R], const float (&l)[4], const FwdLane<R>& fl, float tau,
                                         float inv_tau, uint32_t (&bal)[R]) {
  float qa[R], qb[R];
#pragma unroll
  for (int r = 0; r < R; r++) {
    qa[r] = __shfl_sync(0xffffffffu, m[r], fl.la);
    qb[r] = __shfl_sync(0xffffffffu, m[r], fl.lb);
  }
#pragma unroll
  for (int r = 0; r < R; r++) {
    float p0, p1;
    if constexpr (R == 1) {
      p0 = qa[0];
      p1 = qb[0];
    } else {
      p0 = (2 * r < R) ? qa[2 * r] : qb[2 * r - R];
      p1 = (2 * r < R) ? qa[2 * r + 1] : qb[2 * r - R + 1];
    }
    const float x0 = p0 + bm4(fl.sA[r], l), x1 = p1 + bm4(fl.sB[r], l);
    if constexpr (SOFT) {
      m[r] = lse2(x0, x1, tau, inv_tau);
      bal[r] = 0u;
    } else {
      const bool d = x1 > x0;  // ties keep the lower predecessor
      bal[r] = __ballot_sync(0xffffffffu, fl.live && d);
      m[r] = d ? x1 : x0;
    }
  }
}

// The frame's LLRs of stages [i0, i0 + 32): lane k loads stage i0 + k.
__device__ __forceinline__ void load_block(const MArgs& a, const float* llr, int64_t i0, int lane, float (&lv)[4]) {
#pragma unroll
  for (int b = 0; b < 4; b++) lv[b] = (b < a.beta && i0 + lane < a.n) ? llr[(i0 + lane) * a.beta + b] : 0.f;
}

__device__ __forceinline__ void stage_llr(const float (&lv)[4], int k, float (&l)[4]) {
#pragma unroll
  for (int b = 0; b < 4; b++) l[b] = __shfl_sync(0xffffffffu, lv[b], k);
}

template <int R, bool SOFT>
__global__ void __launch_bounds__(kWarps * 32) metric_fwd_kernel(const MArgs a) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int f = blockIdx.x * kWarps + w;
  if (f >= a.F) return;
  const int S = a.S;
  const float tau = a.tau, inv_tau = SOFT ? 1.f / a.tau : 0.f;
  FwdLane<R> fl;
  fl.init(a, lane);
  float m[R];
#pragma unroll
  for (int r = 0; r < R; r++) m[r] = (R * lane + r == 0) ? 0.f : -INFINITY;  // 0-rooted
  const float* llr = a.llr + (int64_t)f * a.n * a.beta;
  uint8_t* ws = a.ws + (int64_t)f * a.ws_frame;
  double off = 0.0;
  int64_t next_ck = 0;  // next checkpointed stage (soft)
  float* ck = (float*)ws;
  for (int64_t i0 = 0; i0 < a.n; i0 += 32) {
    float lv[4];
    load_block(a, llr, i0, lane, lv);
    const int cnt = (a.n - i0 < 32) ? (int)(a.n - i0) : 32;
    uint32_t keep[R];
#pragma unroll
    for (int r = 0; r < R; r++) keep[r] = 0u;
    for (int k = 0; k < cnt; k++) {
      const int64_t t = i0 + k;
      if (SOFT && t == next_ck) {  // checkpoint of the metrics entering stage t
#pragma unroll
        for (int r = 0; r < R; r++)
          if (fl.live) ck[R * lane + r] = m[r];
        ck += S;
        next_ck += a.C;
      }
      float l[4];
      stage_llr(lv, k, l);
      uint32_t bal[R];
      fwd_step<R, SOFT>(m, l, fl, tau, inv_tau, bal);
      if (!SOFT) {
#pragma unroll
        for (int r = 0; r < R; r++) keep[r] = (lane == k) ? bal[r] : keep[r];
      }
    }
    if (!SOFT && i0 + lane < a.n) {
      uint32_t* dw = (uint32_t*)ws + (i0 + lane) * R;
#pragma unroll
      for (int r = 0; r < R; r++) dw[r] = (S < 32) ? (keep[r] & ((1u << S) - 1u)) : keep[r];
    }
    // re-reference to state 0 (lane 0, register 0; reachable from stage 1 on)
    const float ref = __shfl_sync(0xffffffffu, m[0], 0);
#pragma unroll
    for (int r = 0; r < R; r++) m[r] -= ref;
    off += (double)ref;
  }
  if (lane == 0) a.metric[f] = (float)(off + (double)m[0]);
}

// hard backward: traceback from state 0 through the stored decisions (every
// lane follows the same state; lane k holds stage b0 + k's words), then the
// +-1 branch symbols times the upstream gradient, one stage per lane
template <int R>
__global__ void __launch_bounds__(kWarps * 32) metric_bwd_hard_kernel(const MArgs a) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int f = blockIdx.x * kWarps + w;
  if (f >= a.F) return;
  const uint32_t S = (uint32_t)a.S;
  const uint32_t* dw = (const uint32_t*)(a.ws + (int64_t)f * a.ws_frame);
  const float g = a.gmet[f];
  float* grad = a.grad + (int64_t)f * a.n * a.beta;
  uint32_t J = 0;  // state after the last stage (terminated)
  uint32_t wn[R];   // the next (lower) block's words, loaded one block ahead
  {
    const int64_t my = ((a.n - 1) / 32) * 32 + lane;
#pragma unroll
    for (int r = 0; r < R; r++) wn[r] = (my < a.n) ? dw[my * R + r] : 0u;
  }
  for (int64_t b0 = ((a.n - 1) / 32) * 32; b0 >= 0; b0 -= 32) {
    const int64_t my = b0 + lane;
    uint32_t wv[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
      wv[r] = wn[r];
      wn[r] = (b0 >= 32) ? dw[(b0 - 32 + lane) * R + r] : 0u;
    }
    const int top = (a.n - b0 < 32) ? (int)(a.n - b0) : 32;
    uint32_t myR = 0;
    for (int k = top - 1; k >= 0; k--) {
      uint32_t sel = wv[0];
#pragma unroll
      for (int r = 1; r < R; r++) sel = ((J & (uint32_t)(R - 1)) == (uint32_t)r) ? wv[r] : sel;
      const uint32_t word = __shfl_sync(0xffffffffu, sel, k);
      const uint32_t d = (word >> (J / R)) & 1u;
      const uint32_t Rw = 2u * J + d;  // the branch's register word: predecessor (Rw mod S) -> J
      myR = (lane == k) ? Rw : myR;
      J = Rw & (S - 1u);
    }
    if (my < a.n) {
      const uint32_t o = aout_m(a, myR);
#pragma unroll
      for (int b = 0; b < 4; b++)
        if (b < a.beta) grad[my * a.beta + b] = ((o >> b) & 1u) ? -g : g;
    }
  }
}

// soft backward: beta recursion from the end with lanes holding predecessor
// states i = R l + r (successors i >> 1 and (i >> 1) + S/2, from lanes l >> 1
// and (l >> 1) + 16 -- or + S/2 when R = 1), the alphas of each segment of C
// stages recomputed from its checkpoint into the workspace
template <int R>
__global__ void __launch_bounds__(kWarpsSoft * 32) metric_bwd_soft_kernel(const MArgs a) {
  // [warp][stage of the block][source lane * 5 + (z, g0..g3)]: 165 floats a
  // row, so both the row writes and the column sums are free of bank conflicts
  __shared__ float red[kWarpsSoft][32][32 * 5 + 5];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int f = blockIdx.x * kWarpsSoft + w;
  if (f >= a.F) return;
  const int S = a.S;
  const float tau = a.tau, inv_tau = 1.f / a.tau;
  const float g = a.gmet[f];
  const float* llr = a.llr + (int64_t)f * a.n * a.beta;
  float* grad = a.grad + (int64_t)f * a.n * a.beta;
  float* ck = (float*)(a.ws + (int64_t)f * a.ws_frame);
  float* seg = ck + a.nck * S;  // C rows: alpha entering stage t0 + row
  FwdLane<R> fl;
  fl.init(a, lane);
  // backward-layout constants: branch signs from the lane's states
  const bool live = R * lane < S;
  float s0[R][4], s1[R][4];
#pragma unroll
  for (int r = 0; r < R; r++) {
    const uint32_t i = (uint32_t)(R * lane + r);
    signs(a, aout_m(a, i), s0[r]);
    signs(a, aout_m(a, (uint32_t)S + i), s1[r]);
  }
  const int src0 = lane >> 1, src1 = (R == 1) ? (lane >> 1) + S / 2 : (lane >> 1) + 16;
  float bt[R];  // beta of the lane's states after the current stage
#pragma unroll
  for (int r = 0; r < R; r++) bt[r] = (R * lane + r == 0) ? 0.f : -INFINITY;  // terminated in state 0
  float (*rd)[32 * 5 + 5] = red[w];
  for (int64_t sgi = a.nck - 1; sgi >= 0; sgi--) {
    const int64_t t0 = sgi * a.C;
    const int64_t t1 = (t0 + a.C < a.n) ? t0 + a.C : a.n;
    // alphas of the segment: row 0 is the checkpoint, rows 1.. recomputed
    {
      float m[R];
#pragma unroll
      for (int r = 0; r < R; r++) m[r] = fl.live ? ck[sgi * S + R * lane + r] : -INFINITY;
      for (int64_t b = t0; b < t1; b += 32) {
        float lv[4];
        load_block(a, llr, b, lane, lv);
        const int cnt = (t1 - b < 32) ? (int)(t1 - b) : 32;
        for (int k = 0; k < cnt; k++) {
          const int64_t t = b + k;
#pragma unroll
          for (int r = 0; r < R; r++)
            if (fl.live) seg[(t - t0) * S + R * lane + r] = m[r];
          if (t + 1 < t1) {
            float l[4];
            stage_llr(lv, k, l);
            uint32_t bal[R];
            fwd_step<R, true>(m, l, fl, tau, inv_tau, bal);
          }
        }
      }
    }
    __syncwarp();
    // beta recursion and posteriors, 32 stages at a time from the top; the
    // lane's alphas of the stage below are loaded one stage ahead
    float aln[R];
#pragma unroll
    for (int r = 0; r < R; r++) aln[r] = live ? seg[(t1 - 1 - t0) * S + R * lane + r] : -INFINITY;
    for (int64_t hi = t1; hi > t0; hi -= 32) {
      const int64_t lo = (hi - 32 > t0) ? hi - 32 : t0;
      float lv[4];
      load_block(a, llr, lo, lane, lv);
      for (int64_t t = hi - 1; t >= lo; t--) {
        const int k = (int)(t - lo);
        float l[4];
        stage_llr(lv, k, l);
        float al[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
          al[r] = aln[r];
          aln[r] = (live && t - 1 >= t0) ? seg[(t - 1 - t0) * S + R * lane + r] : -INFINITY;
        }
        float v0[R], v1[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
          v0[r] = __shfl_sync(0xffffffffu, bt[r], src0);
          v1[r] = __shfl_sync(0xffffffffu, bt[r], src1);
        }
        float u0[R], u1[R];
        float mx = -INFINITY;
#pragma unroll
        for (int r = 0; r < R; r++) {
          // successors of i = R l + r: j0 = i >> 1 in register (l & 1) * R/2 + r/2 of
          // lane l >> 1 (R >= 2; register 0 when R == 1), j1 = j0 + S/2
          float bj0, bj1;
          if constexpr (R == 1) {
            bj0 = v0[0];
            bj1 = v1[0];
          } else {
            const int ra = r >> 1, rb = R / 2 + (r >> 1);
            bj0 = (lane & 1) ? v0[rb] : v0[ra];
            bj1 = (lane & 1) ? v1[rb] : v1[ra];
          }
          u0[r] = bm4(s0[r], l) + bj0;
          u1[r] = bm4(s1[r], l) + bj1;
          if (live) mx = fmaxf(mx, fmaxf(al[r] + u0[r], al[r] + u1[r]));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        float z = 0.f, gb[4] = {0.f, 0.f, 0.f, 0.f};
        float bmx = -INFINITY;
#pragma unroll
        for (int r = 0; r < R; r++) {
          if (live) {
            const float q0 = __expf((al[r] + u0[r] - mx) * inv_tau);
            const float q1 = __expf((al[r] + u1[r] - mx) * inv_tau);
            z += q0 + q1;
#pragma unroll
            for (int b = 0; b < 4; b++) gb[b] += q0 * s0[r][b] + q1 * s1[r][b];
          }
          bt[r] = live ? lse2(u0[r], u1[r], tau, inv_tau) : -INFINITY;
          bmx = fmaxf(bmx, bt[r]);
        }
        float* cell = &rd[k][lane * 5];
        cell[0] = z;
#pragma unroll
        for (int b = 0; b < 4; b++) cell[1 + b] = gb[b];
        // re-reference beta to the lane-0 state 0 value every 32 stages
        if (k == 0) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) bmx = fmaxf(bmx, __shfl_xor_sync(0xffffffffu, bmx, o));
          if (bmx != -INFINITY) {
#pragma unroll
            for (int r = 0; r < R; r++) bt[r] -= bmx;
          }
        }
      }
      __syncwarp();
      // lane k sums stage lo + k over the lanes and writes its gradient
      if (lo + lane < hi) {
        float z = 0.f, gb[4] = {0.f, 0.f, 0.f, 0.f};
        for (int q = 0; q < 32; q++) {
          const float* cell = &rd[lane][q * 5];
          z += cell[0];
#pragma unroll
          for (int b = 0; b < 4; b++) gb[b] += cell[1 + b];
        }
#pragma unroll
        for (int b = 0; b < 4; b++)
          if (b < a.beta) grad[(lo + lane) * a.beta + b] = g * gb[b] / z;
      }
      __syncwarp();
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
  const bool soft = tau > 0.f;
  switch (a.spl) {
    case 1: soft ? metric_fwd_kernel<1, true><<<grid, kWarps * 32, 0, s>>>(a)
                 : metric_fwd_kernel<1, false><<<grid, kWarps * 32, 0, s>>>(a); break;
    case 2: soft ? metric_fwd_kernel<2, true><<<grid, kWarps * 32, 0, s>>>(a)
                 : metric_fwd_kernel<2, false><<<grid, kWarps * 32, 0, s>>>(a); break;
    case 4: soft ? metric_fwd_kernel<4, true><<<grid, kWarps * 32, 0, s>>>(a)
                 : metric_fwd_kernel<4, false><<<grid, kWarps * 32, 0, s>>>(a); break;
    default: soft ? metric_fwd_kernel<8, true><<<grid, kWarps * 32, 0, s>>>(a)
                  : metric_fwd_kernel<8, false><<<grid, kWarps * 32, 0, s>>>(a); break;
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
    const unsigned gs = (unsigned)((nframes + kWarpsSoft - 1) / kWarpsSoft);
    switch (a.spl) {
      case 1: metric_bwd_soft_kernel<1><<<gs, kWarpsSoft * 32, 0, s>>>(a); break;
      case 2: metric_bwd_soft_kernel<2><<<gs, kWarpsSoft * 32, 0, s>>>(a); break;
      case 4: metric_bwd_soft_kernel<4><<<gs, kWarpsSoft * 32, 0, s>>>(a); break;
      default: metric_bwd_soft_kernel<8><<<gs, kWarpsSoft * 32, 0, s>>>(a); break;
    }
  } else {
    switch (a.spl) {
      case 1: metric_bwd_hard_kernel<1><<<grid, kWarps * 32, 0, s>>>(a); break;
      case 2: metric_bwd_hard_kernel<2><<<grid, kWarps * 32, 0, s>>>(a); break;
      case 4: metric_bwd_hard_kernel<4><<<grid, kWarps * 32, 0, s>>>(a); break;
      default: metric_bwd_hard_kernel<8><<<grid, kWarps * 32, 0, s>>>(a); break;
    }
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return vit::set_error(VIT_ECUDA, "metric backward launch: %s", cudaGetErrorString(e));
  return VIT_OK;
}

}  // extern "C"
