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
// Every kernel is compiled per (R, beta), so branch metrics, LLR shuffles and
// gradient sums carry exactly beta terms, and the 32 stages of a block are
// unrolled.  The LLRs of 32 stages arrive with one coalesced load (lane k
// holds stage i0 + k) and reach each stage by shuffle.  Every 32 stages the
// metrics are re-referenced to state 0's (the offsets summed in fp64), so
// fp32 keeps its precision over long frames.  Hard decisions are ballots
// (bit l of word r = state R l + r), stored per block of 32 stages.  The soft
// backward checkpoints alpha every C stages, recomputes a segment's alphas
// from its checkpoint, and runs the beta recursion with lanes holding
// predecessor states (segment alphas in shared memory when they fit); the
// per-stage gradient sums go through shared memory, one stage per lane, 32
// stages at a time.  Each block's LLRs are loaded one block ahead, and each
// stage's LLRs are shuffled out one stage ahead.  The soft backward's two
// stage loops are unrolled by four rather than 32 (its code then fits the
// instruction cache: 0.49 against 0.56 ms on 1024 frames of 2054 stages).
//
// Log-sum-exp in base 2: tau log(e^{x/tau} + e^{y/tau}) = max(x, y) +
// tau ln2 log2(1 + 2^{-|x - y| log2(e) / tau}), with the hardware base-2
// approximations (ex2, lg2) and no branch.
//
// Posterior reference.  Every path crosses exactly one branch of a stage, so
// the branch totals x = alpha_t(i) + delta_t(i, j) + beta_{t+1}(j) of a stage
// satisfy sum_branches exp(x / tau) = exp(M_tau / tau): the largest x lies in
// [M_tau - tau ln(2S), M_tau] at every stage.  The backward therefore scales a
// stage's posteriors by exp(-M_tau / tau) (less the offsets that re-reference
// alpha and beta), which needs no reduction over the warp; the forward keeps
// M_tau and its offset at each checkpoint in the workspace for that.  The
// gradient is a ratio of two sums with the same scale, so the reference
// changes no result beyond rounding.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "../../include/vit.h"
#include "vit_internal.h"

namespace {

constexpr int kWarps = 4;      // frames per CTA (forward, hard backward)
constexpr float kLog2e = 1.4426950408889634f;  // log2(e)
constexpr float kLn2 = 0.6931471805599453f;    // ln(2)

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

// Soft workspace of one frame: nck checkpoint rows and C segment rows of S
// floats, then nck + 1 doubles: the forward's re-reference offset at each
// checkpoint, and M_tau.
__host__ __device__ inline size_t soft_offsets_at(int64_t nck, int C, int S) {
  return (size_t)(nck + C) * (size_t)S * sizeof(float);
}

// output pattern of register word Rw (Eq. 1)
__device__ __forceinline__ uint32_t aout_m(const MArgs& a, uint32_t Rw) {
  uint32_t o = 0;
#pragma unroll
  for (int b = 0; b < 4; b++)
    if (b < a.beta) o |= (uint32_t)(__popc(a.polys[b] & Rw) & 1) << b;
  return o;
}

template <int B>
__device__ __forceinline__ void signs(uint32_t c, float (&s)[B]) {
#pragma unroll
  for (int b = 0; b < B; b++) s[b] = ((c >> b) & 1u) ? -1.f : 1.f;
}

// signed branch metric sum_b (-1)^{c_b} l_b
template <int B>
__device__ __forceinline__ float bmv(const float (&s)[B], const float (&l)[B]) {
  float acc = s[0] * l[0];
#pragma unroll
  for (int b = 1; b < B; b++) acc = fmaf(s[b], l[b], acc);
  return acc;
}

__device__ __forceinline__ float ex2a(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float lg2a(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Base-2 constants of the log-sum-exp of temperature tau.
struct Lse {
  float k1;  // log2(e) / tau
  float k2;  // tau ln 2
  __device__ explicit Lse(float tau) : k1(kLog2e / tau), k2(tau * kLn2) {}
};

// tau log(exp(x/tau) + exp(y/tau)).  1 + e lies in [1, 2], where lg2's
// absolute error is ~1e-7.  When both inputs are -inf, |x - y| is NaN and
// fminf returns 1e30 instead, so e = 0 and the result is max = -inf.
__device__ __forceinline__ float lse2(float x, float y, const Lse& c) {
  const float mx = fmaxf(x, y);
  const float d = fminf(fabsf(x - y), 1e30f);
  return fmaf(c.k2, lg2a(1.f + ex2a(-d * c.k1)), mx);
}

// Lane-side constants of the forward layout (lane l holds successor states
// j = R l + r; predecessors 2j, 2j + 1 mod S).
template <int R, int B>
struct FwdLane {
  float sA[R][B], sB[R][B];  // branch signs from 2j (A) and 2j + 1 (B)
  int la, lb;                // source lanes of the predecessors
  bool live;
  __device__ void init(const MArgs& a, int lane) {
    live = R * lane < a.S;
#pragma unroll
    for (int r = 0; r < R; r++) {
      const uint32_t j = (uint32_t)(R * lane + r);
      signs<B>(aout_m(a, 2u * j), sA[r]);
      signs<B>(aout_m(a, 2u * j + 1u), sB[r]);
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
// metrics m; hard: returns the ballots of the decisions in bal.  The branch
// metrics depend only on the LLRs, so they are formed while the shuffles of
// the metrics are in flight.
template <int R, int B, bool SOFT>
__device__ __forceinline__ void fwd_step(float (&m)[R], const float (&l)[B], const FwdLane<R, B>& fl, const Lse& c,
                                         uint32_t (&bal)[R]) {
  float da[R], db[R];
#pragma unroll
  for (int r = 0; r < R; r++) {
    da[r] = bmv<B>(fl.sA[r], l);
    db[r] = bmv<B>(fl.sB[r], l);
  }
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
    const float x0 = p0 + da[r], x1 = p1 + db[r];
    if constexpr (SOFT) {
      m[r] = lse2(x0, x1, c);
      bal[r] = 0u;
    } else {
      const bool d = x1 > x0;  // ties keep the lower predecessor
      bal[r] = __ballot_sync(0xffffffffu, fl.live && d);
      m[r] = d ? x1 : x0;
    }
  }
}

// The frame's LLRs of stages [i0, i0 + 32): lane k loads stage i0 + k.
template <int B>
__device__ __forceinline__ void load_block(const MArgs& a, const float* llr, int64_t i0, int lane, float (&lv)[B]) {
  const bool in = i0 + lane < a.n;
#pragma unroll
  for (int b = 0; b < B; b++) lv[b] = in ? llr[(i0 + lane) * B + b] : 0.f;
}

template <int B>
__device__ __forceinline__ void stage_llr(const float (&lv)[B], int k, float (&l)[B]) {
#pragma unroll
  for (int b = 0; b < B; b++) l[b] = __shfl_sync(0xffffffffu, lv[b], k);
}

// Runs body(k) for k = 0 .. cnt-1 (ascending) or cnt-1 .. 0 (descending).
// kFull: unrolled with constant k for whole blocks of 32 and guarded for a
// partial one (small bodies, R <= 2); otherwise a loop unrolled by four.
template <bool kDown, bool kFull, class F>
__device__ __forceinline__ void block_stages(int cnt, F&& body) {
  if constexpr (kFull) {
    if (cnt == 32) {
#pragma unroll
      for (int q = 0; q < 32; q++) body(kDown ? 31 - q : q);
    } else {
#pragma unroll
      for (int q = 0; q < 32; q++) {
        const int k = kDown ? 31 - q : q;
        if (k < cnt) body(k);
      }
    }
  } else {
#pragma unroll 4
    for (int q = 0; q < cnt; q++) body(kDown ? cnt - 1 - q : q);
  }
}

template <int R, int B, bool SOFT>
__global__ void __launch_bounds__(SOFT ? kWarps * 32 : 32) metric_fwd_kernel(const MArgs a) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int f = blockIdx.x * (blockDim.x >> 5) + w;
  if (f >= a.F) return;
  const int S = a.S;
  const Lse c(SOFT ? a.tau : 1.f);
  FwdLane<R, B> fl;
  fl.init(a, lane);
  float m[R];
#pragma unroll
  for (int r = 0; r < R; r++) m[r] = (R * lane + r == 0) ? 0.f : -INFINITY;  // 0-rooted
  const float* llr = a.llr + (int64_t)f * a.n * B;
  uint8_t* ws = a.ws + (int64_t)f * a.ws_frame;
  double off = 0.0;
  int64_t next_ck = 0;  // next checkpointed stage (soft)
  float* ck = (float*)ws;
  double* cko = (double*)(ws + soft_offsets_at(a.nck, a.C, S));
  const bool ck_blocks = (a.C % 32) == 0;
  float lv[B];
  load_block<B>(a, llr, 0, lane, lv);
  for (int64_t i0 = 0; i0 < a.n; i0 += 32) {
    float lvn[B];  // the next block's LLRs, loaded one block ahead
    load_block<B>(a, llr, i0 + 32, lane, lvn);
    const int cnt = (a.n - i0 < 32) ? (int)(a.n - i0) : 32;
    uint32_t keep[R];
#pragma unroll
    for (int r = 0; r < R; r++) keep[r] = 0u;
    float l[B];
    stage_llr<B>(lv, 0, l);
    auto checkpoint = [&]() {  // the metrics entering stage next_ck, and their offset
#pragma unroll
      for (int r = 0; r < R; r++)
        if (fl.live) ck[R * lane + r] = m[r];
      if (lane == 0) *cko = off;
      ck += S;
      cko++;
      next_ck += a.C;
    };
    auto stage = [&](int k) {
      float ln[B];  // the next stage's LLRs (lane 32 reads lane 0: unused)
      stage_llr<B>(lv, k + 1, ln);
      uint32_t bal[R];
      fwd_step<R, B, SOFT>(m, l, fl, c, bal);
      if (!SOFT) {
#pragma unroll
        for (int r = 0; r < R; r++) keep[r] = (lane == k) ? bal[r] : keep[r];
      }
#pragma unroll
      for (int b = 0; b < B; b++) l[b] = ln[b];
    };
    if (!SOFT || ck_blocks) {
      // checkpoints (C a multiple of 32) fall on block starts: the block's
      // stages form one branch-free sequence
      if (SOFT && i0 == next_ck) checkpoint();
      block_stages<false, (R <= 2)>(cnt, stage);
    } else {
      block_stages<false, (R <= 2)>(cnt, [&](int k) {
        if (i0 + k == next_ck) checkpoint();
        stage(k);
      });
    }
#pragma unroll
    for (int b = 0; b < B; b++) lv[b] = lvn[b];
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
  if (lane == 0) {
    const double M = off + (double)m[0];
    a.metric[f] = (float)M;
    if (SOFT) *(double*)(ws + soft_offsets_at(a.nck, a.C, S) + (size_t)a.nck * sizeof(double)) = M;
  }
}

// hard backward: traceback from state 0 through the stored decisions (every
// lane follows the same state), then the +-1 branch symbols times the
// upstream gradient, one stage per lane.  Lane k holds stage b0 + k's words;
// for R <= 2 every lane takes the block's words by shuffle before the chain
// starts (they do not depend on the state), so a step of the chain is a
// register select, a shift and an add; for R >= 4 the words go through shared
// memory.
template <int R, int B>
__global__ void __launch_bounds__(kWarps * 32) metric_bwd_hard_kernel(const MArgs a) {
  constexpr int RS = R > 2 ? R : 1;
  __shared__ uint32_t sw[kWarps][32][RS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int f = blockIdx.x * kWarps + w;
  if (f >= a.F) return;
  const uint32_t S = (uint32_t)a.S;
  const uint32_t* dw = (const uint32_t*)(a.ws + (int64_t)f * a.ws_frame);
  const float g = a.gmet[f];
  float* grad = a.grad + (int64_t)f * a.n * B;
  uint32_t J = 0;  // state after the last stage (terminated)
  uint32_t wn[R];  // the next (lower) block's words, loaded one block ahead
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
    if constexpr (R <= 2) {
      uint32_t W[32][R];
#pragma unroll
      for (int k = 0; k < 32; k++)
#pragma unroll
        for (int r = 0; r < R; r++) W[k][r] = __shfl_sync(0xffffffffu, wv[r], k);
      block_stages<true, true>(top, [&](int k) {
        const uint32_t word = (R == 1) ? W[k][0] : ((J & 1u) ? W[k][R - 1] : W[k][0]);
        const uint32_t d = (word >> (J / R)) & 1u;
        const uint32_t Rw = 2u * J + d;  // the branch's register word: predecessor (Rw mod S) -> J
        myR = (lane == k) ? Rw : myR;
        J = Rw & (S - 1u);
      });
    } else {
#pragma unroll
      for (int r = 0; r < R; r++) sw[w][lane][r] = wv[r];
      __syncwarp();
      block_stages<true, false>(top, [&](int k) {
        const uint32_t word = sw[w][k][J & (uint32_t)(R - 1)];
        const uint32_t d = (word >> (J / R)) & 1u;
        const uint32_t Rw = 2u * J + d;
        myR = (lane == k) ? Rw : myR;
        J = Rw & (S - 1u);
      });
      __syncwarp();
    }
    if (my < a.n) {
      const uint32_t o = aout_m(a, myR);
#pragma unroll
      for (int b = 0; b < B; b++) grad[my * B + b] = ((o >> b) & 1u) ? -g : g;
    }
  }
}

// soft backward: beta recursion from the end with lanes holding predecessor
// states i = R l + r (successors i >> 1 and (i >> 1) + S/2, from lanes l >> 1
// and (l >> 1) + 16 -- or + S/2 when R = 1), the alphas of each segment of C
// stages recomputed from its checkpoint into shared memory when C S floats
// fit kSegSmemFloats, else into the workspace.  One warp per CTA; dynamic
// shared memory: the reduction buffer, then the segment rows.
//
// Reduction buffer: [stage of the block][source lane * P + (z, g0..g_{B-1})],
// P = B + 1 rounded up to odd and rows of 32 P + 1 floats, so the row writes
// (lane stride P) and the column sums (row stride odd) are free of bank
// conflicts.
constexpr int kSegSmemFloats = 4096;
template <int B>
__host__ __device__ constexpr int red_stride() {
  return ((B + 1) & 1) ? B + 1 : B + 2;
}
template <int B>
__host__ __device__ constexpr int red_floats() {
  return 32 * (32 * red_stride<B>() + 1);
}

template <int R, int B>
__global__ void __launch_bounds__(32) metric_bwd_soft_kernel(const MArgs a) {
  extern __shared__ float dsm[];
  constexpr int P = red_stride<B>(), ROW = 32 * P + 1;
  const int lane = threadIdx.x & 31;
  const int f = blockIdx.x;
  if (f >= a.F) return;
  const int S = a.S;
  const Lse c(a.tau);
  const float g = a.gmet[f];
  const float* llr = a.llr + (int64_t)f * a.n * B;
  float* grad = a.grad + (int64_t)f * a.n * B;
  uint8_t* wsf = a.ws + (int64_t)f * a.ws_frame;
  float* ck = (float*)wsf;
  // C rows: alpha entering stage t0 + row (generic pointer: shared or global)
  float* seg = ((int64_t)a.C * S <= kSegSmemFloats) ? dsm + red_floats<B>() : ck + a.nck * S;
  float* rd = dsm;
  const double* cko = (const double*)(wsf + soft_offsets_at(a.nck, a.C, S));
  const double Mtau = cko[a.nck];
  FwdLane<R, B> fl;
  fl.init(a, lane);
  // backward-layout constants: branch signs from the lane's states
  const bool live = R * lane < S;
  float s0[R][B], s1[R][B];
#pragma unroll
  for (int r = 0; r < R; r++) {
    const uint32_t i = (uint32_t)(R * lane + r);
    signs<B>(aout_m(a, i), s0[r]);
    signs<B>(aout_m(a, (uint32_t)S + i), s1[r]);
  }
  const int src0 = lane >> 1, src1 = (R == 1) ? (lane >> 1) + S / 2 : (lane >> 1) + 16;
  float bt[R];  // beta of the lane's states after the current stage
#pragma unroll
  for (int r = 0; r < R; r++) bt[r] = (R * lane + r == 0) ? 0.f : -INFINITY;  // terminated in state 0
  double boff = 0.0;  // sum of the re-reference offsets taken out of bt
  for (int64_t sgi = a.nck - 1; sgi >= 0; sgi--) {
    const int64_t t0 = sgi * a.C;
    const int64_t t1 = (t0 + a.C < a.n) ? t0 + a.C : a.n;
    // alphas of the segment: row 0 is the checkpoint, rows 1.. recomputed
    {
      float m[R];
#pragma unroll
      for (int r = 0; r < R; r++) m[r] = fl.live ? ck[sgi * S + R * lane + r] : -INFINITY;
      float lv[B];
      load_block<B>(a, llr, t0, lane, lv);
      for (int64_t b = t0; b < t1; b += 32) {
        float lvn[B];  // the next block's LLRs, one block ahead
        load_block<B>(a, llr, b + 32, lane, lvn);
        const int cnt = (t1 - b < 32) ? (int)(t1 - b) : 32;
        float l[B];
        stage_llr<B>(lv, 0, l);
        block_stages<false, false>(cnt, [&](int k) {
          const int64_t t = b + k;
#pragma unroll
          for (int r = 0; r < R; r++)
            if (fl.live) seg[(t - t0) * S + R * lane + r] = m[r];
          float ln[B];
          stage_llr<B>(lv, k + 1, ln);
          // (the step after the segment's last stage is computed and unused,
          // which keeps the block free of branches)
          uint32_t bal[R];
          fwd_step<R, B, true>(m, l, fl, c, bal);
#pragma unroll
          for (int q = 0; q < B; q++) l[q] = ln[q];
        });
#pragma unroll
        for (int q = 0; q < B; q++) lv[q] = lvn[q];
      }
    }
    __syncwarp();
    // M_tau less the offset of this segment's alphas
    const double mrel = Mtau - cko[sgi];
    // beta recursion and posteriors, 32 stages at a time from the top; the
    // lane's alphas of the stage below are loaded one stage ahead
    float aln[R];
#pragma unroll
    for (int r = 0; r < R; r++) aln[r] = live ? seg[(t1 - 1 - t0) * S + R * lane + r] : -INFINITY;
    const int64_t lo0 = (t1 - 32 > t0) ? t1 - 32 : t0;
    float lv[B];
    load_block<B>(a, llr, lo0, lane, lv);
    for (int64_t hi = t1; hi > t0; hi -= 32) {
      const int64_t lo = (hi - 32 > t0) ? hi - 32 : t0;
      const int cnt = (int)(hi - lo);
      float lvn[B];  // the next (lower) block's LLRs, one block ahead
      {
        const int64_t lon = (lo - 32 > t0) ? lo - 32 : t0;
        load_block<B>(a, llr, lon, lane, lvn);
      }
      // the posteriors' common reference, in base-2 exponent units
      const float refk = (float)((mrel - boff) * (double)c.k1);
      float bmx = -INFINITY;
      float l[B];
      stage_llr<B>(lv, cnt - 1, l);
      block_stages<true, false>(cnt, [&](int k) {
        const int64_t t = lo + k;
        float ln[B];  // the next (lower) stage's LLRs (lane -1 reads lane 31: unused)
        stage_llr<B>(lv, k - 1, ln);
        float al[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
          al[r] = aln[r];
          aln[r] = (live && t - 1 >= t0) ? seg[(t - 1 - t0) * S + R * lane + r] : -INFINITY;
        }
        float e0[R], e1[R];  // branch metrics, formed while the shuffles are in flight
#pragma unroll
        for (int r = 0; r < R; r++) {
          e0[r] = bmv<B>(s0[r], l);
          e1[r] = bmv<B>(s1[r], l);
        }
        float v0[R], v1[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
          v0[r] = __shfl_sync(0xffffffffu, bt[r], src0);
          v1[r] = __shfl_sync(0xffffffffu, bt[r], src1);
        }
        float z = 0.f, gb[B];
#pragma unroll
        for (int q = 0; q < B; q++) gb[q] = 0.f;
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
          const float u0 = e0[r] + bj0, u1 = e1[r] + bj1;
          // al = -inf on dead lanes, so their posteriors are 0
          const float q0 = ex2a(fmaf(al[r] + u0, c.k1, -refk));
          const float q1 = ex2a(fmaf(al[r] + u1, c.k1, -refk));
          z += q0 + q1;
#pragma unroll
          for (int q = 0; q < B; q++) gb[q] = fmaf(q0, s0[r][q], fmaf(q1, s1[r][q], gb[q]));
          bt[r] = live ? lse2(u0, u1, c) : -INFINITY;
        }
        float* cell = rd + k * ROW + lane * P;
        cell[0] = z;
#pragma unroll
        for (int q = 0; q < B; q++) cell[1 + q] = gb[q];
        if (k == 0) {
#pragma unroll
          for (int r = 0; r < R; r++) bmx = fmaxf(bmx, bt[r]);
        }
#pragma unroll
        for (int q = 0; q < B; q++) l[q] = ln[q];
      });
#pragma unroll
      for (int q = 0; q < B; q++) lv[q] = lvn[q];
      // re-reference beta to its maximum every 32 stages
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) bmx = fmaxf(bmx, __shfl_xor_sync(0xffffffffu, bmx, o));
      if (bmx != -INFINITY) {
#pragma unroll
        for (int r = 0; r < R; r++) bt[r] -= bmx;
        boff += (double)bmx;
      }
      __syncwarp();
      // lane k sums stage lo + k over the lanes and writes its gradient
      if (lane < cnt) {
        float z = 0.f, gb[B];
#pragma unroll
        for (int q = 0; q < B; q++) gb[q] = 0.f;
        const float* row = rd + lane * ROW;
#pragma unroll 8
        for (int j = 0; j < 32; j++) {
          z += row[j * P];
#pragma unroll
          for (int q = 0; q < B; q++) gb[q] += row[j * P + 1 + q];
        }
        const float gz = g / z;
#pragma unroll
        for (int q = 0; q < B; q++) grad[(lo + lane) * B + q] = gb[q] * gz;
      }
      __syncwarp();
    }
    __syncwarp();
  }
}

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

size_t frame_bytes(const vit_code* c, int64_t n, float tau, int C) {
  const int S = 1 << (c->K - 1);
  if (tau > 0.f) {
    const int64_t nck = (n + C - 1) / C;
    return align_up(soft_offsets_at(nck, C, S) + (size_t)(nck + 1) * sizeof(double));
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

// Launches one kernel of the (R, beta) family: which 0 = forward, 1 = hard
// backward, 2 = soft backward.
template <int R, int B>
void launch_rb(int which, bool soft, const MArgs& a, cudaStream_t s) {
  const unsigned grid = (unsigned)((a.F + kWarps - 1) / kWarps);
  if (which == 0) {
    // the hard forward one frame per CTA, compiled for 32-thread CTAs
    // (1024 frames: 87.4 against 91.7 us with 4-frame CTAs); the soft
    // forward measured 1% slower that way
    if (soft)
      metric_fwd_kernel<R, B, true><<<grid, kWarps * 32, 0, s>>>(a);
    else
      metric_fwd_kernel<R, B, false><<<(unsigned)a.F, 32, 0, s>>>(a);
  } else if (which == 1) {
    metric_bwd_hard_kernel<R, B><<<grid, kWarps * 32, 0, s>>>(a);
  } else {
    // one frame per CTA; the segment rows join the reduction buffer in
    // shared memory when they fit (at most 36 KB, within the default limit)
    static_assert((red_floats<B>() + kSegSmemFloats) * sizeof(float) <= 48 * 1024, "default shared-memory limit");
    const size_t seg = ((int64_t)a.C * a.S <= kSegSmemFloats) ? (size_t)a.C * a.S : 0;
    const size_t bytes = (red_floats<B>() + seg) * sizeof(float);
    metric_bwd_soft_kernel<R, B><<<(unsigned)a.F, 32, bytes, s>>>(a);
  }
}

template <int B>
void launch_b(int which, bool soft, const MArgs& a, cudaStream_t s) {
  switch (a.spl) {
    case 1: launch_rb<1, B>(which, soft, a, s); break;
    case 2: launch_rb<2, B>(which, soft, a, s); break;
    case 4: launch_rb<4, B>(which, soft, a, s); break;
    default: launch_rb<8, B>(which, soft, a, s); break;
  }
}

void launch(int which, bool soft, const MArgs& a, cudaStream_t s) {
  switch (a.beta) {
    case 2: launch_b<2>(which, soft, a, s); break;
    case 3: launch_b<3>(which, soft, a, s); break;
    default: launch_b<4>(which, soft, a, s); break;
  }
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
  launch(0, tau > 0.f, a, (cudaStream_t)stream);
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
  const bool soft = tau > 0.f;
  launch(soft ? 2 : 1, soft, a, (cudaStream_t)stream);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return vit::set_error(VIT_ECUDA, "metric backward launch: %s", cudaGetErrorString(e));
  return VIT_OK;
}

}  // extern "C"
