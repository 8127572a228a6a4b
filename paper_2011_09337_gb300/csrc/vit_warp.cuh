// vit_warp.cuh -- one warp per tile, states spread over the lanes: the
// low-latency decoder for frames with few tiles (K <= 7).
//
// The tile decoder gives each lane two whole tiles, which is the fast way to
// decode many tiles but leaves a warp with one tile 31 idle lanes.  Here lane
// l holds the path metrics of states l and l + 32 (S = 64) or of state l
// (S <= 32) of one tile, so a stage is one butterfly per lane: the metrics of
// the two predecessors (Eq. 3) come from their lanes by shuffle, the
// decisions (Eq. 4) of all states by ballot, and one lane writes them as a
// 64-bit word per stage.  Metrics are 32-bit and compared by signed
// difference, so they may wrap; decisions and the traceback start (argmax,
// ties to the lowest state, Alg. 2) are those of unbounded integers.  The
// decision words of the window stay in the warp's shared memory, so windows
// are limited to kWarpSmemStages stages.
#pragma once
#include "vit_acs.cuh"

namespace vit {

#if defined(__CUDACC__)
// Signed branch metric of pattern c for this stage's LLRs (Eq. 2).
template <class C>
__device__ __forceinline__ int warp_delta(const int (&l)[C::BETA], uint32_t c) {
  int d = 0;
#pragma unroll
  for (int b = 0; b < C::BETA; b++) d += ((c >> b) & 1u) ? -l[b] : l[b];
  return d;
}

// Decodes tile `h` (window [t0, t1), emitted [e0, e1)) with the calling warp.
// dec: the tile's decision words, one 64-bit word per stage of the window
// (shared memory).
template <class C>
__device__ void decode_tile_warp(const Half& h, uint32_t M, uint64_t* dec, int lane) {
  static_assert(C::S <= 64, "states of one tile over the 32 lanes");
  constexpr int S = C::S;
  constexpr int R = S > 32 ? 2 : 1;  // states per lane
  const int L = (int)(h.t1 - h.t0);
  // lane l holds states l + 32 r; state j's predecessors are 2j mod S and
  // 2j+1 mod S, reached by the branches R0 = 2j and R0 + 1 (the two states
  // of a lane share their predecessors: a butterfly)
  uint32_t m[R];
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int j = lane + 32 * r;
    m[r] = (h.known && j != 0) ? 0u - M : 0u;
  }
  const int p0 = (2 * lane) & (S - 1);
  const int src0 = p0 & 31, src1 = (p0 + 1) & 31, reg = p0 >> 5;
  uint32_t cA[R], cB[R];
#pragma unroll
  for (int r = 0; r < R; r++) {
    const uint32_t j = (uint32_t)(lane + 32 * r);
    cA[r] = C::aout(2u * j);
    cB[r] = C::aout(2u * j + 1u);
  }
  const bool live = lane < S;
  const int8_t* llr = h.llr + h.t0 * C::BETA;
  for (int i = 0; i < L; i++) {
    int l[C::BETA];
#pragma unroll
    for (int b = 0; b < C::BETA; b++) l[b] = ld_s8(llr + (int64_t)i * C::BETA + b);
    // metrics of the two predecessors: register `reg` of lanes src0, src1
    uint32_t q0 = __shfl_sync(0xffffffffu, m[0], src0), q1 = __shfl_sync(0xffffffffu, m[0], src1);
    if constexpr (R == 2) {
      const uint32_t u0 = __shfl_sync(0xffffffffu, m[1], src0), u1 = __shfl_sync(0xffffffffu, m[1], src1);
      q0 = reg ? u0 : q0;
      q1 = reg ? u1 : q1;
    }
    uint32_t bal[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
      const uint32_t x0 = q0 + (uint32_t)warp_delta<C>(l, cA[r]), x1 = q1 + (uint32_t)warp_delta<C>(l, cB[r]);
      const bool d = live && (int)(x1 - x0) > 0;  // ties keep the even predecessor
      bal[r] = __ballot_sync(0xffffffffu, d);
      m[r] = d ? x1 : x0;
    }
    if (lane == 0) dec[i] = (uint64_t)bal[0] | (R == 2 ? (uint64_t)bal[R - 1] << 32 : 0ull);
  }
  // traceback start: argmax (ties to the lowest state) relative to state 0
  int best = lane;
  uint32_t bv = m[0];
  if constexpr (R == 2) {
    if ((int)(m[1] - m[0]) > 0) {
      best = lane + 32;
      bv = m[1];
    }
  }
  const uint32_t ref = __shfl_sync(0xffffffffu, m[0], 0);
  int rel = live ? (int)(bv - ref) : (-2147483647 - 1);
  if (!live) best = S;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int orel = __shfl_xor_sync(0xffffffffu, rel, o), ob = __shfl_xor_sync(0xffffffffu, best, o);
    if (orel > rel || (orel == rel && ob < best)) {
      rel = orel;
      best = ob;
    }
  }
  __syncwarp();
  if (lane != 0) return;
  // Alg. 2 over the window, the bytes of [e0, e1) written as they complete;
  // the next 8 decision words are loaded ahead of the dependent steps
  uint32_t j = h.end_zero ? 0u : (uint32_t)best;
  uint32_t acc = 0;
  int i = L - 1;
  const int stop = (int)(h.e0 - h.t0);
  while (i >= stop) {
    uint64_t w[8];
#pragma unroll
    for (int k = 0; k < 8; k++) w[k] = (i - k >= stop) ? dec[i - k] : 0ull;
#pragma unroll
    for (int k = 0; k < 8; k++) {
      if (i < stop) break;
      const int64_t t = h.t0 + i;
      const uint32_t d = (uint32_t)(w[k] >> j) & 1u;
      if (t < h.e1) {
        acc |= ((j >> (C::K - 2)) & 1u) << (t & 7);
        if ((t & 7) == 0 || t == h.e0) {
          h.out[t >> 3] = (uint8_t)acc;
          acc = 0u;
        }
      }
      j = ((j << 1) | d) & (uint32_t)(S - 1);
      i--;
    }
  }
}
#endif

}  // namespace vit
