// vit_warp.cuh -- one warp per tile, states spread over the lanes: the
// low-latency decoder for frames with few tiles (K <= 7).
//
// The tile decoder gives each lane two whole tiles, which is the fast way to
// decode many tiles but leaves a warp with one tile 31 idle lanes.  Here lane
// l holds the path metrics of states 2l and 2l + 1 (S = 64) or of state l
// (S <= 32) of one tile: the two predecessors 2s, 2s + 1 (mod S) of a state
// s (Eq. 3) then sit in one lane and come over by shuffle, and the decisions
// (Eq. 4) of all states are gathered by ballot into a 64-bit word per stage.
// Metrics are 32-bit integers far from overflow (a window of at most
// kWarpSmemStages stages moves them by at most 127 beta per stage), so
// decisions and the traceback start (argmax, ties to the lowest state,
// Alg. 2) are those of unbounded integers.  The decision words of the window
// stay in the warp's shared memory, so windows are limited to
// kWarpSmemStages stages.
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

// The beta LLR bytes of window iteration i (bytes of one 32-bit word).
template <class C>
__device__ __forceinline__ uint32_t warp_llr_word(const int8_t* llr, int i, int L) {
  uint32_t w = 0;
  if (i < L) {
#pragma unroll
    for (int b = 0; b < C::BETA; b++) w |= (uint32_t)(uint8_t)ld_s8(llr + (int64_t)i * C::BETA + b) << (8 * b);
  }
  return w;
}

// Spreads the 32 bits of x to the even bit positions of a 64-bit word.
__device__ __forceinline__ uint64_t spread_even(uint32_t x) {
  uint64_t v = x;
  v = (v | (v << 16)) & 0x0000ffff0000ffffull;
  v = (v | (v << 8)) & 0x00ff00ff00ff00ffull;
  v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0full;
  v = (v | (v << 2)) & 0x3333333333333333ull;
  v = (v | (v << 1)) & 0x5555555555555555ull;
  return v;
}

// One trellis stage (Eq. 3, Eq. 4) of the warp's tile: `pk` holds the
// stage's LLR bytes, m the lane's metrics (states R*lane + r); returns the
// ballot of each register's decisions.  Both predecessors 2s, 2s+1 (mod S)
// of state s sit in one lane: registers 0 and 1 of lane s mod 32 when
// R = 2, register 0 of lanes 2s and 2s+1 (mod S) when R = 1.  The metrics
// stay far from 2^31 (windows of at most kWarpSmemStages stages), so the
// survivor is a plain signed max and the decision compare is off the
// metrics' dependency chain.
template <class C>
__device__ __forceinline__ void warp_stage(int (&m)[C::S > 32 ? 2 : 1], uint32_t pk, int lane, bool live,
                                           const uint32_t (&cA)[C::S > 32 ? 2 : 1],
                                           const uint32_t (&cB)[C::S > 32 ? 2 : 1], uint32_t (&bal)[2]) {
  constexpr int S = C::S;
  constexpr int R = S > 32 ? 2 : 1;
  int l[C::BETA];
#pragma unroll
  for (int b = 0; b < C::BETA; b++) l[b] = (int)(int8_t)(uint8_t)(pk >> (8 * b));
  int q0[R], q1[R];
  if constexpr (R == 2) {
#pragma unroll
    for (int r = 0; r < 2; r++) {
      const int src = (2 * lane + r) & 31;
      q0[r] = __shfl_sync(0xffffffffu, m[0], src);
      q1[r] = __shfl_sync(0xffffffffu, m[1], src);
    }
  } else {
    q0[0] = __shfl_sync(0xffffffffu, m[0], (2 * lane) & (S - 1));
    q1[0] = __shfl_sync(0xffffffffu, m[0], (2 * lane + 1) & (S - 1));
  }
  bal[1] = 0u;
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int x0 = q0[r] + warp_delta<C>(l, cA[r]), x1 = q1[r] + warp_delta<C>(l, cB[r]);
    bal[r] = __ballot_sync(0xffffffffu, live && x1 > x0);  // ties keep the even predecessor
    m[r] = x1 > x0 ? x1 : x0;
  }
}

// Decodes tile `h` (window [t0, t1), emitted [e0, e1)) with the calling warp.
// dec: the tile's decision words, one 64-bit word per stage of the window
// (shared memory, bit s = state s).  The window's LLRs arrive 32 stages at a
// time (lane l loads stage i0 + l, one block ahead) and each stage takes its
// bytes by shuffle, off the metrics' dependency chain; lane l keeps the
// ballots of stage i0 + l and the warp stores a block's words together.
template <class C>
__device__ void decode_tile_warp(const Half& h, uint32_t M, uint64_t* dec, int lane) {
  static_assert(C::S <= 64 && C::BETA <= 4, "states of one tile over the 32 lanes; LLR bytes in one word");
  constexpr int S = C::S;
  constexpr int R = S > 32 ? 2 : 1;  // states per lane: R * lane + r
  const int L = (int)(h.t1 - h.t0);
  int m[R];
  uint32_t cA[R], cB[R];  // output patterns of the branches from 2s and 2s + 1
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int j = R * lane + r;
    m[r] = (h.known && j != 0) ? -(int)M : 0;
    cA[r] = C::aout(2u * (uint32_t)j);
    cB[r] = C::aout(2u * (uint32_t)j + 1u);
  }
  const bool live = R * lane < S;
  const int8_t* llr = h.llr + h.t0 * C::BETA;
  // the stage word of lane l's kept ballots, bit s = state s
  auto word = [](uint32_t kA, uint32_t kB) -> uint64_t {
    if constexpr (R == 2)
      return spread_even(kA) | (spread_even(kB) << 1);
    else
      return (uint64_t)kA;
  };
  uint32_t nxt = warp_llr_word<C>(llr, lane, L);
  int i0 = 0;
  for (; i0 + 32 <= L; i0 += 32) {  // whole blocks of 32 stages
    const uint32_t cur = nxt;
    nxt = warp_llr_word<C>(llr, i0 + 32 + lane, L);
    uint32_t kA = 0u, kB = 0u;
#pragma unroll
    for (int k = 0; k < 32; k++) {
      uint32_t bal[2];
      warp_stage<C>(m, __shfl_sync(0xffffffffu, cur, k), lane, live, cA, cB, bal);
      kA = lane == k ? bal[0] : kA;
      kB = lane == k ? bal[1] : kB;
    }
    dec[i0 + lane] = word(kA, kB);
  }
  if (i0 < L) {  // the last, partial block
    const uint32_t cur = nxt;
    uint32_t kA = 0u, kB = 0u;
    for (int k = 0; k < L - i0; k++) {
      uint32_t bal[2];
      warp_stage<C>(m, __shfl_sync(0xffffffffu, cur, k), lane, live, cA, cB, bal);
      kA = lane == k ? bal[0] : kA;
      kB = lane == k ? bal[1] : kB;
    }
    if (i0 + lane < L) dec[i0 + lane] = word(kA, kB);
  }
  // traceback start: argmax, ties to the lowest state
  int best = R * lane, bv = m[0];
  if constexpr (R == 2) {
    if (m[1] > m[0]) {
      best = R * lane + 1;
      bv = m[1];
    }
  }
  if (!live) {
    best = S;
    bv = -2147483647 - 1;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const int ov = __shfl_xor_sync(0xffffffffu, bv, o), ob = __shfl_xor_sync(0xffffffffu, best, o);
    if (ov > bv || (ov == bv && ob < best)) {
      bv = ov;
      best = ob;
    }
  }
  __syncwarp();
  if (lane != 0 || h.e1 <= h.e0) return;
  // Alg. 2 as in the tile decoder's traceback: following decision d from
  // state j gives 2j + d, so the decision read at iteration i is the decoded
  // bit of iteration i - (K-1); J = 2J + d kept unmasked holds the decoded
  // bits from its low end, and the bytes of [e0, e1) are taken from J at
  // checkpoints every 8 iterations.
  const int r0 = (int)(h.e0 - h.t0), r1 = (int)(h.e1 - h.t0);
  int nb = (r1 - r0 + 7) / 8 - 1;
  uint8_t* const out = h.out + (h.e0 >> 3);
  uint32_t J = h.end_zero ? 0u : (uint32_t)best;
  tb_emit(J, L - C::KM1, r0, r1, nb, out);  // bytes made of start-state bits only
  const int ib = r0 + C::KM1;               // lowest iteration read
  for (int i = L - 1; i >= ib; i -= 8) {
    uint64_t w[8];
#pragma unroll
    for (int k = 0; k < 8; k++) w[k] = (i - k >= ib) ? dec[i - k] : 0ull;
#pragma unroll
    for (int k = 0; k < 8; k++)
      if (i - k >= ib) J = 2u * J + (uint32_t)((w[k] >> (J & (uint32_t)(S - 1))) & 1ull);
    const int lo = (i - 7 > ib ? i - 7 : ib);  // lowest iteration read so far
    tb_emit(J, lo - C::KM1, r0, r1, nb, out);
  }
}
#endif

}  // namespace vit
