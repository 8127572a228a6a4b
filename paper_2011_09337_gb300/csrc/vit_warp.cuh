// vit_warp.cuh -- one warp per tile, states spread over the lanes: the
// low-latency decoder for frames with few tiles (K <= 7).
//
// The tile decoder gives each lane two whole tiles, which is the fast way to
// decode many tiles but leaves a warp with one tile 31 idle lanes.  Here lane
// l holds the path metrics of states l and l + 32 (S = 64) or of state l
// (S <= 32) of one tile, so a stage is one butterfly per lane: the metrics of
// the two predecessors (Eq. 3) come from their lanes by shuffle, the
// decisions (Eq. 4) of all states by ballot, a 64-bit word per stage.
// Metrics are 32-bit and compared by signed
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

// One trellis stage (Eq. 3, Eq. 4) of the warp's tile: `pk` holds the
// stage's LLR bytes, m the lane's metrics; returns the two ballot words.
template <class C>
__device__ __forceinline__ void warp_stage(uint32_t (&m)[C::S > 32 ? 2 : 1], uint32_t pk, int src0, int src1,
                                           int reg, bool live, const uint32_t (&cA)[C::S > 32 ? 2 : 1],
                                           const uint32_t (&cB)[C::S > 32 ? 2 : 1], uint32_t (&bal)[2]) {
  constexpr int R = C::S > 32 ? 2 : 1;
  int l[C::BETA];
#pragma unroll
  for (int b = 0; b < C::BETA; b++) l[b] = (int)(int8_t)(uint8_t)(pk >> (8 * b));
  // metrics of the two predecessors: register `reg` of lanes src0, src1
  uint32_t q0 = __shfl_sync(0xffffffffu, m[0], src0), q1 = __shfl_sync(0xffffffffu, m[0], src1);
  if constexpr (R == 2) {
    const uint32_t u0 = __shfl_sync(0xffffffffu, m[1], src0), u1 = __shfl_sync(0xffffffffu, m[1], src1);
    q0 = reg ? u0 : q0;
    q1 = reg ? u1 : q1;
  }
  bal[1] = 0u;
#pragma unroll
  for (int r = 0; r < R; r++) {
    const uint32_t x0 = q0 + (uint32_t)warp_delta<C>(l, cA[r]), x1 = q1 + (uint32_t)warp_delta<C>(l, cB[r]);
    const bool d = live && (int)(x1 - x0) > 0;  // ties keep the even predecessor
    bal[r] = __ballot_sync(0xffffffffu, d);
    m[r] = d ? x1 : x0;
  }
}

// Decodes tile `h` (window [t0, t1), emitted [e0, e1)) with the calling warp.
// dec: the tile's decision words, one 64-bit word per stage of the window
// (shared memory).  The window's LLRs arrive 32 stages at a time (lane l
// loads stage i0 + l, one block ahead) and each stage takes its bytes by
// shuffle, off the metrics' dependency chain; lane l keeps the decision
// word of stage i0 + l and the warp stores a block's words together.
template <class C>
__device__ void decode_tile_warp(const Half& h, uint32_t M, uint64_t* dec, int lane) {
  static_assert(C::S <= 64 && C::BETA <= 4, "states of one tile over the 32 lanes; LLR bytes in one word");
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
  uint32_t nxt = warp_llr_word<C>(llr, lane, L);
  int i0 = 0;
  for (; i0 + 32 <= L; i0 += 32) {  // whole blocks of 32 stages
    const uint32_t cur = nxt;
    nxt = warp_llr_word<C>(llr, i0 + 32 + lane, L);
    uint32_t kA = 0u, kB = 0u;
#pragma unroll
    for (int k = 0; k < 32; k++) {
      uint32_t bal[2];
      warp_stage<C>(m, __shfl_sync(0xffffffffu, cur, k), src0, src1, reg, live, cA, cB, bal);
      kA = lane == k ? bal[0] : kA;
      kB = lane == k ? bal[1] : kB;
    }
    dec[i0 + lane] = (uint64_t)kA | ((uint64_t)kB << 32);
  }
  if (i0 < L) {  // the last, partial block
    const uint32_t cur = nxt;
    uint32_t kA = 0u, kB = 0u;
    for (int k = 0; k < L - i0; k++) {
      uint32_t bal[2];
      warp_stage<C>(m, __shfl_sync(0xffffffffu, cur, k), src0, src1, reg, live, cA, cB, bal);
      kA = lane == k ? bal[0] : kA;
      kB = lane == k ? bal[1] : kB;
    }
    if (i0 + lane < L) dec[i0 + lane] = (uint64_t)kA | ((uint64_t)kB << 32);
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
