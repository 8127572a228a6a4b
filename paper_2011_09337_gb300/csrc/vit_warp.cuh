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

// Branch-metric multipliers of a lane's two predecessor branches per state:
// delta = sum_b s[b] * l[b] with s[b] = -1 where the branch's output bit b is
// 1 (Eq. 2).  When every generator taps the oldest input (the SYMMETRIC
// codes), the branches from 2s and 2s + 1 carry complementary patterns and
// the second delta is the negated first.
template <class C>
constexpr bool complementary_branches() {
  if constexpr (C::GENERIC)
    return false;  // generators known only at run time
  else
    return C::SYMMETRIC;
}

template <class C>
struct WarpSigns {
  static constexpr int R = C::S > 32 ? 2 : 1;
  static constexpr bool kComplement = complementary_branches<C>();
  int sA[R][C::BETA], sB[R][C::BETA];
  __device__ __forceinline__ void init(const uint32_t (&cA)[R], const uint32_t (&cB)[R]) {
#pragma unroll
    for (int r = 0; r < R; r++)
#pragma unroll
      for (int b = 0; b < C::BETA; b++) {
        sA[r][b] = ((cA[r] >> b) & 1u) ? -1 : 1;
        sB[r][b] = ((cB[r] >> b) & 1u) ? -1 : 1;
      }
  }
};

// One trellis stage (Eq. 3, Eq. 4) of the warp's tile: `pk` holds the
// stage's LLR bytes, m the lane's metrics (states R*lane + r); returns the
// ballot of each register's decisions.  Both predecessors 2s, 2s+1 (mod S)
// of state s sit in one lane: registers 0 and 1 of lane s mod 32 when
// R = 2, register 0 of lanes 2s and 2s+1 (mod S) when R = 1.  The metrics
// stay far from 2^31 (windows of at most kWarpSmemStages stages), so the
// survivor is a plain signed max and the decision compare is off the
// metrics' dependency chain.  The branch metrics depend only on the LLRs, so
// they are formed before the metrics' shuffles and only one add per
// candidate sits on the chain.
template <class C>
__device__ __forceinline__ void warp_stage(int (&m)[C::S > 32 ? 2 : 1], uint32_t pk, int lane, bool live,
                                           const WarpSigns<C>& sg, uint32_t (&bal)[2]) {
  constexpr int S = C::S;
  constexpr int R = S > 32 ? 2 : 1;
  int l[C::BETA];
#pragma unroll
  for (int b = 0; b < C::BETA; b++) l[b] = (int)(int8_t)(uint8_t)(pk >> (8 * b));
  int dA[R], dB[R];
#pragma unroll
  for (int r = 0; r < R; r++) {
    dA[r] = sg.sA[r][0] * l[0];
#pragma unroll
    for (int b = 1; b < C::BETA; b++) dA[r] += sg.sA[r][b] * l[b];
    if constexpr (WarpSigns<C>::kComplement) {
      dB[r] = -dA[r];
    } else {
      dB[r] = sg.sB[r][0] * l[0];
#pragma unroll
      for (int b = 1; b < C::BETA; b++) dB[r] += sg.sB[r][b] * l[b];
    }
  }
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
    const int x0 = q0[r] + dA[r], x1 = q1[r] + dB[r];
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
__device__ void decode_tile_warp(const Half& h, uint32_t M, uint64_t* dec, int lane, const uint32_t* polys) {
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
    if constexpr (C::GENERIC) {
      cA[r] = aout_rt(polys, C::BETA, 2u * (uint32_t)j);
      cB[r] = aout_rt(polys, C::BETA, 2u * (uint32_t)j + 1u);
    } else {
      cA[r] = C::aout(2u * (uint32_t)j);
      cB[r] = C::aout(2u * (uint32_t)j + 1u);
    }
  }
  const bool live = R * lane < S;
  WarpSigns<C> sg;
  sg.init(cA, cB);
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
      warp_stage<C>(m, __shfl_sync(0xffffffffu, cur, k), lane, live, sg, bal);
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
      warp_stage<C>(m, __shfl_sync(0xffffffffu, cur, k), lane, live, sg, bal);
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

// One warp per tile for codes known only at run time (any K in [3, 9]), with
// the tile's decisions in global memory, so any window length and any number
// of tiles.  Lane l holds the 32-bit metrics of states R l + r (R = S / 32
// for S >= 32; R = 1, lanes l < S, for smaller trellises).  The predecessors
// 2s, 2s + 1 (mod S) of state R l + r are registers 2r, 2r + 1 (mod R) of
// lane 2l (r < R/2) or 2l + 1 (mod 32), so a stage takes all R registers of
// those two lanes by shuffle.  The branch patterns of a lane's states (Eq. 1)
// are formed once from the generators.  Decisions (Eq. 4): ballot r of a
// stage has bit l = decision of state R l + r; lane k keeps the R ballots of
// stage i0 + k of each block of 32 stages and the warp stores the block's
// words together (R words per stage).  Metrics are renormalised by state 0's
// metric every 1024 stages, so their differences, which decide every
// comparison, are those of unbounded integers for any window length.
// Traceback (Alg. 2): every lane follows the same state; per block of 32
// stages lane k loads stage k's R words, and each step selects the word of
// the current state's register and takes it from the stage's lane by
// shuffle.
template <class C>
__device__ void decode_tile_warp_gen(const Half& h, uint32_t M, uint32_t* dec, int lane, const uint32_t* polys) {
  constexpr int S = C::S;
  constexpr int R = S >= 32 ? S / 32 : 1;
  const int L = (int)(h.t1 - h.t0);
  const bool live = R * lane < S;
  int m[R];
  int sA[R][C::BETA], sB[R][C::BETA];  // branch-metric multipliers (Eq. 2) of the branches from 2s and 2s + 1
#pragma unroll
  for (int r = 0; r < R; r++) {
    const int j = R * lane + r;
    m[r] = (h.known && j != 0) ? -(int)M : 0;
    const uint32_t cA = aout_rt(polys, C::BETA, 2u * (uint32_t)j);
    const uint32_t cB = aout_rt(polys, C::BETA, 2u * (uint32_t)j + 1u);
#pragma unroll
    for (int b = 0; b < C::BETA; b++) {
      sA[r][b] = ((cA >> b) & 1u) ? -1 : 1;
      sB[r][b] = ((cB >> b) & 1u) ? -1 : 1;
    }
  }
  const int8_t* llr = h.llr + h.t0 * C::BETA;
  const int la = (2 * lane) & (R == 1 ? S - 1 : 31), lb = (2 * lane + 1) & (R == 1 ? S - 1 : 31);
  uint32_t nxt = warp_llr_word<C>(llr, lane, L);
  for (int i0 = 0; i0 < L; i0 += 32) {
    const uint32_t cur = nxt;
    nxt = warp_llr_word<C>(llr, i0 + 32 + lane, L);
    const int cnt = (L - i0 < 32) ? L - i0 : 32;
    uint32_t keep[R];
#pragma unroll
    for (int r = 0; r < R; r++) keep[r] = 0u;
    for (int k = 0; k < cnt; k++) {
      const uint32_t pk = __shfl_sync(0xffffffffu, cur, k);
      int l[C::BETA];
#pragma unroll
      for (int b = 0; b < C::BETA; b++) l[b] = (int)(int8_t)(uint8_t)(pk >> (8 * b));
      int dA[R], dB[R];  // branch metrics, formed before the metrics' shuffles
#pragma unroll
      for (int r = 0; r < R; r++) {
        dA[r] = sA[r][0] * l[0];
        dB[r] = sB[r][0] * l[0];
#pragma unroll
        for (int b = 1; b < C::BETA; b++) {
          dA[r] += sA[r][b] * l[b];
          dB[r] += sB[r][b] * l[b];
        }
      }
      int qa[R], qb[R];
#pragma unroll
      for (int r = 0; r < R; r++) {
        qa[r] = __shfl_sync(0xffffffffu, m[r], la);
        qb[r] = __shfl_sync(0xffffffffu, m[r], lb);
      }
#pragma unroll
      for (int r = 0; r < R; r++) {
        int p0, p1;
        if constexpr (R == 1) {
          p0 = qa[0];
          p1 = qb[0];
        } else {
          p0 = (2 * r < R) ? qa[2 * r] : qb[2 * r - R];
          p1 = (2 * r < R) ? qa[2 * r + 1] : qb[2 * r - R + 1];
        }
        const int x0 = p0 + dA[r], x1 = p1 + dB[r];
        const uint32_t bal = __ballot_sync(0xffffffffu, live && x1 > x0);  // ties keep the even predecessor
        keep[r] = (lane == k) ? bal : keep[r];
        m[r] = x1 > x0 ? x1 : x0;
      }
    }
    if (i0 + lane < L) {
      uint32_t* p = dec + (int64_t)(i0 + lane) * R;
      if constexpr (R == 1) {
        p[0] = keep[0];
      } else if constexpr (R == 2) {
        *reinterpret_cast<uint2*>(p) = make_uint2(keep[0], keep[1]);
      } else {
#pragma unroll
        for (int q = 0; q < R / 4; q++)
          reinterpret_cast<uint4*>(p)[q] = make_uint4(keep[4 * q], keep[4 * q + 1], keep[4 * q + 2], keep[4 * q + 3]);
      }
    }
    if (((i0 >> 5) & 31) == 31) {  // every 1024 stages: subtract state 0's metric
      const int ref = __shfl_sync(0xffffffffu, m[0], 0);
#pragma unroll
      for (int r = 0; r < R; r++) m[r] -= ref;
    }
  }
  // traceback start: argmax, ties to the lowest state
  int best = R * lane, bv = m[0];
#pragma unroll
  for (int r = 1; r < R; r++)
    if (m[r] > bv) {
      bv = m[r];
      best = R * lane + r;
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
  if (h.e1 <= h.e0) return;
  // as in the other tracebacks: the decision read at iteration i is the
  // decoded bit of iteration i - (K-1); J = 2J + d kept unmasked holds the
  // decoded bits from its low end; bytes are taken at checkpoints every 8
  const int r0 = (int)(h.e0 - h.t0), r1 = (int)(h.e1 - h.t0);
  int nb = (r1 - r0 + 7) / 8 - 1;
  uint8_t* const out = h.out + (h.e0 >> 3);
  uint32_t J = h.end_zero ? 0u : (uint32_t)best;
  if (lane == 0) tb_emit(J, L - C::KM1, r0, r1, nb, out);  // bytes made of start-state bits only
  const int ib = r0 + C::KM1;                              // lowest iteration read
  if (ib >= L) return;
  // blocks of 32 stages [b0, b0 + 32) aligned to ib, the highest cut at L
  for (int b0 = ib + 32 * ((L - 1 - ib) / 32); b0 >= ib; b0 -= 32) {
    uint32_t w[R];
    const int my = b0 + lane;
    if (my < L) {
      const uint32_t* p = dec + (int64_t)my * R;
      if constexpr (R == 1) {
        w[0] = p[0];
      } else if constexpr (R == 2) {
        const uint2 v = *reinterpret_cast<const uint2*>(p);
        w[0] = v.x, w[1] = v.y;
      } else {
#pragma unroll
        for (int q = 0; q < R / 4; q++) {
          const uint4 v = reinterpret_cast<const uint4*>(p)[q];
          w[4 * q] = v.x, w[4 * q + 1] = v.y, w[4 * q + 2] = v.z, w[4 * q + 3] = v.w;
        }
      }
    } else {
#pragma unroll
      for (int r = 0; r < R; r++) w[r] = 0u;
    }
    const int top = (L - b0 < 32) ? L - b0 : 32;
    for (int k = top - 1; k >= 0; k--) {
      const uint32_t st = J & (uint32_t)(S - 1);
      uint32_t sel = w[0];
#pragma unroll
      for (int r = 1; r < R; r++) sel = ((st & (uint32_t)(R - 1)) == (uint32_t)r) ? w[r] : sel;
      const uint32_t word = __shfl_sync(0xffffffffu, sel, k);
      J = 2u * J + ((word >> (st / R)) & 1u);
      if (((b0 + k - ib) & 7) == 0 && lane == 0) tb_emit(J, b0 + k - C::KM1, r0, r1, nb, out);
    }
  }
}
#endif

}  // namespace vit
