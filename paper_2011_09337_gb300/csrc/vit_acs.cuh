// vit_acs.cuh -- lane-level soft-decision Viterbi decoding of two tiles at a
// time (arxiv 2011.09337, Eq. 2-4, Alg. 1-3), written for sm_103a.
//
// Data layout.  A lane owns a *pair* of tiles (windows of Fig. relworks).  The
// path metric of state j of tile A and of tile B share one 32-bit register:
//     reg = (sigma_B + 2^15) * 2^16 + (sigma_A + 2^15)
// Both 16-bit fields stay in [0, 2^16) because the metrics are renormalised
// every few stages, so one 32-bit integer add (IADD3, full rate on sm_103a)
// adds a packed branch metric to both tiles exactly, and max.u16x2 (also full
// rate) performs both compare-selects.  All 2^(K-1) states of the pair live in
// the lane's registers (K <= 7), so add-compare-select needs no data exchange.
//
// In-place trellis.  Register ("slot") s holds state rotr(s, r) after r stages
// (rotation over K-1 bits).  The radix-2 butterfly of Eq. 3 then reads and
// writes the same two slots, which differ in bit r mod (K-1); unrolling K-1
// stages turns the permutation into register renaming.  The decoded bit of a
// stage is the pair bit of the traced slot, and the predecessor slot replaces
// that bit with the survivor decision (Eq. 4), so traceback (Alg. 2) is a
// bit-field insert per stage.
//
// Survivor decisions.  decision = [odd-predecessor candidate > even one]
// (ties keep the lower predecessor).  E = X_even - X_odd + 2^15 as one 32-bit
// integer has bit 15 = NOT decision(tile A) and bit 31 = decision(tile B).
// prmt in sign-replicate mode turns two E words into four 0x00/0xff bytes and
// a masked OR places them in the stage's survivor words: bit 16*h + pos(s) of
// word wd(s) is the (A-inverted) decision of slot s, tile h.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define VIT_HD __host__ __device__ __forceinline__
#define VIT_CX __host__ __device__ constexpr
#else
#define VIT_HD inline
#define VIT_CX constexpr
#endif

namespace vit {

// ------------------------------------------------------------ compile time
VIT_CX int cpar(uint32_t x) {
  int p = 0;
  while (x) {
    p ^= 1;
    x &= x - 1u;
  }
  return p;
}
VIT_CX uint32_t rotr_w(uint32_t x, int r, int w) {
  return (r % w) == 0 ? x : (((x >> (r % w)) | (x << (w - (r % w)))) & ((1u << w) - 1u));
}

// A rate-1/beta code with constraint length K and generators G0..G3 (bit K-1
// taps the current input, Eq. 1).
template <int K_, int B_, uint32_t G0, uint32_t G1, uint32_t G2 = 0, uint32_t G3 = 0>
struct Code {
  static constexpr int K = K_, BETA = B_, KM1 = K_ - 1, S = 1 << (K_ - 1);
  static constexpr int NS = S;                       // slots per lane (lane-local trellis)
  static constexpr int WORDS = NS >= 16 ? NS / 16 : 1;  // survivor words per lane per stage
  static constexpr int HALFP = NS >= 16 ? 8 : NS / 2;   // prmt partner offset
  static constexpr int ND = 1 << (B_ - 1);           // branch-metric magnitudes per stage
  // stages per unrolled group: a multiple of K-1 (rotation period)
  static constexpr int U = KM1;
  // renormalise every RN groups (<= 16 stages keeps every field in range)
  static constexpr int RN = (12 / U) > 0 ? (12 / U) : 1;
  static VIT_CX uint32_t poly(int b) { return b == 0 ? G0 : b == 1 ? G1 : b == 2 ? G2 : G3; }
  // branch output alpha_out for register word R (Eq. 1), bit b = coded bit b
  static VIT_CX uint32_t aout(uint32_t R) {
    uint32_t o = 0;
    for (int b = 0; b < B_; b++) o |= (uint32_t)cpar(poly(b) & R) << b;
    return o;
  }
  static_assert(K_ >= 3 && K_ <= 7, "lane-local trellis holds at most 64 states");
  static_assert(B_ >= 2 && B_ <= 4, "beta in [2,4]");
};

// ------------------------------------------------------------ primitives
VIT_HD uint32_t vmaxu2(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
  uint32_t d;
  asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
#else
  const uint32_t lo = ((a & 0xffffu) > (b & 0xffffu)) ? (a & 0xffffu) : (b & 0xffffu);
  const uint32_t hi = ((a >> 16) > (b >> 16)) ? (a >> 16) : (b >> 16);
  return (hi << 16) | lo;
#endif
}

// prmt.b32 default mode: each selector nibble picks one of the 8 bytes of
// {b, a}; nibble bit 3 replicates that byte's sign bit.
VIT_HD uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
#if defined(__CUDA_ARCH__)
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
  return d;
#else
  const uint64_t src = ((uint64_t)b << 32) | a;
  uint32_t d = 0;
  for (int k = 0; k < 4; k++) {
    const uint32_t nib = (sel >> (4 * k)) & 0xfu;
    uint32_t byte = (uint32_t)(src >> (8 * (nib & 7u))) & 0xffu;
    if (nib & 8u) byte = (byte & 0x80u) ? 0xffu : 0u;
    d |= byte << (8 * k);
  }
  return d;
#endif
}

VIT_HD int ld_s8(const int8_t* p) {
#if defined(__CUDA_ARCH__)
  return (int)__ldg((const signed char*)p);
#else
  return (int)*p;
#endif
}

// ------------------------------------------------------- branch metrics
// delta_c for coded pattern c (Eq. 2) from the ND magnitudes D[c'] (c' with
// top bit 0): delta_{~c} = -delta_c.
template <class C>
VIT_HD uint32_t add_bm(uint32_t m, const uint32_t (&D)[C::ND], uint32_t c) {
  return ((c >> (C::BETA - 1)) & 1u) ? m - D[(~c) & (C::ND - 1)] : m + D[c];
}

// Packs the stage's LLRs of both tiles (int8, sign-extended) as
// L_b = l_A[b] + l_B[b] * 2^16 and forms D[c'] = sum_b (-1)^{c'_b} L_b.
template <class C>
VIT_HD void stage_bm(const int (&lA)[C::BETA], const int (&lB)[C::BETA], uint32_t (&D)[C::ND]) {
  int L[C::BETA];
#pragma unroll
  for (int b = 0; b < C::BETA; b++) L[b] = lA[b] + lB[b] * 65536;
#pragma unroll
  for (int c = 0; c < C::ND; c++) {
    int acc = 0;
#pragma unroll
    for (int b = 0; b < C::BETA; b++) acc += ((c >> b) & 1) ? -L[b] : L[b];
    D[c] = (uint32_t)acc;
  }
}

// Survivor-word position of slot s (tile h adds 16).
template <class C>
VIT_HD int surv_word(int s) {
  return C::NS >= 16 ? (s >> 4) : 0;
}
template <class C>
VIT_HD uint32_t pick_word(const uint32_t (&w)[C::WORDS], int s) {
  if constexpr (C::WORDS == 4) {
    const uint32_t lo = (s & 16) ? w[1] : w[0];
    const uint32_t hi = (s & 16) ? w[3] : w[2];
    return (s & 32) ? hi : lo;
  } else if constexpr (C::WORDS == 2) {
    return (s & 16) ? w[1] : w[0];
  } else {
    return w[0];
  }
}
template <class C>
VIT_HD int surv_pos(int s) {
  return (s & (C::HALFP - 1)) + ((s & C::HALFP) ? 8 : 0);
}

// One radix-2 butterfly (Eq. 3, Eq. 4): slots a (even predecessor) and
// b = a | 2^P (odd predecessor) are replaced by the two successors.
template <class C, int P>
VIT_HD void butterfly(uint32_t (&m)[C::NS], const uint32_t (&D)[C::ND], int a, uint32_t& Ea, uint32_t& Eb) {
  const int b = a | (1 << P);
  const uint32_t i0 = rotr_w((uint32_t)a, P, C::KM1);  // even predecessor state in slot a
  const uint32_t c00 = C::aout(i0), c01 = C::aout(i0 | 1u);
  const uint32_t c10 = C::aout(i0 | (uint32_t)C::S), c11 = C::aout(i0 | (uint32_t)C::S | 1u);
  const uint32_t x00 = add_bm<C>(m[a], D, c00), x01 = add_bm<C>(m[b], D, c01);
  const uint32_t x10 = add_bm<C>(m[a], D, c10), x11 = add_bm<C>(m[b], D, c11);
  Ea = x00 - x01 + 0x8000u;
  Eb = x10 - x11 + 0x8000u;
  m[a] = vmaxu2(x00, x01);  // successor state (i0 >> 1) lands in slot a
  m[b] = vmaxu2(x10, x11);  // successor state (i0 >> 1) + S/2 lands in slot b
}

// Places the decisions of slots s and s + HALFP (both tiles) into the
// stage's survivor words.
template <class C>
VIT_HD void gather2(uint32_t (&w)[C::WORDS], int s, uint32_t Es, uint32_t Ep) {
  const uint32_t t = prmt(Es, Ep, 0xFBD9u);
  w[surv_word<C>(s)] |= t & (0x01010101u << (s & (C::HALFP - 1)));
}

// One add-compare-select stage for phase P = stage mod (K-1).  Butterflies
// are visited so that the two slots each prmt combines (s, s + HALFP) are
// finished together, which keeps few decision words live.
template <class C, int P>
VIT_HD void acs_stage(uint32_t (&m)[C::NS], const uint32_t (&D)[C::ND], uint32_t (&w)[C::WORDS]) {
  constexpr int H = C::HALFP;
  constexpr int B = 1 << P;
#pragma unroll
  for (int k = 0; k < C::WORDS; k++) w[k] = 0u;
  if constexpr (B == H) {
    // the butterfly partner is the prmt partner
#pragma unroll
    for (int a = 0; a < C::NS; a++) {
      if (a & B) continue;
      uint32_t Ea, Eb;
      butterfly<C, P>(m, D, a, Ea, Eb);
      gather2<C>(w, a, Ea, Eb);
    }
  } else {
#pragma unroll
    for (int a = 0; a < C::NS; a++) {
      if ((a & B) || (a & H)) continue;
      uint32_t E0, E1, E2, E3;  // slots a, a|B, a|H, a|B|H
      butterfly<C, P>(m, D, a, E0, E1);
      butterfly<C, P>(m, D, a | H, E2, E3);
      gather2<C>(w, a, E0, E2);
      gather2<C>(w, a | B, E1, E3);
    }
  }
}

// Subtracts the metric of slot 0 from every slot (both tiles) and re-biases.
template <class C>
VIT_HD void renorm(uint32_t (&m)[C::NS]) {
  const uint32_t r = m[0];
#pragma unroll
  for (int s = 0; s < C::NS; s++) m[s] = m[s] - r + 0x80008000u;
}

// Initial metrics of one tile (h = 0: low field, 1: high field): state 0 gets
// 0 and the others -M for a known start; all 0 otherwise.
template <class C>
VIT_HD void init_half(uint32_t (&m)[C::NS], int h, bool known, uint32_t M) {
  const uint32_t keep = h ? 0x0000ffffu : 0xffff0000u;
#pragma unroll
  for (int s = 0; s < C::NS; s++) {
    const uint32_t v = (known && s != 0) ? (0x8000u - M) : 0x8000u;
    m[s] = (m[s] & keep) | (v << (16 * h));
  }
}

// One tile handled by one 16-bit half of a lane.
struct Half {
  const int8_t* llr;  // frame LLRs, depunctured, stage-major
  uint8_t* out;       // frame output bits (packed LSB-first)
  int64_t t0, t1;     // window [t0, t1)
  int64_t e0, e1;     // emitted stages [e0, e1)
  int start;          // iteration of stage t0 (end-aligned windows)
  int known;          // known start state 0
  int end_zero;       // traceback starts in state 0
  int active;
};

// A frame and the tiling of Fig. relworks.
struct Frame {
  const int8_t* llr;  // depunctured, stage-major int8
  uint8_t* out;       // packed output bits
  int64_t n;          // trellis stages
  int64_t n_out;      // emitted bits (n, or n - (K-1) when terminated)
  int mode;           // 0 stream, 1 terminated, 2 free start
};
struct Tiling {
  int64_t f, v1, v2;  // f == 0: one tile per frame
};

VIT_HD int64_t tile_len(int64_t n, int64_t f) { return (f == 0 || f > n) ? n : f; }
VIT_HD int64_t tile_count(int64_t n, int64_t f) {
  const int64_t fb = tile_len(n, f);
  return n > 0 ? (n + fb - 1) / fb : 0;
}

// Tile b of a frame: emits [b*f, (b+1)*f) from the window
// [b*f - v1, (b+1)*f + v2), both clipped to [0, n).
VIT_HD Half make_half(const Frame& fr, int64_t b, const Tiling& tl) {
  Half h;
  const int64_t fb = tile_len(fr.n, tl.f);
  const int64_t e0 = b * fb;
  const int64_t e1 = (e0 + fb < fr.n) ? e0 + fb : fr.n;
  h.llr = fr.llr;
  h.out = fr.out;
  h.t0 = (e0 - tl.v1 > 0) ? e0 - tl.v1 : 0;
  h.t1 = (e1 + tl.v2 < fr.n) ? e1 + tl.v2 : fr.n;
  h.e0 = e0;
  h.e1 = (e1 < fr.n_out) ? e1 : fr.n_out;
  h.known = (h.t0 == 0 && fr.mode != 2) ? 1 : 0;
  h.end_zero = (h.t1 == fr.n && fr.mode == 1) ? 1 : 0;
  h.active = 1;
  h.start = 0;
  return h;
}

VIT_HD Half idle_half() {
  Half h;
  h.llr = nullptr;
  h.out = nullptr;
  h.t0 = h.t1 = h.e0 = h.e1 = 0;
  h.known = h.end_zero = h.active = h.start = 0;
  return h;
}

// Survivor store: words of stage i at base + i*stride (+ k).
struct Slab {
  uint32_t* base;
  int64_t stride;
};

template <class C>
VIT_HD void load_stage_llr(const Half (&hw)[2], int i, bool masked, int (&lA)[C::BETA], int (&lB)[C::BETA]) {
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const bool on = !masked || (i >= hw[h].start);
    const int64_t t = hw[h].t0 + (int64_t)(i - hw[h].start);
    const int8_t* p = hw[h].llr + (on ? t : hw[h].t0) * C::BETA;
#pragma unroll
    for (int b = 0; b < C::BETA; b++) {
      const int v = (on && hw[h].active) ? ld_s8(p + b) : 0;
      if (h == 0)
        lA[b] = v;
      else
        lB[b] = v;
    }
  }
}

VIT_HD void store_words4(uint32_t* p, const uint32_t* w, int n) {
#if defined(__CUDA_ARCH__)
  if (n == 4) {
    *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
    return;
  }
  if (n == 2) {
    *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
    return;
  }
#endif
  for (int k = 0; k < n; k++) p[k] = w[k];
}

// Forward procedure over the window of both tiles: Lw iterations (a multiple
// of U), survivor words to the slab.  masked_until: iterations below it may
// contain pre-start stages of some lane of the warp.
template <class C, int P>
VIT_HD void fwd_one(uint32_t (&m)[C::NS], const Half (&hw)[2], int i, bool masked, uint32_t M, Slab sl) {
  int lA[C::BETA], lB[C::BETA];
  load_stage_llr<C>(hw, i, masked, lA, lB);
  if (masked) {
    // a known-start tile begins here: set its initial metrics
#pragma unroll
    for (int h = 0; h < 2; h++)
      if (hw[h].known && i == hw[h].start) init_half<C>(m, h, true, M);
  }
  uint32_t D[C::ND];
  stage_bm<C>(lA, lB, D);
  uint32_t w[C::WORDS];
  acs_stage<C, P>(m, D, w);
  store_words4(sl.base + (int64_t)i * sl.stride, w, C::WORDS);
}

template <class C, int P>
VIT_HD void fwd_group(uint32_t (&m)[C::NS], const Half (&hw)[2], int i0, bool masked, uint32_t M, Slab sl) {
  if constexpr (P < C::KM1) {
    fwd_one<C, P>(m, hw, i0 + P, masked, M, sl);
    fwd_group<C, P + 1>(m, hw, i0, masked, M, sl);
  }
}

// Traceback (Alg. 2) of both tiles from the end of the window.
template <class C, int P>
VIT_HD void tb_one(int i, const uint32_t (&w)[C::WORDS], int (&s)[2], uint32_t (&acc)[2], const Half (&hw)[2]) {
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int64_t t = hw[h].t0 + (int64_t)(i - hw[h].start);
    const int slot = s[h];
    const uint32_t word = pick_word<C>(w, slot);
    const uint32_t d = ((word >> (16 * h + surv_pos<C>(slot))) & 1u) ^ (h == 0 ? 1u : 0u);
    const uint32_t bit = (uint32_t)(slot >> P) & 1u;
    s[h] = (slot & ~(1 << P)) | (int)(d << P);
    if (hw[h].active && t >= hw[h].e0 && t < hw[h].e1) {
      acc[h] |= bit << (t & 7);
      if ((t & 7) == 0 || t == hw[h].e0) {
        hw[h].out[t >> 3] = (uint8_t)acc[h];
        acc[h] = 0;
      }
    }
  }
}

template <class C>
VIT_HD void load_words(const Slab& sl, int i, uint32_t* w) {
#if defined(__CUDA_ARCH__)
  const uint32_t* p = sl.base + (int64_t)i * sl.stride;
  if (C::WORDS == 4) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    w[0] = v.x, w[1] = v.y, w[2] = v.z, w[3] = v.w;
    return;
  }
  if (C::WORDS == 2) {
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    w[0] = v.x, w[1] = v.y;
    return;
  }
  w[0] = p[0];
#else
  for (int k = 0; k < C::WORDS; k++) w[k] = sl.base[(int64_t)i * sl.stride + k];
#endif
}

// stages of a group go from i0 + K-2 down to i0
template <class C, int P>
VIT_HD void tb_group(int i0, const uint32_t (&w)[C::KM1][C::WORDS], int (&s)[2], uint32_t (&acc)[2],
                     const Half (&hw)[2]) {
  if constexpr (P < C::KM1) {
    constexpr int Q = C::KM1 - 1 - P;
    tb_one<C, Q>(i0 + Q, w[Q], s, acc, hw);
    tb_group<C, P + 1>(i0, w, s, acc, hw);
  }
}

// Decodes the two tiles of one lane.  Lw: iterations (multiple of K-1, at
// least every active window length); masked_until: first iteration from which
// every window of the warp has started.
template <class C>
VIT_HD void decode_pair(const Half (&hw)[2], int Lw, int masked_until, uint32_t M, Slab sl) {
  uint32_t m[C::NS];
#pragma unroll
  for (int s = 0; s < C::NS; s++) m[s] = 0x80008000u;
  // tiles that begin at iteration 0 with a known start
#pragma unroll
  for (int h = 0; h < 2; h++)
    if (hw[h].known && hw[h].start == 0) init_half<C>(m, h, true, M);

  const int ngroups = Lw / C::U;
  for (int g = 0; g < ngroups; g++) {
    const int i0 = g * C::U;
    const bool masked = i0 < masked_until;
    fwd_group<C, 0>(m, hw, i0, masked, M, sl);
    if ((g % C::RN) == C::RN - 1) renorm<C>(m);
  }

  // traceback start (Alg. 2): after Lw stages (a multiple of K-1) slot = state
  int s[2];
#pragma unroll
  for (int h = 0; h < 2; h++) {
    int best = 0;
    uint32_t bv = (m[0] >> (16 * h)) & 0xffffu;
#pragma unroll
    for (int q = 1; q < C::NS; q++) {
      const uint32_t v = (m[q] >> (16 * h)) & 0xffffu;
      if (v > bv) {
        bv = v;
        best = q;
      }
    }
    s[h] = hw[h].end_zero ? 0 : best;
  }

  // lowest iteration that still emits a bit, over both tiles
  int stop = Lw;
#pragma unroll
  for (int h = 0; h < 2; h++)
    if (hw[h].active && hw[h].e1 > hw[h].e0) {
      const int it = hw[h].start + (int)(hw[h].e0 - hw[h].t0);
      stop = it < stop ? it : stop;
    }
  const int gstop = stop / C::U;
  uint32_t acc[2] = {0u, 0u};
  for (int g = ngroups - 1; g >= gstop; g--) {
    const int i0 = g * C::U;
    uint32_t w[C::KM1][C::WORDS];
#pragma unroll
    for (int q = 0; q < C::KM1; q++) load_words<C>(sl, i0 + q, w[q]);
    tb_group<C, 0>(i0, w, s, acc, hw);
  }
}

}  // namespace vit
