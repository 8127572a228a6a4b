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
// Trellis layout.  Register j holds state j.  A radix-2 butterfly (Eq. 3)
// reads states 2x and 2x+1 and writes states x and x + S/2 into a second
// register array; the next stage reads that array the same way, so two
// unrolled stages (array A -> B -> A) cover the whole permutation with
// register renaming and a small loop body.  Traceback (Alg. 2) follows
// predecessor (2j + decision) mod S and outputs bit K-2 of each state.
//
// Survivor decisions.  decision = [odd-predecessor candidate > even one]
// (ties keep the lower predecessor).  E = X_even - X_odd + 2^15 as one 32-bit
// integer has bit 15 = NOT decision(tile A) and bit 31 = decision(tile B).
// prmt in sign-replicate mode turns two E words into four 0x00/0xff bytes and
// a masked OR places them in the stage's survivor words: bit 16*h + pos(s) of
// word wd(j) is the (A-inverted) decision of state j, tile h.
#pragma once
#include <stdint.h>
#include <string.h>

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

constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }

// A rate-1/beta code with constraint length K and generators G0..G3 (bit K-1
// taps the current input, Eq. 1).  NSMAX caps the states one lane holds: a
// smaller cap spreads each tile pair over more lanes (S / NSMAX), which
// gives frames with few tiles more warps.
template <int K_, int B_, uint32_t G0, uint32_t G1, uint32_t G2 = 0, uint32_t G3 = 0, int NSMAX = 64>
struct Code {
  static constexpr int K = K_, BETA = B_, KM1 = K_ - 1, S = 1 << (K_ - 1);
  static constexpr int NS = S < NSMAX ? S : NSMAX;      // states (slots) per lane
  static constexpr int G = S / NS;                      // lanes per tile pair
  static constexpr int NSB = ilog2c(NS);                // slot bits held in registers
  static constexpr int WORDS = NS >= 16 ? NS / 16 : 1;  // survivor words per lane per stage
  static constexpr int HALFP = NS >= 16 ? 8 : NS / 2;   // prmt partner offset
  static constexpr int ND = 1 << (B_ - 1);              // branch-metric magnitudes per stage
  // stages per unrolled group: two alternating register arrays (one lane per
  // pair) or the K-1 phases of the rotating slot map (several lanes per pair)
  static constexpr int U = (G == 1) ? 2 : KM1;
  // Renormalise every RN groups.  Path metrics of one tile spread by at most
  // SPREAD = M + 2(K-2)*127*beta < 4(K-1)*127*beta + 1 (M: the finite
  // -infinity of a known start), and each stage moves a metric by at most
  // DMAX = 127*beta, so RN*U stages keep every candidate within
  // SPREAD + (RN*U + 1)*DMAX <= 2^15 - 1 of the reference state.
  static constexpr int DMAX = 127 * B_;
  static constexpr int SPREAD = 4 * KM1 * 127 * B_ + 1;
  static constexpr int RN_MAX = ((32767 - SPREAD) / DMAX - 1) / U;
  static constexpr int RN = RN_MAX < 1 ? 1 : (RN_MAX > 32 ? 32 : RN_MAX);
  static_assert(SPREAD + 2 * DMAX < 32768, "decision differences must fit 16 bits");
  static VIT_CX uint32_t poly(int b) { return b == 0 ? G0 : b == 1 ? G1 : b == 2 ? G2 : G3; }
  // branch output alpha_out for register word R (Eq. 1), bit b = coded bit b
  static VIT_CX uint32_t aout(uint32_t R) {
    uint32_t o = 0;
    for (int b = 0; b < B_; b++) o |= (uint32_t)cpar(poly(b) & R) << b;
    return o;
  }
  // every generator taps both the current and the oldest input: the four
  // branches of a butterfly carry +-delta of one pattern
  static constexpr bool SYMMETRIC = ((G0 & G1 & (B_ > 2 ? G2 : ~0u) & (B_ > 3 ? G3 : ~0u)) & 1u) &&
                                    ((G0 & G1 & (B_ > 2 ? G2 : ~0u) & (B_ > 3 ? G3 : ~0u)) >> (K_ - 1) & 1u);
  static constexpr bool GENERIC = false;  // patterns fixed at compile time
  static_assert(K_ >= 3 && K_ <= 9, "K in [3, 9]");
  static_assert(B_ >= 2 && B_ <= 4, "beta in [2,4]");
  static_assert(G == 1 || SYMMETRIC, "codes spread over several lanes need the butterfly symmetry");
};

// Output pattern of register word R (Eq. 1) for generators known at run time.
VIT_HD uint32_t aout_rt(const uint32_t* polys, int beta, uint32_t R) {
  uint32_t o = 0;
  for (int b = 0; b < beta; b++) o |= (uint32_t)cpar(polys[b] & R) << b;
  return o;
}

// A rate-1/beta code with constraint length K whose generators are known
// only at run time.  It is decoded by the warp-per-tile decoders, whose
// lanes form the branch patterns of their own states from the generators
// once per tile.
template <int K_, int B_>
struct GCode {
  static constexpr int K = K_, BETA = B_, KM1 = K_ - 1, S = 1 << (K_ - 1);
  static constexpr bool GENERIC = true;
  static_assert(K_ >= 3 && K_ <= 9, "K in [3, 9]");
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
// Branch metrics of one stage: D[c'] for the patterns c' with top bit 0,
// integer encoded for both tiles.
template <class C>
struct StageBM {
  uint32_t D[C::ND];
};

template <class C>
VIT_HD uint32_t add_bm(uint32_t m, const StageBM<C>& bm, uint32_t c) {
  return ((c >> (C::BETA - 1)) & 1u) ? m - bm.D[(~c) & (C::ND - 1)] : m + bm.D[c];
}

// Signed branch metric of pattern c (integer encoded for both tiles).
template <class C>
VIT_HD uint32_t bmv(const StageBM<C>& bm, uint32_t c) {
  return ((c >> (C::BETA - 1)) & 1u) ? 0u - bm.D[(~c) & (C::ND - 1)] : bm.D[c];
}

// x + k as one integer multiply-add, x * kOne + k, with the multiplier read
// from constant memory (1; unknown to the compiler, so the add stays an IMAD
// and issues on the FMA pipe, leaving the ALU pipe to max, prmt and lop3).
#if defined(__CUDACC__)
static __constant__ uint32_t kOne = 1u;
// multipliers -4..4 for y + c * x on the FMA pipe (index c + 4)
static __constant__ uint32_t kSmall[9] = {0xfffffffcu, 0xfffffffdu, 0xfffffffeu, 0xffffffffu, 0u, 1u, 2u, 3u, 4u};
#endif
VIT_HD uint32_t add_on_fma(uint32_t x, uint32_t k) {
#if defined(__CUDA_ARCH__)
  uint32_t r;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(kOne), "r"(k));
  return r;
#else
  return x + k;
#endif
}

// y + c * x for a compile-time c in [-4, 4], as one multiply-add whose
// multiplier comes from constant memory (so it issues on the FMA pipe).
template <int c>
VIT_HD uint32_t mad_small(uint32_t x, uint32_t y) {
  static_assert(c >= -4 && c <= 4, "multiplier in [-4, 4]");
#if defined(__CUDA_ARCH__)
  uint32_t r;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(kSmall[c + 4]), "r"(y));
  return r;
#else
  return y + (uint32_t)c * x;
#endif
}

// Packs the stage's LLRs of both tiles (int8, sign-extended) as
// L_b = l_A[b] + l_B[b] * 2^16 and forms D[c'] = sum_b (-1)^{c'_b} L_b.
template <class C>
VIT_HD void stage_bm(const int (&lA)[C::BETA], const int (&lB)[C::BETA], StageBM<C>& D) {
  int L[C::BETA];
#pragma unroll
  for (int b = 0; b < C::BETA; b++) L[b] = lA[b] + lB[b] * 65536;
#pragma unroll
  for (int c = 0; c < C::ND; c++) {
    int acc = 0;
#pragma unroll
    for (int b = 0; b < C::BETA; b++) acc += ((c >> b) & 1) ? -L[b] : L[b];
    D.D[c] = (uint32_t)acc;
  }
}

// Survivor-word position of slot s (tile h adds 16).
template <class C>
VIT_CX int surv_word(int s) {
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

// Coefficient of magnitude D[i] in d(c10) - d(c11) - d(c00) + d(c01), with
// d(c) = D[c] for patterns whose top bit is 0 and -D[~c] otherwise.
template <class C>
VIT_CX int bf_coef(uint32_t c00, uint32_t c01, uint32_t c10, uint32_t c11, int i) {
  auto term = [](uint32_t c, int i) -> int {
    const bool top = ((c >> (C::BETA - 1)) & 1u) != 0;
    const uint32_t idx = top ? ((~c) & (uint32_t)(C::ND - 1)) : c;
    return (idx == (uint32_t)i) ? (top ? -1 : 1) : 0;
  };
  return term(c10, i) - term(c11, i) - term(c00, i) + term(c01, i);
}
template <class C>
VIT_CX int bf_nonzero(uint32_t c00, uint32_t c01, uint32_t c10, uint32_t c11) {
  int n = 0;
  for (int i = 0; i < C::ND; i++) n += bf_coef<C>(c00, c01, c10, c11, i) != 0 ? 1 : 0;
  return n;
}
template <class C>
VIT_CX int bf_index(uint32_t c00, uint32_t c01, uint32_t c10, uint32_t c11) {
  for (int i = 0; i < C::ND; i++)
    if (bf_coef<C>(c00, c01, c10, c11, i) != 0) return i;
  return 0;
}

// One radix-2 butterfly (Eq. 3, Eq. 4): predecessors 2x (even) and 2x+1
// (odd) of mi give successors x and x + S/2 in mo, with their decision words.
template <class C, int x>
VIT_HD void butterfly(const uint32_t (&mi)[C::NS], uint32_t (&mo)[C::NS], const StageBM<C>& D, uint32_t& E0,
                      uint32_t& E1) {
  constexpr int H = C::NS / 2;
  constexpr uint32_t i0 = 2u * (uint32_t)x;
  constexpr uint32_t c00 = C::aout(i0), c01 = C::aout(i0 | 1u);
  constexpr uint32_t c10 = C::aout(i0 | (uint32_t)C::S), c11 = C::aout(i0 | (uint32_t)C::S | 1u);
  const uint32_t x00 = add_bm<C>(mi[2 * x], D, c00), x01 = add_bm<C>(mi[2 * x + 1], D, c01);
  const uint32_t x10 = add_bm<C>(mi[2 * x], D, c10), x11 = add_bm<C>(mi[2 * x + 1], D, c11);
  E0 = x00 - x01 + 0x8000u;
  // x10 - x11 = (x00 - x01) + (d(c10) - d(c11) - d(c00) + d(c01)): the
  // bracket is a sum of the stage's magnitudes D[i] with small integer
  // coefficients; with one nonzero coefficient (every generator tapping the
  // current and the oldest input) it is one multiply-add onto E0, otherwise
  // the bracket is formed once per stage and added
  constexpr int nz = bf_nonzero<C>(c00, c01, c10, c11);
  if constexpr (nz == 1) {
    constexpr int i = bf_index<C>(c00, c01, c10, c11);
    constexpr int k = bf_coef<C>(c00, c01, c10, c11, i);
    E1 = mad_small<k>(D.D[i], E0);
  } else {
    E1 = add_on_fma(E0, bmv<C>(D, c10) - bmv<C>(D, c11) - bmv<C>(D, c00) + bmv<C>(D, c01));
  }
  mo[x] = vmaxu2(x00, x01);
  mo[x + H] = vmaxu2(x10, x11);
}

// Places the decisions of states s and s + HALFP (both tiles) into the
// stage's survivor words.
template <class C>
VIT_HD void gather2(uint32_t (&w)[C::WORDS], int s, uint32_t Es, uint32_t Ep) {
  const uint32_t t = prmt(Es, Ep, 0xFBD9u);
  w[surv_word<C>(s)] |= t & (0x01010101u << (s & (C::HALFP - 1)));
}

// The same when the states of each survivor word arrive in increasing
// position order: the word's first pair (position 0) initialises it, and each
// later pair at position p keeps the word's bits below p of every byte and
// takes the rest from the new sign bytes (one three-input select).
template <class C, int s>
VIT_HD void gather2_ordered(uint32_t (&w)[C::WORDS], uint32_t Es, uint32_t Ep) {
  constexpr int p = s & (C::HALFP - 1);
  constexpr int k = surv_word<C>(s);
  const uint32_t t = prmt(Es, Ep, 0xFBD9u);
  if constexpr (p == 0) {
    w[k] = t;
  } else {
    constexpr uint32_t keep = 0x01010101u * ((1u << p) - 1u);
    w[k] = (w[k] & keep) | (t & ~keep);
  }
}

// One add-compare-select stage from mi to mo.  Butterflies are visited so
// that the two states each prmt combines (s, s + HALFP) are finished
// together, which keeps few decision words live, and so that every survivor
// word receives its positions in increasing order.
template <class C, int x>
VIT_HD void acs_from(const uint32_t (&mi)[C::NS], uint32_t (&mo)[C::NS], const StageBM<C>& D,
                     uint32_t (&w)[C::WORDS]) {
  constexpr int H = C::NS / 2;
  constexpr int HP = C::HALFP;
  if constexpr (x < H) {
    if constexpr (H == HP) {
      // the two successors of a butterfly are a prmt pair
      uint32_t E0, E1;
      butterfly<C, x>(mi, mo, D, E0, E1);
      gather2_ordered<C, x>(w, E0, E1);
    } else if constexpr ((x & HP) == 0) {
      uint32_t Ea, Eb, Ec, Ed;  // successors x, x+H, x+HP, x+HP+H
      butterfly<C, x>(mi, mo, D, Ea, Eb);
      butterfly<C, x + HP>(mi, mo, D, Ec, Ed);
      gather2_ordered<C, x>(w, Ea, Ec);
      gather2_ordered<C, x + H>(w, Eb, Ed);
    }
    acs_from<C, x + 1>(mi, mo, D, w);
  }
}

template <class C>
VIT_HD void acs_stage(const uint32_t (&mi)[C::NS], uint32_t (&mo)[C::NS], const StageBM<C>& D,
                      uint32_t (&w)[C::WORDS]) {
  acs_from<C, 0>(mi, mo, D, w);
}

// Subtracts the metric of state 0 from every state (both tiles) and re-biases.
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

// LLRs of U consecutive stages for both tiles, as sign-extended ints.
template <class C>
struct LlrGroup {
  int v[C::U][2][C::BETA];
};

// Loads the LLRs of the U stages starting at iteration i.  Stages before a
// tile's window start read the window's first stage (always a valid
// address); masking to zero happens at use.
template <class C>
VIT_HD void load_group(const Half (&hw)[2], int i, LlrGroup<C>& g) {
#pragma unroll
  for (int u = 0; u < C::U; u++)
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int it = i + u;
      const int64_t t = hw[h].t0 + (int64_t)((it > hw[h].start ? it : hw[h].start) - hw[h].start);
      const int8_t* p = hw[h].llr + t * C::BETA;
#pragma unroll
      for (int b = 0; b < C::BETA; b++) g.v[u][h][b] = hw[h].active ? ld_s8(p + b) : 0;
    }
}

// Same loads once every window of the warp has started: stage t of tile h is
// at llr + (t0 - start + i) * beta, one base address per group.
template <class C>
VIT_HD void load_group_fast(const Half (&hw)[2], int i, LlrGroup<C>& g) {
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int8_t* p = hw[h].llr + (hw[h].t0 - hw[h].start + (int64_t)i) * C::BETA;
#pragma unroll
    for (int u = 0; u < C::U; u++)
#pragma unroll
      for (int b = 0; b < C::BETA; b++) g.v[u][h][b] = hw[h].active ? ld_s8(p + u * C::BETA + b) : 0;
  }
}

// Word loads: when every tile's group of U stages starts on a 4-byte boundary
// (U*beta a multiple of 4), one 32-bit load per tile fetches the group's
// LLRs, and prmt spreads them; 4x fewer load instructions and L1 wavefronts
// than byte loads.
template <class C>
constexpr bool kWordLoads = (C::U * C::BETA) % 4 == 0;

template <class C>
VIT_HD uint32_t ld_u32(const int8_t* p) {
#if defined(__CUDA_ARCH__)
  return __ldg(reinterpret_cast<const unsigned int*>(p));
#else
  uint32_t v;
  memcpy(&v, p, 4);
  return v;
#endif
}

template <class C>
VIT_HD void load_group_words(const Half (&hw)[2], int i, uint32_t (&w)[2][C::U * C::BETA / 4]) {
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int8_t* p = hw[h].llr + (hw[h].t0 - hw[h].start + (int64_t)i) * C::BETA;
#pragma unroll
    for (int k = 0; k < C::U * C::BETA / 4; k++) w[h][k] = hw[h].active ? ld_u32<C>(p + 4 * k) : 0u;
  }
}

// Sign-extended byte q of the group's words of tile h.
template <class C>
VIT_HD int word_byte(const uint32_t (&w)[2][C::U * C::BETA / 4], int h, int q) {
  return (int)(int8_t)((w[h][q >> 2] >> (8 * (q & 3))) & 0xffu);
}

// Integer-encoded LLR pairs L_b = l_A[b] + l_B[b] * 2^16 of stage u of a
// group, from the group's words: prmt forms the sign-extended 16-bit fields
// [l_B : l_A], and subtracting 2^16 when l_A < 0 turns the field pair into
// the integer encoding.
template <class C, int u>
VIT_HD void pairs_from_words(const uint32_t (&w)[2][C::U * C::BETA / 4], int (&L)[C::BETA]) {
#pragma unroll
  for (int b = 0; b < C::BETA; b++) {
    const int q = u * C::BETA + b;  // byte of the group
    const int k = q >> 2, j = q & 3;
    const uint32_t sel = (uint32_t)j | ((8u | (uint32_t)j) << 4) | ((4u + (uint32_t)j) << 8) |
                         ((8u | (4u + (uint32_t)j)) << 12);
    const uint32_t c = prmt(w[0][k], w[1][k], sel);
    L[b] = (int)(c - ((c & 0x8000u) << 1));
  }
}

// Branch magnitudes of stage u of a group straight from the group's words:
// the prmt fields c_b = [l_B : l_A] (sign-extended halves) with bit 15
// flipped are X_b = L_b + 2^15 in the integer encoding (the flip adds 2^15
// when l_A >= 0 and turns the field's 2^16 - |l_A| into 2^15 - |l_A| when
// l_A < 0), so D[c'] = sum_b (-1)^{c'_b} X_b - (sum_b (-1)^{c'_b}) 2^15.
template <class C, int u>
VIT_HD void bm_from_words(const uint32_t (&w)[2][C::U * C::BETA / 4], StageBM<C>& D) {
  uint32_t X[C::BETA];
#pragma unroll
  for (int b = 0; b < C::BETA; b++) {
    const int q = u * C::BETA + b;  // byte of the group
    const int k = q >> 2, j = q & 3;
    const uint32_t sel = (uint32_t)j | ((8u | (uint32_t)j) << 4) | ((4u + (uint32_t)j) << 8) |
                         ((8u | (4u + (uint32_t)j)) << 12);
    X[b] = prmt(w[0][k], w[1][k], sel) ^ 0x8000u;
  }
#pragma unroll
  for (int c = 0; c < C::ND; c++) {
    uint32_t acc = 0;
    int nsum = 0;
#pragma unroll
    for (int b = 0; b < C::BETA; b++) {
      acc = ((c >> b) & 1) ? acc - X[b] : acc + X[b];
      nsum += ((c >> b) & 1) ? -1 : 1;
    }
    D.D[c] = acc - (uint32_t)nsum * 0x8000u;
  }
}

template <class C>
VIT_HD void bm_from_pairs(const int (&L)[C::BETA], StageBM<C>& D) {
#pragma unroll
  for (int c = 0; c < C::ND; c++) {
    int acc = 0;
#pragma unroll
    for (int b = 0; b < C::BETA; b++) acc += ((c >> b) & 1) ? -L[b] : L[b];
    D.D[c] = (uint32_t)acc;
  }
}

VIT_HD void store_words(uint32_t* p, const uint32_t* w, int n) {
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

template <class C>
VIT_HD void load_words(const Slab& sl, int i, uint32_t (&w)[C::WORDS]) {
#if defined(__CUDA_ARCH__)
  const uint32_t* p = sl.base + (int64_t)i * sl.stride;
  if constexpr (C::WORDS == 4) {
    const uint4 v = *reinterpret_cast<const uint4*>(p);
    w[0] = v.x, w[1] = v.y, w[2] = v.z, w[3] = v.w;
  } else if constexpr (C::WORDS == 2) {
    const uint2 v = *reinterpret_cast<const uint2*>(p);
    w[0] = v.x, w[1] = v.y;
  } else {
    w[0] = p[0];
  }
#else
  for (int k = 0; k < C::WORDS; k++) w[k] = sl.base[(int64_t)i * sl.stride + k];
#endif
}

// One stage: branch metrics of both tiles (masked before a window's start),
// the known-start reset, add-compare-select from mi to mo, survivor store.
template <class C>
VIT_HD void fwd_stage(uint32_t (&mi)[C::NS], uint32_t (&mo)[C::NS], const Half (&hw)[2], int i, bool masked,
                      uint32_t M, const int (&lv)[2][C::BETA], Slab sl) {
  int lA[C::BETA], lB[C::BETA];
#pragma unroll
  for (int b = 0; b < C::BETA; b++) {
    lA[b] = lv[0][b];
    lB[b] = lv[1][b];
  }
  if (masked) {
#pragma unroll
    for (int b = 0; b < C::BETA; b++) {
      lA[b] = (i >= hw[0].start) ? lA[b] : 0;
      lB[b] = (i >= hw[1].start) ? lB[b] : 0;
    }
    // a known-start tile begins at this stage: set its initial metrics
#pragma unroll
    for (int h = 0; h < 2; h++)
      if (hw[h].known && i == hw[h].start) init_half<C>(mi, h, true, M);
  }
  StageBM<C> D;
  stage_bm<C>(lA, lB, D);
  uint32_t w[C::WORDS];
  acs_stage<C>(mi, mo, D, w);
  store_words(sl.base + (int64_t)i * sl.stride, w, C::WORDS);
}

// Forward stage fed by word loads (every window of the warp has started).
template <class C, int u>
VIT_HD void fwd_stage_words(uint32_t (&mi)[C::NS], uint32_t (&mo)[C::NS], int i,
                            const uint32_t (&w)[2][C::U * C::BETA / 4], Slab sl) {
  StageBM<C> D;
  bm_from_words<C, u>(w, D);
  uint32_t wd[C::WORDS];
  acs_stage<C>(mi, mo, D, wd);
  store_words(sl.base + (int64_t)i * sl.stride, wd, C::WORDS);
}

// x >> (n mod 32) (funnel shift of x with itself; only the low 5 bits of n
// are used).
VIT_HD uint32_t rotr32(uint32_t x, uint32_t n) {
#if defined(__CUDA_ARCH__)
  return __funnelshift_r(x, x, n);
#else
  n &= 31u;
  return n ? (x >> n) | (x << (32u - n)) : x;
#endif
}

// Byte store to global memory.
VIT_HD void store_byte(uint8_t* p, uint32_t v) {
#if defined(__CUDA_ARCH__)
  asm volatile("st.global.u8 [%0], %1;" ::"l"(p), "r"(v) : "memory");
#else
  *p = (uint8_t)v;
#endif
}

// Survivor decision of state j (its low K-1 bits) for tile h at one stage.
// Tile h's bit of state s sits at bit 16h + surv_pos(s) of word surv_word(s);
// tile 0's bits are stored inverted.  For 64 states one prmt per word pair
// gathers the tile's 32 bits of states [0, 32) and [32, 64) in state order.
template <class C>
VIT_HD uint32_t tb_decision(const uint32_t (&w)[C::WORDS], uint32_t j, int h) {
  if constexpr (C::WORDS == 4) {
    const uint32_t sel = h ? 0x7632u : 0x5410u;
    const uint32_t x = (j & 32u) ? prmt(w[2], w[3], sel) : prmt(w[0], w[1], sel);
    return (rotr32(x, j) & 1u) ^ (h ? 0u : 1u);
  } else {
    const int sj = (int)(j & (uint32_t)(C::S - 1));
    return ((pick_word<C>(w, sj) >> (16 * h + surv_pos<C>(sj))) & 1u) ^ (h ? 0u : 1u);
  }
}

// Asks L2 to fetch the warp's survivor words of stages [i, i + cnt) (one
// contiguous block of cnt * 32 lanes * WORDS words; lane 0's slab pointer is
// its start).  No effect on the host build.
VIT_HD void slab_prefetch_l2(const Slab& sl, int i, int cnt) {
#if defined(__CUDA_ARCH__)
  if ((threadIdx.x & 31) == 0 && cnt > 0) {
    const uint32_t* p = sl.base + (int64_t)i * sl.stride;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"((uint32_t)(cnt * sl.stride * 4))
                 : "memory");
  }
#endif
}

// Traceback (Alg. 2) of the two tiles of a lane.  Following a decision d at
// iteration i gives state (2j + d) mod S, whose bit K-2 after K-1 further
// steps is d: d is the decoded bit of iteration i - (K-1).  Keeping
// j = 2j + d unmasked therefore leaves the decoded bits of the iterations
// x, x+1, ... in bits 0, 1, ... of j once iteration x + K - 1 is read, and
// the start state's own K-1 bits stand for the top K-1 iterations (as if
// read at iterations Lw .. Lw + K - 2).  Tile h emits iterations
// [r0[h], r1[h]) (r0 at an output byte boundary); its bytes are taken from j
// at checkpoints every 8 iterations, highest byte first, the partial last
// byte masked.  Survivor words: three register buffers of 8 stages, loads
// issued two groups ahead.
template <class C>
VIT_HD void tb_group(uint32_t& j0, uint32_t& j1, const uint32_t (&w)[8][C::WORDS]) {
#pragma unroll
  for (int k = 7; k >= 0; k--) {
    const uint32_t d0 = tb_decision<C>(w[k], j0, 0), d1 = tb_decision<C>(w[k], j1, 1);
    j0 = 2u * j0 + d0;
    j1 = 2u * j1 + d1;
  }
}

template <class C>
VIT_HD void tb_load_group(const Slab& sl, int i, uint32_t (&w)[8][C::WORDS]) {
#pragma unroll
  for (int k = 0; k < 8; k++) load_words<C>(sl, i + k, w[k]);
}

// Emits the bytes of one tile whose lowest output iteration is at least x
// (j holds the outputs from x upward); nb: next byte to emit, descending.
VIT_HD void tb_emit(uint32_t j, int x, int r0, int r1, int& nb, uint8_t* out) {
  int sh = r0 + 8 * nb - x;
  while (nb >= 0 && sh >= 0) {
    const int left = r1 - r0 - 8 * nb;
    const uint32_t mask = left >= 8 ? 0xffu : ((1u << left) - 1u);
    store_byte(out + nb, (j >> sh) & mask);
    nb--;
    sh -= 8;
  }
}

template <class C>
VIT_HD void traceback_pair(const Half (&hw)[2], int Lw, const int (&s0)[2], Slab sl) {
  bool act[2];
  int r0[2], r1[2], nb[2];
  uint8_t* o[2];
#pragma unroll
  for (int h = 0; h < 2; h++) {
    act[h] = hw[h].active && hw[h].e1 > hw[h].e0;
    r0[h] = hw[h].start + (int)(hw[h].e0 - hw[h].t0);
    r1[h] = hw[h].start + (int)(hw[h].e1 - hw[h].t0);
    nb[h] = act[h] ? (r1[h] - r0[h] + 7) / 8 - 1 : -1;
    o[h] = hw[h].out + (hw[h].e0 >> 3);
  }
  if (!act[0] && !act[1]) return;
  const int rmin = act[0] ? (act[1] && r0[1] < r0[0] ? r0[1] : r0[0]) : r0[1];
  const int ib = rmin + C::KM1;  // lowest iteration read
  uint32_t j0 = (uint32_t)s0[0], j1 = (uint32_t)s0[1];
  auto checkpoint = [&](int x) {
    tb_emit(j0, x, r0[0], r1[0], nb[0], o[0]);
    tb_emit(j1, x, r0[1], r1[1], nb[1], o[1]);
  };
  checkpoint(Lw - C::KM1);  // bytes made of start-state bits only
  if (ib >= Lw) return;
  // the partial group below Lw above the last whole group of 8
  const int top = ib + 8 * ((Lw - ib) >> 3);
  for (int i = Lw - 1; i >= top; i--) {
    uint32_t w[C::WORDS];
    load_words<C>(sl, i, w);
    j0 = 2u * j0 + tb_decision<C>(w, j0, 0);
    j1 = 2u * j1 + tb_decision<C>(w, j1, 1);
  }
  if (top < Lw) checkpoint(top - C::KM1);
  int q = ((top - ib) >> 3) - 1;  // highest whole group
  if (q < 0) return;
  uint32_t b0[8][C::WORDS], b1[8][C::WORDS], b2[8][C::WORDS];
  tb_load_group<C>(sl, ib + 8 * q, b0);
  if (q >= 1) tb_load_group<C>(sl, ib + 8 * (q - 1), b1);
  // invariant at the loop top: b0 holds group q, b1 group q-1 (if q >= 1)
  while (true) {
    if (q >= 2) tb_load_group<C>(sl, ib + 8 * (q - 2), b2);
    tb_group<C>(j0, j1, b0);
    checkpoint(rmin + 8 * q);
    if (--q < 0) break;
    if (q >= 2) tb_load_group<C>(sl, ib + 8 * (q - 2), b0);
    tb_group<C>(j0, j1, b1);
    checkpoint(rmin + 8 * q);
    if (--q < 0) break;
    if (q >= 2) tb_load_group<C>(sl, ib + 8 * (q - 2), b1);
    tb_group<C>(j0, j1, b2);
    checkpoint(rmin + 8 * q);
    if (--q < 0) break;
    // b0 holds group q, b1 group q-1: the invariant again
  }
}

// Decodes the two tiles of one lane.  Lw: iterations (a multiple of U, at
// least every active window length); masked_until: first iteration from which
// every window of the warp has started.
template <class C>
VIT_HD void decode_pair(const Half (&hw)[2], int Lw, int masked_until, uint32_t M, Slab sl, bool words_ok) {
  static_assert(C::G == 1 && C::S <= 64, "all states of a tile pair in one lane");
  uint32_t ma[C::NS], mb[C::NS];
#pragma unroll
  for (int s = 0; s < C::NS; s++) ma[s] = 0x80008000u;
#pragma unroll
  for (int h = 0; h < 2; h++)
    if (hw[h].known && hw[h].start == 0) init_half<C>(ma, h, true, M);

  static_assert(C::U == 2, "two register arrays alternate");
  const int ngroups = Lw / C::U;
  bool words = false;
  if constexpr (kWordLoads<C>) words = words_ok;
  if (words) {
    if constexpr (kWordLoads<C>) {
      // groups before every window has started: byte loads, masked
      int g = 0;
      for (; g < ngroups && g * C::U < masked_until; g++) {
        const int i0 = g * C::U;
        LlrGroup<C> lg;
        load_group<C>(hw, i0, lg);
        fwd_stage<C>(ma, mb, hw, i0, true, M, lg.v[0], sl);
        fwd_stage<C>(mb, ma, hw, i0 + 1, true, M, lg.v[1], sl);
        if ((g % C::RN) == C::RN - 1) renorm<C>(ma);
      }
      constexpr int NW = C::U * C::BETA / 4;
      uint32_t wc[2][NW], wn[2][NW];
      if (g < ngroups) load_group_words<C>(hw, g * C::U, wc);
#pragma unroll 2
      for (; g < ngroups; g++) {
        const int i0 = g * C::U;
        if (g + 1 < ngroups) load_group_words<C>(hw, i0 + C::U, wn);  // prefetch the next group
        fwd_stage_words<C, 0>(ma, mb, i0, wc, sl);
        fwd_stage_words<C, 1>(mb, ma, i0 + 1, wc, sl);
        if ((g % C::RN) == C::RN - 1) renorm<C>(ma);
#pragma unroll
        for (int h = 0; h < 2; h++)
#pragma unroll
          for (int k = 0; k < NW; k++) wc[h][k] = wn[h][k];
      }
    }
  } else {
    LlrGroup<C> cur, nxt;
    load_group<C>(hw, 0, cur);
    for (int g = 0; g < ngroups; g++) {
      const int i0 = g * C::U;
      if (g + 1 < ngroups) {  // prefetch the next group
        if (i0 + C::U < masked_until)
          load_group<C>(hw, i0 + C::U, nxt);
        else
          load_group_fast<C>(hw, i0 + C::U, nxt);
      }
      const bool masked = i0 < masked_until;
      fwd_stage<C>(ma, mb, hw, i0, masked, M, cur.v[0], sl);
      fwd_stage<C>(mb, ma, hw, i0 + 1, masked, M, cur.v[1], sl);
      if ((g % C::RN) == C::RN - 1) renorm<C>(ma);
      cur = nxt;
    }
  }

  // traceback start (Alg. 2): best final metric, ties to the lowest state
  int s[2];
#pragma unroll
  for (int h = 0; h < 2; h++) {
    int best = 0;
    uint32_t bv = (ma[0] >> (16 * h)) & 0xffffu;
#pragma unroll
    for (int q = 1; q < C::NS; q++) {
      const uint32_t v = (ma[q] >> (16 * h)) & 0xffffu;
      if (v > bv) {
        bv = v;
        best = q;
      }
    }
    s[h] = hw[h].end_zero ? 0 : best;
  }

  traceback_pair<C>(hw, Lw, s, sl);
}


#if defined(__CUDACC__)
// ---------------------------------------------------------------------------
// Several lanes per tile pair (K = 8, 9): G lanes hold NS = 64 slots each.
// Slot s = (lane-in-group << NSB) | register.  Register s holds state
// rotr(s, r) after r stages (rotation over K-1 bits), so each butterfly reads
// and writes the two slots that differ in bit r mod (K-1): stages whose pair
// bit is a register bit stay inside the lane, the others pair the same
// register of two lanes (one shuffle each).  The part of a butterfly's branch
// pattern that depends on the lane bits is applied by negating LLRs (Eq. 2 is
// linear in the pattern bits), so every instruction is the same for all lanes.
// ---------------------------------------------------------------------------

// Branch-pattern offset (beta bits) contributed by the lane bits of the even
// slot of phase P, for every phase, packed beta bits per phase.
template <class C>
__device__ __forceinline__ uint32_t lane_flip_mask(int lig) {
  uint32_t mask = 0;
#pragma unroll
  for (int P = 0; P < C::KM1; P++) {
    const int la = (P >= C::NSB) ? (lig & ~(1 << (P - C::NSB))) : lig;
    const uint32_t R = rotr_w((uint32_t)la << C::NSB, P, C::KM1);
    mask |= C::aout(R) << (C::BETA * P);
  }
  return mask;
}

template <class C, int P>
__device__ __forceinline__ void rot_butterfly(uint32_t (&m)[C::NS], const StageBM<C>& D, int a, uint32_t& Ea,
                                              uint32_t& Eb) {
  const int b = a | (1 << P);
  const uint32_t i0 = rotr_w((uint32_t)a, P, C::KM1);  // register part of the even predecessor
  const uint32_t c00 = C::aout(i0), c01 = C::aout(i0 | 1u);
  const uint32_t c10 = C::aout(i0 | (uint32_t)C::S), c11 = C::aout(i0 | (uint32_t)C::S | 1u);
  const uint32_t x00 = add_bm<C>(m[a], D, c00), x01 = add_bm<C>(m[b], D, c01);
  const uint32_t x10 = add_bm<C>(m[a], D, c10), x11 = add_bm<C>(m[b], D, c11);
  Ea = x00 - x01 + 0x8000u;
  Eb = add_on_fma(Ea, bmv<C>(D, c10) - bmv<C>(D, c11) - bmv<C>(D, c00) + bmv<C>(D, c01));
  m[a] = vmaxu2(x00, x01);
  m[b] = vmaxu2(x10, x11);
}

// Pair bit P is a register bit: butterflies inside the lane, visited so that
// each prmt pair (s, s + HALFP) is finished together.
template <class C, int P>
__device__ __forceinline__ void rot_local_stage(uint32_t (&m)[C::NS], const StageBM<C>& D,
                                                uint32_t (&w)[C::WORDS]) {
  constexpr int B = 1 << P;
  constexpr int H = C::HALFP;
#pragma unroll
  for (int k = 0; k < C::WORDS; k++) w[k] = 0u;
  if constexpr (B == H) {
#pragma unroll
    for (int a = 0; a < C::NS; a++) {
      if (a & B) continue;
      uint32_t Ea, Eb;
      rot_butterfly<C, P>(m, D, a, Ea, Eb);
      gather2<C>(w, a, Ea, Eb);
    }
  } else {
#pragma unroll
    for (int a = 0; a < C::NS; a++) {
      if ((a & B) || (a & H)) continue;
      uint32_t E0, E1, E2, E3;  // slots a, a|B, a+H, (a+H)|B
      rot_butterfly<C, P>(m, D, a, E0, E1);
      rot_butterfly<C, P>(m, D, a | H, E2, E3);
      gather2<C>(w, a, E0, E2);
      gather2<C>(w, a | B, E1, E3);
    }
  }
}

// Pair bit P is lane bit P - NSB: the partner slot is the same register of
// lane ^ (1 << (P - NSB)).  Both lanes form max(own + d, partner - d); the
// decision polarity of the lane holding the odd slot is reversed (constant
// cb), which the traceback undoes.
template <class C, int P>
__device__ __forceinline__ void rot_cross_stage(uint32_t (&m)[C::NS], const StageBM<C>& D,
                                                uint32_t (&w)[C::WORDS], int lig) {
  constexpr int H = C::HALFP;
  const int xm = 1 << (P - C::NSB);
  const uint32_t cb = (lig & xm) ? 0xffff7fffu : 0x8000u;
  constexpr uint32_t CM = (1u << C::BETA) - 1u;
#pragma unroll
  for (int k = 0; k < C::WORDS; k++) w[k] = 0u;
#pragma unroll
  for (int r0 = 0; r0 < C::NS; r0++) {
    if (r0 & H) continue;
    uint32_t E[2];
#pragma unroll
    for (int q = 0; q < 2; q++) {
      const int r = r0 + q * H;
      const uint32_t pv = __shfl_xor_sync(0xffffffffu, m[r], xm);
      const uint32_t c = C::aout(rotr_w((uint32_t)r, P, C::KM1));
      const uint32_t X = add_bm<C>(m[r], D, c);
      const uint32_t Y = add_bm<C>(pv, D, (~c) & CM);
      E[q] = X - Y + cb;
      m[r] = vmaxu2(X, Y);
    }
    gather2<C>(w, r0, E[0], E[1]);
  }
}

// Branch magnitudes of one stage with the lane's pattern offset for phase P.
template <class C, int P>
__device__ __forceinline__ void rot_stage_bm(int (&lA)[C::BETA], int (&lB)[C::BETA], uint32_t flip,
                                             StageBM<C>& D) {
#pragma unroll
  for (int b = 0; b < C::BETA; b++) {
    const int sgn = 1 - 2 * (int)((flip >> (C::BETA * P + b)) & 1u);
    lA[b] *= sgn;
    lB[b] *= sgn;
  }
  stage_bm<C>(lA, lB, D);
}

template <class C>
__device__ __forceinline__ void load_stage(const Half (&hw)[2], int i, int (&l)[2][C::BETA]) {
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const int64_t t = hw[h].t0 + (int64_t)((i > hw[h].start ? i : hw[h].start) - hw[h].start);
    const int8_t* p = hw[h].llr + t * C::BETA;
#pragma unroll
    for (int b = 0; b < C::BETA; b++) l[h][b] = hw[h].active ? ld_s8(p + b) : 0;
  }
}

template <class C>
__device__ __forceinline__ void rot_init_half(uint32_t (&m)[C::NS], int h, uint32_t M, int lig) {
  const uint32_t keep = h ? 0x0000ffffu : 0xffff0000u;
#pragma unroll
  for (int r = 0; r < C::NS; r++) {
    const uint32_t v = (lig == 0 && r == 0) ? 0x8000u : (0x8000u - M);
    m[r] = (m[r] & keep) | (v << (16 * h));
  }
}

template <class C, int P>
__device__ __forceinline__ void rot_fwd_stage(uint32_t (&m)[C::NS], const Half (&hw)[2], int i, bool masked,
                                              uint32_t M, int (&cur)[2][C::BETA], int (&nxt)[2][C::BETA],
                                              bool more, uint32_t flip, int lig, Slab sl) {
  if (more) load_stage<C>(hw, i + 1, nxt);  // prefetch the next stage
  int lA[C::BETA], lB[C::BETA];
#pragma unroll
  for (int b = 0; b < C::BETA; b++) {
    lA[b] = (!masked || i >= hw[0].start) ? cur[0][b] : 0;
    lB[b] = (!masked || i >= hw[1].start) ? cur[1][b] : 0;
  }
  if (masked) {
#pragma unroll
    for (int h = 0; h < 2; h++)
      if (hw[h].known && i == hw[h].start) rot_init_half<C>(m, h, M, lig);
  }
  StageBM<C> D;
  rot_stage_bm<C, P>(lA, lB, flip, D);
  uint32_t w[C::WORDS];
  if constexpr (P < C::NSB)
    rot_local_stage<C, P>(m, D, w);
  else
    rot_cross_stage<C, P>(m, D, w, lig);
  store_words(sl.base + (int64_t)i * sl.stride, w, C::WORDS);
#pragma unroll
  for (int h = 0; h < 2; h++)
#pragma unroll
    for (int b = 0; b < C::BETA; b++) cur[h][b] = nxt[h][b];
}

// Word-fed stage of the rotating layout (every window of the warp started).
template <class C, int P>
__device__ __forceinline__ void rot_fwd_stage_words(uint32_t (&m)[C::NS], int i,
                                                    const uint32_t (&w)[2][C::U * C::BETA / 4], uint32_t flip,
                                                    int lig, Slab sl) {
  int L[C::BETA];
  pairs_from_words<C, P>(w, L);
#pragma unroll
  for (int b = 0; b < C::BETA; b++)
    if ((flip >> (C::BETA * P + b)) & 1u) L[b] = -L[b];
  StageBM<C> D;
  bm_from_pairs<C>(L, D);
  uint32_t wd[C::WORDS];
  if constexpr (P < C::NSB)
    rot_local_stage<C, P>(m, D, wd);
  else
    rot_cross_stage<C, P>(m, D, wd, lig);
  store_words(sl.base + (int64_t)i * sl.stride, wd, C::WORDS);
}

template <class C, int P>
__device__ __forceinline__ void rot_fwd_group_words(uint32_t (&m)[C::NS], int i0,
                                                    const uint32_t (&w)[2][C::U * C::BETA / 4], uint32_t flip,
                                                    int lig, Slab sl) {
  if constexpr (P < C::KM1) {
    rot_fwd_stage_words<C, P>(m, i0 + P, w, flip, lig, sl);
    rot_fwd_group_words<C, P + 1>(m, i0, w, flip, lig, sl);
  }
}

template <class C, int P>
__device__ __forceinline__ void rot_fwd_group(uint32_t (&m)[C::NS], const Half (&hw)[2], int i0, bool masked,
                                              uint32_t M, int (&cur)[2][C::BETA], int (&nxt)[2][C::BETA],
                                              int Lw, uint32_t flip, int lig, Slab sl) {
  if constexpr (P < C::KM1) {
    rot_fwd_stage<C, P>(m, hw, i0 + P, masked, M, cur, nxt, i0 + P + 1 < Lw, flip, lig, sl);
    rot_fwd_group<C, P + 1>(m, hw, i0, masked, M, cur, nxt, Lw, flip, lig, sl);
  }
}

// Decodes the tile pair of a group of G lanes; lig = lane in group.  Lane
// lig = h (h < 2) traces and emits tile h.  kWords compiles the word-load
// path: groups before every window of the warp has started, or every group
// when the warp's windows are not 4-byte aligned (words_ok false), run the
// masked byte-load stage, the rest the word-fed stage.  Without kWords every
// group runs the byte-load stage.
template <class C, bool kWords>
__device__ void decode_pair_rot(const Half (&hw)[2], int Lw, int masked_until, uint32_t M, Slab sl, int lane,
                                bool words_ok) {
  const int lig = lane & (C::G - 1);
  const int gbase = lane & ~(C::G - 1);
  const uint32_t flip = lane_flip_mask<C>(lig);
  uint32_t m[C::NS];
#pragma unroll
  for (int r = 0; r < C::NS; r++) m[r] = 0x80008000u;
#pragma unroll
  for (int h = 0; h < 2; h++)
    if (hw[h].known && hw[h].start == 0) rot_init_half<C>(m, h, M, lig);
  const int ngroups = Lw / C::U;
  int g = 0;
  auto renorm_group = [&](int gg) {
    if ((gg % C::RN) == C::RN - 1) {
      const uint32_t ref = __shfl_sync(0xffffffffu, m[0], gbase);  // state 0 is slot 0 of the group
#pragma unroll
      for (int r = 0; r < C::NS; r++) m[r] = m[r] - ref + 0x80008000u;
    }
  };
  if constexpr (!(kWordLoads<C> && kWords)) {
    int cur[2][C::BETA], nxt[2][C::BETA];
    load_stage<C>(hw, 0, cur);
    for (; g < ngroups; g++) {
      const int i0 = g * C::U;
      rot_fwd_group<C, 0>(m, hw, i0, i0 < masked_until, M, cur, nxt, Lw, flip, lig, sl);
      renorm_group(g);
    }
  } else {
    // groups before every window has started (all groups without word
    // alignment): byte loads, masked
    const int mu = words_ok ? masked_until : Lw;
    for (; g < ngroups && g * C::U < mu; g++) {
      int cur[2][C::BETA], nxt[2][C::BETA];
      load_stage<C>(hw, g * C::U, cur);
      rot_fwd_group<C, 0>(m, hw, g * C::U, true, M, cur, nxt, Lw, flip, lig, sl);
      renorm_group(g);
    }
    constexpr int NW = C::U * C::BETA / 4;
    uint32_t wc[2][NW], wn[2][NW];
    if (g < ngroups) load_group_words<C>(hw, g * C::U, wc);
    for (; g < ngroups; g++) {
      const int i0 = g * C::U;
      if (g + 1 < ngroups) load_group_words<C>(hw, i0 + C::U, wn);  // prefetch the next group
      rot_fwd_group_words<C, 0>(m, i0, wc, flip, lig, sl);
      renorm_group(g);
#pragma unroll
      for (int h = 0; h < 2; h++)
#pragma unroll
        for (int k = 0; k < NW; k++) wc[h][k] = wn[h][k];
    }
  }

  // traceback start: best final metric of each tile over the group (slot =
  // state after a multiple of K-1 stages), ties to the lowest state
  int s[2];
#pragma unroll
  for (int h = 0; h < 2; h++) {
    int best = 0;
    uint32_t bv = (m[0] >> (16 * h)) & 0xffffu;
#pragma unroll
    for (int r = 1; r < C::NS; r++) {
      const uint32_t v = (m[r] >> (16 * h)) & 0xffffu;
      if (v > bv) {
        bv = v;
        best = r;
      }
    }
    int bs = (lig << C::NSB) | best;
#pragma unroll
    for (int o = 1; o < C::G; o <<= 1) {
      const uint32_t ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int os = __shfl_xor_sync(0xffffffffu, bs, o);
      if (ov > bv || (ov == bv && os < bs)) {
        bv = ov;
        bs = os;
      }
    }
    s[h] = hw[h].end_zero ? 0 : bs;
  }
  const int h = lig < 2 ? lig : 0;  // tile traced by this lane
  // fields of the traced tile, selected without indexing hw at run time
  const bool sel1 = (h == 1);
  const int64_t tt0 = sel1 ? hw[1].t0 : hw[0].t0;
  const int64_t te0 = sel1 ? hw[1].e0 : hw[0].e0;
  const int64_t te1 = sel1 ? hw[1].e1 : hw[0].e1;
  const int tstart = sel1 ? hw[1].start : hw[0].start;
  uint8_t* const tout = (sel1 ? hw[1].out : hw[0].out) + (te0 >> 3);
  const bool tracer = lig < 2 && (sel1 ? hw[1].active : hw[0].active) && te1 > te0;
  int st = sel1 ? s[1] : s[0];
  // The tracer's emitted iterations [r0, r1).  As in the one-lane
  // traceback, the decision read at iteration i (the bit written at slot
  // position i mod (K-1)) is the decoded bit of iteration i - (K-1), so the
  // accumulator a = 2a + d holds decoded bits from its low end, starting with
  // the start state's bits in iteration order (rotated by Lw mod (K-1)).
  const int r0 = tstart + (int)(te0 - tt0), r1 = tstart + (int)(te1 - tt0);
  int nb = tracer ? (r1 - r0 + 7) / 8 - 1 : -1;
  uint32_t acc = rotr_w((uint32_t)st, Lw % C::KM1, C::KM1);
  int rmin = tracer ? r0 : Lw;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int ro = __shfl_xor_sync(0xffffffffu, rmin, o);
    rmin = ro < rmin ? ro : rmin;
  }
  tb_emit(acc, Lw - C::KM1, r0, r1, nb, tout);
  const int ib = rmin + C::KM1;  // lowest iteration read (warp-wide)
  if (ib >= Lw) return;
  constexpr int TB = 8;
  uint32_t wc[TB][C::WORDS], wn[TB][C::WORDS];
  // blocks [lo, lo + TB) aligned to ib, the highest one cut at Lw
  int lo = ib + TB * ((Lw - 1 - ib) / TB);
#pragma unroll
  for (int q = 0; q < TB; q++)
    if (lo + q < Lw) load_words<C>(sl, lo + q, wc[q]);
  while (true) {
    if (lo > ib) {
#pragma unroll
      for (int q = 0; q < TB; q++) load_words<C>(sl, lo - TB + q, wn[q]);
    }
#pragma unroll
    for (int q = TB - 1; q >= 0; q--) {
      const int i = lo + q;
      if (i >= Lw) continue;
      const int P = i % C::KM1;
      const int src = gbase + (st >> C::NSB);
      uint32_t ww[C::WORDS];
#pragma unroll
      for (int k = 0; k < C::WORDS; k++) ww[k] = __shfl_sync(0xffffffffu, wc[q][k], src);
      const int r = st & (C::NS - 1);
      const uint32_t word = pick_word<C>(ww, r);
      const uint32_t pol = (h == 0 ? 1u : 0u) ^ ((P >= C::NSB && ((st >> P) & 1)) ? 1u : 0u);
      const uint32_t d = ((word >> (16 * h + surv_pos<C>(r))) & 1u) ^ pol;
      st = (st & ~(1 << P)) | (int)(d << P);
      acc = 2u * acc + d;
    }
    tb_emit(acc, lo - C::KM1, r0, r1, nb, tout);
    if (lo <= ib) break;
    lo -= TB;
#pragma unroll
    for (int q = 0; q < TB; q++)
#pragma unroll
      for (int k = 0; k < C::WORDS; k++) wc[q][k] = wn[q][k];
  }
}
#endif  // __CUDACC__

}  // namespace vit
