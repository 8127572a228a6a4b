// vit_pt.cuh -- tile decoding with the paper's first parallel traceback
// (Sec. "Parallel Traceback Algorithm", Fig. pt1), for codes whose states
// fit one lane (K <= 7).
//
// A tile's emitted stages [e0, e1) are cut into subframes of f0 stages.
// Subframe k emits [s0, s1) = [e0 + k f0, min(e0 + (k+1) f0, e1)) and is
// traced back from stage u = min(s1 + v2, t1) - 1 (it overlaps its right-hand
// neighbour by v2 stages, whose bits it does not emit).  Its start state is
// the tile's usual one (Alg. 2 argmax, or state 0 at the end of a terminated
// frame) when u is the window's last stage; otherwise the argmax of stage u's
// path metrics, recorded during the forward pass (rule 0), or the top K-1
// bits of SplitMix64 output u under the caller's seed (rule 1).
//
// The forward pass is the tile decoder's (32-bit LLR word loads once every
// window of the warp has started, both tiles of a lane in the two 16-bit
// fields); after every stage at which a subframe of either
// tile starts its traceback, the lane records that tile's argmax state.  The
// traceback then runs per subframe, both tiles of the lane together when
// their subframes line up.
#pragma once
#include "vit_acs.cuh"

namespace vit {

struct PtParams {
  int64_t f0;     // subframe length (a multiple of 8)
  int rule;       // 0: recorded argmax start, 1: SplitMix64 start
  uint64_t seed;  // key of the SplitMix64 start
};

// Output i of SplitMix64 seeded with `seed` (Steele, Lea and Flood, OOPSLA
// 2014): the generator adds 0x9E3779B97F4A7C15 to its state before each
// output and returns the state mixed by two xor-shift-multiply rounds.
VIT_HD uint64_t splitmix64_output(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Subframe k of a tile: emitted [s0, s1) and first traceback stage u.
// e1f: the tile's emitted end before clipping to the frame's output count.
struct Subframe {
  int64_t s0, s1, u;
};
VIT_HD Subframe pt_subframe(const Half& h, int64_t e1f, int64_t f0, int64_t v2, int64_t k) {
  Subframe s;
  s.s0 = h.e0 + k * f0;
  s.s1 = (s.s0 + f0 < e1f) ? s.s0 + f0 : e1f;
  s.u = ((s.s1 + v2 < h.t1) ? s.s1 + v2 : h.t1) - 1;
  return s;
}

// Argmax of tile h's field over the lane's states, ties to the lowest state.
template <class C>
VIT_HD int argmax_field(const uint32_t (&m)[C::NS], int h) {
  uint32_t best = 0u;
#pragma unroll
  for (int q = 0; q < C::NS; q++) {
    const uint32_t key = (((m[q] >> (16 * h)) & 0xffffu) << 8) | (uint32_t)(255 - q);
    best = key > best ? key : best;
  }
  return 255 - (int)(best & 0xffu);
}

// Records the argmax of every subframe of tile h whose traceback starts at
// iteration i (next[h]: the next such iteration, k[h]: its subframe).
template <class C>
VIT_HD void pt_capture(const uint32_t (&m)[C::NS], int i, const Half (&hw)[2], const int64_t (&e1f)[2],
                       const int64_t (&nsub)[2], int64_t v2, const PtParams& pt, uint8_t* const (&st)[2],
                       int (&next)[2], int64_t (&k)[2]) {
#pragma unroll
  for (int h = 0; h < 2; h++) {
    if (next[h] != i) continue;
    const int best = argmax_field<C>(m, h);
    while (k[h] < nsub[h]) {
      const Subframe sf = pt_subframe(hw[h], e1f[h], pt.f0, v2, k[h]);
      const int it = hw[h].start + (int)(sf.u - hw[h].t0);
      if (it > i) {
        next[h] = it;
        break;
      }
      if (it == i) st[h][k[h]] = (uint8_t)best;  // (it < i: a SplitMix64 start)
      k[h]++;
    }
    if (k[h] >= nsub[h]) next[h] = -1;
  }
}

// First capture iteration of tile h (-1: none).  With rule 1 only the
// subframes traced from the window's last stage need their argmax, which the
// capture after the last stage records.
VIT_HD int pt_first_capture(const Half& h, int64_t e1f, int64_t nsub, int64_t v2, const PtParams& pt, int Lw) {
  if (!h.active || nsub <= 0) return -1;
  if (pt.rule != 0) return Lw - 1;
  const Subframe sf = pt_subframe(h, e1f, pt.f0, v2, 0);
  return h.start + (int)(sf.u - h.t0);
}

// Start state of subframe sf of tile hw (k: its index): the tile's usual
// start when sf is traced from the window's last stage, else the recorded
// argmax (rule 0) or the top K-1 bits of SplitMix64 output u (rule 1).
template <class C>
VIT_HD uint32_t pt_start(const Half& hw, const Subframe& sf, int64_t k, const PtParams& pt, const uint8_t* st) {
  if (sf.u == hw.t1 - 1) return hw.end_zero ? 0u : (uint32_t)st[k];
  if (pt.rule == 0) return (uint32_t)st[k];
  return (uint32_t)(splitmix64_output(pt.seed, (uint64_t)sf.u) >> (64 - C::KM1));
}

// Traceback of a lane's tiles, one subframe at a time (last first).  Each
// subframe is the tile decoder's traceback (traceback_pair) over iterations
// up to its stage u, emitting its own stages only.  The two tiles go
// together when their subframes cover the same iterations (every interior
// tile pair), else one after the other.
template <class C>
VIT_HD void pt_traceback_pair(const Half (&hw)[2], const int64_t (&e1f)[2], const int64_t (&nsub)[2], int64_t v2,
                              const PtParams& pt, uint8_t* const (&st)[2], Slab sl) {
  const bool paired = hw[0].active && hw[1].active && nsub[0] == nsub[1] && hw[0].start == hw[1].start &&
                      hw[0].e0 - hw[0].t0 == hw[1].e0 - hw[1].t0 && hw[0].t1 - hw[0].t0 == hw[1].t1 - hw[1].t0 &&
                      e1f[0] - hw[0].e0 == e1f[1] - hw[1].e0 && hw[0].e1 - hw[0].e0 == hw[1].e1 - hw[1].e0;
  for (int pass = 0; pass < (paired ? 1 : 2); pass++) {
    const int lead = paired ? 0 : pass;  // the tile whose geometry drives this pass
    if (!hw[lead].active) continue;
    for (int64_t k = nsub[lead] - 1; k >= 0; k--) {
      const Subframe sf = pt_subframe(hw[lead], e1f[lead], pt.f0, v2, k);
      if (k > 0) {  // the next subframe's survivor words, into L2
        const Subframe nf = pt_subframe(hw[lead], e1f[lead], pt.f0, v2, k - 1);
        slab_prefetch_l2(sl, hw[lead].start + (int)(nf.s0 - hw[lead].t0), (int)(nf.u - nf.s0 + 1));
      }
      Half hs[2];
      int s0[2];
#pragma unroll
      for (int h = 0; h < 2; h++) {
        hs[h] = hw[h];
        s0[h] = 0;
        if (!(paired || h == lead)) {
          hs[h].active = 0;
          continue;
        }
        const Subframe sh = pt_subframe(hw[h], e1f[h], pt.f0, v2, k);
        hs[h].e0 = sh.s0;
        hs[h].e1 = sh.s1 < hw[h].e1 ? sh.s1 : hw[h].e1;
        s0[h] = (int)pt_start<C>(hw[h], sh, k, pt, st[h]);
      }
      traceback_pair<C>(hs, hw[lead].start + (int)(sf.u - hw[lead].t0) + 1, s0, sl);
    }
  }
}

// Decodes the two tiles of one lane with the parallel traceback.  st[h]:
// the tile's recorded start states (one byte per subframe); words_ok: the
// warp's tiles allow the 32-bit LLR word loads of the tile decoder (groups
// before every window has started still use masked byte loads).
template <class C>
VIT_HD void decode_pair_pt(const Half (&hw)[2], const int64_t (&e1f)[2], int Lw, int masked_until, uint32_t M,
                           Slab sl, int64_t v2, const PtParams& pt, uint8_t* const (&st)[2], bool words_ok) {
  static_assert(C::G == 1 && C::U == 2, "one lane per tile pair");
  uint32_t ma[C::NS], mb[C::NS];
#pragma unroll
  for (int s = 0; s < C::NS; s++) ma[s] = 0x80008000u;
#pragma unroll
  for (int h = 0; h < 2; h++)
    if (hw[h].known && hw[h].start == 0) init_half<C>(ma, h, true, M);
  int64_t nsub[2], k[2] = {0, 0};
  int next[2];
#pragma unroll
  for (int h = 0; h < 2; h++) {
    nsub[h] = hw[h].active && e1f[h] > hw[h].e0 ? (e1f[h] - hw[h].e0 + pt.f0 - 1) / pt.f0 : 0;
    next[h] = pt_first_capture(hw[h], e1f[h], nsub[h], v2, pt, Lw);
  }
  // the argmax capture after the stage at iteration i (metrics m)
  auto capture = [&](const uint32_t (&m)[C::NS], int i) {
    if (next[0] == i || next[1] == i) pt_capture<C>(m, i, hw, e1f, nsub, v2, pt, st, next, k);
  };
  const int ngroups = Lw / C::U;
  bool words = false;
  if constexpr (kWordLoads<C>) words = words_ok;
  if (words) {
    if constexpr (kWordLoads<C>) {
      int g = 0;
      for (; g < ngroups && g * C::U < masked_until; g++) {  // masked byte loads
        const int i0 = g * C::U;
        LlrGroup<C> lg;
        load_group<C>(hw, i0, lg);
        fwd_stage<C>(ma, mb, hw, i0, true, M, lg.v[0], sl);
        capture(mb, i0);
        fwd_stage<C>(mb, ma, hw, i0 + 1, true, M, lg.v[1], sl);
        capture(ma, i0 + 1);
        if ((g % C::RN) == C::RN - 1) renorm<C>(ma);
      }
      constexpr int NW = C::U * C::BETA / 4;
      uint32_t wc[2][NW], wn[2][NW];
      if (g < ngroups) load_group_words<C>(hw, g * C::U, wc);
      for (; g < ngroups; g++) {
        const int i0 = g * C::U;
        if (g + 1 < ngroups) load_group_words<C>(hw, i0 + C::U, wn);  // prefetch the next group
        fwd_stage_words<C, 0>(ma, mb, i0, wc, sl);
        capture(mb, i0);
        fwd_stage_words<C, 1>(mb, ma, i0 + 1, wc, sl);
        capture(ma, i0 + 1);
        if ((g % C::RN) == C::RN - 1) renorm<C>(ma);
#pragma unroll
        for (int h = 0; h < 2; h++)
#pragma unroll
          for (int q = 0; q < NW; q++) wc[h][q] = wn[h][q];
      }
    }
  } else {
    LlrGroup<C> cur, nxt;
    load_group<C>(hw, 0, cur);
    for (int g = 0; g < ngroups; g++) {
      const int i0 = g * C::U;
      if (g + 1 < ngroups) {
        if (i0 + C::U < masked_until)
          load_group<C>(hw, i0 + C::U, nxt);
        else
          load_group_fast<C>(hw, i0 + C::U, nxt);
      }
      const bool masked = i0 < masked_until;
      fwd_stage<C>(ma, mb, hw, i0, masked, M, cur.v[0], sl);
      capture(mb, i0);
      fwd_stage<C>(mb, ma, hw, i0 + 1, masked, M, cur.v[1], sl);
      capture(ma, i0 + 1);
      if ((g % C::RN) == C::RN - 1) renorm<C>(ma);
      cur = nxt;
    }
  }
  pt_traceback_pair<C>(hw, e1f, nsub, v2, pt, st, sl);
}

}  // namespace vit
