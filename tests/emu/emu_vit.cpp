// Host build of the lane-level decoder (vit_acs.cuh and the parallel-traceback
// routine of vit_pt.cuh compiled without CUDA):
// runs the kernel's exact packed 16-bit arithmetic, tile pairing, window
// alignment and survivor layout on the CPU, one lane at a time.  Test
// infrastructure only.
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <vector>

#include "../../paper_2011_09337_gb300/csrc/vit_acs.cuh"
#include "../../paper_2011_09337_gb300/csrc/vit_pt.cuh"

using namespace vit;

template <class C>
static int emu(const int8_t* llr, int64_t n, int64_t f, int64_t v1, int64_t v2, int mode, int M, uint8_t* out) {
  Frame fr{llr, out, n, mode == 1 ? n - (C::K - 1) : n, mode};
  Tiling tl{f, v1, v2};
  const int64_t ntiles = tile_count(n, f);
  const int64_t ntasks = (ntiles + 63) / 64;
  for (int64_t task = 0; task < ntasks; task++) {
    Half hw[32][2];
    int64_t maxL = 1;
    for (int l = 0; l < 32; l++)
      for (int h = 0; h < 2; h++) {
        const int64_t b = task * 64 + 2 * l + h;
        hw[l][h] = (b < ntiles) ? make_half(fr, b, tl) : idle_half();
        if (hw[l][h].active && hw[l][h].t1 - hw[l][h].t0 > maxL) maxL = hw[l][h].t1 - hw[l][h].t0;
      }
    const int Lw = (int)(((maxL + C::U - 1) / C::U) * C::U);
    int masked_until = 0;
    for (int l = 0; l < 32; l++)
      for (int h = 0; h < 2; h++)
        if (hw[l][h].active) {
          hw[l][h].start = Lw - (int)(hw[l][h].t1 - hw[l][h].t0);
          if (hw[l][h].start + 1 > masked_until) masked_until = hw[l][h].start + 1;
        }
    std::vector<uint32_t> slab((size_t)Lw * C::WORDS);
    bool words = true;  // the kernel's warp-wide alignment vote
    for (int l = 0; l < 32; l++)
      for (int h = 0; h < 2; h++)
        if (hw[l][h].active)
          words = words && ((reinterpret_cast<uintptr_t>(hw[l][h].llr) +
                             (uintptr_t)((hw[l][h].t0 - hw[l][h].start) * C::BETA)) % 4u == 0u);
    for (int l = 0; l < 32; l++) {
      if (!hw[l][0].active && !hw[l][1].active) continue;
      Slab sl{slab.data(), C::WORDS};
      decode_pair<C>(hw[l], Lw, masked_until, (uint32_t)M, sl, words);
    }
  }
  return 0;
}

// The same with the parallel traceback (subframes of f0, start rule, seed).
template <class C>
static int emu_pt(const int8_t* llr, int64_t n, int64_t f, int64_t v1, int64_t v2, int mode, int M, int64_t f0,
                  int rule, uint64_t seed, uint8_t* out) {
  Frame fr{llr, out, n, mode == 1 ? n - (C::K - 1) : n, mode};
  Tiling tl{f, v1, v2};
  const PtParams pt{f0, rule, seed};
  const int64_t ntiles = tile_count(n, f);
  const int64_t ntasks = (ntiles + 63) / 64;
  const int64_t fb = tile_len(n, f);
  const int64_t nsub = (fb + f0 - 1) / f0;
  std::vector<uint8_t> states((size_t)(ntiles * nsub + 1));
  for (int64_t task = 0; task < ntasks; task++) {
    Half hw[32][2];
    int64_t e1f[32][2];
    int64_t maxL = 1;
    for (int l = 0; l < 32; l++)
      for (int h = 0; h < 2; h++) {
        const int64_t b = task * 64 + 2 * l + h;
        hw[l][h] = (b < ntiles) ? make_half(fr, b, tl) : idle_half();
        e1f[l][h] = (b < ntiles) ? ((b * fb + fb < n) ? b * fb + fb : n) : 0;
        if (hw[l][h].active && hw[l][h].t1 - hw[l][h].t0 > maxL) maxL = hw[l][h].t1 - hw[l][h].t0;
      }
    const int Lw = (int)(((maxL + C::U - 1) / C::U) * C::U);
    int masked_until = 0;
    for (int l = 0; l < 32; l++)
      for (int h = 0; h < 2; h++)
        if (hw[l][h].active) {
          hw[l][h].start = Lw - (int)(hw[l][h].t1 - hw[l][h].t0);
          if (hw[l][h].start + 1 > masked_until) masked_until = hw[l][h].start + 1;
        }
    std::vector<uint32_t> slab((size_t)Lw * C::WORDS);
    bool words = true;  // the kernel's warp-wide alignment vote
    for (int l = 0; l < 32; l++)
      for (int h = 0; h < 2; h++)
        if (hw[l][h].active)
          words = words && ((reinterpret_cast<uintptr_t>(hw[l][h].llr) +
                             (uintptr_t)((hw[l][h].t0 - hw[l][h].start) * C::BETA)) % 4u == 0u);
    for (int l = 0; l < 32; l++) {
      if (!hw[l][0].active && !hw[l][1].active) continue;
      Slab sl{slab.data(), C::WORDS};
      uint8_t* const st[2] = {states.data() + (task * 64 + 2 * l) * nsub,
                              states.data() + (task * 64 + 2 * l + 1) * nsub};
      decode_pair_pt<C>(hw[l], e1f[l], Lw, masked_until, (uint32_t)M, sl, v2, pt, st, words);
    }
  }
  return 0;
}

#define EMU_PT(name, ...)                                                                                    \
  extern "C" int name(const int8_t* llr, int64_t n, int64_t f, int64_t v1, int64_t v2, int mode, int M,      \
                      int64_t f0, int rule, uint64_t seed, uint8_t* out) {                                   \
    return emu_pt<Code<__VA_ARGS__>>(llr, n, f, v1, v2, mode, M, f0, rule, seed, out);                       \
  }
EMU_PT(emu_pt_k7_171_133, 7, 2, 0171, 0133)
EMU_PT(emu_pt_k7_133_171_165, 7, 3, 0133, 0171, 0165)
EMU_PT(emu_pt_k5_23_35, 5, 2, 023, 035)
EMU_PT(emu_pt_k3_7_5, 3, 2, 07, 05)

#define EMU(name, ...)                                                                                      \
  extern "C" int name(const int8_t* llr, int64_t n, int64_t f, int64_t v1, int64_t v2, int mode, int M,     \
                      uint8_t* out) {                                                                       \
    return emu<Code<__VA_ARGS__>>(llr, n, f, v1, v2, mode, M, out);                                         \
  }
EMU(emu_k7_171_133, 7, 2, 0171, 0133)
EMU(emu_k7_133_171_165, 7, 3, 0133, 0171, 0165)
EMU(emu_k5_23_35, 5, 2, 023, 035)
EMU(emu_k3_7_5, 3, 2, 07, 05)
EMU(emu_k4_b4, 4, 4, 013, 015, 017, 011)
EMU(emu_k6_asym, 6, 2, 053, 046)
