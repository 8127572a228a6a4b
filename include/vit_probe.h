/*
 * vit_probe.h -- instruction-rate microbenchmark exported by libvit, the
 * measured denominator of the decoder's roofline (not part of the paper's
 * method).
 *
 * The decoder's add-compare-select is integer arithmetic on packed 16-bit
 * path metrics (IADD3 / IMAD adds, max.u16x2 compare-selects, PRMT / LOP3
 * survivor packing), and the differentiable path metric is FP32 max-plus /
 * log-sum-exp (FADD, FMNMX, MUFU ex2 / lg2).  vit_probe_rate times one
 * instruction class in isolation: every thread runs 8 independent pairs of
 * dependency chains of that instruction (each step updates both registers of
 * a pair from each other and from a neighbouring pair, so no step can be
 * folded away) for `iters` rounds of 16 steps, in a grid of `ctas_per_sm`
 * CTAs of `warps` warps on every SM (all CTAs resident at once).
 */
#ifndef VIT_PROBE_H
#define VIT_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  VIT_PROBE_IADD = 0,     /* add.u32 (IADD3) */
  VIT_PROBE_VMAX16 = 1,   /* max.u16x2 (packed 16-bit compare-select) */
  VIT_PROBE_IMAD = 2,     /* mad.lo.u32 (IMAD) */
  VIT_PROBE_PRMT = 3,     /* prmt.b32 */
  VIT_PROBE_LOP3 = 4,     /* lop3.b32 (a & b) | c */
  VIT_PROBE_FADD = 5,     /* add.f32 */
  VIT_PROBE_FMAX = 6,     /* max.f32 */
  VIT_PROBE_EX2 = 7,      /* ex2.approx.ftz.f32 (MUFU) */
  VIT_PROBE_LG2 = 8,      /* lg2.approx.ftz.f32 (MUFU) */
  VIT_PROBE_KINDS = 9
};

/*
 * Runs the probe of instruction class `kind` on the current device and the
 * given stream (cudaStream_t as void*, NULL = legacy default stream), then
 * synchronises the stream.  Outputs (host pointers):
 *   warp_instr_per_clk_sm: warp-level instructions of that class retired per
 *                          SM clock cycle per SM: the instructions of the CTAs
 *                          that ran on each SM over that SM's clock64 span
 *                          (first CTA start to last CTA end), summed over SMs,
 *   ms:                    wall time of the launch (CUDA events),
 *   sms:                   the device's multiprocessor count.
 * ctas_per_sm in [1, 32], warps in [1, 32], iters in [1, 1<<20]; a grid
 * that cannot be fully resident returns VIT_EINVAL.  Returns VIT_OK or a
 * negative status of include/vit.h (vit_last_error() has the message).
 */
int vit_probe_rate(int kind, int ctas_per_sm, int warps, int iters, void* stream, double* warp_instr_per_clk_sm,
                   double* ms, int* sms);

#ifdef __cplusplus
}
#endif
#endif /* VIT_PROBE_H */
