/*
 * vit_oracle.c -- plain, slow CPU oracle for soft-decision Viterbi decoding
 * (arxiv 2011.09337).  TEST INFRASTRUCTURE ONLY: it is compiled and called by
 * the test-suite, by the smoke check and by the CPU-baseline leg of the
 * benchmark, never by the product library.  It shares no code, header, table
 * or constant with the CUDA path.
 *
 * Everything here is the definition written out, in the paper's order:
 *   encoder ............ Eq. 1 (Fig. 1): out_b = XOR over taps of g_b & R_t
 *   branch metric ...... Eq. 2: delta = sum_b (-1)^{alpha_out[b]} * llr_t[b]
 *   ACS / survivor ..... Eq. 3 and Eq. 4, Alg. 1 (forward procedure)
 *   traceback/decode ... Alg. 2 (backward procedure)
 *   tiling ............. Sec. "Previous GPU methods", Fig. relworks: blocks of
 *                        f output stages with v1/v2 overlaps
 *   de-puncturing ...... Sec. "De-puncturing": zero LLR at removed positions
 *   parallel traceback . Sec. "Parallel Traceback Algorithm" (Fig. pt1):
 *                        subframes of f0 stages, each traced back from v2
 *                        stages to its right
 * plus two quantities the paper does not define (best-path metric and its
 * temperature log-sum-exp relaxation, with gradients) and brute-force ML.
 *
 * Conventions where the paper is silent (each is a reading of the paper):
 *  - Generator g_b is a K-bit word; bit K-1 is the tap on the current input
 *    (Eq. 1 pairs g_{K-1} with in_t).  Register word R_t = in_t*2^(K-1) + s_t.
 *  - State s_t = sum_{m=1}^{K-1} in_{t-m} 2^{K-1-m} (newest input = MSB).
 *    Branch i -> j has R = 2j + (i & 1); predecessors of j are 2j mod S and
 *    2j+1 mod S; alpha_in of every branch into j is bit K-2 of j.
 *  - ACS tie: the lower predecessor index wins (decision 0), i.e. decision 1
 *    only when the odd predecessor's candidate is strictly larger.
 *  - Known start: metric 0 for state 0 and -M for the others (M = 8192 by
 *    default); a window that does not start at stage 0, or FREE_START, starts
 *    with all metrics 0 (Alg. 1 zero-initialises).
 *  - Traceback starts at the argmax of the last stage of the window (ties to
 *    the lowest state index), or at state 0 when the window ends at the end
 *    of a terminated frame.
 *  - Positive LLR means bit 0 is more likely.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-3)

#define ORC_STREAM 0
#define ORC_TERMINATED 1
#define ORC_FREE_START 2

static int parity_u32(uint32_t x) {
  int p = 0;
  while (x) {
    p ^= 1;
    x &= x - 1u;
  }
  return p;
}

static int code_ok(int K, int beta, const uint32_t* polys) {
  if (K < 2 || K > 16 || beta < 1 || beta > 8 || polys == NULL) return 0;
  for (int b = 0; b < beta; b++)
    if (polys[b] >> K) return 0;
  return 1;
}

/* Branch output alpha_out for register word R (Eq. 1), bit b = output b. */
static uint32_t branch_output(int beta, const uint32_t* polys, uint32_t R) {
  uint32_t o = 0;
  for (int b = 0; b < beta; b++) o |= (uint32_t)parity_u32(polys[b] & R) << b;
  return o;
}

/* ------------------------------------------------------------------ Eq. 1 */
int orc_encode(int K, int beta, const uint32_t* polys, const uint8_t* in, int64_t n, uint8_t* out) {
  if (!code_ok(K, beta, polys) || n < 0 || (n > 0 && (!in || !out))) return ORC_EINVAL;
  uint32_t s = 0; /* previous K-1 inputs, newest at bit K-2 */
  for (int64_t t = 0; t < n; t++) {
    uint32_t R = ((uint32_t)(in[t] & 1u) << (K - 1)) | s;
    for (int b = 0; b < beta; b++) out[t * beta + b] = (uint8_t)parity_u32(polys[b] & R);
    s = R >> 1;
  }
  return ORC_OK;
}

/* ---------------------------------------------------- Sec. De-puncturing */
/* rx holds the kept symbols in transmission order (stage-major, coded stream
 * b inside a stage); mask is beta x P row-major, 1 = transmitted; the phase
 * of stage t is t mod P.  Returns the number of symbols consumed, or < 0. */
int64_t orc_depuncture(const int8_t* rx, int64_t n_rx, int64_t n, int beta, const uint8_t* mask, int P, int8_t* llr) {
  if (n < 0 || beta < 1 || P < 1 || !mask || (n > 0 && !llr)) return ORC_EINVAL;
  int64_t k = 0;
  for (int64_t t = 0; t < n; t++) {
    for (int b = 0; b < beta; b++) {
      if (mask[b * P + (int)(t % P)]) {
        if (k >= n_rx) return ORC_EINVAL;
        llr[t * beta + b] = rx[k++];
      } else {
        llr[t * beta + b] = 0;
      }
    }
  }
  return k;
}

/* Decisions as a bitset: one bit per (stage, state). */
static inline void dec_set(uint8_t* d, int64_t idx, int v) {
  if (v) d[idx >> 3] |= (uint8_t)(1u << (idx & 7));
}
static inline int dec_get(const uint8_t* d, int64_t idx) { return (d[idx >> 3] >> (idx & 7)) & 1; }

/*
 * One window of the trellis (Alg. 1 then Alg. 2) over stages [t0, t1) of a
 * de-punctured, stage-major int8 LLR stream.  Bits of stages [e0, e1) are
 * written to bits[t] (indexed by global stage).  end_state < 0 means the
 * traceback starts at the argmax of the last stage.
 */
static int run_window(int K, int beta, const uint32_t* polys, const uint32_t* aout, const int8_t* llr, int64_t t0,
                      int64_t t1, int known_start, int64_t M, int end_state, int64_t e0, int64_t e1, uint8_t* bits,
                      int64_t* metric_out) {
  const int S = 1 << (K - 1);
  const int64_t L = t1 - t0;
  int64_t* pm = (int64_t*)malloc(sizeof(int64_t) * S);
  int64_t* nm = (int64_t*)malloc(sizeof(int64_t) * S);
  uint8_t* dec = (uint8_t*)calloc((size_t)((L * S + 7) / 8 + 1), 1);
  if (!pm || !nm || !dec) {
    free(pm);
    free(nm);
    free(dec);
    return ORC_ENOMEM;
  }
  for (int j = 0; j < S; j++) pm[j] = known_start ? (j == 0 ? 0 : -M) : 0;

  for (int64_t t = t0; t < t1; t++) {
    const int8_t* l = llr + t * beta;
    for (int j = 0; j < S; j++) {
      /* the two branches into j: from i0 = 2j mod S (R = 2j) and
       * i1 = 2j+1 mod S (R = 2j+1); Eq. 2 for each */
      const int i0 = (2 * j) & (S - 1), i1 = i0 | 1;
      const uint32_t R0 = 2u * (uint32_t)j, R1 = R0 + 1u;
      int64_t bm0 = 0, bm1 = 0;
      for (int b = 0; b < beta; b++) {
        bm0 += ((aout[R0] >> b) & 1u) ? -(int64_t)l[b] : (int64_t)l[b];
        bm1 += ((aout[R1] >> b) & 1u) ? -(int64_t)l[b] : (int64_t)l[b];
      }
      const int64_t c0 = pm[i0] + bm0, c1 = pm[i1] + bm1; /* Eq. 3 */
      if (c1 > c0) {                                     /* Eq. 4, tie -> i0 */
        nm[j] = c1;
        dec_set(dec, (t - t0) * S + j, 1);
      } else {
        nm[j] = c0;
      }
    }
    int64_t* tmp = pm;
    pm = nm;
    nm = tmp;
  }

  int j = end_state;
  if (j < 0) { /* Alg. 2: argmax at the last stage, lowest index on ties */
    j = 0;
    for (int s = 1; s < S; s++)
      if (pm[s] > pm[j]) j = s;
  }
  if (metric_out) *metric_out = pm[j];
  for (int64_t t = t1 - 1; t >= t0; t--) {
    if (t >= e0 && t < e1) bits[t] = (uint8_t)((j >> (K - 2)) & 1);
    j = ((j << 1) | dec_get(dec, (t - t0) * S + j)) & (S - 1);
  }
  free(pm);
  free(nm);
  free(dec);
  return ORC_OK;
}

static int make_aout(int K, int beta, const uint32_t* polys, uint32_t** aout) {
  const uint32_t nR = 1u << K;
  *aout = (uint32_t*)malloc(sizeof(uint32_t) * nR);
  if (!*aout) return ORC_ENOMEM;
  for (uint32_t R = 0; R < nR; R++) (*aout)[R] = branch_output(beta, polys, R);
  return ORC_OK;
}

/*
 * Blocked decoding (tiling with overlaps).  Block b emits stages
 * [b*f, min((b+1)*f, n)) and processes [max(0, b*f - v1), min(n, (b+1)*f + v2)).
 * f == 0 means one block spanning the whole frame (full-frame Viterbi).
 * Blocks [b_begin, b_end) are decoded (b_end < 0: all).  bits has n entries.
 */
int orc_viterbi_blocked(int K, int beta, const uint32_t* polys, const int8_t* llr, int64_t n, int64_t f, int64_t v1,
                        int64_t v2, int mode, int64_t M, int64_t b_begin, int64_t b_end, uint8_t* bits,
                        int64_t* metric_out) {
  if (!code_ok(K, beta, polys) || n < 0 || f < 0 || v1 < 0 || v2 < 0 || M <= 0) return ORC_EINVAL;
  if (mode != ORC_STREAM && mode != ORC_TERMINATED && mode != ORC_FREE_START) return ORC_EINVAL;
  if (n == 0) return ORC_OK;
  if (!llr || !bits) return ORC_EINVAL;
  const int64_t fb = (f == 0 || f > n) ? n : f;
  const int64_t B = (n + fb - 1) / fb;
  if (b_end < 0 || b_end > B) b_end = B;
  if (b_begin < 0) b_begin = 0;
  uint32_t* aout = NULL;
  int rc = make_aout(K, beta, polys, &aout);
  if (rc) return rc;
  for (int64_t b = b_begin; b < b_end && rc == ORC_OK; b++) {
    const int64_t e0 = b * fb, e1 = (e0 + fb < n) ? e0 + fb : n;
    const int64_t t0 = (e0 - v1 > 0) ? e0 - v1 : 0;
    const int64_t t1 = (e1 + v2 < n) ? e1 + v2 : n;
    const int known = (t0 == 0 && mode != ORC_FREE_START);
    const int end_state = (t1 == n && mode == ORC_TERMINATED) ? 0 : -1;
    int64_t m = 0;
    rc = run_window(K, beta, polys, aout, llr, t0, t1, known, M, end_state, e0, e1, bits, &m);
    if (metric_out) metric_out[b - b_begin] = m;
  }
  free(aout);
  return rc;
}

/*
 * One window [t0, t1) of a de-punctured stream (Alg. 1 then Alg. 2) with an
 * explicit traceback start: end_state >= 0 starts there, -1 at the argmax of
 * the last stage.  known != 0 starts in state 0 (others -M), else all 0.
 * Bits of stages [e0, e1) are written to bits[t] (global stage index).
 */
int orc_viterbi_window(int K, int beta, const uint32_t* polys, const int8_t* llr, int64_t t0, int64_t t1, int known,
                       int64_t M, int end_state, int64_t e0, int64_t e1, uint8_t* bits) {
  if (!code_ok(K, beta, polys) || t0 < 0 || t1 <= t0 || M <= 0 || !llr || !bits) return ORC_EINVAL;
  if (end_state >= (1 << (K - 1)) || end_state < -1) return ORC_EINVAL;
  uint32_t* aout = NULL;
  if (make_aout(K, beta, polys, &aout)) return ORC_ENOMEM;
  const int rc = run_window(K, beta, polys, aout, llr, t0, t1, known, M, end_state, e0, e1, bits, NULL);
  free(aout);
  return rc;
}

/* ------------------------------------------------- parallel traceback */
/*
 * SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014) used as a counter-based generator: output i under
 * key `seed` is the mix of seed + (i + 1) * 0x9E3779B97F4A7C15 (the state the
 * sequential generator seeded with `seed` holds before its (i+1)-th output).
 */
uint64_t orc_splitmix64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

#define ORC_PT_STORED 0
#define ORC_PT_RANDOM 1

/*
 * Blocked decoding with the paper's first parallel traceback (Sec. "Parallel
 * Traceback Algorithm", Fig. pt1).  Block b's windows are those of
 * orc_viterbi_blocked.  Its emitted range [e0, e1) is cut into subframes of
 * f0 stages: subframe k emits [e0 + k f0, min(e0 + (k+1) f0, e1)).  Subframe
 * k overlaps its right-hand neighbour by v2 stages: its traceback starts at
 * stage u = min(end_k + v2, t1) - 1 and runs down to the subframe's first
 * stage, emitting only the subframe's own stages.  Its start state is
 *   - the window's usual start (Alg. 2 argmax, or state 0 at the end of a
 *     terminated frame) when u is the window's last stage;
 *   - otherwise, with ORC_PT_STORED, the argmax of the path metrics of stage
 *     u (ties to the lowest state), recorded during the forward pass; with
 *     ORC_PT_RANDOM, the top K-1 bits of orc_splitmix64(seed, u).
 * f0 == 0 or f0 >= the block's emitted length gives the serial traceback.
 */
int orc_viterbi_blocked_pt(int K, int beta, const uint32_t* polys, const int8_t* llr, int64_t n, int64_t f,
                           int64_t v1, int64_t v2, int64_t f0, int start_rule, uint64_t seed, int mode, int64_t M,
                           int64_t b_begin, int64_t b_end, uint8_t* bits) {
  if (!code_ok(K, beta, polys) || n < 0 || f < 0 || v1 < 0 || v2 < 0 || f0 < 0 || M <= 0) return ORC_EINVAL;
  if (mode != ORC_STREAM && mode != ORC_TERMINATED && mode != ORC_FREE_START) return ORC_EINVAL;
  if (start_rule != ORC_PT_STORED && start_rule != ORC_PT_RANDOM) return ORC_EINVAL;
  if (n == 0) return ORC_OK;
  if (!llr || !bits) return ORC_EINVAL;
  const int S = 1 << (K - 1);
  const int64_t fb = (f == 0 || f > n) ? n : f;
  const int64_t B = (n + fb - 1) / fb;
  if (b_end < 0 || b_end > B) b_end = B;
  if (b_begin < 0) b_begin = 0;
  uint32_t* aout = NULL;
  if (make_aout(K, beta, polys, &aout)) return ORC_ENOMEM;
  const int64_t Lmax = fb + v1 + v2;
  const int64_t sub = (f0 == 0 || f0 > fb) ? fb : f0;
  const int64_t nsub_max = (fb + sub - 1) / sub;
  int64_t* pm = (int64_t*)malloc(sizeof(int64_t) * S);
  int64_t* nm = (int64_t*)malloc(sizeof(int64_t) * S);
  uint8_t* dec = (uint8_t*)malloc((size_t)((Lmax * S + 7) / 8 + 1));
  int64_t* ustage = (int64_t*)malloc(sizeof(int64_t) * nsub_max);
  int* ustate = (int*)malloc(sizeof(int) * nsub_max);
  int rc = ORC_OK;
  if (!pm || !nm || !dec || !ustage || !ustate) rc = ORC_ENOMEM;
  for (int64_t b = b_begin; b < b_end && rc == ORC_OK; b++) {
    const int64_t e0 = b * fb, e1 = (e0 + fb < n) ? e0 + fb : n;
    const int64_t t0 = (e0 - v1 > 0) ? e0 - v1 : 0;
    const int64_t t1 = (e1 + v2 < n) ? e1 + v2 : n;
    const int known = (t0 == 0 && mode != ORC_FREE_START);
    const int64_t nsub = (e1 - e0 + sub - 1) / sub;
    for (int64_t k = 0; k < nsub; k++) {
      const int64_t end_k = (e0 + (k + 1) * sub < e1) ? e0 + (k + 1) * sub : e1;
      ustage[k] = ((end_k + v2 < t1) ? end_k + v2 : t1) - 1;
      ustate[k] = -1;
    }
    memset(dec, 0, (size_t)(((t1 - t0) * S + 7) / 8 + 1));
    for (int j = 0; j < S; j++) pm[j] = known ? (j == 0 ? 0 : -M) : 0;
    /* forward procedure (Alg. 1, Eq. 2-4) over the window */
    for (int64_t t = t0; t < t1; t++) {
      const int8_t* l = llr + t * beta;
      for (int j = 0; j < S; j++) {
        const int i0 = (2 * j) & (S - 1), i1 = i0 | 1;
        const uint32_t R0 = 2u * (uint32_t)j, R1 = R0 + 1u;
        int64_t bm0 = 0, bm1 = 0;
        for (int bb = 0; bb < beta; bb++) {
          bm0 += ((aout[R0] >> bb) & 1u) ? -(int64_t)l[bb] : (int64_t)l[bb];
          bm1 += ((aout[R1] >> bb) & 1u) ? -(int64_t)l[bb] : (int64_t)l[bb];
        }
        const int64_t c0 = pm[i0] + bm0, c1 = pm[i1] + bm1;
        if (c1 > c0) {
          nm[j] = c1;
          dec_set(dec, (t - t0) * S + j, 1);
        } else {
          nm[j] = c0;
        }
      }
      int64_t* tmp = pm;
      pm = nm;
      nm = tmp;
      /* record the start state of every subframe whose traceback starts here */
      for (int64_t k = 0; k < nsub; k++) {
        if (ustage[k] != t) continue;
        if (t == t1 - 1 && t1 == n && mode == ORC_TERMINATED) {
          ustate[k] = 0;
        } else if (t == t1 - 1 || start_rule == ORC_PT_STORED) {
          int jm = 0;
          for (int s2 = 1; s2 < S; s2++)
            if (pm[s2] > pm[jm]) jm = s2;
          ustate[k] = jm;
        } else {
          ustate[k] = (int)(orc_splitmix64(seed, (uint64_t)t) >> (64 - (K - 1)));
        }
      }
    }
    /* backward procedure (Alg. 2) once per subframe */
    for (int64_t k = nsub - 1; k >= 0; k--) {
      const int64_t s0 = e0 + k * sub;
      const int64_t s1 = (s0 + sub < e1) ? s0 + sub : e1;
      int j = ustate[k];
      for (int64_t t = ustage[k]; t >= s0; t--) {
        if (t < s1) bits[t] = (uint8_t)((j >> (K - 2)) & 1);
        j = ((j << 1) | dec_get(dec, (t - t0) * S + j)) & (S - 1);
      }
    }
  }
  free(aout);
  free(pm);
  free(nm);
  free(dec);
  free(ustage);
  free(ustate);
  return rc;
}

/* -------------------------------------------------- brute-force ML search */
/* Maximises sum_t sum_b (-1)^{c_t[b]} llr_t[b] over every message of n_info
 * bits (plus K-1 zero tail bits when terminated) and, for FREE_START, over
 * every initial state.  Returns the best metric, the number of maximisers and
 * the lowest-numbered maximiser's stage bits (n entries). */
int orc_brute_force(int K, int beta, const uint32_t* polys, const int8_t* llr, int n_info, int mode, int64_t* best,
                    int64_t* n_best, uint8_t* best_bits) {
  if (!code_ok(K, beta, polys) || n_info < 0 || n_info > 20 || !llr || !best || !n_best) return ORC_EINVAL;
  const int tail = (mode == ORC_TERMINATED) ? K - 1 : 0;
  const int n = n_info + tail;
  const int nstart = (mode == ORC_FREE_START) ? (1 << (K - 1)) : 1;
  uint8_t* msg = (uint8_t*)calloc((size_t)n + 1, 1);
  if (!msg) return ORC_ENOMEM;
  int have = 0;
  *n_best = 0;
  for (int s0 = 0; s0 < nstart; s0++) {
    for (int64_t m = 0; m < ((int64_t)1 << n_info); m++) {
      for (int t = 0; t < n; t++) msg[t] = (t < n_info) ? (uint8_t)((m >> t) & 1) : 0;
      uint32_t s = (uint32_t)s0;
      int64_t metric = 0;
      for (int t = 0; t < n; t++) {
        uint32_t R = ((uint32_t)msg[t] << (K - 1)) | s;
        for (int b = 0; b < beta; b++)
          metric += parity_u32(polys[b] & R) ? -(int64_t)llr[t * beta + b] : (int64_t)llr[t * beta + b];
        s = R >> 1;
      }
      if (!have || metric > *best) {
        *best = metric;
        *n_best = 1;
        have = 1;
        if (best_bits) memcpy(best_bits, msg, (size_t)n);
      } else if (metric == *best) {
        (*n_best)++;
      }
    }
  }
  free(msg);
  return ORC_OK;
}

/* ------------------------------------------- best-path metric, FP64 forms */
/*
 * Hard form: M(llr) = max over paths that start and end in state 0 of
 * sum_t delta_t (the survivor metric of state 0 at the last stage, Eq. 3
 * with a -infinity start for states other than 0).  Its subgradient with
 * respect to llr_t[b] is (-1)^{c*_t[b]}, c* the branch outputs of the traced
 * best path (ties as in the decoder).  grad may be NULL.
 */
int orc_metric_hard(int K, int beta, const uint32_t* polys, const double* llr, int64_t n, double* metric,
                    double* grad) {
  if (!code_ok(K, beta, polys) || n <= 0 || !llr || !metric) return ORC_EINVAL;
  const int S = 1 << (K - 1);
  uint32_t* aout = NULL;
  if (make_aout(K, beta, polys, &aout)) return ORC_ENOMEM;
  double* pm = (double*)malloc(sizeof(double) * S);
  double* nm = (double*)malloc(sizeof(double) * S);
  uint8_t* dec = (uint8_t*)calloc((size_t)((n * S + 7) / 8 + 1), 1);
  if (!pm || !nm || !dec) {
    free(aout);
    free(pm);
    free(nm);
    free(dec);
    return ORC_ENOMEM;
  }
  for (int j = 0; j < S; j++) pm[j] = (j == 0) ? 0.0 : -INFINITY;
  for (int64_t t = 0; t < n; t++) {
    const double* l = llr + t * beta;
    for (int j = 0; j < S; j++) {
      const int i0 = (2 * j) & (S - 1), i1 = i0 | 1;
      const uint32_t R0 = 2u * (uint32_t)j, R1 = R0 + 1u;
      double bm0 = 0, bm1 = 0;
      for (int b = 0; b < beta; b++) {
        bm0 += ((aout[R0] >> b) & 1u) ? -l[b] : l[b];
        bm1 += ((aout[R1] >> b) & 1u) ? -l[b] : l[b];
      }
      const double c0 = pm[i0] + bm0, c1 = pm[i1] + bm1;
      if (c1 > c0) {
        nm[j] = c1;
        dec_set(dec, t * S + j, 1);
      } else {
        nm[j] = c0;
      }
    }
    double* tmp = pm;
    pm = nm;
    nm = tmp;
  }
  *metric = pm[0];
  if (grad) {
    int j = 0;
    for (int64_t t = n - 1; t >= 0; t--) {
      const int d = dec_get(dec, t * S + j);
      const uint32_t R = 2u * (uint32_t)j + (uint32_t)d; /* branch taken at t */
      for (int b = 0; b < beta; b++) grad[t * beta + b] = ((aout[R] >> b) & 1u) ? -1.0 : 1.0;
      j = ((j << 1) | d) & (S - 1);
    }
  }
  free(aout);
  free(pm);
  free(nm);
  free(dec);
  return ORC_OK;
}

static double lse2(double a, double b, double tau) {
  const double m = a > b ? a : b;
  if (m == -INFINITY) return -INFINITY;
  return m + tau * log(exp((a - m) / tau) + exp((b - m) / tau));
}

/*
 * Temperature form: M_tau = tau * log sum over 0-rooted, 0-terminated paths
 * of exp(sum_t delta_t / tau).  Forward alpha and backward beta recursions
 * over the same trellis; the gradient is the posterior expectation of the
 * branch symbols (-1)^{alpha_out[b]} at every stage.  grad may be NULL.
 */
int orc_metric_lse(int K, int beta, const uint32_t* polys, const double* llr, int64_t n, double tau, double* metric,
                   double* grad) {
  if (!code_ok(K, beta, polys) || n <= 0 || !llr || !metric || !(tau > 0)) return ORC_EINVAL;
  const int S = 1 << (K - 1);
  uint32_t* aout = NULL;
  if (make_aout(K, beta, polys, &aout)) return ORC_ENOMEM;
  /* alpha[t+1][j] = forward metric after stage t; alpha[0] = start */
  double* alpha = (double*)malloc(sizeof(double) * (size_t)(n + 1) * S);
  double* bet = (double*)malloc(sizeof(double) * (size_t)(n + 1) * S);
  if (!alpha || !bet) {
    free(aout);
    free(alpha);
    free(bet);
    return ORC_ENOMEM;
  }
  for (int j = 0; j < S; j++) alpha[j] = (j == 0) ? 0.0 : -INFINITY;
  for (int64_t t = 0; t < n; t++) {
    const double* l = llr + t * beta;
    const double* a = alpha + t * S;
    double* an = alpha + (t + 1) * S;
    for (int j = 0; j < S; j++) {
      const int i0 = (2 * j) & (S - 1), i1 = i0 | 1;
      const uint32_t R0 = 2u * (uint32_t)j, R1 = R0 + 1u;
      double bm0 = 0, bm1 = 0;
      for (int b = 0; b < beta; b++) {
        bm0 += ((aout[R0] >> b) & 1u) ? -l[b] : l[b];
        bm1 += ((aout[R1] >> b) & 1u) ? -l[b] : l[b];
      }
      an[j] = lse2(a[i0] + bm0, a[i1] + bm1, tau);
    }
  }
  *metric = alpha[n * S + 0];
  if (grad) {
    /* bet[t][j] = backward metric of state j after stage t-1 (i.e. before
     * stage t); bet[n] is the end condition: state 0 only. */
    for (int j = 0; j < S; j++) bet[n * S + j] = (j == 0) ? 0.0 : -INFINITY;
    for (int64_t t = n - 1; t >= 0; t--) {
      const double* l = llr + t * beta;
      for (int i = 0; i < S; i++) {
        double acc = -INFINITY;
        for (int in = 0; in < 2; in++) {
          const uint32_t R = ((uint32_t)in << (K - 1)) | (uint32_t)i;
          const int j = (int)(R >> 1);
          double bm = 0;
          for (int b = 0; b < beta; b++) bm += ((aout[R] >> b) & 1u) ? -l[b] : l[b];
          acc = lse2(acc, bm + bet[(t + 1) * S + j], tau);
        }
        bet[t * S + i] = acc;
      }
    }
    const double Mt = *metric;
    for (int64_t t = 0; t < n; t++) {
      const double* l = llr + t * beta;
      for (int b = 0; b < beta; b++) grad[t * beta + b] = 0.0;
      for (int i = 0; i < S; i++) {
        const double ai = alpha[t * S + i];
        if (ai == -INFINITY) continue;
        for (int in = 0; in < 2; in++) {
          const uint32_t R = ((uint32_t)in << (K - 1)) | (uint32_t)i;
          const int j = (int)(R >> 1);
          const double bj = bet[(t + 1) * S + j];
          if (bj == -INFINITY) continue;
          double bm = 0;
          for (int b = 0; b < beta; b++) bm += ((aout[R] >> b) & 1u) ? -l[b] : l[b];
          const double p = exp((ai + bm + bj - Mt) / tau); /* branch posterior */
          for (int b = 0; b < beta; b++) grad[t * beta + b] += ((aout[R] >> b) & 1u) ? -p : p;
        }
      }
    }
  }
  free(aout);
  free(alpha);
  free(bet);
  return ORC_OK;
}
