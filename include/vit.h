/*
 * vit.h -- C ABI of libvit, a GB300-native (sm_103a) soft-decision Viterbi
 * decoder for rate-1/beta convolutional codes (arxiv 2011.09337).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - All pointers named "device" are CUDA device pointers owned by the
 *    caller; the library never frees them.  Host pointers are read during the
 *    call only.  The library owns vit_code / vit_batch handles and the device
 *    memory they hold.
 *  - Calls that take a stream enqueue work on it and return without
 *    synchronising.  The stream is a cudaStream_t passed as void* (NULL = the
 *    legacy default stream).
 *  - Every call returns VIT_OK (0) or a negative status; nothing aborts.
 *    vit_last_error() returns a thread-local message for the last failure.
 *    A failed launch reports VIT_ECUDA.  Arguments are checked before any
 *    work is enqueued.
 *  - LLRs are int8 in [-127, 127] (decoder) or float32 (path metrics),
 *    stage-major: llr[t*beta + b] is coded bit b of trellis stage t.
 *    Positive means bit 0 is more likely (Sec. "Hard-decision vs.
 *    Soft-decision").  With a puncturing pattern set, the decoder input holds
 *    only the transmitted symbols in the same order.
 *  - Decoded bits are packed LSB-first: bit t is bit (t & 7) of byte t >> 3.
 *
 * Code and trellis (Eq. 1, Fig. 1): generator g_b is a K-bit word whose bit
 * K-1 taps the current input.  The state is the previous K-1 inputs with the
 * newest in bit K-2; every branch into state j carries input bit (j >> (K-2)).
 * Ties in add-compare-select keep the lower-numbered predecessor (decision 0);
 * the traceback of a tile starts at the highest final path metric, ties going
 * to the lowest state, or at state 0 at the end of a terminated frame.
 */
#ifndef VIT_H
#define VIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vit_code vit_code;
typedef struct vit_batch vit_batch;
typedef void* vit_stream_t; /* cudaStream_t */

enum {
  VIT_OK = 0,
  VIT_EINVAL = -1,       /* bad argument (null pointer, size, alignment, range) */
  VIT_EUNSUPPORTED = -2, /* valid code outside the compiled envelope */
  VIT_ENOMEM = -3,       /* host or device allocation failed */
  VIT_ECUDA = -4,        /* a CUDA call or kernel launch failed */
  VIT_ETIMEOUT = -5      /* a bounded device wait gave up (batched queue) */
};

/* Frame start/end handling. */
enum {
  VIT_STREAM = 0,     /* starts in state 0, free end: traceback from the best state */
  VIT_TERMINATED = 1, /* starts in state 0, ends with K-1 zero tail bits: traceback
                         from state 0; the tail bits are not output */
  VIT_FREE_START = 2  /* unknown start (all initial metrics equal, as in Alg. 1) */
};

/* ------------------------------------------------------------------ codes */

/*
 * Creates a code handle.  K in [3, 9], beta in [2, 4], (K-1)*beta <= 32;
 * polys: beta generator words (host array), each nonzero and < 2^K.
 * Tiling (Sec. "Previous GPU methods", Fig. relworks): the stream is cut into
 * tiles of f output stages; tile b decodes stages [b*f, (b+1)*f) from the
 * window [b*f - v1, (b+1)*f + v2) clipped to the frame, with v1 = v2 = v.
 * f = 0 decodes each frame as one tile (full-frame Viterbi, Alg. 1 + 2);
 * otherwise f must be a positive multiple of 8.  A window that does not start
 * at stage 0 starts with all path metrics equal.
 * Every valid code is decoded.  Codes with a compiled kernel (among them
 * (171,133), (133,171), (133,171,165) and (561,753)) run the fast tile
 * decoders; any other generators run decoders that take the generators at
 * run time (one warp per tile, the states over the lanes; slower), which have
 * no parallel traceback.
 */
int vit_create(vit_code** out, int K, int beta, const uint32_t* polys, int64_t f, int64_t v);

/* Sets asymmetric overlaps v1 (left) and v2 (right), both >= 0. */
int vit_set_overlaps(vit_code* code, int64_t v1, int64_t v2);

/*
 * Sets a puncturing pattern (Sec. "De-puncturing"): mask is beta x period,
 * row-major, 1 = transmitted; stage t uses column t mod period.  Removed
 * symbols decode as LLR 0.  period = 0 clears the pattern.  Every column
 * must keep at least one symbol.
 */
int vit_set_puncture(vit_code* code, const uint8_t* mask, int period);

/* Default frame mode used by vit_decode: VIT_STREAM (initial), VIT_TERMINATED
 * or VIT_FREE_START. */
int vit_set_termination(vit_code* code, int mode);

/*
 * Parallel traceback (Sec. "Parallel Traceback Algorithm", Fig. pt1): each
 * tile's emitted stages are cut into subframes of f0 stages, each traced
 * back on its own from v2 stages to its right (the overlap is not emitted).
 * A subframe whose traceback starts at its window's last stage starts from
 * the usual state (argmax, or state 0 at the end of a terminated frame); the
 * others start from the argmax of their first traceback stage's path
 * metrics, recorded during the forward pass (VIT_PT_STORED), or from the top
 * K-1 bits of output u of SplitMix64 seeded with `seed` (VIT_PT_RANDOM; u =
 * the global index of that stage).  The decoded bits differ from the serial
 * traceback's.  f0: 0 (off, the default) or a positive multiple of 8.
 * Returns VIT_EUNSUPPORTED for codes without a compiled parallel-traceback
 * kernel (K > 7, and codes decoded with generators taken at run time).
 */
enum { VIT_PT_STORED = 0, VIT_PT_RANDOM = 1 };
int vit_set_parallel_traceback(vit_code* code, int64_t f0, int rule, uint64_t seed);

/*
 * Decoder choice for vit_decode_ws / vit_decode / vit_decode_noalloc (batches
 * always use the tile decoders).  VIT_DECODER_AUTO (initial): one warp per
 * tile with the decisions in shared memory (Sec. "Unified Kernel": the
 * survivors never leave the SM) for frames of at most 1024 tiles whose
 * windows fit 6144 stages, else the tile decoder (two tiles per lane, 64 per
 * warp, survivor words in the scratch slab), or -- when the frame has too
 * few tiles to keep half of that decoder's resident warps busy and the code
 * has one -- the spread tile decoder (each tile pair over four lanes, 16
 * tiles per warp; compiled for the K=7 rate-1/2 codes (171,133) and
 * (133,171)).  VIT_DECODER_TILES always uses the two-tiles-per-lane decoder,
 * VIT_DECODER_SPREAD the spread one (VIT_EUNSUPPORTED at decode time for
 * codes without it); VIT_DECODER_SHARED always uses the shared-memory
 * decoder (any number of tiles; VIT_EUNSUPPORTED at decode time when a
 * window exceeds 6144 stages or the code has no such decoder: K > 7 with
 * compiled kernels).
 */
enum { VIT_DECODER_AUTO = 0, VIT_DECODER_TILES = 1, VIT_DECODER_SHARED = 2, VIT_DECODER_SPREAD = 3 };
int vit_set_decoder(vit_code* code, int which);

void vit_destroy(vit_code* code);

/* Number of int8 LLRs the decoder reads for n trellis stages. */
int64_t vit_llr_count(const vit_code* code, int64_t n);

/* Number of decoded bits written for n stages (n - (K-1) when terminated). */
int64_t vit_output_bits(const vit_code* code, int64_t n);

/* --------------------------------------------------------------- decoding */

/* Device scratch bytes vit_decode_ws needs for an n-stage frame on the
 * current device.  The tile decoder's survivor slab holds one slot per warp
 * task, but never more slots than warps of that decoder fit on the device at
 * once: beyond one resident wave the warps stride over the tasks and reuse
 * their slots, so the slab stops growing with n. */
size_t vit_decode_workspace(const vit_code* code, int64_t n);

/*
 * Decodes one frame of n >= 1 trellis stages (Alg. 1, Alg. 2 on every tile of
 * Fig. relworks).  llr: device, vit_llr_count(code, n) int8 values.
 * bits_out: device, ceil(vit_output_bits(code, n) / 8) bytes, fully written.
 * ws: device scratch of at least vit_decode_workspace(code, n) bytes,
 * 256-byte aligned, not used concurrently by another call.
 */
int vit_decode_ws(const vit_code* code, const int8_t* llr, int64_t n, uint8_t* bits_out, void* ws, size_t ws_bytes,
                  vit_stream_t stream);

/* Same as vit_decode_ws with scratch taken from the stream-ordered allocator
 * (cudaMallocAsync) and released on the same stream. */
int vit_decode(const vit_code* code, const int8_t* llr, int64_t n, uint8_t* bits_out, vit_stream_t stream);

/*
 * Allocation-free decode (the paper has no counterpart; this is a library
 * service).  Same result as vit_decode_ws, for callers that cannot allocate
 * device memory when they decode: real-time receive loops that must not call
 * cudaMalloc, plugins handed only their input and output buffers, processes
 * with a memory budget fixed at start-up.  The decoder scratch is a 16 MiB
 * array compiled into the library (every GPU that loads it holds the array
 * until exit); frames whose vit_decode_workspace(code, n) exceeds 16 MiB are
 * rejected with VIT_EINVAL.  The first call on each device (with that device
 * current) looks up the array's address and caches it, so make it before any
 * stream capture; after a cudaDeviceReset of that device the cached address
 * is stale and this entry point must not be used there again.  The stream
 * must belong to the current device (VIT_EINVAL otherwise).  All calls on a
 * device share the array: calls whose work overlaps on the GPU (e.g. on
 * different streams) race and must be serialised by the caller.  llr, n and
 * bits_out are as for vit_decode_ws.
 */
int vit_decode_noalloc(const vit_code* code, const int8_t* llr, int64_t n, uint8_t* bits_out, vit_stream_t stream);

/*
 * Convolutional encoder (Eq. 1) starting in state 0: bits is a device array
 * of n bytes (0/1, one input bit per stage); coded receives n*beta bytes
 * (0/1) stage-major.  Puncturing is not applied.
 */
int vit_encode(const vit_code* code, const uint8_t* bits, int64_t n, uint8_t* coded, vit_stream_t stream);

/*
 * Hard-decision input (Sec. "Hard-decision vs. Soft-decision"): a receiver
 * that keeps only the sign of each symbol hands the decoder bits.  Expands
 * `count` received bits (device, packed LSB-first: bit i at byte i >> 3, bit
 * i & 7) into int8 LLRs (device, `count` bytes): bit 0 -> +1, bit 1 -> -1.
 * Decoding those LLRs maximises the agreement with the received bits, i.e.
 * it is minimum-Hamming-distance decoding.  count = vit_llr_count(code, n).
 */
int vit_hard_llr(const uint8_t* bits, int64_t count, int8_t* llr, vit_stream_t stream);

/* ----------------------------------------------------------------- batches */

typedef struct {
  const vit_code* code; /* any created code; frames may mix codes */
  const int8_t* llr;    /* device (page-locked host with VIT_BATCH_HOST), vit_llr_count(code, n) int8 values */
  int64_t n;            /* trellis stages, >= 1 */
  int mode;             /* VIT_STREAM, VIT_TERMINATED or VIT_FREE_START */
  uint8_t* bits_out;    /* device (page-locked host with VIT_BATCH_HOST), ceil(vit_output_bits / 8) bytes */
} vit_frame;

/*
 * Plans a batch: groups the frames by (compiled kernel, tiling), orders each
 * group's frames longest first, sizes the scratch and uploads the frame
 * tables.  Each group is one launch of its code's tile decoder; the groups
 * run concurrently (the costliest on the caller's stream, the others on
 * streams owned by the plan, forked and joined with events).  Frame pointers
 * are recorded: a plan decodes the same buffers every time it runs.  Tiling
 * uses each frame's code (f, v1, v2); the autotuner of the Python package
 * (paper_2011_09337_gb300.tune) picks tilings and CTA sizes by timing plans.
 *
 * flags: VIT_BATCH_GRAPH captures the launches in a CUDA graph on the first
 * run and replays it afterwards.  VIT_BATCH_PERSISTENT: when the batch holds
 * exactly two code groups for which a persistent two-code kernel is
 * compiled, one launch pulls all their warp tasks from a queue ordered
 * longest window first (otherwise ignored).  Bits 8..15 give the CTA size in
 * warps (1..8, 0 = 4).
 *
 * VIT_BATCH_HOST (host-staged batch): every frame's llr and bits_out are
 * HOST pointers to page-locked memory (cudaHostAlloc / cudaHostRegister;
 * anything else gives VIT_EINVAL at plan time).  The plan owns device copies
 * of the frames' LLRs and output bytes, and each run copies the LLRs in,
 * decodes and copies the bits back, pipelined: every group's warp tasks are
 * cut into chunks (bits 16..23: 1..64 chunks, 0 = 8; a chunk count without
 * VIT_BATCH_HOST is VIT_EINVAL); chunk k's input copy (a plan-owned copy
 * stream), its decode launch (one of up to four plan-owned compute streams,
 * in turn) and its output copy (a second copy stream) are ordered by events,
 * so the copies of some chunks overlap the decoding of others.  Each chunk
 * copies the LLR bytes of its tiles' windows that earlier chunks have not
 * copied, and the output bytes its tiles emit (tiles end on byte boundaries,
 * so no byte is shared between chunks).  Punctured frames are copied whole
 * and de-punctured before the first chunk.  All of it is forked from and
 * joined back into the caller's stream: when that stream reaches the end of
 * the run, the host output buffers hold the bits.  VIT_BATCH_PERSISTENT is
 * ignored with VIT_BATCH_HOST.  Other bits: VIT_EINVAL.
 */
enum { VIT_BATCH_GRAPH = 1, VIT_BATCH_PERSISTENT = 4, VIT_BATCH_HOST = 8 };
int vit_batch_plan(vit_batch** out, const vit_frame* frames, int nframes, int flags);
int vit_batch_run(vit_batch* batch, vit_stream_t stream);
void vit_batch_destroy(vit_batch* batch);

/* Plans, runs once and releases the plan after the stream has finished it. */
int vit_decode_batch(const vit_frame* frames, int nframes, vit_stream_t stream);

/* ------------------------------------------------------ path-metric forms */

/*
 * Best-path metric of F zero-terminated frames of n stages each (not defined
 * by the paper; see the oracle): tau == 0 is the hard form
 *   M = max over 0-rooted, 0-terminated paths of sum_t delta_t (Eq. 2),
 * tau > 0 the log-sum-exp form M_tau = tau log sum exp(sum_t delta_t / tau).
 * llr: device float32 [F][n][beta]; metric_out: device float32 [F].
 * ws: device scratch of vit_metric_workspace(...) bytes, kept unchanged
 * between vit_metric_fwd and the matching vit_metric_bwd (it holds the
 * survivor bits, or the forward state metrics every C stages with their fp64
 * offsets and the forward metric, which the backward uses as the common scale
 * of each stage's posteriors).
 */
size_t vit_metric_workspace(const vit_code* code, int nframes, int64_t n, float tau, int C);
int vit_metric_fwd(const vit_code* code, const float* llr, int nframes, int64_t n, float tau, int C,
                   float* metric_out, void* ws, size_t ws_bytes, vit_stream_t stream);
/*
 * Gradient of sum_f grad_metric[f] * M_f with respect to llr: the +-1 code
 * symbols of the traced best path (tau == 0) or their posterior expectation
 * (tau > 0, recomputing forward metrics between checkpoints).
 * grad_metric: device float32 [F]; grad_llr: device float32 [F][n][beta].
 */
int vit_metric_bwd(const vit_code* code, const float* llr, const float* grad_metric, int nframes, int64_t n,
                   float tau, int C, const void* ws, size_t ws_bytes, float* grad_llr, vit_stream_t stream);

/* ------------------------------------------------------------------ misc */

const char* vit_last_error(void);
/* 1 if vit_create accepts (K, beta, polys), i.e. the code is valid, else 0. */
int vit_code_supported(int K, int beta, const uint32_t* polys);

#ifdef __cplusplus
}
#endif
#endif /* VIT_H */
