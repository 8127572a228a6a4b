// vit_api.cu -- host side of the C ABI declared in include/vit.h: argument
// checking, code registry, tiling/workspace arithmetic, launches of the
// tile decoder, de-puncturing and encoder kernels.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/vit.h"
#include "vit_internal.h"

using namespace vit;


namespace {
thread_local std::string g_err;
std::mutex g_reg_mu;
std::vector<CodeEntry>& registry() {
  static std::vector<CodeEntry> r;
  return r;
}

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  return fail(VIT_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

constexpr int kMaxPeriod = 64;
constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

int64_t max_window(const vit_code* c, int64_t n) {
  const int64_t fb = tile_len(n, c->f);
  int64_t w = fb + c->v1 + c->v2;
  return w < n ? w : n;
}
int64_t kept_in(const vit_code* c, int64_t n) {
  if (c->period == 0) return n * c->beta;
  int64_t per = 0, part = 0;
  const int64_t r = n % c->period;
  for (int col = 0; col < c->period; col++)
    for (int b = 0; b < c->beta; b++)
      if (c->mask[b * c->period + col]) {
        per++;
        if (col < r) part++;
      }
  return (n / c->period) * per + part;
}

// ---------------------------------------------------------- small kernels
struct PunctArgs {
  int beta, period;
  int64_t per_period;
  int32_t col_prefix[kMaxPeriod];     // kept symbols before column col
  int8_t rank[4 * kMaxPeriod];        // index of (b, col) inside its column, -1 if removed
};

__global__ void depuncture_kernel(const int8_t* __restrict__ rx, int64_t n, int8_t* __restrict__ out, PunctArgs p) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int col = (int)(t % p.period);
  const int64_t base = (t / p.period) * p.per_period + p.col_prefix[col];
  for (int b = 0; b < p.beta; b++) {
    const int r = p.rank[b * kMaxPeriod + col];
    out[t * p.beta + b] = (r >= 0) ? rx[base + r] : (int8_t)0;
  }
}

__global__ void encode_kernel(const uint8_t* __restrict__ bits, int64_t n, int K, int beta, uint4 polys,
                              uint8_t* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  uint32_t R = 0;  // Eq. 1 register word: bit K-1 = in_t, bit 0 = in_{t-K+1}
  for (int m = 0; m < K; m++) {
    const int64_t s = t - m;
    const uint32_t v = (s >= 0) ? (uint32_t)(bits[s] & 1u) : 0u;
    R |= v << (K - 1 - m);
  }
  const uint32_t g[4] = {polys.x, polys.y, polys.z, polys.w};
  for (int b = 0; b < beta; b++) out[t * beta + b] = (uint8_t)(__popc(g[b] & R) & 1);
}

// Hard-decision input: received bit i (packed LSB-first) -> int8 +1 (bit 0)
// or -1 (bit 1).  One thread per output byte group of 8 symbols.
__global__ void hard_llr_kernel(const uint8_t* __restrict__ bits, int64_t count, int8_t* __restrict__ llr) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g * 8 >= count) return;
  const uint32_t b = bits[g];
  const int64_t lim = (count - g * 8 < 8) ? count - g * 8 : 8;
  for (int k = 0; k < lim; k++) llr[g * 8 + k] = ((b >> k) & 1u) ? (int8_t)-1 : (int8_t)1;
}

bool code_args_ok(int K, int beta, const uint32_t* polys) {
  if (K < 3 || K > 9 || beta < 2 || beta > 4 || polys == nullptr) return false;
  if ((K - 1) * beta > 32) return false;
  for (int b = 0; b < beta; b++)
    if (polys[b] == 0 || (polys[b] >> K) != 0) return false;
  return true;
}

int check_code(const vit_code* c) {
  if (c == nullptr) return fail(VIT_EINVAL, "null code handle");
  return VIT_OK;
}

}  // namespace

namespace vit {
int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}
void register_codes(const CodeEntry* e, int n) {
  std::lock_guard<std::mutex> lk(g_reg_mu);
  for (int i = 0; i < n; i++) registry().push_back(e[i]);
}
namespace mixreg {
struct MixReg {
  MixKey a, b;
  cudaError_t (*launch)(const MixArgs&, int, cudaStream_t);
  MixEntry entry;
};
std::vector<MixReg>& mix_registry() {
  static std::vector<MixReg> r;
  return r;
}
bool key_matches(const MixKey& k, const CodeEntry* e) {
  if (e == nullptr || k.K != e->K || k.beta != e->beta) return false;
  for (int b = 0; b < k.beta; b++)
    if (k.polys[b] != e->polys[b]) return false;
  return true;
}
}  // namespace mixreg
using namespace mixreg;

void register_mixed(const MixKey& a, const MixKey& b, cudaError_t (*launch)(const MixArgs&, int, cudaStream_t)) {
  std::lock_guard<std::mutex> lk(g_reg_mu);
  mix_registry().push_back(MixReg{a, b, launch, MixEntry{{nullptr, nullptr}, launch}});
}

struct PtReg {
  MixKey key;
  LaunchFn launch;
};
std::vector<PtReg>& pt_registry() {
  static std::vector<PtReg> r;
  return r;
}

void register_pt(const MixKey& k, LaunchFn launch) {
  std::lock_guard<std::mutex> lk(g_reg_mu);
  pt_registry().push_back(PtReg{k, launch});
}

std::vector<PtReg>& warp_registry() {
  static std::vector<PtReg> r;
  return r;
}

void register_warp(const MixKey& k, LaunchFn launch) {
  std::lock_guard<std::mutex> lk(g_reg_mu);
  warp_registry().push_back(PtReg{k, launch});
}

struct SpreadReg {
  MixKey key;
  const CodeEntry* entry;
};
std::vector<SpreadReg>& spread_registry() {
  static std::vector<SpreadReg> r;
  return r;
}
void register_spread(const MixKey& k, const CodeEntry* e) {
  std::lock_guard<std::mutex> lk(g_reg_mu);
  spread_registry().push_back(SpreadReg{k, e});
}
const CodeEntry* find_spread(const CodeEntry* e) {
  std::lock_guard<std::mutex> lk(g_reg_mu);
  for (const SpreadReg& r : spread_registry())
    if (key_matches(r.key, e)) return r.entry;
  return nullptr;
}

LaunchFn find_warp(const CodeEntry* e) {
  std::lock_guard<std::mutex> lk(g_reg_mu);
  for (const PtReg& r : warp_registry())
    if (key_matches(r.key, e)) return r.launch;
  return nullptr;
}

LaunchFn find_pt(const CodeEntry* e) {
  std::lock_guard<std::mutex> lk(g_reg_mu);
  for (const PtReg& r : pt_registry())
    if (key_matches(r.key, e)) return r.launch;
  return nullptr;
}

const MixEntry* find_mixed(const CodeEntry* x, const CodeEntry* y, bool* swapped) {
  std::lock_guard<std::mutex> lk(g_reg_mu);
  for (MixReg& r : mix_registry()) {
    if (key_matches(r.a, x) && key_matches(r.b, y)) {
      *swapped = false;
      r.entry.code[0] = x;
      r.entry.code[1] = y;
      return &r.entry;
    }
    if (key_matches(r.a, y) && key_matches(r.b, x)) {
      *swapped = true;
      r.entry.code[0] = y;
      r.entry.code[1] = x;
      return &r.entry;
    }
  }
  return nullptr;
}

struct GenReg {
  int K, beta;
  const CodeEntry* entry;
  LaunchFn warp;
};
std::vector<GenReg>& gen_registry() {
  static std::vector<GenReg> r;
  return r;
}
GenReg* gen_slot(int K, int beta) {
  for (GenReg& r : gen_registry())
    if (r.K == K && r.beta == beta) return &r;
  gen_registry().push_back(GenReg{K, beta, nullptr, nullptr});
  return &gen_registry().back();
}
void register_generic(const CodeEntry* e) {
  std::lock_guard<std::mutex> lk(g_reg_mu);
  gen_slot(e->K, e->beta)->entry = e;
}
void register_warp_generic(int K, int beta, LaunchFn launch) {
  std::lock_guard<std::mutex> lk(g_reg_mu);
  gen_slot(K, beta)->warp = launch;
}
const CodeEntry* find_generic(int K, int beta) {
  std::lock_guard<std::mutex> lk(g_reg_mu);
  for (const GenReg& r : gen_registry())
    if (r.K == K && r.beta == beta) return r.entry;
  return nullptr;
}
LaunchFn find_warp_generic(int K, int beta) {
  std::lock_guard<std::mutex> lk(g_reg_mu);
  for (const GenReg& r : gen_registry())
    if (r.K == K && r.beta == beta) return r.warp;
  return nullptr;
}

const CodeEntry* find_code(int K, int beta, const uint32_t* polys) {
  std::lock_guard<std::mutex> lk(g_reg_mu);
  for (const CodeEntry& e : registry()) {
    if (e.K != K || e.beta != beta) continue;
    bool same = true;
    for (int b = 0; b < beta; b++) same = same && (e.polys[b] == polys[b]);
    if (same) return &e;
  }
  return nullptr;
}
}  // namespace vit

extern "C" {

const char* vit_last_error(void) { return g_err.c_str(); }

int vit_code_supported(int K, int beta, const uint32_t* polys) {
  if (!code_args_ok(K, beta, polys)) return 0;
  return find_code(K, beta, polys) != nullptr || find_generic(K, beta) != nullptr;
}

int vit_create(vit_code** out, int K, int beta, const uint32_t* polys, int64_t f, int64_t v) {
  if (out == nullptr) return fail(VIT_EINVAL, "null output pointer");
  *out = nullptr;
  if (!code_args_ok(K, beta, polys))
    return fail(VIT_EINVAL, "invalid code: need K in [3,9], beta in [2,4], (K-1)*beta <= 32, 0 < g_b < 2^K");
  if (f < 0 || v < 0 || (f % 8) != 0 || f > ((int64_t)1 << 30) || v > ((int64_t)1 << 20))
    return fail(VIT_EINVAL, "invalid tiling f=%lld v=%lld (f: 0 or a positive multiple of 8)", (long long)f,
                (long long)v);
  // a kernel compiled for these generators, else the decoders that take
  // the generators at run time
  const CodeEntry* e = find_code(K, beta, polys);
  if (e == nullptr) e = find_generic(K, beta);
  if (e == nullptr) return fail(VIT_EUNSUPPORTED, "no kernel compiled for K=%d beta=%d", K, beta);
  vit_code* c = new (std::nothrow) vit_code;
  if (c == nullptr) return fail(VIT_ENOMEM, "out of host memory");
  memset(c, 0, sizeof *c);
  c->K = K;
  c->beta = beta;
  for (int b = 0; b < beta; b++) c->polys[b] = polys[b];
  c->f = f;
  c->v1 = c->v2 = v;
  c->mode = VIT_STREAM;
  c->entry = e;
  c->warp_launch = e->generic ? find_warp_generic(K, beta) : find_warp(e);
  c->spread = e->generic ? nullptr : find_spread(e);
  *out = c;
  return VIT_OK;
}

int vit_set_overlaps(vit_code* c, int64_t v1, int64_t v2) {
  if (int r = check_code(c)) return r;
  if (v1 < 0 || v2 < 0 || v1 > ((int64_t)1 << 20) || v2 > ((int64_t)1 << 20))
    return fail(VIT_EINVAL, "invalid overlaps");
  c->v1 = v1;
  c->v2 = v2;
  return VIT_OK;
}

int vit_set_puncture(vit_code* c, const uint8_t* mask, int period) {
  if (int r = check_code(c)) return r;
  if (period == 0) {
    c->period = 0;
    return VIT_OK;
  }
  if (mask == nullptr || period < 1 || period > kMaxPeriod) return fail(VIT_EINVAL, "invalid puncturing pattern");
  for (int col = 0; col < period; col++) {
    int kept = 0;
    for (int b = 0; b < c->beta; b++) kept += mask[b * period + col] ? 1 : 0;
    if (kept == 0) return fail(VIT_EINVAL, "puncturing column %d removes every symbol", col);
  }
  for (int i = 0; i < c->beta * period; i++) c->mask[i] = mask[i] ? 1 : 0;
  c->period = period;
  return VIT_OK;
}

int vit_set_termination(vit_code* c, int mode) {
  if (int r = check_code(c)) return r;
  if (mode != VIT_STREAM && mode != VIT_TERMINATED && mode != VIT_FREE_START) return fail(VIT_EINVAL, "invalid mode");
  c->mode = mode;
  return VIT_OK;
}

int vit_set_parallel_traceback(vit_code* c, int64_t f0, int rule, uint64_t seed) {
  if (int r = check_code(c)) return r;
  if (f0 < 0 || (f0 % 8) != 0 || f0 > ((int64_t)1 << 30))
    return fail(VIT_EINVAL, "invalid subframe length f0=%lld (0 or a positive multiple of 8)", (long long)f0);
  if (rule != VIT_PT_STORED && rule != VIT_PT_RANDOM) return fail(VIT_EINVAL, "invalid traceback start rule");
  if (f0 == 0) {
    c->pt_f0 = 0;
    c->pt_launch = nullptr;
    return VIT_OK;
  }
  const LaunchFn l = c->entry->generic ? nullptr : find_pt(c->entry);
  if (l == nullptr)
    return fail(VIT_EUNSUPPORTED, "no parallel-traceback kernel compiled for K=%d beta=%d with these generators",
                c->K, c->beta);
  c->pt_f0 = f0;
  c->pt_rule = rule;
  c->pt_seed = seed;
  c->pt_launch = l;
  return VIT_OK;
}

int vit_set_decoder(vit_code* c, int which) {
  if (int r = check_code(c)) return r;
  if (which != VIT_DECODER_AUTO && which != VIT_DECODER_TILES && which != VIT_DECODER_SHARED &&
      which != VIT_DECODER_SPREAD)
    return fail(VIT_EINVAL, "invalid decoder choice %d", which);
  c->decoder = which;
  return VIT_OK;
}

void vit_destroy(vit_code* c) { delete c; }

int64_t vit_llr_count(const vit_code* c, int64_t n) {
  if (c == nullptr || n < 0) return -1;
  return kept_in(c, n);
}

int64_t vit_output_bits(const vit_code* c, int64_t n) {
  if (c == nullptr || n < 0) return -1;
  if (c->mode == VIT_TERMINATED) return n > c->K - 1 ? n - (c->K - 1) : 0;
  return n;
}

// Subframes per tile of the parallel traceback (0 when it is off).
static int64_t pt_subframes(const vit_code* c, int64_t n) {
  if (c->pt_f0 <= 0) return 0;
  const int64_t fb = tile_len(n, c->f);
  return (fb + c->pt_f0 - 1) / c->pt_f0;
}

static size_t slab_task_words(const vit_code* c, const CodeEntry* e, int64_t n) {
  const int64_t L = max_window(c, n);
  const int64_t U = e->unroll;
  const int64_t Lr = (L + U - 1) / U * U;
  return (size_t)Lr * e->slab_lanes * e->words;
}

static int64_t task_count(const CodeEntry* e, int64_t tiles) {
  return (tiles + e->tiles_per_task - 1) / e->tiles_per_task;
}

// The tile decoder of a single-frame decode: the code's own, or (when the
// frame's warp tasks would fill at most a quarter of the decoder's resident
// warps, or when asked) the variant with several lanes per tile pair.  Timed
// on a GB300: a 2^24-bit K=7 stream at f=1024 (256 tasks, 14% of the
// resident warps) decodes 1.4x faster spread; a 2^26-bit stream at f=2048
// (512 tasks, 28%) 5-10% slower, so the cut is at a quarter.
static const CodeEntry* tile_entry(const vit_code* c, int64_t n) {
  if (c->spread == nullptr || c->pt_f0 > 0 || c->decoder == VIT_DECODER_TILES) return c->entry;
  if (c->decoder == VIT_DECODER_SPREAD) return c->spread;
  const int64_t r = c->entry->resident ? c->entry->resident(kWarpsPerCta) : 0;
  return (r > 0 && 4 * task_count(c->entry, tile_count(n, c->f)) <= r) ? c->spread : c->entry;
}

// CTA size of a single-frame tile-decoder launch of `tasks` warp tasks that
// fits one wave.  The block scheduler deals CTAs to the SMs in turn, so when
// kWarpsPerCta-warp CTAs do not divide evenly some SMs hold a CTA more than
// others, and the launch lasts as long as its busiest SM.  One CTA of
// ceil(tasks / SMs) warps per SM evens the load; larger CTAs cost ~2% by
// themselves (the 7 x 2^24-bit K=7 batch, 12 warps on every SM either way:
// 0.856 ms with 12-warp CTAs, 0.836 ms with 4), so they are taken when the
// busiest SM loses at least 5% of its warps.  A 2^26-bit K=9 stream (2048
// tasks on 152 SMs): 14-warp CTAs instead of 16 warps on some SMs, 2.77
// against 3.03 ms.
static int balanced_warps(const CodeEntry* e, int64_t tasks) {
  int dev = 0, sms = 0;
  if (e->resident == nullptr || tasks <= 0 || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    return kWarpsPerCta;
  }
  const int64_t w = kWarpsPerCta;
  const int64_t busiest = ((((tasks + w - 1) / w) + sms - 1) / sms) * w;
  const int64_t wb = (tasks + sms - 1) / sms;
  if (wb <= w || wb > kMaxCtaWarps || 100 * busiest < 105 * wb) return kWarpsPerCta;
  // one such CTA must fit an SM (then the launch is one wave)
  if (e->resident((int)wb) < (int64_t)sms * wb) return kWarpsPerCta;
  return (int)wb;
}

// Slab slots of a single-frame decode with the tile decoder: 0 (one per
// warp task) when every task's warp can be resident at once, else the
// number of warps resident on the current device, which then stride over the
// tasks and reuse their slots -- the slab stops growing with n after one
// wave.  The parallel-traceback decoder keeps one slot per task.
static int64_t slab_slots(const vit_code* c, const CodeEntry* e, int64_t tasks) {
  if (c->pt_f0 > 0 || e->resident == nullptr) return 0;
  const int64_t r = e->resident(kWarpsPerCta);
  return (r > 0 && tasks > r) ? r : 0;
}

size_t vit_decode_workspace(const vit_code* c, int64_t n) {
  if (c == nullptr || n <= 0) return 0;
  const int64_t tiles = tile_count(n, c->f);
  const CodeEntry* e = tile_entry(c, n);
  const int64_t tasks = task_count(e, tiles);
  const int64_t slots = slab_slots(c, e, tasks);
  size_t bytes = align_up((size_t)(slots ? slots : tasks) * slab_task_words(c, e, n) * 4);
  if (c->period) bytes += align_up((size_t)n * c->beta);
  bytes += align_up((size_t)(tiles * pt_subframes(c, n)));
  return bytes;
}

static int decode_impl(const vit_code* c, const int8_t* llr, int64_t n, uint8_t* bits_out, void* ws,
                       size_t ws_bytes, cudaStream_t s) {
  const int64_t tiles = tile_count(n, c->f);
  const CodeEntry* te = tile_entry(c, n);
  const int64_t tasks = task_count(te, tiles);
  const size_t tw = slab_task_words(c, te, n);
  const int64_t slots = slab_slots(c, te, tasks);
  uint8_t* p = (uint8_t*)ws;
  uint32_t* slab = (uint32_t*)p;
  p += align_up((size_t)(slots ? slots : tasks) * tw * 4);
  const int8_t* dec_llr = llr;
  if (c->period) {
    int8_t* dep = (int8_t*)p;
    PunctArgs pa;
    memset(&pa, 0, sizeof pa);
    pa.beta = c->beta;
    pa.period = c->period;
    int64_t cum = 0;
    for (int col = 0; col < c->period; col++) {
      pa.col_prefix[col] = (int32_t)cum;
      int r = 0;
      for (int b = 0; b < c->beta; b++) pa.rank[b * kMaxPeriod + col] = c->mask[b * c->period + col] ? r++ : -1;
      cum += r;
    }
    pa.per_period = cum;
    const unsigned grid = (unsigned)((n + 255) / 256);
    depuncture_kernel<<<grid, 256, 0, s>>>(llr, n, dep, pa);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "depuncture launch");
    dec_llr = dep;
    p += align_up((size_t)n * c->beta);
  }
  KArgs a;
  memset(&a, 0, sizeof a);
  a.f0.llr = dec_llr;
  a.f0.out = bits_out;
  a.f0.n = n;
  a.f0.n_out = vit_output_bits(c, n);
  a.f0.mode = c->mode;
  a.frames = nullptr;
  a.tile0 = nullptr;
  a.nframes = 1;
  a.ntiles = tiles;
  a.tl = Tiling{c->f, c->v1, c->v2};
  a.M = (uint32_t)(2 * (c->K - 1) * 127 * c->beta + 1);
  a.ntasks = tasks;
  a.slab = slab;
  a.task_words = (int64_t)tw;
  a.slots = slots;
  a.task_base = 0;
  for (int b = 0; b < c->beta; b++) a.polys[b] = c->polys[b];
  if (c->pt_f0 > 0) {
    a.pt_f0 = c->pt_f0;
    a.pt_rule = c->pt_rule;
    a.pt_seed = c->pt_seed;
    a.pt_nsub = pt_subframes(c, n);
    a.pt_states = p;
  }
  LaunchFn launch = c->pt_f0 > 0 ? c->pt_launch : te->launch;
  // few short tiles: one warp per tile decodes them with lower latency
  const bool fits = c->warp_launch != nullptr && max_window(c, n) <= kWarpSmemStages;
  if (c->pt_f0 == 0 && c->decoder == VIT_DECODER_AUTO && fits && tiles <= kWarpTileLimit) launch = c->warp_launch;
  if (c->decoder == VIT_DECODER_SPREAD && c->spread == nullptr)
    return fail(VIT_EUNSUPPORTED, "no tile decoder with several lanes per tile pair for this code");
  if (c->decoder == VIT_DECODER_SHARED) {
    if (!fits || c->pt_f0 > 0)
      return fail(VIT_EUNSUPPORTED, "the shared-memory decoder needs windows of at most %d stages, no parallel "
                  "traceback and a code with such a decoder", (int)kWarpSmemStages);
    launch = c->warp_launch;
  }
  const int warps = (launch == te->launch && slots == 0) ? balanced_warps(te, tasks) : kWarpsPerCta;
  cudaError_t e = launch(a, warps, s);
  if (e != cudaSuccess) return cuda_fail(e, "decode launch");
  return VIT_OK;
}

}  // extern "C"

namespace vit {
// Decode into a caller-supplied scratch area; shared by the public entry
// points that bring their own device memory.
int decode_into(const vit_code* c, const int8_t* llr, int64_t n, uint8_t* bits_out, void* ws, size_t ws_bytes,
                cudaStream_t s) {
  return decode_impl(c, llr, n, bits_out, ws, ws_bytes, s);
}
}  // namespace vit

extern "C" {

int vit_decode_ws(const vit_code* c, const int8_t* llr, int64_t n, uint8_t* bits_out, void* ws, size_t ws_bytes,
                  vit_stream_t stream) {
  if (int r = check_code(c)) return r;
  if (n <= 0) return fail(VIT_EINVAL, "n must be >= 1");
  if (llr == nullptr || bits_out == nullptr || ws == nullptr) return fail(VIT_EINVAL, "null device pointer");
  if (((uintptr_t)ws % kAlign) != 0) return fail(VIT_EINVAL, "workspace must be 256-byte aligned");
  if (c->mode == VIT_TERMINATED && n <= c->K - 1) return fail(VIT_EINVAL, "terminated frame shorter than its tail");
  const size_t need = vit_decode_workspace(c, n);
  if (ws_bytes < need)
    return fail(VIT_EINVAL, "workspace too small: %zu bytes given, %zu needed", ws_bytes, need);
  return decode_impl(c, llr, n, bits_out, ws, ws_bytes, (cudaStream_t)stream);
}

int vit_decode(const vit_code* c, const int8_t* llr, int64_t n, uint8_t* bits_out, vit_stream_t stream) {
  if (int r = check_code(c)) return r;
  if (n <= 0) return fail(VIT_EINVAL, "n must be >= 1");
  if (llr == nullptr || bits_out == nullptr) return fail(VIT_EINVAL, "null device pointer");
  if (c->mode == VIT_TERMINATED && n <= c->K - 1) return fail(VIT_EINVAL, "terminated frame shorter than its tail");
  const size_t need = vit_decode_workspace(c, n);
  cudaStream_t s = (cudaStream_t)stream;
  void* ws = nullptr;
  cudaError_t e = cudaMallocAsync(&ws, need, s);
  if (e != cudaSuccess) return fail(VIT_ENOMEM, "workspace allocation of %zu bytes failed: %s", need,
                                    cudaGetErrorString(e));
  int r = decode_impl(c, llr, n, bits_out, ws, need, s);
  e = cudaFreeAsync(ws, s);
  if (r == VIT_OK && e != cudaSuccess) r = cuda_fail(e, "workspace release");
  return r;
}

int vit_encode(const vit_code* c, const uint8_t* bits, int64_t n, uint8_t* coded, vit_stream_t stream) {
  if (int r = check_code(c)) return r;
  if (n <= 0) return fail(VIT_EINVAL, "n must be >= 1");
  if (bits == nullptr || coded == nullptr) return fail(VIT_EINVAL, "null device pointer");
  const uint4 g = make_uint4(c->polys[0], c->polys[1], c->polys[2], c->polys[3]);
  const unsigned grid = (unsigned)((n + 255) / 256);
  encode_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(bits, n, c->K, c->beta, g, coded);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "encode launch");
  return VIT_OK;
}

int vit_hard_llr(const uint8_t* bits, int64_t count, int8_t* llr, vit_stream_t stream) {
  if (count <= 0) return fail(VIT_EINVAL, "count must be >= 1");
  if (bits == nullptr || llr == nullptr) return fail(VIT_EINVAL, "null device pointer");
  const int64_t groups = (count + 7) / 8;
  const unsigned grid = (unsigned)((groups + 255) / 256);
  if ((groups + 255) / 256 > 0x7fffffffLL) return fail(VIT_EINVAL, "count too large");
  hard_llr_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(bits, count, llr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "hard-decision expansion launch");
  return VIT_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches
// A plan groups frames that share a compiled kernel and a tiling; each group
// is one launch over a device frame table.  Punctured frames are
// de-punctured into plan-owned buffers first.
struct vit_batch {
  struct Group {
    const CodeEntry* entry;
    LaunchFn launch;  // the code's tile decoder, or its parallel-traceback variant
    int64_t pt_f0 = 0, pt_nsub = 0;
    int pt_rule = 0;
    uint64_t pt_seed = 0;
    uint8_t* d_pt = nullptr;
    Tiling tl;
    uint32_t M;
    uint32_t polys[4] = {0, 0, 0, 0};
    int nframes;
    int64_t ntiles, ntasks, task_words;
    Frame* d_frames = nullptr;
    int64_t* d_tile0 = nullptr;
    uint32_t* d_slab = nullptr;
    std::vector<int64_t> task_len;  // host estimate of each task's window length
    std::vector<Frame> hframes;     // host copy of the frame table
    std::vector<int64_t> htile0;
    struct IO {                     // VIT_BATCH_HOST: host buffers and their device copies
      const int8_t* h_llr;
      uint8_t* h_out;
      int8_t* d_llr;
      uint8_t* d_out;
      int64_t llr_bytes, out_bytes;
      bool punctured;
    };
    std::vector<IO> io;
  };
  struct Dep {
    const int8_t* src;
    int8_t* dst;
    int64_t n;
    PunctArgs pa;
  };
  // host-staged runs (VIT_BATCH_HOST): one contiguous copy of host memory
  struct Copy {
    const void* src;
    void* dst;
    size_t bytes;
  };
  // a chunk: warp tasks [lo, hi) of one group, the LLR bytes they need that
  // earlier chunks have not copied, and the output bytes they complete
  struct Chunk {
    int group;
    int64_t lo, hi;
    std::vector<Copy> in, out;
  };
  std::vector<Group> groups;
  std::vector<Dep> deps;
  std::vector<Copy> host_in;  // whole punctured frames, copied before the chunks
  std::vector<Chunk> chunks;
  cudaStream_t copy_in = nullptr, copy_out = nullptr;
  std::vector<cudaStream_t> comp;        // compute streams, chunks in turn
  std::vector<cudaEvent_t> ev_in, ev_dec;  // per chunk
  cudaEvent_t ev_end = nullptr;
  // one stream and completion event per group after the first: the groups
  // run concurrently (fork/join with events, also inside a captured graph)
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> done;
  cudaEvent_t fork = nullptr;
  std::vector<void*> allocs;
  int flags = 0;
  int warps = kWarpsPerCta;
  const MixEntry* mix = nullptr;  // persistent two-code kernel, when available
  int mix_group[2] = {0, 1};
  MixTask* d_queue = nullptr;
  int64_t nqueue = 0;
  unsigned long long* d_counter = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {
PunctArgs make_punct(const vit_code* c) {
  PunctArgs pa;
  memset(&pa, 0, sizeof pa);
  pa.beta = c->beta;
  pa.period = c->period;
  int64_t cum = 0;
  for (int col = 0; col < c->period; col++) {
    pa.col_prefix[col] = (int32_t)cum;
    int r = 0;
    for (int b = 0; b < c->beta; b++) pa.rank[b * kMaxPeriod + col] = c->mask[b * c->period + col] ? r++ : -1;
    cum += r;
  }
  pa.per_period = cum;
  return pa;
}

void batch_free(vit_batch* b) {
  if (b == nullptr) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaStream_t x : b->side) cudaStreamDestroy(x);
  for (cudaEvent_t x : b->done) cudaEventDestroy(x);
  for (cudaStream_t x : b->comp) cudaStreamDestroy(x);
  for (cudaEvent_t x : b->ev_in) cudaEventDestroy(x);
  for (cudaEvent_t x : b->ev_dec) cudaEventDestroy(x);
  if (b->copy_in) cudaStreamDestroy(b->copy_in);
  if (b->copy_out) cudaStreamDestroy(b->copy_out);
  if (b->ev_end) cudaEventDestroy(b->ev_end);
  if (b->fork) cudaEventDestroy(b->fork);
  for (void* p : b->allocs) cudaFree(p);
  delete b;
}

KArgs group_args(const vit_batch::Group& g) {
  KArgs a;
  memset(&a, 0, sizeof a);
  a.frames = g.d_frames;
  a.tile0 = g.d_tile0;
  a.nframes = g.nframes;
  a.ntiles = g.ntiles;
  a.tl = g.tl;
  a.M = g.M;
  a.ntasks = g.ntasks;
  a.slab = g.d_slab;
  a.task_words = g.task_words;
  a.pt_f0 = g.pt_f0;
  a.pt_rule = g.pt_rule;
  a.pt_seed = g.pt_seed;
  a.pt_nsub = g.pt_nsub;
  a.pt_states = g.d_pt;
  for (int b = 0; b < 4; b++) a.polys[b] = g.polys[b];
  return a;
}

// Host-staged run: input copies on copy_in, chunk launches on the compute
// streams in turn, output copies on copy_out, ordered per chunk by events;
// forked from and joined back into the caller's stream.
int batch_enqueue_host(vit_batch* b, cudaStream_t s) {
  cudaError_t e = cudaEventRecord(b->fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->copy_in, b->fork, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(b->copy_out, b->fork, 0);
  for (size_t j = 0; j < b->comp.size() && e == cudaSuccess; j++) e = cudaStreamWaitEvent(b->comp[j], b->fork, 0);
  for (const auto& c : b->host_in)
    if (e == cudaSuccess) e = cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyHostToDevice, b->copy_in);
  if (e != cudaSuccess) return cuda_fail(e, "host batch input");
  for (const auto& d : b->deps) {
    const unsigned grid = (unsigned)((d.n + 255) / 256);
    depuncture_kernel<<<grid, 256, 0, b->copy_in>>>(d.src, d.n, d.dst, d.pa);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "depuncture launch");
  }
  for (size_t k = 0; k < b->chunks.size() && e == cudaSuccess; k++) {
    const auto& ch = b->chunks[k];
    for (const auto& c : ch.in)
      if (e == cudaSuccess) e = cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyHostToDevice, b->copy_in);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_in[k], b->copy_in);
    cudaStream_t cs = b->comp[k % b->comp.size()];
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, b->ev_in[k], 0);
    if (e == cudaSuccess) {
      KArgs a = group_args(b->groups[(size_t)ch.group]);
      a.task_base = ch.lo;
      a.ntasks = ch.hi;
      e = b->groups[(size_t)ch.group].launch(a, b->warps, cs);
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_dec[k], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->copy_out, b->ev_dec[k], 0);
    for (const auto& c : ch.out)
      if (e == cudaSuccess) e = cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost, b->copy_out);
  }
  // join every plan stream back into the caller's stream (copy_out's end
  // already follows all of them; the direct joins keep graph capture happy)
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_end, b->copy_out);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->ev_end, 0);
  const size_t nk = b->chunks.size();
  if (e == cudaSuccess && nk > 0) e = cudaStreamWaitEvent(s, b->ev_in[nk - 1], 0);
  for (size_t j = 0; j < b->comp.size() && j < nk && e == cudaSuccess; j++) {
    const size_t last = j + (nk - 1 - j) / b->comp.size() * b->comp.size();  // last chunk on comp[j]
    e = cudaStreamWaitEvent(s, b->ev_dec[last], 0);
  }
  if (e != cudaSuccess) return cuda_fail(e, "host batch");
  return VIT_OK;
}

int batch_enqueue(vit_batch* b, cudaStream_t s) {
  if (b->flags & VIT_BATCH_HOST) return batch_enqueue_host(b, s);
  for (const auto& d : b->deps) {
    const unsigned grid = (unsigned)((d.n + 255) / 256);
    depuncture_kernel<<<grid, 256, 0, s>>>(d.src, d.n, d.dst, d.pa);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "depuncture launch");
  }
  if (b->mix) {
    cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "queue reset");
    MixArgs m;
    memset(&m, 0, sizeof m);
    m.g[0] = group_args(b->groups[b->mix_group[0]]);
    m.g[1] = group_args(b->groups[b->mix_group[1]]);
    m.queue = b->d_queue;
    m.nqueue = b->nqueue;
    m.counter = b->d_counter;
    e = b->mix->launch(m, b->warps, s);
    if (e != cudaSuccess) return cuda_fail(e, "persistent decode launch");
    return VIT_OK;
  }
  // group 0 (the costliest) on the caller's stream, the others forked onto
  // the plan's side streams and joined back before the batch completes
  cudaError_t e = cudaSuccess;
  if (b->groups.size() > 1) e = cudaEventRecord(b->fork, s);
  for (size_t k = 1; k < b->groups.size() && e == cudaSuccess; k++) {
    e = cudaStreamWaitEvent(b->side[k - 1], b->fork, 0);
    if (e == cudaSuccess) e = b->groups[k].launch(group_args(b->groups[k]), b->warps, b->side[k - 1]);
    if (e == cudaSuccess) e = cudaEventRecord(b->done[k - 1], b->side[k - 1]);
  }
  if (e == cudaSuccess) e = b->groups[0].launch(group_args(b->groups[0]), b->warps, s);
  for (size_t k = 1; k < b->groups.size() && e == cudaSuccess; k++) e = cudaStreamWaitEvent(s, b->done[k - 1], 0);
  if (e != cudaSuccess) return cuda_fail(e, "batched decode launch");
  return VIT_OK;
}
// Cuts every group's warp tasks into up to `nchunks` chunks (round-robin over
// the groups) and lists each chunk's copies; creates the plan's streams and
// events for host-staged runs.
int plan_host_chunks(vit_batch* b, int nchunks) {
  for (auto& g : b->groups)
    for (const auto& io : g.io)
      if (io.punctured) b->host_in.push_back(vit_batch::Copy{io.h_llr, io.d_llr, (size_t)io.llr_bytes});
  std::vector<std::vector<int64_t>> mark(b->groups.size());  // LLR bytes copied so far, per frame
  for (size_t gi = 0; gi < b->groups.size(); gi++) mark[gi].assign(b->groups[gi].io.size(), 0);
  for (int c = 0; c < nchunks; c++) {
    for (size_t gi = 0; gi < b->groups.size(); gi++) {
      const auto& g = b->groups[gi];
      const int64_t ng = g.ntasks < nchunks ? g.ntasks : nchunks;
      if (c >= ng) continue;
      vit_batch::Chunk ch;
      ch.group = (int)gi;
      ch.lo = g.ntasks * c / ng;
      ch.hi = g.ntasks * (c + 1) / ng;
      const int64_t tpt = g.entry->tiles_per_task;
      const int64_t t_lo = ch.lo * tpt, t_hi = ch.hi * tpt < g.ntiles ? ch.hi * tpt : g.ntiles;
      for (size_t j = 0; j < g.hframes.size(); j++) {
        const Frame& fr = g.hframes[j];
        const auto& io = g.io[j];
        const int64_t ft0 = g.htile0[j], nt = tile_count(fr.n, g.tl.f);
        const int64_t a = (t_lo > ft0 ? t_lo : ft0) - ft0, z = (t_hi < ft0 + nt ? t_hi : ft0 + nt) - ft0;
        if (a >= z) continue;
        const Half ha = make_half(fr, a, g.tl), hz = make_half(fr, z - 1, g.tl);
        if (!io.punctured) {
          const int beta = g.entry->beta;
          int64_t lo = ha.t0 * beta;
          const int64_t hi = hz.t1 * beta;
          lo = lo > mark[gi][j] ? lo : mark[gi][j];
          if (hi > lo) ch.in.push_back(vit_batch::Copy{io.h_llr + lo, io.d_llr + lo, (size_t)(hi - lo)});
          if (hi > mark[gi][j]) mark[gi][j] = hi;
        }
        if (hz.e1 > ha.e0) {
          const int64_t o0 = ha.e0 / 8, o1 = (hz.e1 + 7) / 8;
          ch.out.push_back(vit_batch::Copy{io.d_out + o0, io.h_out + o0, (size_t)(o1 - o0)});
        }
      }
      b->chunks.push_back(std::move(ch));
    }
  }
  const size_t nk = b->chunks.size();
  const size_t ncomp = nk < 4 ? nk : 4;
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_end, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->copy_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->copy_out, cudaStreamNonBlocking);
  for (size_t j = 0; j < ncomp && e == cudaSuccess; j++) {
    cudaStream_t x = nullptr;
    e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->comp.push_back(x);
  }
  for (size_t k = 0; k < nk && e == cudaSuccess; k++) {
    cudaEvent_t x = nullptr, y = nullptr;
    e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
    if (e == cudaSuccess) b->ev_in.push_back(x);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&y, cudaEventDisableTiming);
    if (e == cudaSuccess) b->ev_dec.push_back(y);
  }
  if (e != cudaSuccess) return cuda_fail(e, "host batch streams");
  return VIT_OK;
}
}  // namespace

extern "C" {

int vit_batch_plan(vit_batch** out, const vit_frame* frames, int nframes, int flags) {
  if (out == nullptr) return fail(VIT_EINVAL, "null output pointer");
  *out = nullptr;
  if (frames == nullptr || nframes <= 0) return fail(VIT_EINVAL, "empty batch");
  for (int i = 0; i < nframes; i++) {
    const vit_frame& f = frames[i];
    if (f.code == nullptr || f.llr == nullptr || f.bits_out == nullptr || f.n <= 0)
      return fail(VIT_EINVAL, "frame %d: null pointer or empty frame", i);
    if (f.mode != VIT_STREAM && f.mode != VIT_TERMINATED && f.mode != VIT_FREE_START)
      return fail(VIT_EINVAL, "frame %d: invalid mode", i);
    if (f.mode == VIT_TERMINATED && f.n <= f.code->K - 1)
      return fail(VIT_EINVAL, "frame %d: terminated frame shorter than its tail", i);
  }
  if (flags & ~(VIT_BATCH_GRAPH | VIT_BATCH_PERSISTENT | VIT_BATCH_HOST | 0xff00 | 0xff0000))
    return fail(VIT_EINVAL, "unknown batch flag");
  const int warps = (flags >> 8) & 0xff;
  if (warps != 0 && (warps < 1 || warps > 8)) return fail(VIT_EINVAL, "warps per CTA must be in [1, 8]");
  const bool host = (flags & VIT_BATCH_HOST) != 0;
  int nchunks = (flags >> 16) & 0xff;
  if (nchunks != 0 && !host) return fail(VIT_EINVAL, "a chunk count needs VIT_BATCH_HOST");
  if (nchunks > 64) return fail(VIT_EINVAL, "chunks must be in [1, 64]");
  if (nchunks == 0) nchunks = 8;
  if (host) {
    // page-locked host memory only: pageable buffers would make the copies
    // synchronous, and device buffers belong to the ordinary batch
    auto pinned = [](const void* p) {
      cudaPointerAttributes at;
      if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
      }
      return at.type == cudaMemoryTypeHost;
    };
    for (int i = 0; i < nframes; i++)
      if (!pinned(frames[i].llr) || !pinned(frames[i].bits_out))
        return fail(VIT_EINVAL, "frame %d: VIT_BATCH_HOST wants page-locked host buffers", i);
  }
  vit_batch* b = new (std::nothrow) vit_batch;
  if (b == nullptr) return fail(VIT_ENOMEM, "out of host memory");
  b->flags = flags;
  b->warps = warps ? warps : kWarpsPerCta;
  // group frames by (kernel, tiling); inside a group, longest frames first so
  // that the tiles of one warp task have similar windows
  std::vector<std::vector<int>> members;
  std::vector<const vit_code*> leaders;
  for (int i = 0; i < nframes; i++) {
    const vit_code* c = frames[i].code;
    int gi = -1;
    for (size_t k = 0; k < leaders.size(); k++) {
      const vit_code* l = leaders[k];
      if (l->entry == c->entry && l->f == c->f && l->v1 == c->v1 && l->v2 == c->v2 && l->pt_f0 == c->pt_f0 &&
          (c->pt_f0 == 0 || (l->pt_rule == c->pt_rule && l->pt_seed == c->pt_seed)) &&
          (!c->entry->generic || memcmp(l->polys, c->polys, sizeof c->polys) == 0))
        gi = (int)k;
    }
    if (gi < 0) {
      leaders.push_back(c);
      members.emplace_back();
      gi = (int)leaders.size() - 1;
    }
    members[gi].push_back(i);
  }
  for (auto& m : members)
    std::stable_sort(m.begin(), m.end(), [&](int x, int y) { return frames[x].n > frames[y].n; });
  int rc = VIT_OK;
  auto dalloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes ? bytes : 1) != cudaSuccess) return nullptr;
    b->allocs.push_back(p);
    return p;
  };
  for (size_t k = 0; k < leaders.size() && rc == VIT_OK; k++) {
    const vit_code* c = leaders[k];
    vit_batch::Group g;
    g.entry = c->entry;
    g.launch = c->pt_f0 > 0 ? c->pt_launch : c->entry->launch;  // replaced below for short frames
    for (int q = 0; q < c->beta; q++) g.polys[q] = c->polys[q];
    g.pt_f0 = c->pt_f0;
    g.pt_rule = c->pt_rule;
    g.pt_seed = c->pt_seed;
    g.tl = Tiling{c->f, c->v1, c->v2};
    g.M = (uint32_t)(2 * (c->K - 1) * 127 * c->beta + 1);
    g.nframes = (int)members[k].size();
    std::vector<Frame> hf(g.nframes);
    std::vector<int64_t> ht0(g.nframes);
    std::vector<int64_t> tile_len_host;  // window length of every tile, in order
    int64_t tiles = 0, maxw = 1;
    for (int j = 0; j < g.nframes; j++) {
      const vit_frame& f = frames[members[k][j]];
      const vit_code* fc = f.code;
      const int8_t* llr = f.llr;
      uint8_t* out = f.bits_out;
      const int64_t n_out = (f.mode == VIT_TERMINATED) ? f.n - (fc->K - 1) : f.n;
      if (host) {
        vit_batch::Group::IO io{f.llr, f.bits_out, nullptr, nullptr, kept_in(fc, f.n), (n_out + 7) / 8,
                                fc->period != 0};
        io.d_llr = (int8_t*)dalloc((size_t)io.llr_bytes);
        io.d_out = (uint8_t*)dalloc((size_t)io.out_bytes);
        if (io.d_llr == nullptr || io.d_out == nullptr) {
          rc = fail(VIT_ENOMEM, "device allocation failed");
          break;
        }
        llr = io.d_llr;
        out = io.d_out;
        g.io.push_back(io);
      }
      if (fc->period) {
        int8_t* dst = (int8_t*)dalloc((size_t)f.n * fc->beta);
        if (dst == nullptr) {
          rc = fail(VIT_ENOMEM, "device allocation failed");
          break;
        }
        b->deps.push_back(vit_batch::Dep{llr, dst, f.n, make_punct(fc)});
        llr = dst;
      }
      hf[j].llr = llr;
      hf[j].out = out;
      hf[j].n = f.n;
      hf[j].n_out = n_out;
      hf[j].mode = f.mode;
      ht0[j] = tiles;
      const int64_t nt = tile_count(f.n, c->f);
      for (int64_t t = 0; t < nt; t++) {
        const Half h = make_half(hf[j], t, g.tl);
        tile_len_host.push_back(h.t1 - h.t0);
      }
      tiles += nt;
      const int64_t w = max_window(c, f.n);
      if (w > maxw) maxw = w;
      if (g.pt_f0 > 0) {
        const int64_t ns = (tile_len(f.n, c->f) + g.pt_f0 - 1) / g.pt_f0;
        if (ns > g.pt_nsub) g.pt_nsub = ns;
      }
    }
    if (rc != VIT_OK) break;
    g.ntiles = tiles;
    // frames shorter than a warp task on average: most groups of a warp are
    // loaded with masking, and the byte-load kernel runs them faster
    if (g.pt_f0 == 0 && tiles < (int64_t)g.nframes * c->entry->tiles_per_task) g.launch = c->entry->launch_bytes;
    const int64_t tpt = c->entry->tiles_per_task;
    g.ntasks = (tiles + tpt - 1) / tpt;
    g.task_len.assign((size_t)g.ntasks, 0);
    for (int64_t t = 0; t < tiles; t++) {
      int64_t& L = g.task_len[(size_t)(t / tpt)];
      L = tile_len_host[(size_t)t] > L ? tile_len_host[(size_t)t] : L;
    }
    const int64_t U = c->entry->unroll;
    g.task_words = ((maxw + U - 1) / U * U) * c->entry->slab_lanes * c->entry->words;
    g.d_frames = (Frame*)dalloc(sizeof(Frame) * g.nframes);
    g.d_tile0 = (int64_t*)dalloc(sizeof(int64_t) * g.nframes);
    g.d_slab = (uint32_t*)dalloc((size_t)g.ntasks * g.task_words * 4);
    if (g.pt_f0 > 0) g.d_pt = (uint8_t*)dalloc((size_t)(g.ntiles * g.pt_nsub));
    if (!g.d_frames || !g.d_tile0 || !g.d_slab || (g.pt_f0 > 0 && !g.d_pt)) {
      rc = fail(VIT_ENOMEM, "device allocation failed");
      break;
    }
    cudaError_t e = cudaMemcpy(g.d_frames, hf.data(), sizeof(Frame) * g.nframes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g.d_tile0, ht0.data(), sizeof(int64_t) * g.nframes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "plan upload");
      break;
    }
    g.hframes = hf;
    g.htile0 = ht0;
    b->groups.push_back(std::move(g));
  }
  // costliest group first (it is launched on the caller's stream, first)
  if (rc == VIT_OK) {
    auto cost = [](const vit_batch::Group& g) {
      int64_t c = 0;
      for (int64_t L : g.task_len) c += L;
      return (double)c * (double)(1 << (g.entry->K - 1));
    };
    std::stable_sort(b->groups.begin(), b->groups.end(),
                     [&](const vit_batch::Group& x, const vit_batch::Group& y) { return cost(x) > cost(y); });
  }
  // with VIT_BATCH_PERSISTENT, two code groups with a compiled persistent
  // kernel become one launch over a queue of all their tasks, longest first
  if (rc == VIT_OK && host) rc = plan_host_chunks(b, nchunks);
  if (rc == VIT_OK && !host && (flags & VIT_BATCH_PERSISTENT) && b->groups.size() == 2 && b->groups[0].pt_f0 == 0 &&
      b->groups[1].pt_f0 == 0) {
    bool swapped = false;
    const MixEntry* mx = find_mixed(b->groups[0].entry, b->groups[1].entry, &swapped);
    if (mx != nullptr) {
      b->mix = mx;
      b->mix_group[0] = swapped ? 1 : 0;
      b->mix_group[1] = swapped ? 0 : 1;
      std::vector<MixTask> q;
      std::vector<int64_t> cost;
      for (int slot = 0; slot < 2; slot++) {
        const auto& g = b->groups[b->mix_group[slot]];
        for (int64_t t = 0; t < g.ntasks; t++) {
          q.push_back(MixTask{slot, 0, t});
          cost.push_back(g.task_len[(size_t)t]);
        }
      }
      std::vector<size_t> ord(q.size());
      for (size_t i = 0; i < ord.size(); i++) ord[i] = i;
      std::stable_sort(ord.begin(), ord.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
      std::vector<MixTask> qs(q.size());
      for (size_t i = 0; i < ord.size(); i++) qs[i] = q[ord[i]];
      b->nqueue = (int64_t)qs.size();
      b->d_queue = (MixTask*)dalloc(sizeof(MixTask) * qs.size());
      b->d_counter = (unsigned long long*)dalloc(sizeof(unsigned long long));
      if (!b->d_queue || !b->d_counter) {
        rc = fail(VIT_ENOMEM, "device allocation failed");
      } else {
        cudaError_t e = cudaMemcpy(b->d_queue, qs.data(), sizeof(MixTask) * qs.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = cuda_fail(e, "queue upload");
      }
    }
  }
  if (rc == VIT_OK && !host && b->mix == nullptr && b->groups.size() > 1) {
    cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (size_t k = 1; k < b->groups.size() && e == cudaSuccess; k++) {
      cudaStream_t x = nullptr;
      cudaEvent_t ev = nullptr;
      e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
      if (e == cudaSuccess) b->side.push_back(x);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) b->done.push_back(ev);
    }
    if (e != cudaSuccess) rc = cuda_fail(e, "group streams");
  }
  if (rc != VIT_OK) {
    batch_free(b);
    return rc;
  }
  *out = b;
  return VIT_OK;
}

int vit_batch_run(vit_batch* b, vit_stream_t stream) {
  if (b == nullptr) return fail(VIT_EINVAL, "null batch");
  cudaStream_t s = (cudaStream_t)stream;
  if (!(b->flags & VIT_BATCH_GRAPH)) return batch_enqueue(b, s);
  if (b->exec == nullptr) {
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "capture stream");
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaStreamDestroy(cs);
      return cuda_fail(e, "begin capture");
    }
    int rc = batch_enqueue(b, cs);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (rc != VIT_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_fail(e, "graph instantiate");
    }
    b->graph = g;
  }
  cudaError_t e = cudaGraphLaunch(b->exec, s);
  if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  return VIT_OK;
}

void vit_batch_destroy(vit_batch* b) {
  if (b == nullptr) return;
  cudaDeviceSynchronize();  // plan buffers may still be in use by enqueued work
  batch_free(b);
}

int vit_decode_batch(const vit_frame* frames, int nframes, vit_stream_t stream) {
  vit_batch* b = nullptr;
  int rc = vit_batch_plan(&b, frames, nframes, 0);
  if (rc != VIT_OK) return rc;
  rc = vit_batch_run(b, stream);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  batch_free(b);
  if (rc == VIT_OK && e != cudaSuccess) rc = cuda_fail(e, "batch");
  return rc;
}

}  // extern "C"
