// C ABI and host runtime: detector handles, device memory, guard constants, launches.
#include <algorithm>
#include <cfloat>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <cmath>
#include <cstdlib>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "ace_internal.h"
#include "gemm_plan.h"
#include "tc_plan.h"
#include "tc_ptx.cuh"
#include "fwht_plan.h"
#include "admission.h"

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(ACE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define ACE_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

}  // namespace

struct ace_detector {
  int d = 0, K = 0, L = 0, KL = 0, device = 0;
  int precision = ACE_PROJ_AUTO;
  int last_precision = ACE_PROJ_FP32;
  int last_products = 0;  // tensor-core products per accumulation in the last hash (0: SIMT)
  float* W = nullptr;       // [d][KL]
  float* Wt = nullptr;      // [KL][d]
  float* cB = nullptr;      // [KL]
  float xfac = 1.f, xabs = 0.f, babs = 0.f;
  float dot2c = 0.f, dot2abs = 0.f;  // Dot2 filter constants for this d
  float runc = 0.f, run64 = 0.f, runabs = 0.f;  // the SIMT engine's warp recheck (running bound)
  uint32_t* counts = nullptr;  // [L][2^K]
  ace::DevStats* st = nullptr;
  void* ids = nullptr;
  size_t ids_cap = 0;  // bytes
  uint32_t* sums = nullptr;
  size_t sums_cap = 0;  // bytes
  // host-buffer entry: two X staging slots, so the copy of one batch overlaps the work of the
  // previous one; each with its per-chunk copy events and a "batch done" event on the stream
  struct HostSlot {
    void* x = nullptr;
    size_t cap = 0;  // bytes
    cudaEvent_t done = nullptr;
    cudaEvent_t chunk[16] = {};
    bool busy = false;
  } hs[2];
  int hs_next = 0;
  cudaStream_t hs_stream = nullptr;  // stream of the batches in flight
  double* scstage = nullptr;
  uint8_t* flstage = nullptr;
  size_t stage_cap = 0;  // elements
  cudaStream_t cstream = nullptr;  // copy stream of the host-buffer entry (created on first use)
  uint64_t n_ins = 0;
  // sliding window (ace_window_enable): the ids of the points held, table-major [L][win_cap],
  // a ring whose oldest point sits at slot win_start; n_ins = points held
  void* ring = nullptr;
  long long win_cap = 0, win_start = 0;
  ace::DivConst div{};    // constants of the score division by L
  std::vector<float> Wh;  // host copy of W
  // tensor-core path
  int num_sms = 0;
  bool tc_ok = false;
  ace::TcArgs tc{};           // constant part of the launch (plan, guard constants, layout)
  uint8_t* bimg = nullptr;    // resident operand image of W' (device)
  unsigned long long* defer = nullptr;
  size_t defer_bytes = 0;
  unsigned int* defer_counts = nullptr;  // one per CTA of the tensor-core kernel
  float* wpad = nullptr;                 // [KL][dp] W, columns contiguous, zero-padded (recheck)
  float* wnorm = nullptr;                // [KL] ||w_c|| in binary32 (ace_project, tensor-core engine)
  uint32_t* hist = nullptr;              // [L][2^K] histogram of a batch being deleted
  unsigned int* dflag = nullptr;         // deletion check flag
  // insert path of the tensor-core engine: the deferred tables are resolved (and counted) on
  // rstream while the insert pass runs on the caller's stream
  cudaStream_t rstream = nullptr;
  cudaEvent_t ev_hashed = nullptr, ev_resolved = nullptr;
  // streaming tensor-core path (large d, bfloat16 input; hash_gemm.cu)
  // ACE_W_HADAMARD: the structured engine (hash_fwht.cu)
  bool hadamard = false, fwht_ok = false;
  ace::FwhtArgs fw{};
  uint32_t* gdsign = nullptr;   // [nblk][dp/32] sign words of the blocks' diagonals
  bool wgen = false;             // ACE_W_COUNTER: the SIMT engine regenerates W tiles from wseed
  uint64_t wseed = 0;
  bool seeded = false;           // created from a seed (the seed kept to refuse it as a noise seed)
  uint64_t seed = 0;
  // privacy noise (ace_set_privacy): sigma, the noise seed, and the noise index of the next
  // point hashed (points hashed with noise so far)
  float nsig = 0.f;
  uint64_t nseed = 0, nbase = 0;
  bool gemm_ok = false;
  ace::GemmArgs gm{};           // constant part of the launch
  uint16_t* gimg = nullptr;     // [2 klp][dp] bfloat16 image of W' (hi rows, then lo rows)
  float* gprof = nullptr;       // [2][dp/16] prefix and block norm maxima of the hi image
  float* gcolf = nullptr;       // [klp] image column norms (single-product image only)
  uint16_t* gwt16 = nullptr;    // [KL][d] bfloat16 W, columns contiguous (single-product only)
  CUtensorMap tm_img{};         // TMA description of gimg
  // E4M3 variant of the streaming engine (ACE_PROJ_FP8; bfloat16-valued W only)
  bool gemm8_ok = false;
  ace::GemmArgs gm8{};
  uint8_t* gimg8 = nullptr;     // [nunits][nkb][W1, W2][256 x 64] canonical E4M3 blocks
  float* gprof8 = nullptr;      // [2][nkb] W1 profile (K = 32 instructions folded per k-block)
  float* gcolf8 = nullptr;      // [klp] norms of the scaled image columns
  float* gwnorm8 = nullptr;     // [KL] accumulator scale back to x.w_c (ace_project)
  // graph replay (ace_set_graph): the launches of a repeated score / insert_score call are
  // captured once and replayed while its arguments and buffers stay the same
  struct GraphKey {
    const void* X = nullptr;
    long long n = -1;
    int dtype = -1, precision = -2;
    double alpha = 0.0;
    const void *sc = nullptr, *su = nullptr, *fl = nullptr, *ids = nullptr, *sums = nullptr, *defer = nullptr;
    cudaStream_t s = nullptr;
    bool insert = false;
    bool operator==(const GraphKey& o) const {
      return X == o.X && n == o.n && dtype == o.dtype && precision == o.precision && alpha == o.alpha && sc == o.sc &&
             su == o.su && fl == o.fl && ids == o.ids && sums == o.sums && defer == o.defer && s == o.s &&
             insert == o.insert;
    }
  };
  bool graph_on = false;
  GraphKey gkey{};
  bool gseen = false;                   // the key's call ran once uncaptured (buffers sized)
  cudaGraphExec_t gexec = nullptr;
  uint64_t glaunch[ACE_NPHASE] = {};    // kernels the captured graph launches, per phase
  int gprec = ACE_PROJ_FP32, gprod = 0; // engine the captured call used
  // profiling hook
  bool prof = false;
  unsigned prof_mask = ~0u;  // phases bracketed while profiling
  uint64_t launches[ACE_NPHASE] = {0, 0, 0, 0, 0, 0};
  struct Mark {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<Mark> marks;
  std::vector<cudaEvent_t> pool;
};

namespace {

// Brackets one library kernel launch with events when profiling is on.
struct PhaseScope {
  ace_detector* h;
  int phase;
  cudaStream_t s;
  cudaEvent_t b = nullptr;
  cudaEvent_t take() {
    if (!h->pool.empty()) {
      cudaEvent_t e = h->pool.back();
      h->pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  PhaseScope(ace_detector* h_, int phase_, cudaStream_t s_) : h(h_), phase(phase_), s(s_) {
    h->launches[phase] += 1;
    if (h->prof && ((h->prof_mask >> phase) & 1u)) {
      cudaEvent_t a = take();
      b = take();
      cudaEventRecord(a, s);
      h->marks.push_back({phase, a, b});
    }
  }
  ~PhaseScope() {
    if (b) cudaEventRecord(b, s);
  }
};

size_t count_elems(const ace_detector* h) { return (static_cast<size_t>(1) << h->K) * static_cast<size_t>(h->L); }

void free_all(ace_detector* h) {
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  h->gexec = nullptr;
  if (h->ev_hashed) cudaEventDestroy(h->ev_hashed);
  if (h->ev_resolved) cudaEventDestroy(h->ev_resolved);
  if (h->rstream) cudaStreamDestroy(h->rstream);
  for (auto& m : h->marks) {
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  for (auto e : h->pool) cudaEventDestroy(e);
  h->marks.clear();
  h->pool.clear();
  cudaFree(h->bimg);
  cudaFree(h->ring);
  cudaFree(h->gimg);
  cudaFree(h->gprof);
  cudaFree(h->gcolf);
  cudaFree(h->gwt16);
  cudaFree(h->gdsign);
  cudaFree(h->gimg8);
  cudaFree(h->gprof8);
  cudaFree(h->gcolf8);
  cudaFree(h->gwnorm8);
  cudaFree(h->defer);
  cudaFree(h->defer_counts);
  cudaFree(h->wpad);
  cudaFree(h->wnorm);
  cudaFree(h->hist);
  cudaFree(h->dflag);
  cudaFree(h->W);
  cudaFree(h->Wt);
  cudaFree(h->cB);
  cudaFree(h->counts);
  cudaFree(h->st);
  cudaFree(h->ids);
  cudaFree(h->sums);
  for (auto& sl : h->hs) {
    for (auto& e : sl.chunk)
      if (e) cudaEventDestroy(e);
    if (sl.done) cudaEventDestroy(sl.done);
    cudaFree(sl.x);
  }
  if (h->cstream) cudaStreamDestroy(h->cstream);
  cudaFree(h->scstage);
  cudaFree(h->flstage);
}

// Guard constants of the binary32 paths (see hash_simt.cu): both gammas, ||w_c|| rounded
// up, and a 2% margin that covers the few binary32 roundings of the bound itself.
void guard_constants(const std::vector<float>& W, int d, int KL, std::vector<float>& cB, float& xfac, float& xabs,
                     float& babs, float& dot2c, float& dot2abs, float& runc, float& run64, float& runabs) {
  const double u32 = std::ldexp(1.0, -24), u64 = std::ldexp(1.0, -53);
  const double g32 = d * u32 / (1.0 - d * u32);
  const double g64 = d * u64 / (1.0 - d * u64);
  const double gam = (g32 + g64) * 1.02;
  cB.resize(KL);
  for (int c = 0; c < KL; ++c) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) {
      const double w = W[static_cast<size_t>(i) * KL + c];
      s += w * w;
    }
    const double nw = std::sqrt(s) * (1.0 + 1e-12);
    cB[c] = std::nextafter(static_cast<float>(gam * nw), FLT_MAX);
  }
  xfac = std::nextafter(static_cast<float>(1.0 + 2.0 * g32 + std::ldexp(1.0, -20)), FLT_MAX);
  xabs = static_cast<float>(std::ldexp(static_cast<double>(d), -149));
  babs = static_cast<float>(std::ldexp(static_cast<double>(d), -148));
  if (xabs == 0.f) xabs = std::ldexp(1.0f, -149);
  if (babs == 0.f) babs = std::ldexp(1.0f, -148);
  // Dot2 filter: (gamma_d^2 + gamma64_d) (1 + u) sum|x_i w_i|, with sum|x_i w_i| <=
  // a / ((1 - u)(1 - gamma_d)) for the binary32 sum a of the rounded |products|; underflow
  // (each product error and each sum below 2^-126 off by at most 2^-150) in dot2abs.
  dot2c = std::nextafter(static_cast<float>((g32 * g32 + g64) * (1.0 + u32) / ((1.0 - u32) * (1.0 - g32)) * 1.01),
                         FLT_MAX);
  dot2abs = static_cast<float>(4.0 * d * std::ldexp(1.0, -149));
  // Running error bound of the SIMT engine's warp recheck: d FMAs spread over 32 lane chains
  // and 31 additions joining them, each rounding step r^ = RN(r) off by at most u |r^| / (1 - u)
  // plus 2^-150 below 2^-126; the binary32 tree sum R^ of the d + 31 terms |r^| has
  // sum |r^| <= R^ / (1 - gamma_(d+64)) (generous: no term passes through more additions).  The
  // binary64 definition's own error, gamma64_d ||x|| ||w_c||, is a multiple of cB[c].
  const double gr = (d + 64) * u32 / (1.0 - (d + 64) * u32);
  runc = std::nextafter(static_cast<float>(u32 / ((1.0 - u32) * (1.0 - gr)) * 1.01), FLT_MAX);
  run64 = std::nextafter(static_cast<float>(g64 / (1.02 * (g32 + g64)) * 1.01), FLT_MAX);
  runabs = static_cast<float>(std::ldexp(static_cast<double>(d + 31), -149));
}

uint16_t bf16_rn(float f) {  // round to nearest even (finite inputs)
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return static_cast<uint16_t>((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}
float bf16_value(uint16_t b) {
  const uint32_t u = static_cast<uint32_t>(b) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
constexpr uint32_t kmajor_off(int r, int k, int kt) {
  return static_cast<uint32_t>((r >> 3) * (kt * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Plans the tensor-core path (hash_tc.cu): chunks of whole tables, the resident operand
// image of the unit-column matrix W' (bfloat16 hi and lo parts, K-major canonical layout),
// the shared-memory layout, and the guard constants.  Leaves tc_ok false when the device
// is not sm_103 or the shape does not fit the resident design.
int plan_tc(ace_detector* h) {
  h->tc_ok = false;
  cudaDeviceProp p;
  cudaError_t e = cudaGetDeviceProperties(&p, h->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  h->num_sms = p.multiProcessorCount;
  if (p.major != 10 || p.minor != 3) return ACE_OK;
  const int d = h->d, K = h->K, L = h->L, KL = h->KL;
  if (d > ace::kMaxD) return ACE_OK;
  const int d_pad = (d + 15) / 16 * 16;
  const int tpc = std::min(ace::kTcBufCols / K, 32);  // N <= kTcBufCols per chunk, at most 32 tables (32-bit masks)
  const int nch = (L + tpc - 1) / tpc;
  if (nch > ace::kTcMaxChunks) return ACE_OK;
  ace::TcArgs& t = h->tc;
  t = ace::TcArgs{};
  t.d = d;
  t.d_pad = d_pad;
  t.K = K;
  t.L = L;
  t.nchunks = nch;
  uint32_t off = 0;
  for (int c = 0; c < nch; ++c) {
    ace::TcChunk& ch = t.chunk[c];
    ch.tab0 = c * tpc;
    ch.ntab = std::min(tpc, L - ch.tab0);
    ch.N = (ch.ntab * K + 15) / 16 * 16;
    ch.boff_hi = off;
    off += static_cast<uint32_t>(ch.N) * d_pad * 2;
    ch.boff_lo = off;
    off += static_cast<uint32_t>(ch.N) * d_pad * 2;
  }
  t.bimg_bytes = static_cast<int>(off);
  auto up = [](int v, int a) { return (v + a - 1) / a * a; };
  t.a_bytes = 128 * d_pad * 2;
  t.off_a = up(t.bimg_bytes, 1024);
  t.off_stage = t.off_a + 4 * t.a_bytes;
  t.off_bnd = t.off_stage + up(128 * d * 4, 128);
  t.off_bits = t.off_bnd + 2 * 128 * 4;
  t.off_ctl = t.off_bits;
  t.smem_bytes = t.off_ctl + 256;
  if (t.smem_bytes > static_cast<int>(p.sharedMemPerBlockOptin)) return ACE_OK;

  // W' = w_c / ||w_c|| (binary32), split into bfloat16 hi + lo, laid out per chunk
  std::vector<uint16_t> img(off / 2, 0);
  std::vector<double> inv(KL, 0.0);
  for (int c = 0; c < KL; ++c) {
    double s2 = 0.0;
    for (int i = 0; i < d; ++i) {
      const double w = h->Wh[static_cast<size_t>(i) * KL + c];
      s2 += w * w;
    }
    inv[c] = s2 > 0.0 ? 1.0 / std::sqrt(s2) : 0.0;
  }
  for (int c = 0; c < nch; ++c) {
    const ace::TcChunk& ch = t.chunk[c];
    for (int r = 0; r < ch.ntab * K; ++r) {
      const int col = ch.tab0 * K + r;
      for (int k = 0; k < d; ++k) {
        const float wn = static_cast<float>(static_cast<double>(h->Wh[static_cast<size_t>(k) * KL + col]) * inv[col]);
        const uint16_t hi = bf16_rn(wn);
        const uint16_t lo = bf16_rn(wn - bf16_value(hi));
        img[(ch.boff_hi + kmajor_off(r, k, d_pad)) / 2] = hi;
        img[(ch.boff_lo + kmajor_off(r, k, d_pad)) / 2] = lo;
      }
    }
  }
  cudaFree(h->bimg);
  h->bimg = nullptr;
  if ((e = cudaMalloc(&h->bimg, off)) != cudaSuccess) return cuda_fail(e, "cudaMalloc W' image");
  if ((e = cudaMemcpy(h->bimg, img.data(), off, cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "copy W' image");
  if (!h->defer_counts &&
      (e = cudaMalloc(&h->defer_counts, sizeof(unsigned int) * static_cast<size_t>(h->num_sms))) != cudaSuccess)
    return cuda_fail(e, "cudaMalloc deferred counters");
  t.bimg = h->bimg;

  // guard constants (relative to ||x||; see hash_tc.cu)
  const double u32 = std::ldexp(1.0, -24), u64 = std::ldexp(1.0, -53);
  // MMA instructions accumulating into one result: the two small products first (each
  // addend at most 2^-8 (1 + 2^-8)^2 |x_i w'_i|, so each instruction's addends sum to at most
  // about 2^-7 sum|x_i w'_i|; 2^-6 is used), then x_hi . w'_hi (addends at most about
  // sum|x_i w'_i|)
  const int S_small = 2 * d_pad / 16, S_big = d_pad / 16;
  const double t_split = 3.0 * std::ldexp(1.0, -16) * (1.0 + std::ldexp(1.0, -6));
  const double t_acc = 5.25 * 1.5 * ((S_big + 1) + S_small * std::ldexp(1.0, -6)) * std::ldexp(1.0, -23) *
                       (1.0 + std::ldexp(1.0, -6));
  const double t_norm = std::ldexp(1.0, -23);
  const double g64 = d * u64 / (1.0 - d * u64);
  t.tau = std::nextafter(static_cast<float>((t_split + t_acc + t_norm + g64) * 1.01), FLT_MAX);
  t.tau_abs = static_cast<float>(3.0 * d_pad * std::ldexp(1.0, -125));
  const double g32 = d_pad * u32 / (1.0 - d_pad * u32);
  t.xfac = std::nextafter(static_cast<float>(1.0 + 2.0 * g32 + std::ldexp(1.0, -20)), FLT_MAX);
  t.qmin = std::ldexp(1.0f, -60);
  t.dot2c = h->dot2c;  // the Dot2 filter's constants depend on d only (guard_constants)
  t.dot2abs = h->dot2abs;
  // Running error bound of the recheck's binary32 FMA chain over dp steps (zero padding
  // included): each step s^_k = RN(s^_(k-1) + x_k w_k) is off by at most u |s^_k| / (1 - u)
  // plus 2^-150 below 2^-126, so |s^ - s| <= u / (1 - u) sum_k |s^_k| + dp 2^-150 / (1 - u);
  // the binary32 sum R^ of the |s^_k| has sum_k |s^_k| <= R^ / (1 - gamma_dp).  The binary64
  // definition's own error, gamma64_d sum|x_i w_i| <= gamma64_d ||x|| ||w_c||, is a multiple of
  // the a priori coefficient cB32[c] = 1.02 (gamma_d + gamma64_d) ||w_c||^.
  {
    const int dp = (d + 3) / 4 * 4;
    const double g32p = dp * u32 / (1.0 - dp * u32);
    const double g32a = d * u32 / (1.0 - d * u32);
    t.runc = std::nextafter(static_cast<float>(u32 / ((1.0 - u32) * (1.0 - g32p)) * 1.01), FLT_MAX);
    t.run64 = std::nextafter(static_cast<float>(g64 / (1.02 * (g32a + g64)) * 1.01), FLT_MAX);
    t.runabs = static_cast<float>(std::ldexp(static_cast<double>(dp), -149));
  }
  t.Wt = h->Wt;
  t.W = h->W;
  // W with contiguous, zero-padded columns for the recheck's 16-byte loads
  t.dp = (d + 3) / 4 * 4;
  {
    std::vector<float> wp(static_cast<size_t>(KL) * t.dp, 0.f);
    for (int c = 0; c < KL; ++c)
      for (int i = 0; i < d; ++i) wp[static_cast<size_t>(c) * t.dp + i] = h->Wh[static_cast<size_t>(i) * KL + c];
    cudaFree(h->wpad);
    h->wpad = nullptr;
    if ((e = cudaMalloc(&h->wpad, wp.size() * sizeof(float))) != cudaSuccess) return cuda_fail(e, "cudaMalloc padded W");
    if ((e = cudaMemcpy(h->wpad, wp.data(), wp.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail(e, "copy padded W");
  }
  t.Wp = h->wpad;
  {
    std::vector<float> wn(KL);
    for (int c = 0; c < KL; ++c) wn[c] = inv[c] > 0.0 ? static_cast<float>(1.0 / inv[c]) : 0.f;
    cudaFree(h->wnorm);
    h->wnorm = nullptr;
    if ((e = cudaMalloc(&h->wnorm, KL * sizeof(float))) != cudaSuccess) return cuda_fail(e, "cudaMalloc column norms");
    if ((e = cudaMemcpy(h->wnorm, wn.data(), KL * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail(e, "copy column norms");
  }
  t.wnorm = h->wnorm;
  t.cB32 = h->cB;
  t.xfac32 = h->xfac;
  t.xabs32 = h->xabs;
  t.babs32 = h->babs;
  t.counts = h->counts;
  t.st = h->st;
  t.defer_counts = h->defer_counts;
  h->tc_ok = true;
  return ACE_OK;
}

// cuTensorMapEncodeTiled from the driver (through the runtime, so the library does not link
// libcuda itself).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// A 2-D bfloat16 tensor map: rows x cols (cols innermost, row pitch cols * 2 bytes), boxes of
// box_rows x 64 elements, 128-byte swizzle, zero fill outside the tensor.
int encode_bf16_map(CUtensorMap* m, const void* base, uint64_t cols, uint64_t rows, uint32_t box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return fail(ACE_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const cuuint64_t gdim[2] = {cols, rows};
  const cuuint64_t gstride[1] = {cols * 2};
  const cuuint32_t box[2] = {static_cast<cuuint32_t>(ace::kGemmBK), box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), gdim, gstride, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ACE_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
  return ACE_OK;
}

// E4M3 (1 sign, 4 exponent bits with bias 7, 3 mantissa bits; no infinities, largest 448):
// round to nearest even, saturating beyond 448, and the value of a code.
uint8_t e4m3_rn(double v) {
  const uint8_t sg = std::signbit(v) ? 0x80 : 0x00;
  const double a = std::fabs(v);
  if (a == 0.0) return sg;
  if (a > 448.0) return sg | 0x7E;
  int ex = 0;
  std::frexp(a, &ex);
  int E = ex - 1;  // a in [2^E, 2^(E+1))
  if (E < -6) {    // subnormal: m 2^-9, m in 0..8 (8 is the smallest normal, code 0x08)
    return sg | static_cast<uint8_t>(std::nearbyint(std::ldexp(a, 9)));
  }
  double m = std::nearbyint(std::ldexp(a, 3 - E));  // 8 .. 16
  if (m == 16.0) {
    m = 8.0;
    ++E;
  }
  if (E > 8 || (E == 8 && m > 14.0)) return sg | 0x7E;
  return sg | static_cast<uint8_t>(((E + 7) << 3) | (static_cast<int>(m) - 8));
}
double e4m3_value(uint8_t b) {
  const int e = (b >> 3) & 15, m = b & 7;
  const double v = e == 0 ? std::ldexp(static_cast<double>(m), -9) : std::ldexp(8.0 + m, e - 10);
  return (b & 0x80) ? -v : v;
}

// Plans the E4M3 variant from the single-product bfloat16 image (every W entry a bfloat16
// value; columns already scaled by 2^-e_c to norms in [1/2, 1)).  Each image column v is scaled
// again by 2^f (its largest |v_i| to [128, 256)) and split as W1 = e4m3(2^f v), W2 = e4m3(2^f v
// - W1), W3 = the rest (nonzero only where an element falls into E4M3's subnormal range).  The
// accumulator of column c then holds 2^(s + f) x.v for a row scaled by 2^s.  Guard terms
// (normalised-column units, the bound of column c being B colf[c]).  One kind::f8f6f4
// instruction adds 33 addends (32 products and the accumulator): aligned to the largest
// exponent 2^E with two bits kept below its last place, each loses less than 2^(E-25), and the
// truncation of the sum to binary32 less than one unit in its last place, so the error is at
// most (33/4 + 1) 2^-23 = 9.25 2^-23 times the sum of their magnitudes (the same model as the
// 5.25 of kind::f16's 17 addends; tests/test_gpu_tc_model.py checks it on the device):
//   pass 1 (X1.W1, S8 = dp/32 instructions): E over y's prefix and block norms with W1's
//     profile, plus (||X2|| + ||X3||) sum_t (WP_t^1/2 + WB_t^1/2) for ||X1_S|| <= ||y_S|| +
//     ||y - X1||, plus S8 T0 for the pass-0 total the accumulator carries;
//   pass 0 (3 S8 instructions): at most (3 S8 + 1) T0, T0 bounding the magnitudes of all the
//     small products;
//   dropped: ||X3|| ||v|| + ||X1 + X2|| ||W3|| <= (||X3|| + rres (||y|| + ||X3||)) colf;
//   the binary64 reference (gamma64_d ||y||).
constexpr double kF8Acc = 9.25;
int plan_gemm_fp8(ace_detector* h, const std::vector<uint16_t>& img, const std::vector<int>& cexp, int dp, int tpu,
                  int nunits, int klp) {
  h->gemm8_ok = false;
  const int d = h->d, K = h->K, KL = h->KL;
  const int nkb = dp / ace::kGemmBK, S8 = dp / 32;
  const size_t plane = static_cast<size_t>(ace::kGemmBN) * ace::kGemmBK;
  std::vector<uint8_t> img8(static_cast<size_t>(nunits) * nkb * 2 * plane, 0);
  std::vector<float> colf8(klp, 0.f);
  std::vector<int> fexp(klp, 0);
  std::vector<double> wp(S8, 0.0), wb(S8, 0.0);
  double w1m = 0.0, w2m = 0.0, rres = 0.0;
  std::vector<double> vs(dp), w1(dp), w2(dp);
  for (int row = 0; row < klp; ++row) {
    double mx = 0.0;
    for (int i = 0; i < dp; ++i) mx = std::max(mx, std::fabs(static_cast<double>(bf16_value(img[static_cast<size_t>(row) * dp + i]))));
    if (mx == 0.0) continue;  // a padding row: zero planes
    int ex = 0;
    std::frexp(mx, &ex);
    const int f = 8 - ex;  // mx 2^f in [128, 256)
    fexp[row] = f;
    double n2 = 0.0, n1 = 0.0, n22 = 0.0, n3 = 0.0;
    for (int i = 0; i < dp; ++i) {
      vs[i] = std::ldexp(static_cast<double>(bf16_value(img[static_cast<size_t>(row) * dp + i])), f);
      const uint8_t b1 = e4m3_rn(vs[i]);
      w1[i] = e4m3_value(b1);
      const uint8_t b2 = e4m3_rn(vs[i] - w1[i]);
      w2[i] = e4m3_value(b2);
      const double r3 = vs[i] - w1[i] - w2[i];  // exact in binary64
      n2 += vs[i] * vs[i];
      n1 += w1[i] * w1[i];
      n22 += w2[i] * w2[i];
      n3 += r3 * r3;
      const int u = row / ace::kGemmBN, rr = row % ace::kGemmBN, kb = i / ace::kGemmBK, k = i % ace::kGemmBK;
      const size_t blk = (static_cast<size_t>(u) * nkb + kb) * 2 * plane;
      img8[blk + ace::tc::kmajor_offset8(rr, k, ace::kGemmBK)] = b1;
      img8[blk + plane + ace::tc::kmajor_offset8(rr, k, ace::kGemmBK)] = b2;
    }
    const double nrm = std::sqrt(n2);
    colf8[row] = std::nextafter(static_cast<float>(nrm * (1.0 + 1e-12)), FLT_MAX);
    w1m = std::max(w1m, std::sqrt(n1) / nrm);
    w2m = std::max(w2m, std::sqrt(n22) / nrm);
    rres = std::max(rres, std::sqrt(n3) / nrm);
    double pre = 0.0;
    for (int t = 0; t < S8; ++t) {
      wp[t] = std::max(wp[t], pre);
      double blk = 0.0;
      for (int i = 32 * t; i < 32 * t + 32; ++i) blk += (w1[i] / nrm) * (w1[i] / nrm);
      wb[t] = std::max(wb[t], blk);
      pre += blk;
    }
  }
  std::vector<float> prof(2 * static_cast<size_t>(nkb), 0.f);
  double sumw = 0.0;
  for (int kb = 0; kb < nkb; ++kb) {
    double sp = 0.0, sb = 0.0;
    for (int t = 2 * kb; t < 2 * kb + 2; ++t) {
      sp += std::sqrt(wp[t]);
      sb += wb[t];
      sumw += std::sqrt(wp[t]) + std::sqrt(wb[t]);
    }
    prof[kb] = std::nextafter(static_cast<float>(sp * (1.0 + 1e-12)), FLT_MAX);
    prof[nkb + kb] = std::nextafter(static_cast<float>(std::sqrt(sb) * (1.0 + 1e-12)), FLT_MAX);
  }
  std::vector<float> wn8(KL, 0.f);
  for (int c = 0; c < KL; ++c) {
    const int j = c / K, k = c % K;
    const int row = (j / tpu) * ace::kGemmBN + (j % tpu) * K + k;
    wn8[c] = std::ldexp(1.0f, cexp[c] - fexp[row]);
  }
  cudaError_t e;
  auto upload = [&](auto** dst, const auto& v, const char* what) -> int {
    cudaFree(*dst);
    *dst = nullptr;
    const size_t bytes = v.size() * sizeof(v[0]);
    if ((e = cudaMalloc(dst, bytes)) != cudaSuccess) return cuda_fail(e, what);
    if ((e = cudaMemcpy(*dst, v.data(), bytes, cudaMemcpyHostToDevice)) != cudaSuccess) return cuda_fail(e, what);
    return ACE_OK;
  };
  if (int rc = upload(&h->gimg8, img8, "E4M3 image")) return rc;
  if (int rc = upload(&h->gprof8, prof, "E4M3 norm profile")) return rc;
  if (int rc = upload(&h->gcolf8, colf8, "E4M3 column norms")) return rc;
  if (int rc = upload(&h->gwnorm8, wn8, "E4M3 column scales")) return rc;
  ace::GemmArgs g = h->gm;
  g.fp8 = 1;
  g.img8 = h->gimg8;
  g.nprod = 2;
  g.S = S8;
  g.wprof = h->gprof8;
  g.colf = h->gcolf8;
  g.wnorm = h->gwnorm8;
  const double u64 = std::ldexp(1.0, -53);
  const double g64 = d * u64 / (1.0 - d * u64);
  const double ca = kF8Acc * std::ldexp(1.0, -23) * 1.25;
  auto up = [](double v) { return std::nextafter(static_cast<float>(v * 1.01), FLT_MAX); };
  g.ca = up(ca);
  g.cx = up(rres * (1.0 + 1e-9) + g64);
  g.ksw = up(ca * sumw);
  g.kt0 = up(ca * (4.0 * S8 + 1.0));
  g.c3 = up(1.0 + rres);
  g.w1m = up(w1m);
  g.w2m = up(w2m);
  h->gm8 = g;
  h->gemm8_ok = true;
  return ACE_OK;
}

// Plans the streaming tensor-core path (hash_gemm.cu) for d > 64: the image of W' = w_c/||w_c||
// split into bfloat16 hi and lo parts, laid out per 256-column unit of whole tables
// (floor(256/K) tables per unit, zero rows after the last table), hi rows first, each row
// d zero-padded to a multiple of 64; its tensor map; and the guard constants (see hash_gemm.cu).
// Leaves gemm_ok false when the device is not sm_103 or the shape does not fit (d must be a
// multiple of 8: the TMA engine needs the row pitch of X in whole 16-byte units).
int plan_gemm(ace_detector* h) {
  h->gemm_ok = false;
  cudaDeviceProp p;
  cudaError_t e = cudaGetDeviceProperties(&p, h->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  h->num_sms = p.multiProcessorCount;
  if (p.major != 10 || p.minor != 3) return ACE_OK;
  const int d = h->d, K = h->K, L = h->L, KL = h->KL;
  if (d <= ace::kMaxD || d % 8 != 0) return ACE_OK;
  if (ace::gemm_smem_bytes() > static_cast<int>(p.sharedMemPerBlockOptin)) return ACE_OK;
  if (!tensor_map_encoder()) return ACE_OK;
  const int dp = (d + ace::kGemmBK - 1) / ace::kGemmBK * ace::kGemmBK;
  const int tpu = ace::kGemmBN / K;
  const int nunits = (L + tpu - 1) / tpu;
  const int klp = nunits * ace::kGemmBN;
  // Single product when every W entry is a bfloat16 value (ace_create_ex with ACE_W_BF16, or an
  // explicit W that happens to be): each column is scaled by a power of two to a norm in
  // [1/2, 1) (exact), and x_i w_i is then one exact bfloat16 product.  Otherwise each column is
  // normalised to unit length in binary32 and split into bfloat16 hi + lo parts (two products).
  bool one = true;
  std::vector<int> cexp(KL, 0);
  for (int c = 0; c < KL && one; ++c) {
    double s2 = 0.0;
    for (int i = 0; i < d; ++i) {
      const double w = h->Wh[static_cast<size_t>(i) * KL + c];
      s2 += w * w;
    }
    int e = 0;
    if (s2 > 0.0) std::frexp(std::sqrt(s2), &e);
    cexp[c] = e;
    for (int i = 0; i < d && one; ++i) {
      const float ws = std::ldexp(h->Wh[static_cast<size_t>(i) * KL + c], -e);
      one = std::isfinite(ws) && bf16_value(bf16_rn(ws)) == ws &&
            (h->Wh[static_cast<size_t>(i) * KL + c] == 0.f || ws != 0.f);
    }
  }
  const int nprod = one ? 1 : 2;
  std::vector<uint16_t> img(static_cast<size_t>(nprod) * klp * dp, 0);
  std::vector<float> wn(KL, 0.f);
  double rmax2 = 0.0;  // largest ||w' - w_hi - w_lo||^2 over the columns (exact in binary64)
  for (int c = 0; c < KL; ++c) {
    const int j = c / K, k = c % K;
    const size_t row = static_cast<size_t>(j / tpu) * ace::kGemmBN + static_cast<size_t>(j % tpu) * K + k;
    if (one) {
      wn[c] = std::ldexp(1.0f, cexp[c]);  // the scale back to x.w_c (ace_project)
      for (int i = 0; i < d; ++i)
        img[row * dp + i] = bf16_rn(std::ldexp(h->Wh[static_cast<size_t>(i) * KL + c], -cexp[c]));
      continue;
    }
    double s2 = 0.0;
    for (int i = 0; i < d; ++i) {
      const double w = h->Wh[static_cast<size_t>(i) * KL + c];
      s2 += w * w;
    }
    const double inv = s2 > 0.0 ? 1.0 / std::sqrt(s2) : 0.0;
    wn[c] = s2 > 0.0 ? static_cast<float>(std::sqrt(s2)) : 0.f;
    double r2 = 0.0;
    for (int i = 0; i < d; ++i) {
      const float w1 = static_cast<float>(static_cast<double>(h->Wh[static_cast<size_t>(i) * KL + c]) * inv);
      const uint16_t hi = bf16_rn(w1);
      const uint16_t lo = bf16_rn(w1 - bf16_value(hi));
      img[row * dp + i] = hi;
      img[(static_cast<size_t>(klp) + row) * dp + i] = lo;
      const double r = static_cast<double>(w1) - bf16_value(hi) - bf16_value(lo);
      r2 += r * r;
    }
    rmax2 = std::max(rmax2, r2);
  }
  cudaFree(h->gimg);
  h->gimg = nullptr;
  const size_t bytes = img.size() * sizeof(uint16_t);
  if ((e = cudaMalloc(&h->gimg, bytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc W' image");
  if ((e = cudaMemcpy(h->gimg, img.data(), bytes, cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "copy W' image");
  if (int rc = encode_bf16_map(&h->tm_img, h->gimg, static_cast<uint64_t>(dp), static_cast<uint64_t>(nprod) * klp,
                               ace::kGemmBN))
    return rc;
  // WP_t = max over columns of ||w'_hi[0, 16t)||, WB_t = max of ||w'_hi[16t, 16t + 16)||, for
  // the S = dp/16 MMA instructions of one pass, folded per k-block (rounded up).  The single-product image's
  // columns (norms in [1/2, 1)) are normalised for the profile, and each column's norm goes to
  // colf, which scales the row bound per column.
  const int S = dp / 16;
  std::vector<float> prof(2 * static_cast<size_t>(S), 0.f);
  std::vector<float> colf(one ? klp : 0, 0.f);
  {
    std::vector<double> wp(S, 0.0), wb(S, 0.0);
    for (int row = 0; row < klp; ++row) {
      double nrm2 = 0.0;
      for (int i = 0; i < dp; ++i) {
        const double v = bf16_value(img[static_cast<size_t>(row) * dp + i]);
        nrm2 += v * v;
      }
      const double sc = one && nrm2 > 0.0 ? 1.0 / std::sqrt(nrm2) : 1.0;
      if (one) colf[row] = nrm2 > 0.0 ? std::nextafter(static_cast<float>(std::sqrt(nrm2) * (1.0 + 1e-12)), FLT_MAX) : 0.f;
      double pre = 0.0;
      for (int t = 0; t < S; ++t) {
        wp[t] = std::max(wp[t], pre);
        double blk = 0.0;
        for (int i = 16 * t; i < 16 * t + 16; ++i) {
          const double v = bf16_value(img[static_cast<size_t>(row) * dp + i]) * sc;
          blk += v * v;
        }
        wb[t] = std::max(wb[t], blk);
        pre += blk;
      }
    }
    // per k-block of four instructions: sum of the four WP_t, and sqrt of the sum of the four
    // WB_t^2 (the kernel bounds the k-block's terms with these; see hash_gemm.cu)
    const int nkb = dp / ace::kGemmBK;
    for (int kb = 0; kb < nkb; ++kb) {
      double sp = 0.0, sb = 0.0;
      for (int t = 4 * kb; t < 4 * kb + 4; ++t) {
        sp += std::sqrt(wp[t]);
        sb += wb[t];
      }
      prof[kb] = std::nextafter(static_cast<float>(sp * (1.0 + 1e-12)), FLT_MAX);
      prof[nkb + kb] = std::nextafter(static_cast<float>(std::sqrt(sb) * (1.0 + 1e-12)), FLT_MAX);
    }
  }
  cudaFree(h->gprof);
  h->gprof = nullptr;
  if ((e = cudaMalloc(&h->gprof, prof.size() * sizeof(float))) != cudaSuccess) return cuda_fail(e, "cudaMalloc norm profile");
  if ((e = cudaMemcpy(h->gprof, prof.data(), prof.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "copy norm profile");
  cudaFree(h->gcolf);
  h->gcolf = nullptr;
  cudaFree(h->gwt16);
  h->gwt16 = nullptr;
  if (one) {
    std::vector<uint16_t> wt16(static_cast<size_t>(KL) * d);
    for (int c = 0; c < KL; ++c)
      for (int i = 0; i < d; ++i) wt16[static_cast<size_t>(c) * d + i] = bf16_rn(h->Wh[static_cast<size_t>(i) * KL + c]);
    if ((e = cudaMalloc(&h->gwt16, wt16.size() * 2)) != cudaSuccess) return cuda_fail(e, "cudaMalloc bfloat16 W");
    if ((e = cudaMemcpy(h->gwt16, wt16.data(), wt16.size() * 2, cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail(e, "copy bfloat16 W");
    if ((e = cudaMalloc(&h->gcolf, colf.size() * sizeof(float))) != cudaSuccess) return cuda_fail(e, "cudaMalloc column norms");
    if ((e = cudaMemcpy(h->gcolf, colf.data(), colf.size() * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail(e, "copy column norms");
  }
  if (!h->wnorm) {
    if ((e = cudaMalloc(&h->wnorm, KL * sizeof(float))) != cudaSuccess) return cuda_fail(e, "cudaMalloc column norms");
    if ((e = cudaMemcpy(h->wnorm, wn.data(), KL * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail(e, "copy column norms");
  }
  if (!h->defer_counts &&
      (e = cudaMalloc(&h->defer_counts, sizeof(unsigned int) * static_cast<size_t>(h->num_sms))) != cudaSuccess)
    return cuda_fail(e, "cudaMalloc deferred counters");

  ace::GemmArgs& g = h->gm;
  g = ace::GemmArgs{};
  g.d = d;
  g.dp = dp;
  g.nkb = dp / ace::kGemmBK;
  g.K = K;
  g.L = L;
  g.KL = KL;
  g.tpu = tpu;
  g.nunits = nunits;
  g.nprod = nprod;
  g.klp = klp;
  // guard constants (unit columns; see hash_gemm.cu): B = ca E + cx ||x||_up + tau_abs with
  // ca = 5.25 2^-23 (1.25 margin), cx = ca (2^-6 S + 1) + split + normalisation + gamma64_d.
  // The split term |x . (w' - w_hi - w_lo)| <= ||x|| ||w' - w_hi - w_lo|| uses the largest
  // residual norm over the columns (each residual element is at most 2^-16 |w'_i|).
  const double u32 = std::ldexp(1.0, -24), u64 = std::ldexp(1.0, -53);
  const double ca = 5.25 * std::ldexp(1.0, -23) * 1.25;
  const double t_split = std::sqrt(rmax2) * (1.0 + 1e-12);
  const double t_norm = one ? 0.0 : std::ldexp(1.0, -23);  // power-of-two scaling is exact
  const double g64 = d * u64 / (1.0 - d * u64);
  g.ca = std::nextafter(static_cast<float>(ca * 1.01), FLT_MAX);
  g.cx = std::nextafter(static_cast<float>((ca * (std::ldexp(1.0, -6) * S + 1.0) + t_split + t_norm + g64) * 1.01),
                        FLT_MAX);
  g.S = S;
  g.wprof = h->gprof;
  g.colf = h->gcolf;
  g.Wt16 = h->gwt16;
  g.tau_abs = static_cast<float>(2.0 * dp * std::ldexp(1.0, -125));
  const double g32 = d * u32 / (1.0 - d * u32);
  g.xfac = std::nextafter(static_cast<float>(1.0 + 2.0 * g32 + std::ldexp(1.0, -20)), FLT_MAX);
  g.qmin = std::ldexp(1.0f, -60);
  g.wnorm = h->wnorm;
  g.st = h->st;
  g.Wt = h->Wt;
  g.cB32 = h->cB;
  g.xfac32 = h->xfac;
  g.xabs32 = h->xabs;
  g.babs32 = h->babs;
  g.dot2c = h->dot2c;
  g.dot2abs = h->dot2abs;
  g.runc = h->runc;
  g.run64 = h->run64;
  g.runabs = h->runabs;
  g.defer_counts = h->defer_counts;
  g.smem_bytes = ace::gemm_smem_bytes();
  h->gemm_ok = true;
  if (one) return plan_gemm_fp8(h, img, cexp, dp, tpu, nunits, klp);
  return ACE_OK;
}

int make_detector(int d, int K, int L, const float* Wsrc, uint64_t seed, bool from_seed, unsigned flags,
                  ace_handle* out) {
  if (!out) return fail(ACE_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (flags & ~static_cast<unsigned>(ACE_W_BF16 | ACE_W_COUNTER | ACE_W_HADAMARD))
    return fail(ACE_ERR_ARG, "unknown creation flags 0x%x", flags);
  if ((flags & (ACE_W_COUNTER | ACE_W_HADAMARD)) && !from_seed)
    return fail(ACE_ERR_ARG, "ACE_W_COUNTER and ACE_W_HADAMARD need a seed");
  if ((flags & ACE_W_COUNTER) && (flags & ACE_W_HADAMARD))
    return fail(ACE_ERR_ARG, "ACE_W_COUNTER and ACE_W_HADAMARD exclude each other");
  if (d < 1 || K < 1 || K > 24 || L < 1 || static_cast<long long>(K) * L > 65536)
    return fail(ACE_ERR_ARG, "invalid shape d=%d K=%d L=%d (need d>=1, 1<=K<=24, L>=1, K*L<=65536)", d, K, L);
  if (!from_seed && !Wsrc) return fail(ACE_ERR_ARG, "W_host is NULL");
  ace_detector* h = new (std::nothrow) ace_detector();
  if (!h) return fail(ACE_ERR_OOM, "host allocation failed");
  h->d = d;
  h->K = K;
  h->L = L;
  h->KL = K * L;
  h->seeded = from_seed;
  h->seed = from_seed ? seed : 0u;
  h->div = ace::make_div_const(static_cast<uint32_t>(L));
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "cudaGetDevice");
  }
  const size_t dkl = static_cast<size_t>(d) * h->KL;
  try {
    h->Wh.resize(dkl);
  } catch (...) {
    delete h;
    return fail(ACE_ERR_OOM, "host allocation of W failed");
  }
  std::vector<uint32_t> dsign;
  if (flags & ACE_W_HADAMARD) {
    const int dp = ace::fwht_order(d);
    dsign.assign(static_cast<size_t>((h->KL + dp - 1) / dp) * (dp / 32), 0u);
    ace::generate_projection_hadamard(d, K, L, seed, h->Wh.data(), dsign.data());
    h->hadamard = true;
  } else if (flags & ACE_W_COUNTER) {
    ace::generate_projection_counter(d, K, L, seed, h->Wh.data());
    h->wgen = true;
    h->wseed = seed;
  } else if (from_seed) {
    ace::generate_projection(d, K, L, seed, h->Wh.data());
    if (flags & ACE_W_BF16) ace::round_projection_bf16(h->Wh.data(), dkl);
  } else {
    std::memcpy(h->Wh.data(), Wsrc, dkl * sizeof(float));
    if (flags & ACE_W_BF16) ace::round_projection_bf16(h->Wh.data(), dkl);
  }
  for (size_t i = 0; i < dkl; ++i)
    if (!std::isfinite(h->Wh[i])) {
      delete h;
      return fail(ACE_ERR_ARG, "W has a non-finite entry at flat index %zu", i);
    }
  std::vector<float> Wt(dkl), cB;
  for (int i = 0; i < d; ++i)
    for (int c = 0; c < h->KL; ++c) Wt[static_cast<size_t>(c) * d + i] = h->Wh[static_cast<size_t>(i) * h->KL + c];
  guard_constants(h->Wh, d, h->KL, cB, h->xfac, h->xabs, h->babs, h->dot2c, h->dot2abs, h->runc, h->run64,
                  h->runabs);

  auto bad = [&](cudaError_t err, const char* what) {
    free_all(h);
    delete h;
    return err == cudaErrorMemoryAllocation ? fail(ACE_ERR_OOM, "%s: out of device memory", what)
                                            : cuda_fail(err, what);
  };
  // (a regenerated W needs no row-major device copy: only the SIMT engine's tiles read it)
  if (!h->wgen && (e = cudaMalloc(&h->W, dkl * sizeof(float))) != cudaSuccess) return bad(e, "cudaMalloc W");
  if ((e = cudaMalloc(&h->Wt, dkl * sizeof(float))) != cudaSuccess) return bad(e, "cudaMalloc Wt");
  if ((e = cudaMalloc(&h->cB, h->KL * sizeof(float))) != cudaSuccess) return bad(e, "cudaMalloc cB");
  if ((e = cudaMalloc(&h->counts, count_elems(h) * sizeof(uint32_t))) != cudaSuccess) return bad(e, "cudaMalloc counts");
  if ((e = cudaMalloc(&h->st, sizeof(ace::DevStats))) != cudaSuccess) return bad(e, "cudaMalloc stats");
  if (h->W && (e = cudaMemcpy(h->W, h->Wh.data(), dkl * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
    return bad(e, "copy W");
  if ((e = cudaMemcpy(h->Wt, Wt.data(), dkl * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
    return bad(e, "copy Wt");
  if ((e = cudaMemcpy(h->cB, cB.data(), h->KL * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess)
    return bad(e, "copy cB");
  if ((e = cudaMemset(h->counts, 0, count_elems(h) * sizeof(uint32_t))) != cudaSuccess) return bad(e, "zero counts");
  if ((e = cudaMemset(h->st, 0, sizeof(ace::DevStats))) != cudaSuccess) return bad(e, "zero stats");
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bad(e, "create sync");
  if (int rc = plan_tc(h)) {
    free_all(h);
    delete h;
    return rc;
  }
  if (int rc = plan_gemm(h)) {
    free_all(h);
    delete h;
    return rc;
  }
  if (h->hadamard) {
    // the structured engine: the transform's order dp, its sign words, and the guard constant
    // (gamma_m of the m-level addition tree + gamma64_d of the binary64 definition, 1 % margin)
    ace::FwhtArgs& f = h->fw;
    f = ace::FwhtArgs{};
    f.d = d;
    f.dp = ace::fwht_order(d);
    f.m = 0;
    while ((1 << f.m) < f.dp) ++f.m;
    f.K = K;
    f.L = L;
    f.KL = h->KL;
    f.nblk = (h->KL + f.dp - 1) / f.dp;
    const double u = std::ldexp(1.0, -24), u64 = std::ldexp(1.0, -53);
    const double gm = f.m * u / (1.0 - f.m * u), g64 = d * u64 / (1.0 - d * u64);
    f.cband = std::nextafter(static_cast<float>((gm + g64) * 1.01), FLT_MAX);
    f.babs = static_cast<float>(f.m * std::ldexp(1.0, -146));
    f.Wt = h->Wt;
    f.st = h->st;
    h->fwht_ok = f.dp <= ace::kFwhtMaxDp && f.nblk * (f.dp / 32) <= ace::kFwhtMaxWords;
    if ((e = cudaMalloc(&h->gdsign, dsign.size() * sizeof(uint32_t))) != cudaSuccess) return bad(e, "cudaMalloc signs");
    if ((e = cudaMemcpy(h->gdsign, dsign.data(), dsign.size() * sizeof(uint32_t), cudaMemcpyHostToDevice)) != cudaSuccess)
      return bad(e, "copy signs");
    f.dsign = h->gdsign;
    if (h->fwht_ok) h->precision = ACE_PROJ_AUTO;
  }
  if (h->tc_ok) {
    if ((e = cudaStreamCreateWithFlags(&h->rstream, cudaStreamNonBlocking)) != cudaSuccess) return bad(e, "recheck stream");
    if ((e = cudaEventCreateWithFlags(&h->ev_hashed, cudaEventDisableTiming)) != cudaSuccess) return bad(e, "event");
    if ((e = cudaEventCreateWithFlags(&h->ev_resolved, cudaEventDisableTiming)) != cudaSuccess) return bad(e, "event");
    h->precision = ACE_PROJ_AUTO;
  }
  *out = h;
  return ACE_OK;
}

int check_x(ace_handle h, const void* X, long long n, int dtype) {
  if (!h) return fail(ACE_ERR_ARG, "handle is NULL");
  if (n < 0) return fail(ACE_ERR_ARG, "n < 0");
  if (dtype != ACE_F32 && dtype != ACE_BF16) return fail(ACE_ERR_ARG, "unknown dtype %d", dtype);
  if (n > 0 && !X) return fail(ACE_ERR_ARG, "X is NULL");
  const size_t esz = dtype == ACE_F32 ? 4 : 2;
  if (reinterpret_cast<uintptr_t>(X) % esz) return fail(ACE_ERR_ARG, "X is not aligned to its element size");
  if (n > (1LL << 40)) return fail(ACE_ERR_ARG, "n too large");
  return ACE_OK;
}

// Grow a device buffer (synchronises `s` before freeing the old one).
int grow(void** p, size_t* cap, size_t need, cudaStream_t s, const char* what) {
  if (need <= *cap) return ACE_OK;
  size_t ncap = need + need / 2;
  if (*p) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, what);
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
  }
  cudaError_t e = cudaMalloc(p, ncap);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    if (e == cudaErrorMemoryAllocation) return fail(ACE_ERR_OOM, "%s: out of device memory (%zu bytes)", what, ncap);
    return cuda_fail(e, what);
  }
  *cap = ncap;
  return ACE_OK;
}

// Launch arguments for hashing n points of X.  With privacy noise on (and ids, not
// projections, asked for) the next n noise indices are reserved for these points, in order;
// `noise` = false (the autotuner's scratch runs) reserves none and adds no noise.
ace::HashArgs hash_args(ace_handle h, const void* X, long long n, int dtype, int mode, bool noise = true) {
  ace::HashArgs a{};
  if (noise && h->nsig != 0.f && !(mode & ace::kStoreProj)) {
    a.nsig = h->nsig;
    a.nseed = h->nseed;
    a.nbase = static_cast<long long>(h->nbase);
    h->nbase += static_cast<uint64_t>(n);
  }
  a.X = X;
  a.x_bf16 = dtype == ACE_BF16;
  a.n = n;
  a.d = h->d;
  a.K = h->K;
  a.L = h->L;
  a.KL = h->KL;
  a.W = h->W;
  a.wseed = h->wseed;
  a.wgen = h->wgen ? 1 : 0;
  a.Wt = h->Wt;
  a.cB = h->cB;
  a.xfac = h->xfac;
  a.xabs = h->xabs;
  a.babs = h->babs;
  a.dot2c = h->dot2c;
  a.dot2abs = h->dot2abs;
  a.runc = h->runc;
  a.run64 = h->run64;
  a.runabs = h->runabs;
  a.mode = mode;
  a.ids = h->ids;
  a.ld = n;
  a.ids_rm = nullptr;
  a.counts = h->counts;
  a.st = h->st;
  return a;
}

size_t id_bytes(ace_handle h) { return h->K <= 16 ? 2 : 4; }

// Hashes a.n points into the ids scratch (a.ids, leading dimension a.ld).  With kInsert the
// counts are incremented too: fused in the SIMT engine; on the tensor-core path by a pass over
// the stored ids, which `tc_insert` = false leaves to the caller (chunked hashing of one batch).
enum class Engine { kSimt, kResident, kStreaming, kFwht };

// The engine that hashes X: binary32 SIMT when asked for, or when no tensor-core design fits;
// the resident tensor-core design for d <= 64 (any input type); the streaming one for larger
// d with bfloat16 input at a 16-byte-aligned address (the TMA engine's rule).
Engine pick_engine(ace_handle h, int x_bf16, const void* X) {
  if (h->precision == ACE_PROJ_FP32) return Engine::kSimt;
  if (h->precision == ACE_PROJ_FWHT || (h->precision == ACE_PROJ_AUTO && h->fwht_ok)) return Engine::kFwht;
  if (h->nsig != 0.f) return Engine::kSimt;  // privacy noise: the tensor-core engines add none
  if (h->precision == ACE_PROJ_FP8)
    return h->gemm8_ok && x_bf16 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0 ? Engine::kStreaming : Engine::kSimt;
  if (h->tc_ok) return Engine::kResident;
  if (h->gemm_ok && x_bf16 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0) return Engine::kStreaming;
  return Engine::kSimt;
}

// Bytes of table-major ids for n points (plus a word of slack: the streaming engine's recheck
// flips bits of 16-bit ids with 32-bit atomics).
size_t ids_need(ace_handle h, long long n) { return static_cast<size_t>(n) * h->L * (h->K <= 16 ? 2 : 4) + 16; }

// Sliding window, before a batch of n points is inserted: the batch must fit, and the oldest
// points beyond the window are removed (§3.4.1 deletion: their counts decremented).
int window_prepare(ace_handle h, long long n, cudaStream_t s) {
  if (!h->ring || n == 0) return ACE_OK;
  if (n > h->win_cap)
    return fail(ACE_ERR_ARG, "a batch of %lld points is larger than the window of %lld", n, h->win_cap);
  const long long held = static_cast<long long>(h->n_ins);
  const long long m = std::max(0LL, held + n - h->win_cap);
  if (m == 0) return ACE_OK;
  cudaError_t e;
  {
    PhaseScope ps(h, ACE_PHASE_OTHER, s);
    e = ace::launch_window_evict(h->ring, h->K <= 16, h->win_cap, h->win_start, m, h->K, h->L, h->counts, h->num_sms > 0 ? h->num_sms : 152, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "window eviction launch");
  h->win_start = (h->win_start + m) % h->win_cap;
  h->n_ins -= static_cast<uint64_t>(m);
  return ACE_OK;
}

// Sliding window, after the batch's ids are in `ids` (table-major, leading dimension ld): they
// go to the ring slots after the newest point (the slots of the points just removed).
int window_commit(ace_handle h, const void* ids, long long ld, long long n, cudaStream_t s) {
  if (!h->ring || n == 0) return ACE_OK;
  const size_t idb = h->K <= 16 ? 2 : 4;
  long long dst = (h->win_start + static_cast<long long>(h->n_ins)) % h->win_cap;
  long long done = 0;
  while (done < n) {
    const long long len = std::min(n - done, h->win_cap - dst);
    ACE_CUDA(cudaMemcpy2DAsync(static_cast<char*>(h->ring) + static_cast<size_t>(dst) * idb, h->win_cap * idb,
                               static_cast<const char*>(ids) + static_cast<size_t>(done) * idb, ld * idb, len * idb,
                               static_cast<size_t>(h->L), cudaMemcpyDeviceToDevice, s));
    done += len;
    dst = (dst + len) % h->win_cap;
  }
  return ACE_OK;
}

// Streaming tensor-core engine (hash_gemm.cu): ids (or projections), then the exact
// resolution of the deferred (point, column) entries, then the count increments from the
// stored ids when inserting.
int run_gemm(ace_handle h, const ace::HashArgs& a, cudaStream_t s, bool tc_insert) {
  if (a.n > 0x7FFFFFFFLL) return fail(ACE_ERR_UNSUPPORTED, "the streaming engine takes at most 2^31-1 points per call");
  const bool insert = (a.mode & ace::kInsert) != 0;
  const bool proj = (a.mode & ace::kStoreProj) != 0;
  void* ids = a.ids;
  if (insert && (!ids || ids == h->ids)) {
    if (int rc = grow(&h->ids, &h->ids_cap, ids_need(h, a.n), s, "ids scratch")) return rc;
    ids = h->ids;
  }
  const long long ntiles = (a.n + ace::kGemmBM - 1) / ace::kGemmBM;
  const long long grid = std::min(static_cast<long long>(h->num_sms), ntiles);
  const size_t cap = static_cast<size_t>(a.n) * 4 + static_cast<size_t>(grid) * 4096;
  void* p = h->defer;
  if (int rc = grow(&p, &h->defer_bytes, cap * 8, s, "deferred list")) return rc;
  h->defer = static_cast<unsigned long long*>(p);
  const bool f8 = h->precision == ACE_PROJ_FP8;
  ace::GemmArgs g = f8 ? h->gm8 : h->gm;
  g.X = a.X;
  g.n = a.n;
  g.ntiles = ntiles;
  g.mode = (a.mode & ~ace::kInsert) | (insert ? ace::kStoreIds : 0);
  g.ids = ids;
  g.ld = a.ld;
  g.ids_rm = a.ids_rm;
  g.proj = a.proj;
  g.defer = h->defer;
  g.seg_cap = h->defer_bytes / 8 / static_cast<size_t>(grid);
  alignas(128) CUtensorMap tmx;
  if (int rc = encode_bf16_map(&tmx, a.X, static_cast<uint64_t>(h->d), static_cast<uint64_t>(a.n), ace::kGemmBM))
    return rc;
  cudaError_t e;
  if (!proj) {
    h->last_precision = f8 ? ACE_PROJ_FP8 : ACE_PROJ_BF16;
    h->last_products = f8 ? 4 : g.nprod;
  }
  {
    PhaseScope ps(h, ACE_PHASE_HASH, s);
    e = ace::launch_hash_gemm(g, &tmx, &h->tm_img, h->num_sms, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "streaming tensor-core hash kernel launch");
  if (proj) return ACE_OK;
  {
    PhaseScope ps(h, ACE_PHASE_RECHECK, s);
    e = ace::launch_recheck_cols(g, static_cast<int>(grid), h->num_sms, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "column recheck kernel launch");
  if (insert && tc_insert) {
    PhaseScope ps(h, ACE_PHASE_INSERT, s);
    e = ace::launch_insert_from_ids(ids, h->K <= 16, a.ld, a.n, h->K, h->L, h->counts, h->num_sms, s);
    if (e != cudaSuccess) return cuda_fail(e, "insert kernel launch");
  }
  return ACE_OK;
}

int run_hash(ace_handle h, const ace::HashArgs& a, cudaStream_t s, bool tc_insert = true) {
  const Engine eng = pick_engine(h, a.x_bf16, a.X);
  if (eng == Engine::kSimt && (h->precision == ACE_PROJ_BF16 || h->precision == ACE_PROJ_FP8))
    return fail(ACE_ERR_UNSUPPORTED, "the tensor-core engine at d=%d needs bfloat16 input at a 16-byte-aligned address",
                h->d);
  if (eng == Engine::kSimt) {
    h->last_precision = ACE_PROJ_FP32;
    h->last_products = 0;
    PhaseScope ps(h, ACE_PHASE_HASH, s);
    cudaError_t e = ace::launch_hash_simt(a, s);
    if (e != cudaSuccess) return cuda_fail(e, "hash kernel launch");
    return ACE_OK;
  }
  if (eng == Engine::kStreaming) return run_gemm(h, a, s, tc_insert);
  if (eng == Engine::kFwht) {  // structured engine: ids (or projections), then the count increments
    const bool insert = (a.mode & ace::kInsert) != 0;
    void* ids = a.ids;
    if (insert && (!ids || ids == h->ids)) {
      if (int rc = grow(&h->ids, &h->ids_cap, ids_need(h, a.n), s, "ids scratch")) return rc;
      ids = h->ids;
    }
    ace::FwhtArgs f = h->fw;
    f.X = a.X;
    f.x_bf16 = a.x_bf16;
    f.n = a.n;
    f.mode = (a.mode & ~ace::kInsert) | (insert ? ace::kStoreIds : 0);
    f.ids = ids;
    f.ld = a.ld;
    f.ids_rm = a.ids_rm;
    f.proj = a.proj;
    f.nsig = a.nsig;
    f.nseed = a.nseed;
    f.nbase = a.nbase;
    if (!(a.mode & ace::kStoreProj)) {
      h->last_precision = ACE_PROJ_FWHT;
      h->last_products = 0;
    }
    cudaError_t e;
    {
      PhaseScope ps(h, ACE_PHASE_HASH, s);
      e = ace::launch_hash_fwht(f, h->num_sms, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "structured hash kernel launch");
    if (insert && tc_insert) {
      PhaseScope ps(h, ACE_PHASE_INSERT, s);
      e = ace::launch_insert_from_ids(ids, h->K <= 16, a.ld, a.n, h->K, h->L, h->counts, h->num_sms, s);
      if (e != cudaSuccess) return cuda_fail(e, "insert kernel launch");
    }
    return ACE_OK;
  }
  // tensor-core engine (ids only), the binary64 resolution of the deferred tables, then the
  // count increments from the stored ids.  With 16-bit ids and K <= 15 the deferred tables are
  // tagged (kTagDeferred): their resolution, which counts them too, runs on rstream while the
  // insert pass counts the rest; the caller's stream joins it before anything reads the ids.
  const bool insert = (a.mode & ace::kInsert) != 0;
  const bool overlap = insert && tc_insert && h->K <= 15 && !a.ids_rm && h->rstream;
  void* ids = a.ids;
  if (insert && (!ids || ids == h->ids)) {
    if (int rc = grow(&h->ids, &h->ids_cap, ids_need(h, a.n), s, "ids scratch")) return rc;
    ids = h->ids;
  }
  const size_t cap = static_cast<size_t>(a.n) + 65536;
  void* p = h->defer;
  if (int rc = grow(&p, &h->defer_bytes, cap * 8, s, "deferred list")) return rc;
  h->defer = static_cast<unsigned long long*>(p);
  ace::TcArgs t = h->tc;
  t.X = a.X;
  t.x_bf16 = a.x_bf16;
  t.n = a.n;
  t.ntiles = (a.n + 127) / 128;
  const long long grid = std::min(static_cast<long long>(h->num_sms), t.ntiles);
  t.mode = (a.mode & ~ace::kInsert) | (insert ? ace::kStoreIds : 0) | (overlap ? ace::kTagDeferred : 0);
  t.ids = ids;
  t.ld = a.ld;
  t.ids_rm = a.ids_rm;
  t.defer = h->defer;
  t.seg_cap = h->defer_bytes / 8 / static_cast<size_t>(grid);
  h->last_precision = ACE_PROJ_BF16;
  h->last_products = 3;
  cudaError_t e;
  {
    PhaseScope ps(h, ACE_PHASE_HASH, s);
    e = ace::launch_hash_tc(t, h->num_sms, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core hash kernel launch");
  if (overlap) {
    ACE_CUDA(cudaEventRecord(h->ev_hashed, s));
    {
      PhaseScope ps(h, ACE_PHASE_INSERT, s);  // launched first: its blocks need the most shared memory
      e = ace::launch_insert_from_ids(ids, 1, a.ld, a.n, h->K, h->L, h->counts, h->num_sms, s);
      if (e != cudaSuccess) return cuda_fail(e, "insert kernel launch");
    }
    ACE_CUDA(cudaStreamWaitEvent(h->rstream, h->ev_hashed, 0));
    {
      PhaseScope ps(h, ACE_PHASE_RECHECK, h->rstream);
      e = ace::launch_recheck(t, h->num_sms, h->rstream);
    }
    if (e != cudaSuccess) return cuda_fail(e, "recheck kernel launch");
    ACE_CUDA(cudaEventRecord(h->ev_resolved, h->rstream));
    ACE_CUDA(cudaStreamWaitEvent(s, h->ev_resolved, 0));
    return ACE_OK;
  }
  {
    PhaseScope ps(h, ACE_PHASE_RECHECK, s);
    e = ace::launch_recheck(t, h->num_sms, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "recheck kernel launch");
  if (insert && tc_insert) {
    PhaseScope ps(h, ACE_PHASE_INSERT, s);
    e = ace::launch_insert_from_ids(ids, h->K <= 16, a.ld, a.n, h->K, h->L, h->counts, h->num_sms, s);
    if (e != cudaSuccess) return cuda_fail(e, "insert kernel launch");
  }
  return ACE_OK;
}

// Query phase and §5.3 rule over the n ids already in the scratch.
int score_tail(ace_handle h, long long n, double alpha, double* scores, uint32_t* sum_out, uint8_t* flags,
               cudaStream_t s) {
  cudaError_t e;
  {
    PhaseScope ps(h, ACE_PHASE_SCORE, s);
    e = ace::launch_score_gather(h->ids, h->K <= 16, n, n, h->K, h->L, alpha, h->counts, sum_out, h->st, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "score kernel launch");
  {
    PhaseScope ps(h, ACE_PHASE_FLAGS, s);
    e = ace::launch_flags(sum_out, n, h->div, h->st, scores, flags, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "flags kernel launch");
  return ACE_OK;
}

int score_common_direct(ace_handle h, const void* X, long long n, int dtype, double alpha, double* scores,
                        uint32_t* sums, uint8_t* flags, cudaStream_t s, bool insert);

// score / insert_score with graph replay (ace_set_graph): the first call with a given set of
// arguments runs directly (its buffers grow to size), the second captures its launches into a
// CUDA graph, later ones replay it.  The host bookkeeping (n_ins, the overflow check) is
// arithmetic on the arguments and runs on every call; nothing in the kernels depends on it.
int score_common(ace_handle h, const void* X, long long n, int dtype, double alpha, double* scores, uint32_t* sums,
                 uint8_t* flags, cudaStream_t s, bool insert) {
  // (the legacy default stream cannot be captured, and a stream someone is capturing already
  // records these launches in that capture)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (!h || !h->graph_on || h->ring || h->prof || h->nsig != 0.f || n <= 0 || s == nullptr || s == cudaStreamLegacy ||
      s == cudaStreamPerThread || cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
    return score_common_direct(h, X, n, dtype, alpha, scores, sums, flags, s, insert);
  int rc = check_x(h, X, n, dtype);
  if (rc) return rc;
  if (!std::isfinite(alpha)) return fail(ACE_ERR_ARG, "alpha must be finite");
  if (insert && h->n_ins + static_cast<uint64_t>(n) > 0xFFFFFFFFull)
    return fail(ACE_ERR_OVERFLOW, "inserting %lld points would allow a count above 2^32-1", n);
  ace_detector::GraphKey k;
  k.X = X;
  k.n = n;
  k.dtype = dtype;
  k.precision = h->precision;
  k.alpha = alpha;
  k.sc = scores;
  k.su = sums;
  k.fl = flags;
  k.ids = h->ids;
  k.sums = h->sums;
  k.defer = h->defer;
  k.s = s;
  k.insert = insert;
  if (h->gexec && k == h->gkey) {
    ACE_CUDA(cudaGraphLaunch(h->gexec, s));
    for (int p = 0; p < ACE_NPHASE; ++p) h->launches[p] += h->glaunch[p];
    if (insert) h->n_ins += static_cast<uint64_t>(n);
    h->last_precision = h->gprec;
    h->last_products = h->gprod;
    return ACE_OK;
  }
  if (!(h->gseen && k == h->gkey)) {  // first call with these arguments: run it directly
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    rc = score_common_direct(h, X, n, dtype, alpha, scores, sums, flags, s, insert);
    k.ids = h->ids;  // the call may have grown the scratch
    k.sums = h->sums;
    k.defer = h->defer;
    h->gkey = k;
    h->gseen = rc == ACE_OK;
    return rc;
  }
  // second call: capture (the buffers are already sized, so nothing allocates or synchronises)
  uint64_t before[ACE_NPHASE];
  for (int p = 0; p < ACE_NPHASE; ++p) before[p] = h->launches[p];
  const uint64_t nins = h->n_ins;
  ACE_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
  rc = score_common_direct(h, X, n, dtype, alpha, scores, sums, flags, s, insert);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  h->n_ins = nins;  // the captured call did not run: the replay below does
  cudaGraphExec_t ex = nullptr;
  if (rc == ACE_OK && e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
  if (g) cudaGraphDestroy(g);
  if (rc != ACE_OK || e != cudaSuccess) {
    // nothing captured has run: turn graph replay off for this handle and run the call directly
    cudaGetLastError();
    for (int p = 0; p < ACE_NPHASE; ++p) h->launches[p] = before[p];
    h->graph_on = false;
    h->gseen = false;
    return score_common_direct(h, X, n, dtype, alpha, scores, sums, flags, s, insert);
  }
  h->gexec = ex;
  for (int p = 0; p < ACE_NPHASE; ++p) {
    h->glaunch[p] = h->launches[p] - before[p];
    h->launches[p] = before[p];
  }
  h->gprec = h->last_precision;
  h->gprod = h->last_products;
  ACE_CUDA(cudaGraphLaunch(h->gexec, s));
  for (int p = 0; p < ACE_NPHASE; ++p) h->launches[p] += h->glaunch[p];
  if (insert) h->n_ins += static_cast<uint64_t>(n);
  return ACE_OK;
}

int score_common_direct(ace_handle h, const void* X, long long n, int dtype, double alpha, double* scores,
                        uint32_t* sums, uint8_t* flags, cudaStream_t s, bool insert) {
  int rc = check_x(h, X, n, dtype);
  if (rc) return rc;
  if (!std::isfinite(alpha)) return fail(ACE_ERR_ARG, "alpha must be finite");
  if (insert && h->n_ins + static_cast<uint64_t>(n) > 0xFFFFFFFFull)
    return fail(ACE_ERR_OVERFLOW, "inserting %lld points would allow a count above 2^32-1", n);
  if (n == 0) return ACE_OK;
  if (insert && h->ring && n > h->win_cap)
    return fail(ACE_ERR_ARG, "a batch of %lld points is larger than the window of %lld", n, h->win_cap);
  if ((rc = grow(&h->ids, &h->ids_cap, ids_need(h, n), s, "ids scratch"))) return rc;
  uint32_t* sum_out = sums;
  if (!sum_out) {
    void* p = h->sums;
    if ((rc = grow(&p, &h->sums_cap, static_cast<size_t>(n) * sizeof(uint32_t), s, "sums scratch"))) return rc;
    h->sums = static_cast<uint32_t*>(p);
    sum_out = h->sums;
  }
  if (insert && (rc = window_prepare(h, n, s))) return rc;
  ace::HashArgs a = hash_args(h, X, n, dtype, ace::kStoreIds | (insert ? ace::kInsert : 0));
  if ((rc = run_hash(h, a, s))) return rc;
  if (insert && (rc = window_commit(h, h->ids, n, n, s))) return rc;
  if (insert) h->n_ins += static_cast<uint64_t>(n);
  return score_tail(h, n, alpha, scores, sum_out, flags, s);
}

using u128 = unsigned __int128;

// ---------------------------------------------------------------------------------------
// Autotuner of the binary32 engine's tile for batched detectors: per (d rounded up to a
// power of two, K, L, input type), the first batch that meets the shape times the four tile
// variants (128 or 64 points x 128 or 64 columns per block) on 131,072 points (the detector's
// rows, repeated; enough blocks for many waves, as in a batch, where every block is a full
// one), hashing into a scratch with a scratch statistics block (no state of the detector
// changes).  A variant replaces the default 128 x 128 tile only if it is at least 5% faster;
// the choice is kept for the rest of the process.
// ---------------------------------------------------------------------------------------
struct TuneKey {
  int dcls, K, L, dtype;
  bool operator<(const TuneKey& o) const {
    return dcls != o.dcls ? dcls < o.dcls : K != o.K ? K < o.K : L != o.L ? L < o.L : dtype < o.dtype;
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;

TuneKey tune_key(int d, int K, int L, int dtype) {
  int c = 0;
  while ((1 << c) < d) ++c;
  return TuneKey{c, K, L, dtype};
}

// The tile for detector h's shape (tuned on X's first points the first time); -1 on a CUDA
// error (message set).
int tuned_tile(ace_handle h, const void* X, long long n, int dtype, cudaStream_t s) {
  const TuneKey key = tune_key(h->d, h->K, h->L, dtype);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(key);
  if (it != g_tune.end()) return it->second;
  if (n < 1024) return 0;  // too few points to sample: the default tile
  const long long nt = 131072;
  unsigned char* buf = nullptr;
  const size_t row = static_cast<size_t>(h->d) * (dtype == ACE_F32 ? 4 : 2);
  const size_t ib = static_cast<size_t>(nt) * h->L * 4, xb = static_cast<size_t>(nt) * row;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&buf), ib + xb + sizeof(ace::DevStats), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf + ib + xb, 0, sizeof(ace::DevStats), s);
  for (long long c0 = 0; c0 < nt && e == cudaSuccess; c0 += n)  // the detector's rows, repeated
    e = cudaMemcpyAsync(buf + ib + static_cast<size_t>(c0) * row, X, static_cast<size_t>(std::min(n, nt - c0)) * row,
                        cudaMemcpyDeviceToDevice, s);
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  int best = 0;
  float best_ms = 0.f;
  for (int t = 0; t < 4 && e == cudaSuccess; ++t) {
    ace::HashArgs a = hash_args(h, buf + ib, nt, dtype, ace::kStoreIds, false);
    a.ids = buf;
    a.ld = nt;
    a.st = reinterpret_cast<ace::DevStats*>(buf + ib + xb);
    a.tile = t;
    e = ace::launch_hash_simt(a, s);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = ace::launch_hash_simt(a, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    if (e == cudaSuccess && (t == 0 || ms < best_ms * (best == 0 ? 0.95f : 1.0f))) {
      best = t;
      best_ms = ms;
    }
  }
  if (buf) cudaFreeAsync(buf, s);
  for (auto v : ev)
    if (v) cudaEventDestroy(v);
  if (e != cudaSuccess) {
    cuda_fail(e, "tile autotuning");
    return -1;
  }
  g_tune[key] = best;
  return best;
}

}  // namespace

extern "C" {

int ace_create(int d, int K, int L, uint64_t seed, ace_handle* out) {
  return make_detector(d, K, L, nullptr, seed, true, 0u, out);
}

int ace_create_ex(int d, int K, int L, uint64_t seed, unsigned flags, ace_handle* out) {
  return make_detector(d, K, L, nullptr, seed, true, flags, out);
}

int ace_create_with_projection(int d, int K, int L, const float* W_host, ace_handle* out) {
  return make_detector(d, K, L, W_host, 0, false, 0u, out);
}

int ace_destroy(ace_handle h) {
  if (!h) return ACE_OK;
  cudaDeviceSynchronize();
  free_all(h);
  delete h;
  return ACE_OK;
}

int ace_reset(ace_handle h, void* stream) {
  if (!h) return fail(ACE_ERR_ARG, "handle is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ACE_CUDA(cudaMemsetAsync(h->counts, 0, count_elems(h) * sizeof(uint32_t), s));
  ACE_CUDA(cudaMemsetAsync(h->st, 0, sizeof(ace::DevStats), s));
  h->n_ins = 0;
  h->win_start = 0;
  return ACE_OK;
}

int ace_window_enable(ace_handle h, int64_t window_points) {
  if (!h) return fail(ACE_ERR_ARG, "handle is NULL");
  if (window_points < 0) return fail(ACE_ERR_ARG, "window_points < 0");
  if (h->n_ins != 0) return fail(ACE_ERR_ARG, "the window must be set while the detector holds no points");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "window");
  cudaFree(h->ring);
  h->ring = nullptr;
  h->win_cap = 0;
  h->win_start = 0;
  if (window_points == 0) return ACE_OK;
  if (window_points > 0xFFFFFFFFLL) return fail(ACE_ERR_ARG, "window_points above 2^32-1");
  const size_t bytes = static_cast<size_t>(window_points) * h->L * (h->K <= 16 ? 2 : 4);
  e = cudaMalloc(&h->ring, bytes);
  if (e != cudaSuccess) {
    h->ring = nullptr;
    cudaGetLastError();
    return fail(ACE_ERR_OOM, "window ring of %zu bytes: %s", bytes, cudaGetErrorString(e));
  }
  h->win_cap = window_points;
  return ACE_OK;
}

int ace_set_graph(ace_handle h, int enable) {
  if (!h) return fail(ACE_ERR_ARG, "handle is NULL");
  h->graph_on = enable != 0;
  if (!h->graph_on) {
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
    h->gseen = false;
  }
  return ACE_OK;
}

int ace_set_precision(ace_handle h, int precision) {
  if (!h) return fail(ACE_ERR_ARG, "handle is NULL");
  if (precision != ACE_PROJ_AUTO && precision != ACE_PROJ_FP32 && precision != ACE_PROJ_BF16 &&
      precision != ACE_PROJ_FP8 && precision != ACE_PROJ_FWHT)
    return fail(ACE_ERR_ARG, "unknown precision %d", precision);
  if (precision == ACE_PROJ_FWHT && !h->fwht_ok)
    return fail(ACE_ERR_UNSUPPORTED, "the structured engine needs a detector created with ACE_W_HADAMARD, d <= %d "
                                     "and ceil(K*L / dp) dp <= %d (d=%d K=%d L=%d)", ace::kFwhtMaxDp,
                ace::kFwhtMaxWords * 32, h->d, h->K, h->L);
  if (precision == ACE_PROJ_FP8 && !h->gemm8_ok)
    return fail(ACE_ERR_UNSUPPORTED, "the E4M3 projection needs the streaming tensor-core engine (an sm_103 device, "
                                     "d > 64 and a multiple of 8) and a W whose entries are all bfloat16 values "
                                     "(ACE_W_BF16); d=%d K=%d L=%d", h->d, h->K, h->L);
  if (precision == ACE_PROJ_BF16 && !h->tc_ok && !h->gemm_ok)
    return fail(ACE_ERR_UNSUPPORTED, "the tensor-core paths need an sm_103 device and either d <= 64 or d a multiple "
                                     "of 8 (d=%d K=%d L=%d)", h->d, h->K, h->L);
  if ((precision == ACE_PROJ_BF16 || precision == ACE_PROJ_FP8) && h->nsig != 0.f)
    return fail(ACE_ERR_UNSUPPORTED, "privacy noise is on: the tensor-core engines add no noise");
  h->precision = precision;
  return ACE_OK;
}

int ace_set_privacy(ace_handle h, float sigma, uint64_t noise_seed) {
  if (!h) return fail(ACE_ERR_ARG, "handle is NULL");
  if (!(sigma == 0.f || (sigma >= 0x1p-60f && sigma <= 0x1p60f)))
    return fail(ACE_ERR_ARG, "sigma must be 0 or in [2^-60, 2^60] (got %g)", static_cast<double>(sigma));
  if (sigma != 0.f && h->seeded && noise_seed == h->seed)
    return fail(ACE_ERR_ARG, "the noise seed must differ from the detector's projection seed");
  if (sigma != 0.f && (h->precision == ACE_PROJ_BF16 || h->precision == ACE_PROJ_FP8))
    return fail(ACE_ERR_UNSUPPORTED, "the tensor-core engines add no noise: set ACE_PROJ_AUTO, ACE_PROJ_FP32 or "
                                     "ACE_PROJ_FWHT first");
  h->nsig = sigma;
  h->nseed = sigma != 0.f ? noise_seed : 0u;
  h->nbase = 0;
  if (h->gexec) cudaGraphExecDestroy(h->gexec);  // a captured call holds the noise-free arguments
  h->gexec = nullptr;
  h->gseen = false;
  return ACE_OK;
}

int ace_get_privacy(ace_handle h, float* sigma, uint64_t* noise_seed, uint64_t* next_index) {
  if (!h) return fail(ACE_ERR_ARG, "handle is NULL");
  if (sigma) *sigma = h->nsig;
  if (noise_seed) *noise_seed = h->nseed;
  if (next_index) *next_index = h->nbase;
  return ACE_OK;
}

int ace_insert(ace_handle h, const void* X_dev, int64_t n, int dtype, void* stream) {
  int rc = check_x(h, X_dev, n, dtype);
  if (rc) return rc;
  if (h->n_ins + static_cast<uint64_t>(n) > 0xFFFFFFFFull)
    return fail(ACE_ERR_OVERFLOW, "inserting %lld points would allow a count above 2^32-1", static_cast<long long>(n));
  if (n == 0) return ACE_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->ring) {  // the window keeps the batch's ids: they go through the scratch
    if (n > h->win_cap)
      return fail(ACE_ERR_ARG, "a batch of %lld points is larger than the window of %lld", static_cast<long long>(n),
                  h->win_cap);
    if ((rc = grow(&h->ids, &h->ids_cap, ids_need(h, n), s, "ids scratch"))) return rc;
    if ((rc = window_prepare(h, n, s))) return rc;
  }
  ace::HashArgs a = hash_args(h, X_dev, n, dtype, ace::kInsert | (h->ring ? ace::kStoreIds : 0));
  if ((rc = run_hash(h, a, s))) return rc;
  if (h->ring && (rc = window_commit(h, h->ids, n, n, s))) return rc;
  h->n_ins += static_cast<uint64_t>(n);
  return ACE_OK;
}

int ace_score(ace_handle h, const void* X_dev, int64_t n, int dtype, double alpha, double* scores_dev,
              uint32_t* sums_dev, uint8_t* flags_dev, void* stream) {
  return score_common(h, X_dev, n, dtype, alpha, scores_dev, sums_dev, flags_dev, static_cast<cudaStream_t>(stream),
                      false);
}

int ace_insert_score(ace_handle h, const void* X_dev, int64_t n, int dtype, double alpha, double* scores_dev,
                     uint32_t* sums_dev, uint8_t* flags_dev, void* stream) {
  return score_common(h, X_dev, n, dtype, alpha, scores_dev, sums_dev, flags_dev, static_cast<cudaStream_t>(stream),
                      true);
}

int ace_host_wait(ace_handle h) {
  if (!h) return fail(ACE_ERR_ARG, "handle is NULL");
  int rc = ACE_OK;
  for (auto& sl : h->hs) {
    if (!sl.busy) continue;
    cudaError_t e = cudaEventSynchronize(sl.done);
    sl.busy = false;
    if (e != cudaSuccess && rc == ACE_OK) rc = cuda_fail(e, "host batch");
  }
  return rc;
}

// A piece of host X: n rows at X.
struct HostSeg {
  const void* X;
  int64_t n;
};

// One host-buffer batch on `stream`: op ACE_OP_INSERT, ACE_OP_SCORE or ACE_OP_INSERT_SCORE.
// With `segs` (inserts only), the batch is the concatenation of nseg pieces of host X (n
// their total; X_host unused): each piece is copied to its place in the staging buffer and
// the batch is hashed and counted as one, which gives the counts of inserting the pieces one
// after another (counts do not depend on the order of points).
static int enqueue_host_batch(ace_handle h, int op, const void* X_host, int64_t n, int dtype, double alpha,
                              double* scores_host, uint32_t* sums_host, uint8_t* flags_host, void* stream,
                              const HostSeg* segs = nullptr, int nseg = 0) {
  if (op != ACE_OP_INSERT && op != ACE_OP_SCORE && op != ACE_OP_INSERT_SCORE)
    return fail(ACE_ERR_ARG, "unknown operation %d", op);
  if (segs && op != ACE_OP_INSERT) return fail(ACE_ERR_ARG, "only inserts take several pieces");
  const bool do_insert = op != ACE_OP_SCORE, do_score = op != ACE_OP_INSERT;
  int rc = check_x(h, segs ? segs[0].X : X_host, n, dtype);
  if (rc) return rc;
  if (!std::isfinite(alpha)) return fail(ACE_ERR_ARG, "alpha must be finite");
  if (do_insert && h->n_ins + static_cast<uint64_t>(n) > 0xFFFFFFFFull)
    return fail(ACE_ERR_OVERFLOW, "inserting %lld points would allow a count above 2^32-1", static_cast<long long>(n));
  if (n == 0) return ACE_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // batches in flight share the ids scratch and rely on the order of one stream
  if (s != h->hs_stream) {
    if ((rc = ace_host_wait(h))) return rc;
    h->hs_stream = s;
  }
  ace_detector::HostSlot& sl = h->hs[h->hs_next];
  if (sl.busy) {  // at most two batches in flight
    cudaError_t e = cudaEventSynchronize(sl.done);
    sl.busy = false;
    if (e != cudaSuccess) return cuda_fail(e, "host batch");
  }
  const size_t row = static_cast<size_t>(h->d) * (dtype == ACE_F32 ? 4 : 2);
  const size_t xbytes = static_cast<size_t>(n) * row;
  const size_t need_ids = ids_need(h, n);
  // The slot's own staging buffer is idle here; sums and ids are used on `s` only (grow
  // synchronises it); the output staging is replaced below only once nothing is in flight.
  if (xbytes > sl.cap) {
    cudaFree(sl.x);
    sl.x = nullptr;
    sl.cap = 0;
    const size_t cap = xbytes + xbytes / 2;
    cudaError_t e = cudaMalloc(&sl.x, cap);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(ACE_ERR_OOM, "X staging: %s", cudaGetErrorString(e));
    }
    sl.cap = cap;
  }
  if (do_score && static_cast<size_t>(n) > h->stage_cap) {
    if ((rc = ace_host_wait(h))) return rc;
    ACE_CUDA(cudaStreamSynchronize(s));
    cudaFree(h->scstage);
    cudaFree(h->flstage);
    h->scstage = nullptr;
    h->flstage = nullptr;
    h->stage_cap = 0;
    const size_t cap = static_cast<size_t>(n) + static_cast<size_t>(n) / 2;
    cudaError_t e = cudaMalloc(&h->scstage, cap * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&h->flstage, cap);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(ACE_ERR_OOM, "output staging: %s", cudaGetErrorString(e));
    }
    h->stage_cap = cap;
  }
  if (do_score) {
    void* p = h->sums;
    if ((rc = grow(&p, &h->sums_cap, static_cast<size_t>(n) * sizeof(uint32_t), s, "sums scratch"))) return rc;
    h->sums = static_cast<uint32_t*>(p);
  }
  if ((rc = grow(&h->ids, &h->ids_cap, need_ids, s, "ids scratch"))) return rc;
  if (!h->cstream) ACE_CUDA(cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking));
  if (!sl.done) ACE_CUDA(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
  for (auto& ev : sl.chunk)
    if (!ev) ACE_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));

  // X goes up in chunks on the copy stream (after the slot's previous batch is done with its
  // staging buffer); each chunk is hashed on `s` as soon as it has landed, so the copy of
  // chunk c + 1 — and of the next batch — overlaps the hashing of chunk c.  Hashing is per
  // point, so the ids of the whole batch are the same as from one launch; the count
  // increments (tensor-core path), the query phase and the flags then run once over the batch.
  constexpr long long kMinChunk = 32768;
  const int kMaxChunks = static_cast<int>(sizeof(sl.chunk) / sizeof(sl.chunk[0]));
  long long chunk = std::max<long long>(kMinChunk, (static_cast<long long>(n) + 7) / 8);
  chunk = (chunk + 127) / 128 * 128;
  int nch = static_cast<int>(std::min<long long>((n + chunk - 1) / chunk, kMaxChunks));
  chunk = (n + nch - 1) / nch;
  chunk = (chunk + 127) / 128 * 128;
  // With the other slot's batch still in flight, that batch's work overlaps this batch's copy
  // already, and chunks would only cost link time (measured end to end at 500,000 points:
  // 1.05 G points/s with eight chunks, 1.21 with two, 1.24 with one copy): one copy.
  if (h->hs[h->hs_next ^ 1].busy) {
    nch = 1;
    chunk = n;
  }
  if (segs) {  // pieces: one copy each, then the batch is hashed as one chunk
    nch = 1;
    chunk = n;
  }
  if (do_insert && h->ring && n > h->win_cap)
    return fail(ACE_ERR_ARG, "a batch of %lld points is larger than the window of %lld", static_cast<long long>(n),
                h->win_cap);
  // A small single-chunk batch copies X on `s` itself: there is no later chunk whose copy
  // could overlap its hashing, and the copy stream would cost three more driver calls (two
  // waits and an event) per batch, which is what limits the rate of small requests.  The
  // slot's staging buffer is free on `s`: its previous batch ran on `s` (a change of stream
  // waits for every batch above), and that batch's hashing, its last use of the buffer, came
  // after its copy on either stream.
  constexpr size_t kDirectCopyMax = size_t(4) << 20;
  const bool direct = nch == 1 && xbytes <= kDirectCopyMax;
  cudaStream_t xs = direct ? s : h->cstream;
  if (!direct) ACE_CUDA(cudaStreamWaitEvent(h->cstream, sl.done, 0));
  if (segs) {
    size_t off = 0;
    for (int i = 0; i < nseg; ++i) {
      if (segs[i].n > 0)
        ACE_CUDA(cudaMemcpyAsync(static_cast<char*>(sl.x) + off, segs[i].X, static_cast<size_t>(segs[i].n) * row,
                                 cudaMemcpyHostToDevice, xs));
      off += static_cast<size_t>(segs[i].n) * row;
    }
    if (!direct) ACE_CUDA(cudaEventRecord(sl.chunk[0], h->cstream));
  } else {
    for (int c = 0; c < nch; ++c) {
      const long long c0 = c * chunk, nc = std::min<long long>(chunk, n - c0);
      if (nc <= 0) break;
      ACE_CUDA(cudaMemcpyAsync(static_cast<char*>(sl.x) + c0 * row, static_cast<const char*>(X_host) + c0 * row,
                               static_cast<size_t>(nc) * row, cudaMemcpyHostToDevice, xs));
      if (!direct) ACE_CUDA(cudaEventRecord(sl.chunk[c], h->cstream));
    }
  }
  const bool simt = pick_engine(h, dtype == ACE_BF16, sl.x) == Engine::kSimt;
  if (do_insert && (rc = window_prepare(h, n, s))) return rc;
  for (int c = 0; c < nch; ++c) {
    const long long c0 = c * chunk, nc = std::min<long long>(chunk, n - c0);
    if (nc <= 0) break;
    if (!direct) ACE_CUDA(cudaStreamWaitEvent(s, sl.chunk[c], 0));
    ace::HashArgs a = hash_args(h, static_cast<const char*>(sl.x) + c0 * row, nc, dtype,
                                ace::kStoreIds | (simt && do_insert ? ace::kInsert : 0));
    a.ids = static_cast<char*>(h->ids) + static_cast<size_t>(c0) * id_bytes(h);
    a.ld = n;
    if ((rc = run_hash(h, a, s, false))) return rc;
  }
  if (do_insert && !simt) {
    PhaseScope ps(h, ACE_PHASE_INSERT, s);
    cudaError_t e = ace::launch_insert_from_ids(h->ids, h->K <= 16, n, n, h->K, h->L, h->counts, h->num_sms, s);
    if (e != cudaSuccess) return cuda_fail(e, "insert kernel launch");
  }
  if (do_insert && (rc = window_commit(h, h->ids, n, n, s))) return rc;
  if (do_insert) h->n_ins += static_cast<uint64_t>(n);
  if (do_score) {
    if ((rc = score_tail(h, n, alpha, scores_host ? h->scstage : nullptr, h->sums, flags_host ? h->flstage : nullptr,
                         s)))
      return rc;
    if (scores_host) ACE_CUDA(cudaMemcpyAsync(scores_host, h->scstage, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (sums_host) ACE_CUDA(cudaMemcpyAsync(sums_host, h->sums, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    if (flags_host) ACE_CUDA(cudaMemcpyAsync(flags_host, h->flstage, n, cudaMemcpyDeviceToHost, s));
  }
  ACE_CUDA(cudaEventRecord(sl.done, s));
  sl.busy = true;
  h->hs_next ^= 1;
  return ACE_OK;
}

int ace_insert_score_host_async(ace_handle h, const void* X_host, int64_t n, int dtype, double alpha,
                                double* scores_host, uint32_t* sums_host, uint8_t* flags_host, void* stream) {
  return enqueue_host_batch(h, ACE_OP_INSERT_SCORE, X_host, n, dtype, alpha, scores_host, sums_host, flags_host,
                            stream);
}

int ace_insert_score_host(ace_handle h, const void* X_host, int64_t n, int dtype, double alpha, double* scores_host,
                          uint32_t* sums_host, uint8_t* flags_host, void* stream) {
  int rc = ace_insert_score_host_async(h, X_host, n, dtype, alpha, scores_host, sums_host, flags_host, stream);
  if (rc) return rc;
  return ace_host_wait(h);
}

// ---------------------------------------------------------------------------------------
// Request server (continuous batching over several detectors).  The detectors are divided
// among the scheduler threads (one by default; detector i belongs to thread i mod W); each
// detector keeps its waiting requests in submission order, and a thread admits the earliest
// admissible one among its detectors whenever a slot or memory frees up: at most two per
// detector are in flight (its two staging slots), the staged bytes of all threads stay within
// the budget, and a detector whose oldest waiting request cannot start keeps its later
// requests waiting too, so each detector sees its requests in submission order — its results
// are the same alone and in any mix.
// Inserts that follow one another in a detector's order (no other request of that detector
// between them) are admitted together as one launch set (their points copied side by side,
// hashed and counted once), which gives the same counts as inserting them one by one.  Each
// detector runs on its own stream, so different detectors' work overlaps on the device;
// completion is stamped by a host callback on that stream.
// ---------------------------------------------------------------------------------------
}  // extern "C"

struct ace_server_s {
  struct Req {
    uint64_t id = 0;
    int det = 0, op = 0, dtype = 0;
    const void* X = nullptr;
    int64_t n = 0;
    double alpha = 1.0;
    double* scores = nullptr;
    uint32_t* sums = nullptr;
    uint8_t* flags = nullptr;
    size_t bytes = 0;
    std::chrono::steady_clock::time_point t_sub, t_done;
    int rc = ACE_OK;
    bool done = false;
    ace_server_s* srv = nullptr;
    std::vector<Req*> merged;  // inserts admitted with this one (completed with it)
  };
  static constexpr int kMaxWorkers = 4;
  std::vector<ace_handle> dets;
  std::vector<cudaStream_t> streams;
  ace::Admission<Req> adm;  // queues, slots and the memory budget (admission.h)
  std::unordered_map<uint64_t, Req*> reqs;
  uint64_t next_id = 1;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv;  // waiters (ace_server_wait / drain)
  std::vector<std::unique_ptr<std::condition_variable>> wcv;  // one per scheduler thread
  std::vector<std::thread> workers;
  bool stop = false;

  void wake_workers() {
    for (auto& c : wcv) c->notify_one();
  }

  int nworkers() const { return adm.nthreads(); }

  static void CUDART_CB on_done(void* p) {
    Req* r = static_cast<Req*>(p);
    ace_server_s* s = r->srv;
    std::lock_guard<std::mutex> lk(s->mu);
    const auto now = std::chrono::steady_clock::now();
    s->adm.finish(r);
    r->t_done = now;
    r->done = true;
    for (Req* q : r->merged) {
      q->t_done = now;
      q->done = true;
    }
    s->cv.notify_all();
    s->wake_workers();  // a slot and memory are free again
  }

  // The request thread w starts next (caller holds mu), with the inserts that join it.
  Req* pick(int w) {
    return adm.pick(w, ACE_OP_INSERT, [&](int d) { return !dets[static_cast<size_t>(d)]->ring; });
  }

  void release(Req* r, int rc) {  // caller holds mu: a request that could not be enqueued
    const auto now = std::chrono::steady_clock::now();
    adm.finish(r);
    r->rc = rc;
    r->t_done = now;
    r->done = true;
    for (Req* q : r->merged) {
      q->rc = rc;
      q->t_done = now;
      q->done = true;
    }
    cv.notify_all();
    wake_workers();
  }

  void run(int w) {
    cudaSetDevice(device);
    std::vector<HostSeg> segs;
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      Req* r = nullptr;
      wcv[w]->wait(lk, [&] {
        return (r = pick(w)) != nullptr || (stop && adm.npending[static_cast<size_t>(w)] == 0);
      });
      if (!r) break;
      adm.start(r);
      lk.unlock();
      int rc;
      if (r->merged.empty()) {
        rc = enqueue_host_batch(dets[r->det], r->op, r->X, r->n, r->dtype, r->alpha, r->scores, r->sums, r->flags,
                                streams[r->det]);
      } else {
        segs.clear();
        int64_t n = r->n;
        segs.push_back({r->X, r->n});
        for (Req* q : r->merged) {
          segs.push_back({q->X, q->n});
          n += q->n;
        }
        rc = enqueue_host_batch(dets[r->det], ACE_OP_INSERT, nullptr, n, r->dtype, 1.0, nullptr, nullptr, nullptr,
                                streams[r->det], segs.data(), static_cast<int>(segs.size()));
      }
      if (rc == ACE_OK && cudaLaunchHostFunc(streams[r->det], on_done, r) != cudaSuccess) rc = ACE_ERR_CUDA;
      lk.lock();
      if (rc != ACE_OK) release(r, rc);
    }
  }
};

extern "C" {

int ace_server_create(const ace_handle* dets, int n_dets, size_t mem_budget_bytes, ace_server* out) {
  if (!out || !dets || n_dets < 1) return fail(ACE_ERR_ARG, "invalid server arguments");
  *out = nullptr;
  for (int i = 0; i < n_dets; ++i)
    if (!dets[i]) return fail(ACE_ERR_ARG, "detector %d is NULL", i);
  for (int i = 0; i < n_dets; ++i)
    for (int j = 0; j < i; ++j)
      if (dets[i] == dets[j]) return fail(ACE_ERR_ARG, "detector %d appears twice", i);
  ace_server_s* s = new (std::nothrow) ace_server_s();
  if (!s) return fail(ACE_ERR_OOM, "host allocation failed");
  s->dets.assign(dets, dets + n_dets);
  // scheduler threads: ACE_SERVER_THREADS (1 .. 4) if set, else 1 (measured: four threads
  // issuing CUDA calls at once gave 0.7x the capacity of one), at most one per detector
  int nw = 1;
  if (const char* env = std::getenv("ACE_SERVER_THREADS"))
    nw = std::max(1, std::min(ace_server_s::kMaxWorkers, std::atoi(env)));
  s->adm.init(n_dets, std::min(n_dets, nw), mem_budget_bytes);
  for (int w = 0; w < s->nworkers(); ++w) s->wcv.emplace_back(new std::condition_variable());
  cudaGetDevice(&s->device);
  s->streams.assign(n_dets, nullptr);
  for (int i = 0; i < n_dets; ++i) {
    cudaError_t e = cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      for (auto st : s->streams)
        if (st) cudaStreamDestroy(st);
      delete s;
      return cuda_fail(e, "server stream");
    }
  }
  for (int w = 0; w < s->nworkers(); ++w) s->workers.emplace_back([s, w] { s->run(w); });
  *out = s;
  return ACE_OK;
}

int ace_server_submit(ace_server s, int det, int op, const void* X_host, int64_t n, int dtype, double alpha,
                      double* scores_host, uint32_t* sums_host, uint8_t* flags_host, uint64_t* ticket) {
  if (!s || !ticket) return fail(ACE_ERR_ARG, "NULL argument");
  if (det < 0 || det >= static_cast<int>(s->dets.size())) return fail(ACE_ERR_ARG, "detector index %d out of range", det);
  if (op != ACE_OP_INSERT && op != ACE_OP_SCORE && op != ACE_OP_INSERT_SCORE)
    return fail(ACE_ERR_ARG, "unknown operation %d", op);
  if (int rc = check_x(s->dets[det], X_host, n, dtype)) return rc;
  auto* r = new (std::nothrow) ace_server_s::Req();
  if (!r) return fail(ACE_ERR_OOM, "host allocation failed");
  r->det = det;
  r->op = op;
  r->dtype = dtype;
  r->X = X_host;
  r->n = n;
  r->alpha = alpha;
  r->scores = scores_host;
  r->sums = sums_host;
  r->flags = flags_host;
  r->srv = s;
  const size_t row = static_cast<size_t>(s->dets[det]->d) * (dtype == ACE_F32 ? 4 : 2);
  r->bytes = static_cast<size_t>(n) * (row + static_cast<size_t>(s->dets[det]->L) * 4 + 13);
  r->t_sub = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    s->reqs[r->id] = r;
    s->adm.submit(r);
  }
  s->wcv[det % s->nworkers()]->notify_one();
  *ticket = r->id;
  return ACE_OK;
}

int ace_server_wait(ace_server s, uint64_t ticket, double* latency_s) {
  if (!s) return fail(ACE_ERR_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return fail(ACE_ERR_ARG, "unknown ticket %llu", static_cast<unsigned long long>(ticket));
  ace_server_s::Req* r = it->second;
  s->cv.wait(lk, [&] { return r->done; });
  if (latency_s) latency_s[0] = std::chrono::duration<double>(r->t_done - r->t_sub).count();
  const int rc = r->rc;
  s->reqs.erase(it);
  delete r;
  if (rc != ACE_OK) return fail(rc, "request %llu failed", static_cast<unsigned long long>(ticket));
  return ACE_OK;
}

int ace_server_drain(ace_server s) {
  if (!s) return fail(ACE_ERR_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv.wait(lk, [&] { return s->adm.idle(); });
  return ACE_OK;
}

int ace_server_info(ace_server s, int* threads, uint64_t* coalesced) {
  if (!s) return fail(ACE_ERR_ARG, "server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  if (threads) *threads = s->nworkers();
  if (coalesced) *coalesced = s->adm.coalesced;
  return ACE_OK;
}

int ace_server_destroy(ace_server s) {
  if (!s) return ACE_OK;
  ace_server_drain(s);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->wake_workers();
  for (auto& t : s->workers)
    if (t.joinable()) t.join();
  for (auto st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
  return ACE_OK;
}

int ace_delete(ace_handle h, const void* X_dev, int64_t n, int dtype, void* stream) {
  int rc = check_x(h, X_dev, n, dtype);
  if (rc) return rc;
  if (h->ring) return fail(ACE_ERR_ARG, "a windowed detector removes its oldest points itself");
  if (h->nsig != 0.f)
    return fail(ACE_ERR_UNSUPPORTED, "privacy noise is on: a point hashes to other ids than when it was inserted");
  if (n == 0) return ACE_OK;
  if (static_cast<uint64_t>(n) > h->n_ins)
    return fail(ACE_ERR_ARG, "deleting %lld points from a detector holding %llu", static_cast<long long>(n),
                static_cast<unsigned long long>(h->n_ins));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((rc = grow(&h->ids, &h->ids_cap, ids_need(h, n), s, "ids scratch"))) return rc;
  const long long total = static_cast<long long>(count_elems(h));
  if (!h->hist) {
    cudaError_t e = cudaMalloc(&h->hist, static_cast<size_t>(total) * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&h->dflag, sizeof(unsigned int));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(ACE_ERR_OOM, "deletion scratch: %s", cudaGetErrorString(e));
    }
  }
  // the batch's ids (no count change), then its histogram into the scratch
  ace::HashArgs a = hash_args(h, X_dev, n, dtype, ace::kStoreIds);
  if ((rc = run_hash(h, a, s))) return rc;
  ACE_CUDA(cudaMemsetAsync(h->hist, 0, static_cast<size_t>(total) * sizeof(uint32_t), s));
  ACE_CUDA(cudaMemsetAsync(h->dflag, 0, sizeof(unsigned int), s));
  cudaError_t e;
  {
    PhaseScope ps(h, ACE_PHASE_INSERT, s);
    e = ace::launch_insert_from_ids(h->ids, h->K <= 16, n, n, h->K, h->L, h->hist, h->num_sms, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "deletion histogram launch");
  {
    PhaseScope ps(h, ACE_PHASE_OTHER, s);
    e = ace::launch_delete_check(h->hist, h->counts, total, h->dflag, h->num_sms, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "deletion check launch");
  unsigned int bad = 0;
  ACE_CUDA(cudaMemcpyAsync(&bad, h->dflag, sizeof bad, cudaMemcpyDeviceToHost, s));
  ACE_CUDA(cudaStreamSynchronize(s));
  if (bad) return fail(ACE_ERR_ARG, "deleting points that were not inserted (a count would go below zero)");
  {
    PhaseScope ps(h, ACE_PHASE_OTHER, s);
    e = ace::launch_delete_apply(h->hist, h->counts, total, h->num_sms, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "deletion launch");
  h->n_ins -= static_cast<uint64_t>(n);
  return ACE_OK;
}

int ace_batch_insert_score(const ace_handle* dets, int count, const void* const* X_dev, const int64_t* n, int dtype,
                           double alpha, double* const* scores_dev, uint32_t* const* sums_dev,
                           uint8_t* const* flags_dev, void* stream) {
  if (!dets || !X_dev || !n || count < 1) return fail(ACE_ERR_ARG, "invalid batch arguments");
  if (!std::isfinite(alpha)) return fail(ACE_ERR_ARG, "alpha must be finite");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool id16 = dets[0] && dets[0]->K <= 16;
  std::vector<ace_handle> seen(dets, dets + count);
  std::sort(seen.begin(), seen.end());
  if (std::adjacent_find(seen.begin(), seen.end()) != seen.end())
    return fail(ACE_ERR_ARG, "a detector appears twice in one batch");
  for (int g = 0; g < count; ++g) {
    ace_handle h = dets[g];
    if (int rc = check_x(h, X_dev[g], n[g], dtype)) return rc;
    if ((h->K <= 16) != id16) return fail(ACE_ERR_ARG, "a batch mixes K <= 16 and K > 16");
    if (h->ring) return fail(ACE_ERR_ARG, "detector %d has a window (not supported in batches)", g);
    if (h->n_ins + static_cast<uint64_t>(n[g]) > 0xFFFFFFFFull)
      return fail(ACE_ERR_OVERFLOW, "detector %d: inserting %lld points would allow a count above 2^32-1", g,
                  static_cast<long long>(n[g]));
  }
  // per detector: scratch, hash arguments (SIMT engine, ids stored and counts incremented, the
  // tile the autotuner picked for its shape) and its query job; then the item prefixes of the
  // persistent launch
  std::vector<ace::HashArgs> ha(count);
  std::vector<ace::ScoreJob> sj(count);
  std::vector<long long> hstart(count + 1, 0), sstart(count + 1, 0);
  for (int g = 0; g < count; ++g) {
    ace_handle h = dets[g];
    const long long ng = n[g];
    uint32_t* sum_out = sums_dev ? sums_dev[g] : nullptr;
    if (ng > 0) {
      if (int rc = grow(&h->ids, &h->ids_cap, static_cast<size_t>(ng) * h->L * id_bytes(h), s, "ids scratch")) return rc;
      if (!sum_out) {
        void* p = h->sums;
        if (int rc = grow(&p, &h->sums_cap, static_cast<size_t>(ng) * sizeof(uint32_t), s, "sums scratch")) return rc;
        h->sums = static_cast<uint32_t*>(p);
        sum_out = h->sums;
      }
    }
    ha[g] = hash_args(h, X_dev[g], ng, dtype, ace::kStoreIds | ace::kInsert);
    ha[g].tile = tuned_tile(h, X_dev[g], ng, dtype, s);
    if (ha[g].tile < 0) return ACE_ERR_CUDA;
    sj[g] = ace::ScoreJob{h->ids, ng, ng, h->K, h->L, alpha, h->counts, sum_out, h->st, h->div,
                          scores_dev ? scores_dev[g] : nullptr, flags_dev ? flags_dev[g] : nullptr};
    hstart[g + 1] = hstart[g] + ace::hash_simt_blocks(ha[g]);
    sstart[g + 1] = sstart[g] + (ng + 255) / 256;
  }
  // one device table: arguments, jobs, prefixes, then the dispensing counter and the
  // per-detector progress flags (zeroed)
  const size_t b_ha = sizeof(ace::HashArgs) * count, b_sj = sizeof(ace::ScoreJob) * count;
  const size_t b_st = sizeof(long long) * (count + 1);
  const size_t b_sync = 8 + sizeof(unsigned int) * 2 * static_cast<size_t>(count);
  std::vector<unsigned char> host(b_ha + b_sj + 2 * b_st + b_sync, 0);
  std::memcpy(host.data(), ha.data(), b_ha);
  std::memcpy(host.data() + b_ha, sj.data(), b_sj);
  std::memcpy(host.data() + b_ha + b_sj, hstart.data(), b_st);
  std::memcpy(host.data() + b_ha + b_sj + b_st, sstart.data(), b_st);
  unsigned char* dev = nullptr;
  ACE_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&dev), host.size(), s));
  cudaError_t e = cudaMemcpyAsync(dev, host.data(), host.size(), cudaMemcpyHostToDevice, s);
  const auto* d_ha = reinterpret_cast<const ace::HashArgs*>(dev);
  const auto* d_sj = reinterpret_cast<const ace::ScoreJob*>(dev + b_ha);
  const auto* d_hs = reinterpret_cast<const long long*>(dev + b_ha + b_sj);
  const auto* d_ss = reinterpret_cast<const long long*>(dev + b_ha + b_sj + b_st);
  auto* d_next = reinterpret_cast<unsigned long long*>(dev + b_ha + b_sj + 2 * b_st);
  auto* d_hdone = reinterpret_cast<unsigned int*>(dev + b_ha + b_sj + 2 * b_st + 8);
  auto* d_sready = d_hdone + count;
  const int sms = dets[0]->num_sms > 0 ? dets[0]->num_sms : 152;
  bool noisy = false;
  for (const auto& a : ha) noisy = noisy || a.nsig != 0.f;
  if (e == cudaSuccess) {
    ace_detector* h0 = dets[0];
    PhaseScope ps(h0, ACE_PHASE_HASH, s);  // the one launch (all phases of all detectors)
    e = ace::launch_batch(d_ha, d_sj, d_hs, d_ss, count, d_next, d_hdone, d_sready, dtype == ACE_BF16, id16, noisy, sms, s);
  }
  cudaFreeAsync(dev, s);
  if (e != cudaSuccess) return cuda_fail(e, "batched launch");
  for (int g = 0; g < count; ++g) {
    dets[g]->n_ins += static_cast<uint64_t>(n[g]);
    dets[g]->last_precision = ACE_PROJ_FP32;
    dets[g]->last_products = 0;
  }
  return ACE_OK;
}

int ace_project(ace_handle h, const void* X_dev, int64_t n, int dtype, float* proj_dev, void* stream) {
  int rc = check_x(h, X_dev, n, dtype);
  if (rc) return rc;
  if (n > 0 && !proj_dev) return fail(ACE_ERR_ARG, "proj_dev is NULL");
  if (n == 0) return ACE_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ace::HashArgs a = hash_args(h, X_dev, n, dtype, ace::kStoreProj);
  a.proj = proj_dev;
  cudaError_t e;
  const Engine eng = pick_engine(h, a.x_bf16, X_dev);
  if (eng == Engine::kStreaming) return run_gemm(h, a, s, false);
  if (eng == Engine::kSimt) {
    e = ace::launch_hash_simt(a, s);
  } else {
    const size_t cap = static_cast<size_t>(n) + 65536;
    void* p = h->defer;
    if ((rc = grow(&p, &h->defer_bytes, cap * 8, s, "deferred list"))) return rc;
    h->defer = static_cast<unsigned long long*>(p);
    ace::TcArgs t = h->tc;
    t.X = X_dev;
    t.x_bf16 = dtype == ACE_BF16;
    t.n = n;
    t.ntiles = (n + 127) / 128;
    const long long grid = std::min(static_cast<long long>(h->num_sms), t.ntiles);
    t.mode = ace::kStoreProj;
    t.ids = nullptr;
    t.ids_rm = nullptr;
    t.proj = proj_dev;
    t.defer = h->defer;
    t.seg_cap = h->defer_bytes / 8 / static_cast<size_t>(grid);
    e = ace::launch_hash_tc(t, h->num_sms, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "projection launch");
  return ACE_OK;
}

int ace_hash(ace_handle h, const void* X_dev, int64_t n, int dtype, uint32_t* ids_dev, void* stream) {
  int rc = check_x(h, X_dev, n, dtype);
  if (rc) return rc;
  if (n > 0 && !ids_dev) return fail(ACE_ERR_ARG, "ids_dev is NULL");
  if (n == 0) return ACE_OK;
  ace::HashArgs a = hash_args(h, X_dev, n, dtype, ace::kStoreIdsRowMajor);
  a.ids_rm = ids_dev;
  return run_hash(h, a, static_cast<cudaStream_t>(stream));
}

int ace_stats(ace_handle h, void* stream, ace_stats_t* out) {
  if (!h || !out) return fail(ACE_ERR_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ACE_CUDA(cudaMemsetAsync(h->st->Q, 0, sizeof(h->st->Q), s));
  cudaError_t e;
  {
    PhaseScope ps(h, ACE_PHASE_OTHER, s);
    e = ace::launch_sum_squares(h->counts, static_cast<long long>(count_elems(h)), h->st, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "sum of squares launch");
  ace::DevStats st;
  ACE_CUDA(cudaMemcpyAsync(&st, h->st, sizeof st, cudaMemcpyDeviceToHost, s));
  ACE_CUDA(cudaStreamSynchronize(s));
  std::memset(out, 0, sizeof *out);
  out->n_ins = h->n_ins;
  out->n_scored = st.n_scored;
  out->Q_lo = st.Q[0];
  out->Q_hi = st.Q[1];
  out->S1_lo = st.S1[0];
  out->S1_hi = st.S1[1];
  out->S2_lo = st.S2[0];
  out->S2_hi = st.S2[1];
  const u128 Q = (static_cast<u128>(st.Q[1]) << 64) | st.Q[0];
  out->mu_ins = h->n_ins ? static_cast<double>(Q) / (static_cast<double>(h->n_ins) * static_cast<double>(h->L)) : 0.0;
  // mu and sigma from the exact sums, the same binary64 steps as the flags kernel
  const u128 S1 = (static_cast<u128>(st.S1[1]) << 64) | st.S1[0];
  const u128 S2 = (static_cast<u128>(st.S2[1]) << 64) | st.S2[0];
  const uint64_t N = st.n_scored;
  if (N > 0 && (S2 == 0 || static_cast<u128>(N) <= (~static_cast<u128>(0)) / S2)) {
    const double NL = static_cast<double>(N) * static_cast<double>(h->L);
    out->mu = static_cast<double>(S1) / NL;
    out->sigma = std::sqrt(static_cast<double>(static_cast<u128>(N) * S2 - S1 * S1)) / NL;
  } else if (N > 0) {
    out->mu = out->sigma = std::nan("");
  }
  out->rechecks = st.rechecks;
  out->nonfinite_points = st.nonfinite;
  out->deferred = st.deferred;
  out->status = st.status;
  out->precision = h->last_precision;
  out->tc_products = h->last_products;
  return ACE_OK;
}

int ace_get_counts(ace_handle h, uint32_t* counts_host, void* stream) {
  if (!h || !counts_host) return fail(ACE_ERR_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ACE_CUDA(cudaMemcpyAsync(counts_host, h->counts, count_elems(h) * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  ACE_CUDA(cudaStreamSynchronize(s));
  return ACE_OK;
}

int ace_get_projection(ace_handle h, float* W_host) {
  if (!h || !W_host) return fail(ACE_ERR_ARG, "NULL argument");
  std::memcpy(W_host, h->Wh.data(), h->Wh.size() * sizeof(float));
  return ACE_OK;
}

// ---------------------------------------------------------------------------------------
// Checkpoint blob (ace_save / ace_load).  Little-endian, 8-byte fields:
//   "ACEDET01", version, d, K, L, flags (bit 0: W is bfloat16-valued), n_ins,
//   n_scored, S1 lo/hi, S2 lo/hi, rechecks, nonfinite, deferred, status, 0,
//   [version 2: the privacy noise's sigma (binary32 bits), noise seed, next noise index, 0,]
//   W (d*K*L binary32, row-major), counts (L*2^K uint32), FNV-1a 64 of everything before it.
// ace_save writes version 2; ace_load reads both.
// ---------------------------------------------------------------------------------------
namespace {
constexpr char kBlobMagic[8] = {'A', 'C', 'E', 'D', 'E', 'T', '0', '1'};
constexpr int kBlobHeaderWords1 = 16;  // after the magic, version 1
constexpr int kBlobHeaderWords = 20;   // version 2

uint64_t fnv1a64(const unsigned char* p, size_t n) {
  uint64_t h = 0xCBF29CE484222325ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 0x100000001B3ull;
  }
  return h;
}

size_t blob_bytes(int d, int K, int L, int words = kBlobHeaderWords) {
  return 8 + 8 * static_cast<size_t>(words) + static_cast<size_t>(d) * K * L * 4 +
         (static_cast<size_t>(1) << K) * L * 4 + 8;
}
}  // namespace

int ace_save_size(ace_handle h, size_t* bytes) {
  if (!h || !bytes) return fail(ACE_ERR_ARG, "NULL argument");
  *bytes = blob_bytes(h->d, h->K, h->L);
  return ACE_OK;
}

int ace_save(ace_handle h, void* buf, size_t cap, void* stream) {
  if (!h || !buf) return fail(ACE_ERR_ARG, "NULL argument");
  if (h->ring) return fail(ACE_ERR_ARG, "checkpoints of windowed detectors are not supported");
  const size_t need = blob_bytes(h->d, h->K, h->L);
  if (cap < need) return fail(ACE_ERR_ARG, "buffer of %zu bytes; the checkpoint needs %zu", cap, need);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* out = static_cast<unsigned char*>(buf);
  const size_t wbytes = static_cast<size_t>(h->d) * h->KL * 4, cbytes = count_elems(h) * 4;
  unsigned char* wdst = out + 8 + 8 * kBlobHeaderWords;
  ace::DevStats st;
  ACE_CUDA(cudaMemcpyAsync(&st, h->st, sizeof st, cudaMemcpyDeviceToHost, s));
  ACE_CUDA(cudaMemcpyAsync(wdst + wbytes, h->counts, cbytes, cudaMemcpyDeviceToHost, s));
  ACE_CUDA(cudaStreamSynchronize(s));
  bool wb = true;
  for (float w : h->Wh) wb = wb && bf16_value(bf16_rn(w)) == w;
  uint32_t nsig_bits;
  std::memcpy(&nsig_bits, &h->nsig, 4);
  uint64_t hdr[kBlobHeaderWords] = {2u,
                                    static_cast<uint64_t>(h->d),
                                    static_cast<uint64_t>(h->K),
                                    static_cast<uint64_t>(h->L),
                                    wb ? 1u : 0u,
                                    h->n_ins,
                                    st.n_scored,
                                    st.S1[0],
                                    st.S1[1],
                                    st.S2[0],
                                    st.S2[1],
                                    st.rechecks,
                                    st.nonfinite,
                                    st.deferred,
                                    st.status,
                                    0u,
                                    nsig_bits,
                                    h->nseed,
                                    h->nbase,
                                    0u};
  std::memcpy(out, kBlobMagic, 8);
  std::memcpy(out + 8, hdr, sizeof hdr);
  std::memcpy(wdst, h->Wh.data(), wbytes);
  const uint64_t sum = fnv1a64(out, need - 8);
  std::memcpy(out + need - 8, &sum, 8);
  return ACE_OK;
}

int ace_load(const void* buf, size_t bytes, ace_handle* out) {
  if (!buf || !out) return fail(ACE_ERR_ARG, "NULL argument");
  *out = nullptr;
  const unsigned char* in = static_cast<const unsigned char*>(buf);
  if (bytes < 8 + 8 * kBlobHeaderWords1 + 8 || std::memcmp(in, kBlobMagic, 8) != 0)
    return fail(ACE_ERR_ARG, "not an ACE checkpoint");
  uint64_t hdr[kBlobHeaderWords] = {};
  std::memcpy(hdr, in + 8, 8 * kBlobHeaderWords1);
  if (hdr[0] != 1u && hdr[0] != 2u)
    return fail(ACE_ERR_ARG, "checkpoint version %llu is not supported", static_cast<unsigned long long>(hdr[0]));
  const int words = hdr[0] == 1u ? kBlobHeaderWords1 : kBlobHeaderWords;
  if (words > kBlobHeaderWords1) {
    if (bytes < 8 + 8 * static_cast<size_t>(words) + 8) return fail(ACE_ERR_ARG, "checkpoint header truncated");
    std::memcpy(hdr, in + 8, 8 * static_cast<size_t>(words));
  }
  const uint64_t d = hdr[1], K = hdr[2], L = hdr[3];
  if (d < 1 || d > (1u << 30) || K < 1 || K > 24 || L < 1 || K * L > 65536)
    return fail(ACE_ERR_ARG, "checkpoint shape d=%llu K=%llu L=%llu is invalid", static_cast<unsigned long long>(d),
                static_cast<unsigned long long>(K), static_cast<unsigned long long>(L));
  const size_t need = blob_bytes(static_cast<int>(d), static_cast<int>(K), static_cast<int>(L), words);
  if (bytes != need) return fail(ACE_ERR_ARG, "checkpoint of %zu bytes; its shape needs %zu", bytes, need);
  float nsig = 0.f;
  if (words > kBlobHeaderWords1) {
    const uint32_t nb = static_cast<uint32_t>(hdr[16]);
    std::memcpy(&nsig, &nb, 4);
    if (!(nsig == 0.f || (nsig >= 0x1p-60f && nsig <= 0x1p60f)) || hdr[16] > 0xFFFFFFFFull)
      return fail(ACE_ERR_ARG, "checkpoint privacy sigma is invalid");
  }
  uint64_t sum;
  std::memcpy(&sum, in + need - 8, 8);
  if (sum != fnv1a64(in, need - 8)) return fail(ACE_ERR_ARG, "checkpoint checksum mismatch (corrupted blob)");
  const size_t wbytes = static_cast<size_t>(d) * K * L * 4;
  std::vector<float> W(static_cast<size_t>(d) * K * L);
  const size_t hbytes = 8 + 8 * static_cast<size_t>(words);
  std::memcpy(W.data(), in + hbytes, wbytes);
  ace_handle h = nullptr;
  if (int rc = make_detector(static_cast<int>(d), static_cast<int>(K), static_cast<int>(L), W.data(), 0, false, 0u, &h))
    return rc;
  ace::DevStats st{};
  st.n_scored = hdr[6];
  st.S1[0] = hdr[7];
  st.S1[1] = hdr[8];
  st.S2[0] = hdr[9];
  st.S2[1] = hdr[10];
  st.rechecks = hdr[11];
  st.nonfinite = hdr[12];
  st.deferred = hdr[13];
  st.status = static_cast<unsigned int>(hdr[14]);
  cudaError_t e = cudaMemcpy(h->counts, in + hbytes + wbytes, count_elems(h) * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->st, &st, sizeof st, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    ace_destroy(h);
    return cuda_fail(e, "checkpoint upload");
  }
  h->n_ins = hdr[5];
  h->nsig = nsig;
  h->nseed = nsig != 0.f ? hdr[17] : 0u;
  h->nbase = nsig != 0.f ? hdr[18] : 0u;
  *out = h;
  return ACE_OK;
}

int ace_get_shape(ace_handle h, int* d, int* K, int* L) {
  if (!h) return fail(ACE_ERR_ARG, "handle is NULL");
  if (d) *d = h->d;
  if (K) *K = h->K;
  if (L) *L = h->L;
  return ACE_OK;
}

int ace_profile_enable(ace_handle h, int enable) {
  if (!h) return fail(ACE_ERR_ARG, "handle is NULL");
  h->prof = enable != 0;
  return ACE_OK;
}

int ace_profile_phases(ace_handle h, unsigned mask) {
  if (!h) return fail(ACE_ERR_ARG, "handle is NULL");
  h->prof_mask = mask ? mask : ~0u;
  return ACE_OK;
}

int ace_profile_read(ace_handle h, ace_profile_t* out) {
  if (!h || !out) return fail(ACE_ERR_ARG, "NULL argument");
  std::memset(out, 0, sizeof *out);
  for (int p = 0; p < ACE_NPHASE; ++p) out->launches[p] = h->launches[p];
  int rc = ACE_OK;
  for (auto& m : h->marks) {
    float ms = 0.f;
    cudaError_t e = cudaEventSynchronize(m.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, m.a, m.b);
    if (e != cudaSuccess && rc == ACE_OK) rc = cuda_fail(e, "profile event");
    out->ms[m.phase] += ms;
    out->timed[m.phase] += 1;
    h->pool.push_back(m.a);
    h->pool.push_back(m.b);
  }
  h->marks.clear();
  for (int p = 0; p < ACE_NPHASE; ++p) h->launches[p] = 0;
  return rc;
}

int ace_batch_tile(int d, int K, int L, int dtype, int* points, int* columns) {
  if (!points || !columns) return fail(ACE_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(tune_key(d, K, L, dtype));
  if (it == g_tune.end()) {
    *points = *columns = 0;
    return ACE_OK;
  }
  *points = 16 * ace::simt_tile_rows(it->second);
  *columns = 16 * ace::simt_tile_cols(it->second);
  return ACE_OK;
}

namespace {
int tc_probe_any(const void* A_host, const void* B_host, int kdim, int ncols, float* D_host, bool fp8) {
  if (!A_host || !B_host || !D_host) return fail(ACE_ERR_ARG, "NULL argument");
  const int kq = fp8 ? 32 : 16;
  if (kdim < kq || kdim > 256 || kdim % kq || ncols < 16 || ncols > 256 || ncols % 16)
    return fail(ACE_ERR_ARG, "kdim must be a multiple of %d and ncols of 16, both in [%d, 256] (got %d, %d)", kq, kq,
                kdim, ncols);
  int dev = 0;
  ACE_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp p;
  ACE_CUDA(cudaGetDeviceProperties(&p, dev));
  if (p.major != 10 || p.minor != 3) return fail(ACE_ERR_UNSUPPORTED, "the tensor-core probe needs an sm_103 device");
  const size_t eb = fp8 ? 1 : 2;
  const size_t ab = static_cast<size_t>(128) * kdim * eb, bb = static_cast<size_t>(ncols) * kdim * eb;
  const size_t db = static_cast<size_t>(128) * ncols * 4;
  unsigned char* buf = nullptr;
  ACE_CUDA(cudaMalloc(&buf, ab + bb + db + 16));
  unsigned char* A = buf;
  unsigned char* B = buf + ab;
  float* D = reinterpret_cast<float*>(buf + ab + bb);
  int* status = reinterpret_cast<int*>(buf + ab + bb + db);
  cudaError_t e = cudaMemcpy(A, A_host, ab, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(B, B_host, bb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(status, 0, sizeof(int));
  if (e == cudaSuccess) e = ace::launch_tc_probe(A, B, kdim, ncols, fp8, D, status, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int st = 0;
  if (e == cudaSuccess) e = cudaMemcpy(D_host, D, db, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&st, status, sizeof st, cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core probe");
  if (st) return fail(ACE_ERR_TIMEOUT, "tensor-core probe: the MMA completion wait gave up");
  return ACE_OK;
}
}  // namespace

int ace_exact_score(const void* Q_dev, int64_t nq, const void* D_dev, int64_t nd, int d, int dtype, int K,
                    double* S_dev, void* stream) {
  if (nq < 0 || nd < 0) return fail(ACE_ERR_ARG, "nq and nd must be >= 0");
  if (nq == 0) return ACE_OK;
  if (!Q_dev || !S_dev || (nd > 0 && !D_dev)) return fail(ACE_ERR_ARG, "NULL argument");
  if (d < 1 || K < 1 || K > 64) return fail(ACE_ERR_ARG, "need d >= 1 and 1 <= K <= 64 (got d=%d K=%d)", d, K);
  if (dtype != ACE_F32 && dtype != ACE_BF16) return fail(ACE_ERR_ARG, "unknown dtype %d", dtype);
  if (nq > 65535) return fail(ACE_ERR_ARG, "at most 65535 queries per call (got %lld)", static_cast<long long>(nq));
  if (nd > (1LL << 38)) return fail(ACE_ERR_ARG, "nd too large");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* part = nullptr;
  const size_t bytes = std::max<size_t>(ace::exact_score_scratch(nq, nd), 8);
  cudaError_t e = cudaMalloc(&part, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ACE_ERR_OOM, "exact score scratch: %s", cudaGetErrorString(e));
  }
  e = ace::launch_exact_score(Q_dev, nq, D_dev, nd, d, dtype == ACE_BF16 ? 1 : 0, K, static_cast<double*>(part),
                              S_dev, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(part);
  if (e != cudaSuccess) return cuda_fail(e, "exact score");
  return ACE_OK;
}

int ace_wait_probe(int kind, int64_t limit_cycles, uint32_t* status, int64_t* cycles_out) {
  if (!status || (kind != 0 && kind != 1) || limit_cycles < 100000 || limit_cycles > 1000000000)
    return fail(ACE_ERR_ARG, "kind must be 0 or 1, limit_cycles in [1e5, 1e9] and status non-NULL");
  int dev = 0;
  ACE_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp p;
  ACE_CUDA(cudaGetDeviceProperties(&p, dev));
  if (kind == 0 && (p.major != 10 || p.minor != 3))
    return fail(ACE_ERR_UNSUPPORTED, "the tensor-core wait probe needs an sm_103 device");
  unsigned char* buf = nullptr;
  const size_t bytes = 16 + sizeof(ace::DevStats) + 2 * sizeof(long long);
  ACE_CUDA(cudaMalloc(&buf, bytes));
  unsigned int* flag = reinterpret_cast<unsigned int*>(buf);
  auto* st = reinterpret_cast<ace::DevStats*>(buf + 16);
  auto* cyc = reinterpret_cast<long long*>(buf + 16 + sizeof(ace::DevStats));
  cudaError_t e = cudaMemset(buf, 0, bytes);
  if (e == cudaSuccess) e = ace::launch_wait_probe(kind, limit_cycles, flag, st, cyc, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  ace::DevStats hs{};
  long long hc[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpy(&hs, st, sizeof hs, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(hc, cyc, sizeof hc, cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "wait probe");
  *status = hs.status;
  if (cycles_out) {
    cycles_out[0] = hc[0];
    cycles_out[1] = hc[1];
  }
  return ACE_OK;
}

int ace_tc_probe(const uint16_t* A_host, const uint16_t* B_host, int kdim, int ncols, float* D_host) {
  return tc_probe_any(A_host, B_host, kdim, ncols, D_host, false);
}

int ace_tc_probe_fp8(const uint8_t* A_host, const uint8_t* B_host, int kdim, int ncols, float* D_host) {
  return tc_probe_any(A_host, B_host, kdim, ncols, D_host, true);
}

const char* ace_last_error(void) { return g_err.c_str(); }

const char* ace_version(void) { return "ace-gb300 0.1 (sm_103a)"; }

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Allocation-free variant of ace_insert_score (for callers that cannot call cudaMalloc).
//
// The scratch is a file-scope device array.  Host code may not use the array's name as a
// device address (on the host it is only a stand-in), so its real address is looked up
// once per device with cudaGetSymbolAddress while that device is current, and that
// pointer is what the kernels receive.
// ---------------------------------------------------------------------------------------
#include <mutex>

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[ACE_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch on `device` (looked up on first use, with that device
// current; the previously current device is restored).
int noalloc_scratch(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return fail(ACE_ERR_ARG, "device %d out of range", device);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    int cur = -1;
    ACE_CUDA(cudaGetDevice(&cur));
    if (cur != device) ACE_CUDA(cudaSetDevice(device));
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (cur != device) cudaSetDevice(cur);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    if (!p) return fail(ACE_ERR_CUDA, "scratch has no device address");
    g_noalloc_ptr[device] = p;
  }
  *out = g_noalloc_ptr[device];
  return ACE_OK;
}

}  // namespace

extern "C" int ace_insert_score_noalloc(ace_handle h, const void* X_dev, int64_t n, int dtype, double alpha,
                                        double* scores_dev, uint32_t* sums_dev, uint8_t* flags_dev, void* stream) {
  int rc = check_x(h, X_dev, n, dtype);
  if (rc) return rc;
  if (!std::isfinite(alpha)) return fail(ACE_ERR_ARG, "alpha must be finite");
  if (h->ring) return fail(ACE_ERR_ARG, "a windowed detector is not supported by the allocation-free entry point");
  if (h->n_ins + static_cast<uint64_t>(n) > 0xFFFFFFFFull)
    return fail(ACE_ERR_OVERFLOW, "inserting %lld points would allow a count above 2^32-1", static_cast<long long>(n));
  const size_t ids_bytes = (static_cast<size_t>(n) * h->L * id_bytes(h) + 255) & ~static_cast<size_t>(255);
  const size_t need = ids_bytes + (sums_dev ? 0 : static_cast<size_t>(n) * sizeof(uint32_t));
  if (need > ACE_NOALLOC_SCRATCH_BYTES)
    return fail(ACE_ERR_ARG,
                "batch of %lld points needs %zu bytes of scratch; the static scratch holds %u bytes "
                "(split the batch)",
                static_cast<long long>(n), need, static_cast<unsigned>(ACE_NOALLOC_SCRATCH_BYTES));
  if (n == 0) return ACE_OK;
  void* base = nullptr;
  if ((rc = noalloc_scratch(h->device, &base))) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* ids = base;
  uint32_t* sum_out = sums_dev ? sums_dev : reinterpret_cast<uint32_t*>(static_cast<unsigned char*>(base) + ids_bytes);
  ace::HashArgs a = hash_args(h, X_dev, n, dtype, ace::kStoreIds | ace::kInsert);
  a.ids = ids;
  a.ld = n;
  h->last_precision = ACE_PROJ_FP32;
  // each launch is counted, and bracketed by events while the timing hook is on (the events
  // come from the handle's pool; no device memory is allocated)
  cudaError_t e;
  {
    PhaseScope ps(h, ACE_PHASE_HASH, s);
    e = ace::launch_hash_simt(a, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "hash kernel launch");
  h->n_ins += static_cast<uint64_t>(n);
  {
    PhaseScope ps(h, ACE_PHASE_SCORE, s);
    e = ace::launch_score_gather(ids, h->K <= 16, n, n, h->K, h->L, alpha, h->counts, sum_out, h->st, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "score kernel launch");
  {
    PhaseScope ps(h, ACE_PHASE_FLAGS, s);
    e = ace::launch_flags(sum_out, n, h->div, h->st, scores_dev, flags_dev, s);
  }
  if (e != cudaSuccess) return cuda_fail(e, "flags kernel launch");
  return ACE_OK;
}
