// SRP hashing on the tcgen05 tensor cores (BF16 operands, FP32 accumulators in TMEM).
//
// Projection (Eq. 1) of a 128-point tile onto a chunk of whole tables (floor(256/K) tables,
// N <= 256 columns) as three BF16 products accumulated in one TMEM accumulator:
//     x.w'  ~  x_hi.w'_hi + x_hi.w'_lo + x_lo.w'_hi
// where x_hi = bf16(x), x_lo = bf16(x - x_hi), and w' = w_c / ||w_c|| (unit columns, so the
// guard bound is one number per point) split the same way on the host.  The sign of x.w'
// is the sign of x.w_c.  Error bound relative to ||x|| (all terms rigorous; see the host
// constants in ace_abi.cu):
//   - split: the dropped terms x_lo w_lo + (x - x_hi - x_lo) w' + x (w' - w_hi - w_lo) are at
//     most 3 u^2 |x_i w'_i| per term, u = 2^-8 (bfloat16 unit roundoff);
//   - accumulation: tcgen05 aligns the 17 addends of one MMA instruction (16 products and
//     the accumulator) to the largest exponent keeping two bits below its last place, and
//     truncates the sum to binary32, i.e. at most 5.25 * 2^-23 * (sum of |addends|) per
//     instruction.  The two small products go first: their instructions see addends of at
//     most about 2^-7 sum |x_i w'_i|, the last product's at most about sum |x_i w'_i|, so
//     over S_small + S_big instructions at most 5.25 * 2^-23 * (S_big + 1 + 2^-6 S_small)
//     * sum |x_i w'_i| (a 1.5x margin is applied);
//   - normalisation: w' is w_c / ||w_c|| rounded to binary32 elementwise (2^-24);
//   - the binary64 reference itself (gamma64_d).
// A (point, table) pair with a projection inside the bound on some column is appended to a
// deferred list; recheck_kernel recomputes that table's K bits exactly (binary32 with the
// SIMT bound, binary64 inside it) and stores the final id, so every id equals the binary64
// definition.
//
// Roles (one CTA per SM, persistent over 128-point tiles):
//   warp 0       TMEM allocation, B image load (resident W'), MMA issue (one lane)
//   warps 1-4    converters: X tile bulk-copied into a staging buffer (TMA engine), one
//                row per thread -> bf16 hi/lo operand images + per-row bound
//   warps 5-12   epilogue, two groups alternating TMEM buffers: tcgen05.ld, guard
//                classification, streaming bit packing, id store, deferral of ambiguous
//                tables to this CTA's segment of the deferred list
// The count increments (Algorithm 1 counting phase) run afterwards in insert_hist_kernel,
// from the stored ids, with per-table shared-memory histograms.
#include "guard.cuh"
#include "tc_ptx.cuh"
#include "tc_plan.h"

#include <type_traits>
#include "launch_cache.h"

namespace ace {
namespace {

using namespace tc;

constexpr int kBufs = kTcBufs;        // TMEM accumulator buffers, one epilogue group each
constexpr int kBufCols = kTcBufCols;  // largest chunk N
constexpr int kThreads = 32 * (5 + 4 * kBufs);  // MMA, 4 converters, kBufs x 4 epilogue warps
constexpr int kConv0 = 32;     // first converter thread
constexpr int kEpi0 = 160;     // first epilogue thread
constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz

struct Smem {
  uint64_t st_full;
  uint64_t b_full;
  uint64_t drain;
  uint64_t a_full[2], a_empty[2];
  uint64_t bnd_full[2], bnd_empty[2];
  uint64_t t_full[kBufs], t_empty[kBufs];
  uint32_t taddr;
  int abort;
  unsigned int ndef;  // entries in this CTA's deferred segment
};

__device__ __forceinline__ void set_abort(Smem* S, DevStats* st) {
  S->abort = 1;
  atomicOr(&st->status, static_cast<unsigned>(ACE_STATUS_TIMEOUT));
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Named barrier 1 over the 128 converter threads, returning the OR of `v` over them (so a
// decision to stop is the same in every converter thread).
__device__ __forceinline__ bool conv_bar_or(bool v) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 1, 128, p;\n\tselp.u32 %0, 1, 0, q;\n}"
      : "=r"(out)
      : "r"(static_cast<uint32_t>(v))
      : "memory");
  return out != 0;
}

template <bool BF16>
__device__ __forceinline__ float xval(const void* p, long long idx) {
  if constexpr (BF16) return __uint_as_float(static_cast<unsigned>(reinterpret_cast<const unsigned short*>(p)[idx]) << 16);
  else return reinterpret_cast<const float*>(p)[idx];
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);  // .x = a (low half), .y = b
  return *reinterpret_cast<const uint32_t*>(&v);
}

// The exact bucket id of table j for point i, for the rare path where a CTA's deferred list
// is full: each of the K projections in binary32 with the SIMT engine's bound, binary64
// (the definition) when inside it.
template <bool BF16>
__device__ __noinline__ uint32_t exact_table_id(const void* X, long long i, int d, int K, int j, const float* Wt,
                                                const float* cB32, float xfac32, float xabs32, float babs32,
                                                DevStats* st) {
  float q = 0.f;
  for (int t = 0; t < d; ++t) {
    const float x = load_x<BF16>(X, i * d + t);
    q = fmaf(x, x, q);
  }
  const float xu = norm_upper(q, xfac32, xabs32);
  uint32_t id = 0u;
  for (int k = 0; k < K; ++k) {
    const int col = j * K + k;
    const float* wc = Wt + static_cast<size_t>(col) * d;
    float s32 = 0.f;
    for (int t = 0; t < d; ++t) s32 = fmaf(load_x<BF16>(X, i * d + t), __ldg(wc + t), s32);
    bool bit;
    if (fabsf(s32) > fmaf(__ldg(cB32 + col), xu, babs32)) bit = s32 > 0.f;
    else bit = exact_bit<BF16>(X, i, d, Wt, col);
    id |= (bit ? 1u : 0u) << k;
  }
  atomicAdd(&st->rechecks, static_cast<unsigned long long>(K));
  return id;
}

// KC > 0: the kernel is specialised for K = KC (the table offsets inside a chunk are then
// compile-time constants and the pack is a fully unrolled, branch-free sequence); KC = 0
// handles any K with a streaming extractor.
template <bool BF16, typename IdT, int KC, bool PROJ = false>
__global__ void __launch_bounds__(kThreads, 1) hash_tc_kernel(const __grid_constant__ TcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* Bimg = smem;
  uint8_t* stage = smem + a.off_stage;
  // A stage s: hi image at off_a + 2 s a_bytes, lo image right after it
  auto a_hi = [&](int st) { return smem + a.off_a + 2 * st * a.a_bytes; };
  auto a_lo = [&](int st) { return smem + a.off_a + (2 * st + 1) * a.a_bytes; };
  float* bnd = reinterpret_cast<float*>(smem + a.off_bnd);          // [2][128]
  Smem* S = reinterpret_cast<Smem*>(smem + a.off_ctl);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long ntiles = a.ntiles;

  if (tid == 0) {
    S->abort = 0;
    S->ndef = 0;
    mbar_init(&S->st_full, 1);
    mbar_init(&S->b_full, 1);
    mbar_init(&S->drain, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(&S->a_full[s], 128);
      mbar_init(&S->a_empty[s], 1);
      mbar_init(&S->bnd_full[s], 128);
      mbar_init(&S->bnd_empty[s], 128 * kBufs);
    }
    for (int b = 0; b < kBufs; ++b) {
      mbar_init(&S->t_full[b], 1);
      mbar_init(&S->t_empty[b], 128);
    }
    mbar_fence_init();
  }
  // zero both A stages once: the padding columns k >= d are never written again
  for (int i = tid; i < a.a_bytes; i += kThreads) {
    a_hi(0)[i] = 0;
    a_lo(0)[i] = 0;
    a_hi(1)[i] = 0;
    a_lo(1)[i] = 0;
  }
  fence_proxy_async();
  if (warp == 0) {
    tmem_alloc(&S->taddr, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S->taddr;

  if (warp == 0) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      mbar_expect_tx(&S->b_full, static_cast<uint32_t>(a.bimg_bytes));
      for (int off = 0; off < a.bimg_bytes; off += 32768) {
        const int sz = min(32768, a.bimg_bytes - off);
        bulk_g2s(Bimg + off, a.bimg + off, static_cast<uint32_t>(sz), &S->b_full);
      }
      bool ok = mbar_wait(&S->b_full, 0, &S->abort, kWaitCycles);
      if (!ok) set_abort(S, a.st);
      const uint32_t a_sbo = static_cast<uint32_t>(a.d_pad) * 16u;
      const int ksteps = a.d_pad / 16;
      long long item = 0;
      int tl = 0;
      for (long long m = blockIdx.x; ok && m < ntiles; m += gridDim.x, ++tl) {
        const int s = tl & 1;
        if (!mbar_wait(&S->a_full[s], (tl >> 1) & 1, &S->abort, kWaitCycles)) { ok = false; set_abort(S, a.st); break; }
        tc_fence_after();
        const uint32_t ahi = smem_u32(a_hi(s)), alo = smem_u32(a_lo(s));
        for (int c = 0; c < a.nchunks; ++c, ++item) {
          const int b = static_cast<int>(item % kBufs);
          if (item >= kBufs && !mbar_wait(&S->t_empty[b], ((item / kBufs) + 1) & 1, &S->abort, kWaitCycles)) {
            ok = false;
            set_abort(S, a.st);
            break;
          }
          tc_fence_after();
          const TcChunk& ch = a.chunk[c];
          const uint32_t idesc = idesc_bf16(128, ch.N);
          const uint32_t bhi = smem_u32(Bimg) + ch.boff_hi, blo = smem_u32(Bimg) + ch.boff_lo;
          const uint32_t dt = tmem + static_cast<uint32_t>(b * kBufCols);
          uint32_t acc = 0;
          // x_hi . w_lo and x_lo . w_hi first, x_hi . w_hi last: while the small products
          // accumulate, the accumulator stays small, and so does the accumulation error (the
          // guard band on the host counts only the last product's instructions at full size)
          for (int p = 0; p < 3; ++p) {
            const uint32_t as = (p == 1) ? alo : ahi;
            const uint32_t bs = (p == 0) ? blo : bhi;
            for (int k = 0; k < ksteps; ++k) {
              mma_bf16(dt, smem_desc(as + 256u * k, 128, a_sbo), smem_desc(bs + 256u * k, 128, a_sbo), idesc, acc);
              acc = 1;
            }
          }
          mma_commit(&S->t_full[b]);
        }
        if (!ok) break;
        mma_commit(&S->a_empty[s]);
      }
      // drain: every MMA this thread issued has completed before TMEM is released
      // (bounded by time only)
      const int never = 0;
      mma_commit(&S->drain);
      if (!mbar_wait(&S->drain, 0, &never, kWaitCycles)) set_abort(S, a.st);
    }
    __syncwarp();
  } else if (warp >= 1 && warp <= 4) {
    // ------------------------------------------------------------------ converters
    // Tiles arrive in a staging buffer by bulk copy (the TMA engine); thread r converts row r
    // of the tile into its bfloat16 hi/lo operand rows (16-byte stores) and derives the row's
    // bound.  The tail tile (and an unaligned X) is read with plain loads instead.
    const int r = tid - kConv0;
    const int d = a.d, d_pad = a.d_pad;
    const long long n = a.n;
    const void* const X = a.X;
    const float tau = a.tau, tau_abs = a.tau_abs, xfac = a.xfac, qmin = a.qmin;
    DevStats* const st = a.st;
    const bool aligned = (reinterpret_cast<uintptr_t>(X) & 15u) == 0;
    const uint32_t tile_bytes = static_cast<uint32_t>(128) * d * (BF16 ? 2 : 4);
    auto full_tile = [&](long long m) { return aligned && (m + 1) * 128 <= n; };
    auto issue_copy = [&](long long m) {
      mbar_expect_tx(&S->st_full, tile_bytes);
      bulk_g2s(stage, static_cast<const uint8_t*>(X) + static_cast<size_t>(m) * tile_bytes, tile_bytes, &S->st_full);
    };
    int staged = 0;        // staging phases consumed
    bool pending = false;  // (r == 0) a copy is in flight
    if (r == 0 && blockIdx.x < ntiles && full_tile(blockIdx.x)) {
      pending = true;
      issue_copy(blockIdx.x);
    }
    // Odd d: rows of the staging buffer sit d words apart, an odd stride, so thread r reading
    // its own row is free of bank conflicts; the whole row is read into registers first (the
    // compiler cannot move a later load of the staging buffer above an earlier store to the A
    // stage, so reading while converting would serialise the groups), and the next tile's
    // copy is issued as soon as every converter has read the buffer, overlapping the
    // conversion.  Even d: the group order is rotated across rows (banks) and the buffer is
    // read group by group while converting.
    const bool odd = (d & 1) != 0;
    const int ngrp = d_pad / 8;
    const int rot = odd ? 0 : r % ngrp;
    const float* const stagef = reinterpret_cast<const float*>(stage);
    const unsigned short* const stageh = reinterpret_cast<const unsigned short*>(stage);
    auto staged_x = [&](int k) {
      return BF16 ? __uint_as_float(static_cast<unsigned>(stageh[r * d + k]) << 16) : stagef[r * d + k];
    };
    // hi = bf16(v), lo = bf16(v - hi) for a pair, as two packed bfloat16x2 words
    auto split2 = [](float v0, float v1, uint32_t& hi, uint32_t& lo) {
      hi = pack_bf16x2(v0, v1);
      const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xFFFF0000u);
      lo = pack_bf16x2(v0 - h0, v1 - h1);
    };
    int tl = 0;
    for (long long m = blockIdx.x; m < ntiles; m += gridDim.x, ++tl) {
      const int s = tl & 1;
      const bool full = full_tile(m);
      const long long i = m * 128 + r;
      const bool valid = i < n;
      const long long mn = m + gridDim.x;
      bool ok = S->abort == 0;
      if (ok && full) {
        if (mbar_wait(&S->st_full, staged & 1, &S->abort, kWaitCycles)) {
          ++staged;
          if (r == 0) pending = false;
        } else {
          ok = false;
          set_abort(S, a.st);
        }
      }
      float xr[kMaxD];
      if (odd) {
        if (conv_bar_or(!ok)) break;
#pragma unroll
        for (int k = 0; k < kMaxD; ++k) xr[k] = 0.f;
        if (valid) {
          if (full) {
#pragma unroll
            for (int k = 0; k < kMaxD; ++k)
              if (k < d) xr[k] = staged_x(k);
          } else {
#pragma unroll
            for (int k = 0; k < kMaxD; ++k)
              if (k < d) xr[k] = xval<BF16>(X, i * d + k);
          }
        }
        conv_bar_or(false);  // every converter has read the staging buffer
        if (r == 0 && mn < ntiles && full_tile(mn)) {
          pending = true;
          issue_copy(mn);
        }
      }
      if (ok && tl >= 2) {
        if (!mbar_wait(&S->a_empty[s], ((tl >> 1) + 1) & 1, &S->abort, kWaitCycles) ||
            !mbar_wait(&S->bnd_empty[s], ((tl >> 1) + 1) & 1, &S->abort, kWaitCycles)) {
          ok = false;
          set_abort(S, a.st);
        }
      }
      // every converter reaches the barrier; stopping is decided for all of them at once
      if (conv_bar_or(!ok)) break;
      float q = 0.f;
      if (odd) {
#pragma unroll
        for (int k = 0; k < kMaxD; ++k) q = fmaf(xr[k], xr[k], q);
#pragma unroll
        for (int g = 0; g < kMaxD / 8; ++g) {
          if (g < ngrp) {
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) split2(xr[8 * g + 2 * e], xr[8 * g + 2 * e + 1], hi[e], lo[e]);
            const uint32_t off = kmajor_offset(r, g * 8, d_pad);
            *reinterpret_cast<uint4*>(a_hi(s) + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4*>(a_lo(s) + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
          }
        }
      } else {
        for (int gi = 0; gi < ngrp; ++gi) {
          int g = gi + rot;
          if (g >= ngrp) g -= ngrp;
          float v[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int k = g * 8 + e;
            float x = 0.f;
            if (valid && k < d) x = full ? staged_x(k) : xval<BF16>(X, i * d + k);
            v[e] = x;
            q = fmaf(x, x, q);
          }
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) split2(v[2 * e], v[2 * e + 1], hi[e], lo[e]);
          const uint32_t off = kmajor_offset(r, g * 8, d_pad);
          *reinterpret_cast<uint4*>(a_hi(s) + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<uint4*>(a_lo(s) + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
      }
      // row bound: tau * ||x||_up + tau_abs; +inf makes every column of the row a recheck
      float B;
      if (!isfinite(q) || q < qmin) B = __int_as_float(0x7f800000);
      else B = fmaf(tau, sqrtf(q * xfac) * 1.00000095367431640625f, tau_abs);
      bnd[s * 128 + r] = B;
      if (valid && !isfinite(q) && !(a.mode & kStoreProj)) atomicAdd(&st->nonfinite, 1ull);
      fence_proxy_async();
      mbar_arrive(&S->a_full[s]);
      mbar_arrive(&S->bnd_full[s]);
      if (!odd) {
        conv_bar_or(false);  // every converter is done with the staging buffer
        if (r == 0 && mn < ntiles && full_tile(mn)) {
          pending = true;
          issue_copy(mn);
        }
      }
    }
    // leave no bulk copy in flight (bounded wait that ignores the abort flag)
    if (r == 0 && pending) {
      const int never = 0;
      mbar_wait(&S->st_full, staged & 1, &never, kWaitCycles);
    }
  } else {
    // ------------------------------------------------------------------ epilogue
    // Two groups of four warps; group wg takes the work items whose TMEM buffer is wg.
    // Every parameter is copied into registers first: the loop stores to global memory, and
    // a field re-read from the parameter block after each store would cost a load each time.
    const int et = tid - kEpi0;
    const int wg = et >> 7;
    const int q4 = warp & 3;
    const int r = q4 * 32 + lane;  // TMEM lane = tile row
    const int K = KC > 0 ? KC : a.K;
    const int L = a.L, mode = a.mode, nch = a.nchunks, d = a.d;
    const bool st_tm = (mode & kStoreIds) != 0, st_rm = (mode & kStoreIdsRowMajor) != 0;
    const uint32_t tag = (mode & kTagDeferred) ? 0x8000u : 0u;  // 16-bit ids only
    const int tpc = min(kBufCols / K, 32);  // tables per chunk (the host plans chunks the same way)
    const long long n = a.n, ld = a.ld;
    IdT* const ids = reinterpret_cast<IdT*>(a.ids);
    uint32_t* const ids_rm = a.ids_rm;
    const unsigned long long seg_cap = a.seg_cap;
    const void* const X = a.X;
    const float* const Wt = a.Wt;
    const float* const cB32 = a.cB32;
    const float xfac32 = a.xfac32, xabs32 = a.xabs32, babs32 = a.babs32;
    DevStats* const st = a.st;
    const uint32_t kmask = (1u << K) - 1u;
    unsigned long long* seg = a.defer + seg_cap * blockIdx.x;
    long long item = 0;
    int tl = 0;
    bool ok = true;
    for (long long m = blockIdx.x; ok && m < ntiles; m += gridDim.x, ++tl) {
      const int s = tl & 1;
      ok = mbar_wait(&S->bnd_full[s], (tl >> 1) & 1, &S->abort, kWaitCycles);
      if (!__all_sync(0xFFFFFFFFu, ok)) {
        ok = false;
        set_abort(S, st);
        break;
      }
      const float B = bnd[s * 128 + r];
      mbar_arrive(&S->bnd_empty[s]);
      const long long i = m * 128 + r;
      const bool valid = i < n;
      for (int c = 0; c < nch; ++c, ++item) {
        const int b = static_cast<int>(item % kBufs);
        if (b != wg) continue;
        ok = mbar_wait(&S->t_full[b], (item / kBufs) & 1, &S->abort, kWaitCycles);
        if (!__all_sync(0xFFFFFFFFu, ok)) {
          ok = false;
          set_abort(S, st);
          break;
        }
        tc_fence_after();
        const int tab0 = c * tpc;
        const int ntab = min(tpc, L - tab0);
        const int ncols = ntab * K;
        const int ng = (ncols + 31) >> 5;
        const uint32_t tbase = tmem + (static_cast<uint32_t>(q4 * 32) << 16) + static_cast<uint32_t>(b * kBufCols);
        // Classify the chunk's columns.  bw[g] bit k = [column 32g+k > 0].  A table with any
        // column inside the bound (|projection| <= B, compared on bit patterns: both are
        // non-negative floats; Bi = all ones for a row whose bound is +inf, so that row is
        // deferred whatever the minimum, NaN included) is deferred whole to the recheck
        // kernel.  Columns come from TMEM 64 at a time, each load waited for at once: fewer,
        // larger loads measured faster than double-buffered 32-column loads, and overlapping
        // the loads with the classification (or handing the buffer back before the last
        // columns are classified) measured no faster.  Signs are packed by four independent
        // funnel-shift chains.
        const uint32_t Bi = isinf(B) ? 0xFFFFFFFFu : __float_as_uint(B);
        constexpr int NG = kBufCols / 32;  // 32-column groups of a buffer
        uint32_t bw[NG];
        uint32_t defmask = 0u;  // bit t: table t of the chunk has a column inside the bound
        constexpr int TPC = KC > 0 ? kBufCols / KC : 1;
        float tmin[TPC];  // per table: smallest |projection| (a min with |.| operands)
        uint32_t aw[NG];
        uint32_t v64[64];
        // Pairs of groups: a pair past the chunk's last column is skipped, and a pair's second
        // group past it is classified too (those bits and minima are never read).
#pragma unroll
        for (int h = 0; h < NG / 2; ++h) {
          bw[2 * h] = bw[2 * h + 1] = 0u;
          aw[2 * h] = aw[2 * h + 1] = 0u;
          if (2 * h >= ng) continue;
          tmem_ld64(tbase + 64u * h, v64);
          tmem_ld_wait(v64);
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int g = 2 * h + q;
            const uint32_t* v = v64 + 32 * q;
            uint32_t c0 = 0u, c1 = 0u, c2 = 0u, c3 = 0u;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              c0 = __funnelshift_l(v[k], c0, 1);
              c1 = __funnelshift_l(v[8 + k], c1, 1);
              c2 = __funnelshift_l(v[16 + k], c2, 1);
              c3 = __funnelshift_l(v[24 + k], c3, 1);
            }
            // column k's sign sits at bit 31 - k of the concatenation
            bw[g] = ~__brev((c0 << 24) | (c1 << 16) | (c2 << 8) | c3);
            if constexpr (KC > 0) {
#pragma unroll
              for (int k = 0; k < 32; ++k) {
                const int col = 32 * g + k, t = col / KC;  // compile-time
                if (t < TPC) {
                  const float av = fabsf(__uint_as_float(v[k]));
                  tmin[t] = col % KC == 0 ? av : fminf(tmin[t], av);
                }
              }
            } else {
              if constexpr (PROJ) {  // measurement path: the accumulators, scaled back by ||w_c||
                if (valid) {
#pragma unroll
                  for (int k = 0; k < 32; ++k) {
                    const int col = 32 * g + k;
                    if (col < ncols)
                      a.proj[i * static_cast<long long>(K * L) + tab0 * K + col] =
                          __uint_as_float(v[k]) * a.wnorm[tab0 * K + col];
                  }
                }
              }
              bool any = false;
#pragma unroll
              for (int k = 0; k < 32; ++k) any |= (v[k] & 0x7FFFFFFFu) <= Bi;
              if (any) {
                uint32_t am = 0u;
#pragma unroll
                for (int k = 0; k < 32; ++k) am |= ((v[k] & 0x7FFFFFFFu) <= Bi ? 1u : 0u) << k;
                aw[g] = am;
              }
            }
          }
        }
        tc_fence_before();
        mbar_arrive(&S->t_empty[b]);
        auto store = [&](uint32_t id, int j) {
          if (st_tm) ids[static_cast<size_t>(j) * ld + i] = static_cast<IdT>(id);
          if (st_rm) ids_rm[i * L + j] = id;
        };
        if constexpr (KC > 0) {
          constexpr uint32_t KM = (1u << KC) - 1u;
#pragma unroll
          for (int t = 0; t < TPC; ++t)
            if (t < ntab && __float_as_uint(tmin[t]) <= Bi) defmask |= 1u << t;
          if (!valid) defmask = 0u;
          // table t is bits [t KC, t KC + KC) of the chunk: compile-time word and shift.  Every
          // table's id is stored, deferred ones too: the recheck kernel, which runs after this
          // one, overwrites those.  One pointer steps through the tables (no per-table multiply).
          if (valid) {
            IdT* pt = ids + static_cast<size_t>(tab0) * ld + i;
            uint32_t* pr = ids_rm + i * L + tab0;
#pragma unroll
            for (int t = 0; t < TPC; ++t) {
              if (t < ntab) {
                const int cb = t * KC, wi = cb >> 5, sh = cb & 31;
                uint32_t id = bw[wi] >> sh;
                if (sh + KC > 32) id |= bw[wi + 1] << (32 - sh);
                id &= KM;
                if (st_tm) *pt = static_cast<IdT>(id);
                if (st_rm) pr[t] = id;
                pt += ld;
              }
            }
          }
        } else {
          // any K: streaming extraction, table t is bits [tK, tK + K) of the chunk
          unsigned long long accb = 0ull, acca = 0ull;
          int nacc = 0, t = 0;
#pragma unroll
          for (int g = 0; g < NG; ++g) {
            if (g < ng) {
              accb |= static_cast<unsigned long long>(bw[g]) << nacc;
              acca |= static_cast<unsigned long long>(aw[g]) << nacc;
              nacc += 32;
              while (nacc >= K && t < ntab) {
                const uint32_t id = static_cast<uint32_t>(accb) & kmask;
                const uint32_t amb = static_cast<uint32_t>(acca) & kmask;
                accb >>= K;
                acca >>= K;
                nacc -= K;
                if (amb != 0u) defmask |= 1u << t;
                else if (valid) store(id, tab0 + t);
                ++t;
              }
            }
          }
          if (!valid) defmask = 0u;
        }
        // append the deferred (point, table) pairs to this CTA's segment (one shared-memory
        // atomic per row that has any) and, with kTagDeferred, replace their stored ids by the
        // tag; beyond the segment's capacity, resolve them here (untagged: counted by the insert
        // pass)
        if (__any_sync(0xFFFFFFFFu, defmask != 0u) && defmask != 0u) {
          unsigned int idx = atomicAdd(&S->ndef, static_cast<unsigned int>(__popc(defmask)));
          uint32_t dm = defmask;
          while (dm) {
            const int t = __ffs(dm) - 1;
            dm &= dm - 1u;
            const int j = tab0 + t;
            if (idx < seg_cap) {
              seg[idx] = (static_cast<unsigned long long>(i) << 24) | static_cast<unsigned long long>(j);
              if (tag) ids[static_cast<size_t>(j) * ld + i] = static_cast<IdT>(tag);
            } else store(exact_table_id<BF16>(X, i, d, K, j, Wt, cB32, xfac32, xabs32, babs32, st), j);
            ++idx;
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    a.defer_counts[blockIdx.x] = static_cast<unsigned int>(min(static_cast<unsigned long long>(S->ndef), a.seg_cap));
    if (S->ndef) atomicAdd(&a.st->deferred, static_cast<unsigned long long>(S->ndef));
  }
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

}  // namespace

cudaError_t launch_hash_tc(const TcArgs& a, int num_sms, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const long long grid = min(static_cast<long long>(num_sms), a.ntiles);
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = smem_limit(kern, a.smem_bytes);
    if (e != cudaSuccess) return e;
    kern<<<static_cast<unsigned>(grid), kThreads, a.smem_bytes, s>>>(a);
    return cudaGetLastError();
  };
  auto pick = [&](auto bf16_tag) -> cudaError_t {
    constexpr bool B = decltype(bf16_tag)::value;
    if (a.mode & kStoreProj) return a.K > 16 ? go(hash_tc_kernel<B, uint32_t, 0, true>) : go(hash_tc_kernel<B, uint16_t, 0, true>);
    if (a.K > 16) return go(hash_tc_kernel<B, uint32_t, 0>);
    switch (a.K) {
      case 10: return go(hash_tc_kernel<B, uint16_t, 10>);
      case 12: return go(hash_tc_kernel<B, uint16_t, 12>);
      case 15: return go(hash_tc_kernel<B, uint16_t, 15>);
      case 16: return go(hash_tc_kernel<B, uint16_t, 16>);
      default: return go(hash_tc_kernel<B, uint16_t, 0>);
    }
  };
  if (a.x_bf16) return pick(std::true_type{});
  return pick(std::false_type{});
}

}  // namespace ace
