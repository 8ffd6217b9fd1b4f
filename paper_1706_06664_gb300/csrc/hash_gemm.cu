// SRP hashing of large-d bfloat16 batches on the tcgen05 tensor cores, streamed.
//
// Eq. 1 for every point and every column is a dense contraction X (n x d) . W (d x KL); at
// d = 1024 neither X nor W fits in shared memory, so both stream through a ring of
// 128-byte-swizzled k-blocks loaded by the TMA engine (cp.async.bulk.tensor), and each
// 128-point tile meets the projection image one 256-column unit at a time:
//     acc(128 x 256, binary32, TMEM) = x . w'_lo  (all k-blocks)  then  + x . w'_hi
// where w' = w_c / ||w_c|| (unit columns, rounded to binary32) is split on the host into
// bfloat16 hi + lo parts.  x is bfloat16, so x_i w'_hi,i and x_i w'_lo,i are exact products
// and the only errors are the dropped third part of w', the accumulation, and the
// normalisation.  Error bound of a point's accumulator (host constants in plan_gemm):
//   - split: |w' - w_hi - w_lo| <= 2^-16 |w'| elementwise (two round-to-nearest steps with the
//     bfloat16 unit roundoff 2^-8); the dropped term is at most ||x|| ||w' - w_hi - w_lo||,
//     and the host uses the largest residual norm over the columns (about 2^-18 in practice);
//   - accumulation: tcgen05 aligns the 17 addends of one MMA instruction (16 products and the
//     accumulator) to the largest exponent keeping two bits below its last place and truncates
//     the sum to binary32 (a model of the hardware that tests/test_gpu_tc_model.py checks on
//     the device): at most 5.25 * 2^-23 * (sum of |addends|) per instruction.  The lo product
//     goes first over all of d, so its instructions see addends of at most about
//     2^-8 ||x||.  Instruction t of the hi product adds the block B_t = [16t, 16t + 16) to an
//     accumulator that holds the partial sum over [0, 16t) (plus the small lo total and the
//     error so far), so by Cauchy-Schwarz its addends sum to at most
//     ||x_<16t|| WP_t + ||x_Bt|| WB_t + 2^-7 ||x||, with WP_t and WB_t the largest norms of
//     w'_hi's prefix and block over the columns.  Summed over the instructions:
//     5.25 * 2^-23 * (E + (2^-6 S + 1) ||x||), E = sum_t ||x_<16t|| WP_t + ||x_Bt|| WB_t, a
//     1.25x margin applied.  E is evaluated per k-block of four instructions (the prefix at the
//     k-block's end for all four, Cauchy-Schwarz over the four block terms).  For a point whose
//     energy is spread over d, E is about S/2 ||x|| instead of the S ||x|| that bounding every
//     partial sum by ||x|| would give;
//   - normalisation (2^-23 ||x||) and the binary64 reference itself (gamma64_d ||x||).
// The bound is one number per point, computed by the row-bound warps with upward rounding.
// A column whose |accumulator| <= B is deferred as a (point, column) entry; recheck_cols
// recomputes its bit exactly and flips the stored id bit if the tensor cores had it wrong.
//
// Roles (one CTA per SM, persistent over tiles; 8 warps):
//   warp 0      TMA producer: one (X k-block, image k-block) pair per ring stage
//   warp 1      TMEM allocation and MMA issue (one lane): 4 MMAs of 128 x 256 x 16 per stage
//   warps 2-3   row bounds: block and prefix norms of each point of the tile from global
//               memory (the TMA loads then find the rows in L2), the bound B, exact-zero and
//               non-finite rows
//   warps 4-7   epilogue: tcgen05.ld of the accumulator (thread = point), sign bits, guard
//               classification, deferral entries, bucket ids (Eq. 2) stored table-major
#include <cuda.h>
#include <cuda_fp8.h>

#include "gemm_plan.h"
#include "guard.cuh"
#include "tc_ptx.cuh"
#include "launch_cache.h"

namespace ace {
namespace {

using namespace tc;

constexpr int kThreads = 320;   // 10 warps
constexpr int kBndWarps = 4;    // row-bound warps (2 .. 5): one thread per tile row
constexpr int kStages = kGemmStages;
constexpr uint32_t kABytes = kGemmBM * kGemmBK * 2;  // 16 KB
constexpr uint32_t kBBytes = kGemmBN * kGemmBK * 2;  // 32 KB
constexpr uint32_t kStageBytes = kABytes + kBBytes;
// E4M3 stage: the bfloat16 X k-block (TMA, as above), the image's W1 and W2 planes (256 rows x
// 64 bytes each, bulk copies of canonical blocks) and the X1 and X2 planes the row warps
// convert (128 rows x 64 bytes each)
constexpr int kStagesF8 = kGemmStagesF8;
constexpr uint32_t kPlaneBytes = kGemmBN * kGemmBK;   // 16 KB
constexpr uint32_t kXPlaneBytes = kGemmBM * kGemmBK;  // 8 KB
constexpr uint32_t kOffW1 = kABytes, kOffW2 = kABytes + kPlaneBytes;
constexpr uint32_t kOffX1 = kABytes + 2 * kPlaneBytes, kOffX2 = kOffX1 + kXPlaneBytes;
constexpr uint32_t kStageBytesF8 = kOffX2 + kXPlaneBytes;  // 64 KB
static_assert(kStagesF8 * kStageBytesF8 == kStages * kStageBytes, "both rings span the same bytes");
constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz
static_assert(kStages * kStageBytes + 4096 * 4 + 4096 + 1024 <= 227 * 1024, "shared memory");

struct GSmem {
  uint64_t full[kStages], empty[kStages];
  uint64_t a_ready[kStages];  // E4M3: the stage's X1/X2 planes are written (one arrival per row)
  uint64_t t_full[2], t_empty[2];
  uint64_t b_full[2], b_empty[2];
  uint64_t drain;
  uint32_t taddr;
  int abort;
  unsigned int ndef;
  uint32_t bthr[2][kGemmBM];  // per tile slot and row: the row bound B (bit pattern)
  uint32_t bzero[2][kGemmBM]; // per tile slot and row: the row is exactly zero
  float bunscale[2][kGemmBM]; // E4M3: 2^-s of the row's scale 2^s (projection output only)
};

constexpr int kColfMax = 4096;  // per-column norms kept in shared memory (16 units)
constexpr int kSmemBytes = static_cast<int>(kStages * kStageBytes + sizeof(GSmem) + kColfMax * 4 + 1024);

__device__ __forceinline__ void set_abort(GSmem* S, DevStats* st) {
  S->abort = 1;
  atomicOr(&st->status, static_cast<unsigned>(ACE_STATUS_TIMEOUT));
}

__device__ __forceinline__ void expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// 2-D tiled TMA load (box of the tensor map at coordinates (c0 = innermost, c1)) into shared
// memory, completing `bytes` on the mbarrier.  c0 * 2 bytes is a multiple of 16 (c0 is a
// multiple of 64 here).
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

// 1-D bulk copy global -> shared (both 16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// Two binary32 values to E4M3 (round to nearest even, saturating to +-448): the first in the
// low byte.  And back (exact: every E4M3 value is a binary16 value).
__device__ __forceinline__ uint32_t to_e4m3x2(float a, float b) {
  return static_cast<uint32_t>(__nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3));
}
__device__ __forceinline__ float2 from_e4m3x2(uint32_t v) {
  const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(v), __NV_E4M3);
  return __half22float2(__half2(h));
}

// The leading four significant bits of y by Veltkamp's splitting (Dekker, "A floating-point
// technique for extending the available precision", 1971): with c = RN((2^20 + 1) y),
// h = RN(c - RN(c - y)) has at most 24 - 20 = 4 significant bits and y - h is exact in
// binary32.  Three FMA-pipe operations instead of integer ones.  Where |y| < 2^-6 (E4M3's
// subnormal range) h need not be an E4M3 value: its conversion then rounds, and the measuring
// pass takes the converted values, so the remainder X3 is still exact.
__device__ __forceinline__ float split4(float y) {
  const float c = __fmul_rn(y, 1048577.0f);
  return __fsub_rn(c, __fsub_rn(c, y));
}

__device__ __forceinline__ void tma_prefetch(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Shared-memory descriptor of a K-major operand in the 128-byte swizzled layout written by
// the TMA engine: rows of 128 bytes, 8-row groups 1024 bytes apart (SBO), swizzle mode 2.
// The tile base is 1024-byte aligned, so the k-th 16-element slice starts 32 k bytes in.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
  d |= static_cast<uint64_t>(1) << 16;           // LBO (not used by swizzled K-major layouts)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;   // SBO
  d |= static_cast<uint64_t>(1) << 46;           // descriptor version
  d |= static_cast<uint64_t>(2) << 61;           // 128-byte swizzle
  return d;
}

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// The exact bit of column c for point i (bfloat16 row): a binary32 FMA chain decided by the
// SIMT engine's a priori bound, then Dot2, then the binary64 definition.  The slow path of a
// CTA whose deferred segment is full.
__device__ __noinline__ bool exact_col_bit(const GemmArgs& a, long long i, int c) {
  const int d = a.d;
  const float* wc = a.Wt + static_cast<size_t>(c) * d;
  float q = 0.f, s32 = 0.f;
  for (int t = 0; t < d; ++t) {
    const float x = load_x<true>(a.X, i * d + t);
    q = fmaf(x, x, q);
    s32 = fmaf(x, __ldg(wc + t), s32);
  }
  const float xu = norm_upper(q, a.xfac32, a.xabs32);
  atomicAdd(&a.st->rechecks, 1ull);
  if (fabsf(s32) > fmaf(__ldg(a.cB32 + c), xu, a.babs32)) return s32 > 0.f;
  const int sg = dot2_sign<true>(a.X, i, d, wc, 1, a.dot2c, a.dot2abs);
  return sg != 0 ? sg > 0 : exact_bit<true>(a.X, i, d, a.Wt, c);
}

// KC > 0: specialised for K = KC (compile-time table offsets); KC = 0 handles any K.
// F8: E4M3 operands (see the notes at launch_hash_gemm).
template <typename IdT, int KC, bool PROJ, bool F8>
__global__ void __launch_bounds__(kThreads, 1)
    hash_gemm_kernel(const __grid_constant__ GemmArgs a, const __grid_constant__ CUtensorMap tmX,
                     const __grid_constant__ CUtensorMap tmW) {
  extern __shared__ uint8_t smem_raw[];
  constexpr int ST = F8 ? kStagesF8 : kStages;
  constexpr uint32_t SB = F8 ? kStageBytesF8 : kStageBytes;
  // the swizzled tiles need 1024-byte alignment
  const uint32_t raw = smem_u32(smem_raw);
  uint8_t* const smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  const uint32_t sbase = smem_u32(smem);
  GSmem* const S = reinterpret_cast<GSmem*>(smem + kStages * kStageBytes);
  float* const colf_s = reinterpret_cast<float*>(smem + kStages * kStageBytes + sizeof(GSmem));

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long ntiles = a.ntiles, n = a.n;
  const int nunits = a.nunits, nkb = a.nkb, nprod = a.nprod;
  const int ksteps = nprod * nkb;

  if (tid == 0) {
    S->abort = 0;
    S->ndef = 0;
    for (int s = 0; s < ST; ++s) {
      mbar_init(&S->full[s], 1);
      // the MMA commit and each row-bound warp; E4M3: the MMA commit only (it follows the
      // row warps' arrivals on a_ready, after they have read the stage's X k-block)
      mbar_init(&S->empty[s], F8 ? 1 : 1 + kBndWarps);
      mbar_init(&S->a_ready[s], kGemmBM);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&S->t_full[b], 1);
      mbar_init(&S->t_empty[b], 128);
      mbar_init(&S->b_full[b], 32 * kBndWarps);
      mbar_init(&S->b_empty[b], 128);
    }
    mbar_init(&S->drain, 1);
    mbar_fence_init();
  }
  if (warp == 1) {
    tmem_alloc(&S->taddr, 512);
    tmem_relinquish();
  }
  const bool colf_in_smem = a.colf && nunits * kGemmBN <= kColfMax;
  if (colf_in_smem)
    for (int c = tid; c < nunits * kGemmBN; c += kThreads) colf_s[c] = a.colf[c];
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = S->taddr;

  if (warp == 0) {
    // ------------------------------------------------------------------ TMA producer
    if (lane == 0) {
      tma_prefetch(&tmX);
      tma_prefetch(&tmW);
      long long it = 0;
      bool ok = true;
      for (long long m = blockIdx.x; ok && m < ntiles; m += gridDim.x) {
        for (int u = 0; ok && u < nunits; ++u) {
          for (int ks = 0; ks < ksteps; ++ks, ++it) {
            const int s = static_cast<int>(it % ST);
            if (it >= ST && !mbar_wait(&S->empty[s], static_cast<uint32_t>(((it / ST) + 1) & 1), &S->abort,
                                       kWaitCycles)) {
              ok = false;
              set_abort(S, a.st);
              break;
            }
            const int p = ks / nkb, kb = ks - p * nkb;
            const uint32_t sa = sbase + static_cast<uint32_t>(s) * SB;
            if constexpr (F8) {
              // pass 0 (the small products) needs both image planes, pass 1 (X1.W1) only W1
              const uint8_t* blk = a.img8 + (static_cast<size_t>(u) * nkb + kb) * 2 * kPlaneBytes;
              expect_tx(&S->full[s], kABytes + (p == 0 ? 2u : 1u) * kPlaneBytes);
              tma_load_2d(sa, &tmX, kb * kGemmBK, static_cast<int>(m * kGemmBM), &S->full[s]);
              bulk_load(sa + kOffW1, blk, kPlaneBytes, &S->full[s]);
              if (p == 0) bulk_load(sa + kOffW2, blk + kPlaneBytes, kPlaneBytes, &S->full[s]);
            } else {
              // the lo part (rows klp.. of the image) first, then the hi part
              const int brow = (nprod == 2 && p == 0 ? a.klp : 0) + u * kGemmBN;
              expect_tx(&S->full[s], kStageBytes);
              tma_load_2d(sa, &tmX, kb * kGemmBK, static_cast<int>(m * kGemmBM), &S->full[s]);
              tma_load_2d(sa + kABytes, &tmW, kb * kGemmBK, brow, &S->full[s]);
            }
          }
        }
      }
      // leave no copy in flight: the newest phase of every stage used has completed (bounded
      // waits that ignore the abort flag)
      const int never = 0;
      for (long long k = it - 1; k >= 0 && k >= it - ST; --k)
        mbar_wait(&S->full[k % ST], static_cast<uint32_t>((k / ST) & 1), &never, kWaitCycles);
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = F8 ? idesc_e4m3(kGemmBM, kGemmBN) : idesc_bf16(kGemmBM, kGemmBN);
      long long it = 0, u = 0;
      bool ok = true;
      for (long long m = blockIdx.x; ok && m < ntiles; m += gridDim.x) {
        for (int un = 0; ok && un < nunits; ++un, ++u) {
          const int b = static_cast<int>(u & 1);
          if (u >= 2 && !mbar_wait(&S->t_empty[b], static_cast<uint32_t>(((u >> 1) + 1) & 1), &S->abort, kWaitCycles)) {
            ok = false;
            set_abort(S, a.st);
            break;
          }
          tc_fence_after();
          const uint32_t dt = tmem + static_cast<uint32_t>(b * kGemmBN);
          uint32_t acc = 0;
          for (int ks = 0; ks < ksteps; ++ks, ++it) {
            const int s = static_cast<int>(it % ST);
            const uint32_t par = static_cast<uint32_t>((it / ST) & 1);
            if (!mbar_wait(&S->full[s], par, &S->abort, kWaitCycles) ||
                (F8 && !mbar_wait(&S->a_ready[s], par, &S->abort, kWaitCycles))) {
              ok = false;
              set_abort(S, a.st);
              break;
            }
            tc_fence_after();
            const uint32_t sa = sbase + static_cast<uint32_t>(s) * SB;
            if constexpr (F8) {
              // two K = 32 slices per k-block; no-swizzle canonical planes (8-row groups 512
              // bytes apart, K-adjacent core matrices 128 bytes apart).  Pass 0 accumulates the
              // small products X2.W2, X2.W1, X1.W2; pass 1 adds X1.W1.
              const bool small = ks < nkb;
#pragma unroll
              for (int kk = 0; kk < kGemmBK / 32; ++kk) {
                const uint32_t ko = 256u * kk;
                const uint64_t x1 = smem_desc(sa + kOffX1 + ko, 128, 512), w1 = smem_desc(sa + kOffW1 + ko, 128, 512);
                if (small) {
                  const uint64_t x2 = smem_desc(sa + kOffX2 + ko, 128, 512), w2 = smem_desc(sa + kOffW2 + ko, 128, 512);
                  mma_e4m3(dt, x2, w2, idesc, acc);
                  mma_e4m3(dt, x2, w1, idesc, 1u);
                  mma_e4m3(dt, x1, w2, idesc, 1u);
                } else {
                  mma_e4m3(dt, x1, w1, idesc, acc);
                }
                acc = 1;
              }
            } else {
              const uint64_t ad = sdesc_sw128(sa), bd = sdesc_sw128(sa + kABytes);
#pragma unroll
              for (int kk = 0; kk < kGemmBK / 16; ++kk) {
                mma_bf16(dt, ad + 2u * kk, bd + 2u * kk, idesc, acc);
                acc = 1;
              }
            }
            mma_commit(&S->empty[s]);
          }
          if (!ok) break;
          mma_commit(&S->t_full[b]);
        }
      }
      // every MMA issued has completed before TMEM is released (bounded by time only)
      const int never = 0;
      mma_commit(&S->drain);
      if (!mbar_wait(&S->drain, 0, &never, kWaitCycles)) set_abort(S, a.st);
    }
    __syncwarp();
  } else if (warp < 2 + kBndWarps) {
    // ------------------------------------------------------------------ row bounds
    // Thread r owns row r of the tile.  It follows the ring like the MMA issuer and releases
    // every stage it has seen (one arrival per warp); during the first pass of the first unit
    // of a tile, the stage's X k-block is the row's coordinates [64 kb, 64 kb + 64): the thread
    // reads its 128 bytes from the swizzled tile (chunk j of row r sits at chunk j ^ (r mod 8)),
    // and updates, in k order, the squared norms b_t of MMA blocks t = 4 kb .. 4 kb + 3, their
    // running prefix P, and E = sum_t sqrt(P_t) WP_t + sqrt(b_t) WB_t, every step rounded up
    // (xfac covers the binary32 sums of squares).  The row's bound is ready after the pass, long
    // before the epilogue of that unit needs it.
    const int r = tid - 64;  // 0 .. 127
    const float ca = a.ca, cx = a.cx, tau_abs = a.tau_abs, xfac = a.xfac, qmin = a.qmin;
    const float* const WP = a.wprof;           // per k-block: sum of the four WP_t
    const float* const WB = a.wprof + a.nkb;   // per k-block: sqrt of the sum of the four WB_t^2
    const bool count_nonfinite = !(a.mode & kStoreProj);
    const uint32_t rsw = static_cast<uint32_t>(r & 7);
    const uint32_t roff = static_cast<uint32_t>((r >> 3) * 1024 + (r & 7) * 128);
    long long it = 0;
    int ml = 0;
    bool ok = true;
    // E4M3: this row's 16-byte chunks in the stage's canonical X1 / X2 planes (chunk j2, the
    // coordinates [16 j2, 16 j2 + 16) of the k-block, 128 j2 bytes further)
    const uint32_t xoff = static_cast<uint32_t>((r >> 3) * 512 + (r & 7) * 16);
    for (long long m = blockIdx.x; ok && m < ntiles; m += gridDim.x, ++ml) {
      const int t = ml & 1;
      if (ml >= 2) ok = mbar_wait(&S->b_empty[t], static_cast<uint32_t>(((ml >> 1) + 1) & 1), &S->abort, kWaitCycles);
      if (!__all_sync(0xFFFFFFFFu, ok)) {
        ok = false;
        if (lane == 0) set_abort(S, a.st);
        break;
      }
      float P = 0.f, E = 0.f;
      uint32_t nz = 0u;
      float sc = 1.f, q2 = 0.f, q3 = 0.f;  // E4M3: the row's scale 2^s, ||X2||^2, ||X3||^2 (rounded up)
      bool big = false;                    // E4M3: an element of the scaled row reached 2^15
      for (int un = 0; ok && un < nunits; ++un) {
        for (int ks = 0; ks < ksteps; ++ks, ++it) {
          const int s = static_cast<int>(it % ST);
          ok = mbar_wait(&S->full[s], static_cast<uint32_t>((it / ST) & 1), &S->abort, kWaitCycles);
          if (!__all_sync(0xFFFFFFFFu, ok)) {
            ok = false;
            if (lane == 0) set_abort(S, a.st);
            break;
          }
          if constexpr (F8) {
            // Convert row r's k-block to E4M3 planes.  y = 2^s x (exact).  h = y split to four
            // significant bits (split4), X1 = e4m3(h) (exact where |y| >= 2^-6), X2 =
            // e4m3(y - h) (y - h is exact with at most four significant bits: its conversion is
            // exact too, except in E4M3's subnormal range, spacing 2^-9), X3 = y - X1 - X2, the
            // part the products miss.  The scale comes from the row's first k-block (its largest
            // |x| to [32, 64)); a row with |y| >= 448 anywhere (beyond E4M3's range) has every
            // column resolved exactly.  During pass 0 of the first unit the row is also
            // measured: the norms of y's blocks (E, as in the bfloat16 path), ||X2|| and ||X3||
            // from the converted values (exact differences in binary32).
            uint8_t* const stg = smem + static_cast<uint32_t>(s) * SB;
            const uint8_t* arow = stg + roff;
            const bool small = ks < nkb, first = un == 0 && small;
            if (un == 0 && ks == 0) {
              float mx = 0.f;
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const uint4 v = *reinterpret_cast<const uint4*>(arow + ((static_cast<uint32_t>(j) ^ rsw) << 4));
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) mx = fmaxf(mx, fmaxf(fabsf(bf16_lo(w[e])), fabsf(bf16_hi(w[e]))));
              }
              int sx = 0;
              if (mx > 0.f && isfinite(mx)) sx = min(100, max(-100, 5 - ilogbf(mx)));
              sc = __uint_as_float(static_cast<uint32_t>(127 + sx) << 23);
              S->bunscale[t][r] = __uint_as_float(static_cast<uint32_t>(127 - sx) << 23);
            }
            float bq[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int j2 = 0; j2 < 4; ++j2) {
              uint32_t o1[4] = {0u, 0u, 0u, 0u}, o2[4] = {0u, 0u, 0u, 0u};
#pragma unroll
              for (int hh = 0; hh < 2; ++hh) {
                const int j = 2 * j2 + hh;
                const uint4 v = *reinterpret_cast<const uint4*>(arow + ((static_cast<uint32_t>(j) ^ rsw) << 4));
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  const float y0 = bf16_lo(w[e]) * sc, y1 = bf16_hi(w[e]) * sc;
                  const float h0 = split4(y0), h1 = split4(y1);
                  const uint32_t b1 = to_e4m3x2(h0, h1);
                  // elements 8 hh + 2e and 8 hh + 2e + 1 of the chunk: bytes of word 2 hh + e / 2
                  o1[2 * hh + (e >> 1)] |= b1 << (16 * (e & 1));
                  if (small) {
                    const float r0 = y0 - h0, r1 = y1 - h1;
                    const uint32_t b2 = to_e4m3x2(r0, r1);
                    o2[2 * hh + (e >> 1)] |= b2 << (16 * (e & 1));
                    if (first) {
                      const float2 f1 = from_e4m3x2(b1), f2 = from_e4m3x2(b2);
                      const float t0 = (y0 - f1.x) - f2.x, t1 = (y1 - f1.y) - f2.y;
                      bq[j >> 1] = fmaf(y0, y0, bq[j >> 1]);
                      bq[j >> 1] = fmaf(y1, y1, bq[j >> 1]);
                      q2 = __fmaf_ru(f2.x, f2.x, q2);
                      q2 = __fmaf_ru(f2.y, f2.y, q2);
                      q3 = __fmaf_ru(t0, t0, q3);
                      q3 = __fmaf_ru(t1, t1, q3);
                      nz |= w[e] & 0x7FFF7FFFu;
                      big |= !(fabsf(y0) < 448.f) || !(fabsf(y1) < 448.f);
                    }
                  }
                }
              }
              *reinterpret_cast<uint4*>(stg + kOffX1 + xoff + 128u * j2) = make_uint4(o1[0], o1[1], o1[2], o1[3]);
              if (small)
                *reinterpret_cast<uint4*>(stg + kOffX2 + xoff + 128u * j2) = make_uint4(o2[0], o2[1], o2[2], o2[3]);
            }
            fence_proxy_async();
            mbar_arrive(&S->a_ready[s]);
            if (first) {
              // the E terms of the k-block, as in the bfloat16 path below (with y for x)
              const float bk = __fadd_ru(__fadd_ru(bq[0], bq[1]), __fadd_ru(bq[2], bq[3]));
              P = __fadd_ru(P, bk);
              const float sp = __fmul_ru(sqrtf(__fmul_ru(P, xfac)), 1.00000023841857910156f);
              const float sb = __fmul_ru(sqrtf(__fmul_ru(bk, xfac)), 1.00000023841857910156f);
              E = __fmaf_ru(sp, __ldg(WP + ks), E);
              E = __fmaf_ru(sb, __ldg(WB + ks), E);
              if (ks == nkb - 1) {
                uint32_t thr, zero = 0u;
                if (nz == 0u) {
                  thr = 0u;
                  zero = 1u;
                } else if (!isfinite(P) || !isfinite(E) || !isfinite(q2) || !isfinite(q3) || big || P < qmin) {
                  thr = 0xFFFFFFFFu;
                } else {
                  // B = ca E + cx ||y|| + ksw (||X2|| + ||X3||) + kt0 T0 + c3 ||X3|| + tau_abs,
                  // T0 = ||X2|| (w1m + w2m) + ||X1|| w2m, ||X1|| <= ||y|| + ||X2|| + ||X3||
                  const float yu = __fsqrt_ru(__fmul_ru(P, xfac));
                  const float x2u = __fsqrt_ru(q2), x3u = __fsqrt_ru(q3);
                  const float x1u = __fadd_ru(__fadd_ru(yu, x2u), x3u);
                  const float T0 = __fmaf_ru(x2u, __fadd_ru(a.w1m, a.w2m), __fmul_ru(x1u, a.w2m));
                  float B = __fmaf_ru(ca, E, __fmaf_ru(cx, yu, tau_abs));
                  B = __fmaf_ru(a.ksw, __fadd_ru(x2u, x3u), B);
                  B = __fmaf_ru(a.kt0, T0, B);
                  B = __fmaf_ru(a.c3, x3u, B);
                  thr = __float_as_uint(B);
                }
                S->bthr[t][r] = thr;
                S->bzero[t][r] = zero;
                if (count_nonfinite && m * kGemmBM + r < n && !isfinite(P)) atomicAdd(&a.st->nonfinite, 1ull);
                mbar_arrive(&S->b_full[t]);
              }
            }
            continue;
          }
          if (un == 0 && ks < nkb) {
            const uint8_t* arow = smem + static_cast<uint32_t>(s) * SB + roff;
            float bq[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const uint4 v = *reinterpret_cast<const uint4*>(arow + ((static_cast<uint32_t>(j) ^ rsw) << 4));
              const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float lo = bf16_lo(w[e]), hi = bf16_hi(w[e]);
                bq[j >> 1] = fmaf(lo, lo, bq[j >> 1]);
                bq[j >> 1] = fmaf(hi, hi, bq[j >> 1]);
                nz |= w[e] & 0x7FFF7FFFu;
              }
            }
            // per k-block (four MMA blocks): sum_t sqrt(P_t) WP_t <= sqrt(P_end) sum_t WP_t with
            // P_end the prefix through this k-block, and sum_t sqrt(b_t) WB_t <=
            // sqrt(sum_t b_t) sqrt(sum_t WB_t^2) (Cauchy-Schwarz over the four blocks); the host
            // folds the two sums into WP[kb] and WB[kb].  sqrtf is correctly rounded, so
            // (1 + 2^-22) makes each square root an upper bound.
            const float bk = __fadd_ru(__fadd_ru(bq[0], bq[1]), __fadd_ru(bq[2], bq[3]));
            P = __fadd_ru(P, bk);
            const float sp = __fmul_ru(sqrtf(__fmul_ru(P, xfac)), 1.00000023841857910156f);
            const float sb = __fmul_ru(sqrtf(__fmul_ru(bk, xfac)), 1.00000023841857910156f);
            E = __fmaf_ru(sp, __ldg(WP + ks), E);
            E = __fmaf_ru(sb, __ldg(WB + ks), E);
            if (ks == nkb - 1) {
              uint32_t thr, zero = 0u;
              if (nz == 0u) {  // every coordinate is +-0: every projection is exactly 0, bit 0
                thr = 0u;
                zero = 1u;
              } else if (!isfinite(P) || !isfinite(E) || P < qmin) {
                thr = 0xFFFFFFFFu;  // every column of the row is resolved exactly
              } else {
                const float xu = __fsqrt_ru(__fmul_ru(P, xfac));
                thr = __float_as_uint(__fmaf_ru(ca, E, __fmaf_ru(cx, xu, tau_abs)));
              }
              S->bthr[t][r] = thr;
              S->bzero[t][r] = zero;
              if (count_nonfinite && m * kGemmBM + r < n && !isfinite(P)) atomicAdd(&a.st->nonfinite, 1ull);
              mbar_arrive(&S->b_full[t]);
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive(&S->empty[s]);
        }
      }
    }
  } else {
    // ------------------------------------------------------------------ epilogue
    const int q4 = warp & 3;
    const int r = q4 * 32 + lane;  // TMEM lane = tile row
    const int K = KC > 0 ? KC : a.K;
    const int L = a.L, tpu = a.tpu, mode = a.mode;
    const long long ld = a.ld;
    const bool st_tm = (mode & kStoreIds) != 0, st_rm = (mode & kStoreIdsRowMajor) != 0;
    IdT* const ids = reinterpret_cast<IdT*>(a.ids);
    uint32_t* const ids_rm = a.ids_rm;
    const unsigned long long seg_cap = a.seg_cap;
    unsigned long long* const seg = a.defer + seg_cap * blockIdx.x;
    const uint32_t kmask = K >= 32 ? 0xFFFFFFFFu : (1u << K) - 1u;
    const float* const colf = colf_in_smem ? colf_s : a.colf;
    long long u = 0;
    int ml = 0;
    bool ok = true;
    for (long long m = blockIdx.x; ok && m < ntiles; m += gridDim.x, ++ml) {
      const int tslot = ml & 1;
      ok = mbar_wait(&S->b_full[tslot], static_cast<uint32_t>((ml >> 1) & 1), &S->abort, kWaitCycles);
      if (!__all_sync(0xFFFFFFFFu, ok)) {
        ok = false;
        if (lane == 0) set_abort(S, a.st);
        break;
      }
      // B of the row (bit pattern); all ones: every column is resolved exactly
      const uint32_t Bb = S->bthr[tslot][r];
      const bool zero_row = S->bzero[tslot][r] != 0u;
      const bool every = Bb == 0xFFFFFFFFu;
      const uint32_t thr1 = (every || zero_row) ? 0u : Bb + 1u;  // |v| <= B  <=>  bits(|v|) < bits(B) + 1
      const float Bf = (every || zero_row) ? 0.f : __uint_as_float(Bb);
      const float unscale = F8 ? S->bunscale[tslot][r] : 1.f;  // E4M3: the accumulators carry 2^s
      mbar_arrive(&S->b_empty[tslot]);
      const long long i = m * kGemmBM + r;
      const bool valid = i < n;
      for (int un = 0; un < nunits; ++un, ++u) {
        const int b = static_cast<int>(u & 1);
        ok = mbar_wait(&S->t_full[b], static_cast<uint32_t>((u >> 1) & 1), &S->abort, kWaitCycles);
        if (!__all_sync(0xFFFFFFFFu, ok)) {
          ok = false;
          if (lane == 0) set_abort(S, a.st);
          break;
        }
        tc_fence_after();
        const int j0 = un * tpu;
        const int ntab = min(tpu, L - j0);
        const int ncols = ntab * K;
        const int c0 = j0 * K;  // detector column of unit column 0
        const uint32_t tbase = tmem + (static_cast<uint32_t>(q4 * 32) << 16) + static_cast<uint32_t>(b * kGemmBN);
        uint32_t sw[8], aw[8];
        uint32_t v[64];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          tmem_ld64(tbase + 64u * h, v);
          tmem_ld_wait(v);
#pragma unroll
          for (int qh = 0; qh < 2; ++qh) {
            const int g = 2 * h + qh;
            const uint32_t* vv = v + 32 * qh;
            // sign bits: four funnel-shift chains, column k's sign at bit 31 - k, then reversed
            uint32_t c_0 = 0u, c_1 = 0u, c_2 = 0u, c_3 = 0u;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              c_0 = __funnelshift_l(vv[k], c_0, 1);
              c_1 = __funnelshift_l(vv[8 + k], c_1, 1);
              c_2 = __funnelshift_l(vv[16 + k], c_2, 1);
              c_3 = __funnelshift_l(vv[24 + k], c_3, 1);
            }
            sw[g] = ~__brev((c_0 << 24) | (c_1 << 16) | (c_2 << 8) | c_3);
            uint32_t am = 0u;
            if (colf) {  // columns of unequal norms: column c's bound is B * colf[c]
#pragma unroll
              for (int k = 0; k < 32; ++k) {
                const float tc = __fmul_ru(Bf, colf[un * kGemmBN + 32 * g + k]);
                am |= (fabsf(__uint_as_float(vv[k])) <= tc ? 1u : 0u) << k;
              }
            } else {
#pragma unroll
              for (int k = 0; k < 32; ++k) am |= ((vv[k] & 0x7FFFFFFFu) < thr1 ? 1u : 0u) << k;
            }
            aw[g] = every ? 0xFFFFFFFFu : (zero_row ? 0u : am);
            if constexpr (PROJ) {
              if (valid) {
#pragma unroll
                for (int k = 0; k < 32; ++k) {
                  const int uc = 32 * g + k;
                  if (uc < ncols)
                    a.proj[i * static_cast<long long>(a.KL) + c0 + uc] =
                        __uint_as_float(vv[k]) * unscale * __ldg(a.wnorm + c0 + uc);
                }
              }
            }
          }
        }
        tc_fence_before();
        mbar_arrive(&S->t_empty[b]);
        if constexpr (PROJ) continue;
        // columns past the unit's last table (zero image rows) carry no bit
        uint32_t cnt = 0u;
#pragma unroll
        for (int g = 0; g < 8; ++g) {
          const int lo = 32 * g;
          const uint32_t cm = ncols >= lo + 32 ? 0xFFFFFFFFu : (ncols > lo ? (1u << (ncols - lo)) - 1u : 0u);
          if (zero_row) sw[g] = 0u;
          aw[g] = valid ? (aw[g] & cm) : 0u;
          cnt += __popc(aw[g]);
        }
        // deferred (point, column) entries: one shared-memory atomic per row that has any; past
        // the segment's capacity the bit is resolved here
        if (cnt) {
          unsigned long long idx = atomicAdd(&S->ndef, cnt);
#pragma unroll
          for (int g = 0; g < 8; ++g) {
            uint32_t mm = aw[g];
            while (mm) {
              const int k = __ffs(mm) - 1;
              mm &= mm - 1u;
              const int c = c0 + 32 * g + k;
              const uint32_t tb = (sw[g] >> k) & 1u;
              if (idx < seg_cap) {
                seg[idx] = (static_cast<unsigned long long>(i) << kGemmEntryShift) |
                           (static_cast<unsigned long long>(c) << 1) | tb;
              } else {
                const uint32_t eb = exact_col_bit(a, i, c) ? 1u : 0u;
                sw[g] ^= (eb ^ tb) << k;
              }
              ++idx;
            }
          }
        }
        if (!valid) continue;
        // bucket ids (Eq. 2): table t of the unit is bits [t K, t K + K)
        if constexpr (KC == 16) {
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            if (t < ntab) {
              const uint32_t id = (sw[t >> 1] >> ((t & 1) * 16)) & 0xFFFFu;
              if (st_tm) ids[static_cast<size_t>(j0 + t) * ld + i] = static_cast<IdT>(id);
              if (st_rm) ids_rm[i * L + j0 + t] = id;
            }
          }
        } else {
          unsigned long long accb = 0ull;
          int nacc = 0, t = 0;
#pragma unroll
          for (int g = 0; g < 8; ++g) {
            accb |= static_cast<unsigned long long>(sw[g]) << nacc;
            nacc += 32;
            while (nacc >= K && t < ntab) {
              const uint32_t id = static_cast<uint32_t>(accb) & kmask;
              accb >>= K;
              nacc -= K;
              if (st_tm) ids[static_cast<size_t>(j0 + t) * ld + i] = static_cast<IdT>(id);
              if (st_rm) ids_rm[i * L + j0 + t] = id;
              ++t;
            }
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (tid == 0) {
    a.defer_counts[blockIdx.x] = static_cast<unsigned int>(min(static_cast<unsigned long long>(S->ndef), a.seg_cap));
    if (S->ndef && !(a.mode & kStoreProj)) atomicAdd(&a.st->deferred, static_cast<unsigned long long>(S->ndef));
  }
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

constexpr int kMaxDeferSegs = 1024;  // deferral segments (one per hash CTA)

// Exact resolution of the deferred (point, column) entries.  One warp per entry: the lanes
// split the dot product (lane l: 16-byte chunks l, l + 32, ... of the bfloat16 row and the
// matching binary32 W column), each as a binary32 FMA chain, join the sums by a butterfly of
// shuffles and keep the binary32 sum R of the magnitudes of every rounded partial result.
// u R / ((1 - u)(1 - gamma_(d+64))) plus underflow and the binary64 sum's own error bounds the
// distance to the definition whatever the summation tree (the SIMT engine's warp recheck),
// and the a priori gamma_d bound holds as well; the smaller decides.  What neither decides
// goes to Dot2 and then to the binary64 definition (one lane).  A bit that differs from the
// stored one is flipped in the id with an atomic XOR (other columns of the same id may be
// resolved by other warps at the same time).  The entries of all segments form one index
// space (segment prefixes in shared memory) that every warp strides through, so that the work
// is balanced whatever the segments' sizes.
template <typename IdT, bool W16>
__global__ void __launch_bounds__(256, W16 ? 3 : 2) recheck_cols_kernel(const __grid_constant__ GemmArgs a, int nseg) {
  __shared__ unsigned long long pre[kMaxDeferSegs + 1];  // pre[s]: entries of segments < s
  const int lane = threadIdx.x & 31;
  const unsigned nwarps = gridDim.x * (blockDim.x >> 5);
  const unsigned gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (threadIdx.x < 32) {  // warp 0: inclusive scan of the segment counts, 32 at a time
    unsigned long long run = 0;
    if (lane == 0) pre[0] = 0;
    for (int b = 0; b < nseg; b += 32) {
      const int sg = b + lane;
      unsigned long long v =
          sg < nseg ? min(static_cast<unsigned long long>(a.defer_counts[sg]), a.seg_cap) : 0ull;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const unsigned long long o = __shfl_up_sync(0xFFFFFFFFu, v, off);
        if (lane >= off) v += o;
      }
      if (sg < nseg) pre[sg + 1] = run + v;
      run += __shfl_sync(0xFFFFFFFFu, v, 31);
    }
  }
  __syncthreads();
  const unsigned long long total = pre[nseg];
  const int d = a.d, K = a.K, L = a.L, mode = a.mode;
  const int nch = d / 8;
  const long long ld = a.ld;
  unsigned long long nre = 0;
  int lo = 0;  // the segment holding g (pre[lo] <= g < pre[lo + 1]); g only grows
  for (unsigned long long g = gw; g < total; g += nwarps) {
    while (pre[lo + 1] <= g) ++lo;
    const unsigned long long w = a.defer[a.seg_cap * static_cast<unsigned long long>(lo) + (g - pre[lo])];
    const long long i = static_cast<long long>(w >> kGemmEntryShift);
    const int c = static_cast<int>((w >> 1) & 0xFFFFull);
    const uint32_t tb = static_cast<uint32_t>(w & 1ull);
    const uint4* xr = reinterpret_cast<const uint4*>(a.X) + i * nch;
    const float4* wr = reinterpret_cast<const float4*>(a.Wt + static_cast<size_t>(c) * d);
    const uint4* wr16 = reinterpret_cast<const uint4*>(a.Wt16) + static_cast<size_t>(c) * nch;
    float s = 0.f, run = 0.f, q = 0.f;
    // lane l's chunks l, l + 32, ..., four at a time: the loads of a round are all issued
    // before its arithmetic (one memory latency per round instead of one per chunk)
    constexpr int kRound = 4;
    for (int c0 = lane; c0 < nch; c0 += 32 * kRound) {
      uint4 xv[kRound], wa[kRound], wb[kRound];  // wb: the second half of a binary32 W chunk
#pragma unroll
      for (int u = 0; u < kRound; ++u) {
        const int ch = c0 + 32 * u;
        if (ch < nch) {
          xv[u] = __ldg(xr + ch);
          if constexpr (W16) {  // bfloat16-valued W: the same binary32 values from half the bytes
            wa[u] = __ldg(wr16 + ch);
          } else {
            wa[u] = __ldg(reinterpret_cast<const uint4*>(wr) + 2 * ch);
            wb[u] = __ldg(reinterpret_cast<const uint4*>(wr) + 2 * ch + 1);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < kRound; ++u) {
        if (c0 + 32 * u < nch) {
          float ws[8];
          if constexpr (W16) {
            ws[0] = bf16_lo(wa[u].x); ws[1] = bf16_hi(wa[u].x); ws[2] = bf16_lo(wa[u].y); ws[3] = bf16_hi(wa[u].y);
            ws[4] = bf16_lo(wa[u].z); ws[5] = bf16_hi(wa[u].z); ws[6] = bf16_lo(wa[u].w); ws[7] = bf16_hi(wa[u].w);
          } else {
            ws[0] = __uint_as_float(wa[u].x); ws[1] = __uint_as_float(wa[u].y);
            ws[2] = __uint_as_float(wa[u].z); ws[3] = __uint_as_float(wa[u].w);
            ws[4] = __uint_as_float(wb[u].x); ws[5] = __uint_as_float(wb[u].y);
            ws[6] = __uint_as_float(wb[u].z); ws[7] = __uint_as_float(wb[u].w);
          }
          const float xs[8] = {bf16_lo(xv[u].x), bf16_hi(xv[u].x), bf16_lo(xv[u].y), bf16_hi(xv[u].y),
                               bf16_lo(xv[u].z), bf16_hi(xv[u].z), bf16_lo(xv[u].w), bf16_hi(xv[u].w)};
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            s = fmaf(xs[k], ws[k], s);
            run = __fadd_rn(run, fabsf(s));
            q = fmaf(xs[k], xs[k], q);
          }
        }
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float so = __shfl_xor_sync(0xFFFFFFFFu, s, off);
      const float ro = __shfl_xor_sync(0xFFFFFFFFu, run, off);
      q += __shfl_xor_sync(0xFFFFFFFFu, q, off);
      s = __fadd_rn(s, so);
      run = __fadd_rn(__fadd_rn(run, ro), fabsf(s));
    }
    const float xu = norm_upper(q, a.xfac32, a.xabs32);
    const float cb = __ldg(a.cB32 + c);
    const float brun = __fmaf_ru(a.runc, run, __fmaf_ru(__fmul_ru(a.run64, cb), xu, a.runabs));
    const float bpri = fmaf(cb, xu, a.babs32);
    bool bit;
    if (fabsf(s) > fminf(brun, bpri)) {
      bit = s > 0.f;
    } else {
      // Warp-cooperative exact sum.  x is bfloat16 (8 significant bits); a bfloat16-valued w
      // makes every product x_t w_t exact in binary64, and a binary32 w is split into w_hi =
      // its bfloat16 rounding and w_lo = w - w_hi (exact), whose products are summed apart.
      // When the bits from the lowest set bit of any product of a sum up to d times its largest
      // product fit in 53, every binary64 sum of those products is exact, in any order: the
      // lanes' sums joined by a butterfly are exact, and so is the sign of their total (one
      // rounded addition keeps it) -- the definition's.  Otherwise (products spanning too many
      // binades) Dot2 and the binary64 definition on one lane.
      double sh = 0.0, sl = 0.0;
      int emh = -4096, elh = 4096, eml = -4096, ell = 4096;
      // em: the largest biased exponent; el: the lowest set bit of any product is 2^(el - 1023)
      auto track = [](double pr, int& em, int& el) {
        const long long b = __double_as_longlong(pr);
        const int ef = static_cast<int>((b >> 52) & 0x7FF);
        if (ef == 0x7FF) {
          em = 1 << 20;  // inf or NaN: not this tier
        } else if (pr != 0.0) {
          const long long sig = (b & 0xFFFFFFFFFFFFFLL) | (ef ? (1LL << 52) : 0LL);
          em = max(em, ef);
          el = min(el, max(ef, 1) - 52 + (__ffsll(sig) - 1));
        }
      };
      for (int ch = lane; ch < nch; ch += 32) {
        const uint4 xv = __ldg(xr + ch);
        float ws[8];
        if constexpr (W16) {
          const uint4 wv = __ldg(wr16 + ch);
          ws[0] = bf16_lo(wv.x); ws[1] = bf16_hi(wv.x); ws[2] = bf16_lo(wv.y); ws[3] = bf16_hi(wv.y);
          ws[4] = bf16_lo(wv.z); ws[5] = bf16_hi(wv.z); ws[6] = bf16_lo(wv.w); ws[7] = bf16_hi(wv.w);
        } else {
          const float4 w0 = __ldg(wr + 2 * ch), w1 = __ldg(wr + 2 * ch + 1);
          ws[0] = w0.x; ws[1] = w0.y; ws[2] = w0.z; ws[3] = w0.w;
          ws[4] = w1.x; ws[5] = w1.y; ws[6] = w1.z; ws[7] = w1.w;
        }
        const float xs[8] = {bf16_lo(xv.x), bf16_hi(xv.x), bf16_lo(xv.y), bf16_hi(xv.y),
                             bf16_lo(xv.z), bf16_hi(xv.z), bf16_lo(xv.w), bf16_hi(xv.w)};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const double xd = static_cast<double>(xs[k]);
          if constexpr (W16) {
            const double pr = __dmul_rn(xd, static_cast<double>(ws[k]));
            sh = __dadd_rn(sh, pr);
            track(pr, emh, elh);
          } else {
            const float whi = __bfloat162float(__float2bfloat16_rn(ws[k]));
            const double ph = __dmul_rn(xd, static_cast<double>(whi));
            const double pl = __dmul_rn(xd, static_cast<double>(__fsub_rn(ws[k], whi)));
            sh = __dadd_rn(sh, ph);
            sl = __dadd_rn(sl, pl);
            track(ph, emh, elh);
            track(pl, eml, ell);
          }
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        sh = __dadd_rn(sh, __shfl_xor_sync(0xFFFFFFFFu, sh, off));
        emh = max(emh, __shfl_xor_sync(0xFFFFFFFFu, emh, off));
        elh = min(elh, __shfl_xor_sync(0xFFFFFFFFu, elh, off));
        if constexpr (!W16) {
          sl = __dadd_rn(sl, __shfl_xor_sync(0xFFFFFFFFu, sl, off));
          eml = max(eml, __shfl_xor_sync(0xFFFFFFFFu, eml, off));
          ell = min(ell, __shfl_xor_sync(0xFFFFFFFFu, ell, off));
        }
      }
      // (biased exponents) every partial sum is below d 2^(em - 1022) <= 2^(em - 1022 + lg) and a
      // multiple of 2^(el - 1023): at most em - el + lg + 1 bits
      const int lg = 32 - __clz(d - 1);
      const bool exh = emh < 0 || emh - elh + lg + 1 <= 53;
      const bool exl = W16 || eml < 0 || eml - ell + lg + 1 <= 53;
      if (exh && exl) {
        bit = __dadd_rn(sh, sl) > 0.0;
      } else {
        int sg = 0;
        bool eb = false;
        if (lane == 0) {
          sg = dot2_sign<true>(a.X, i, d, a.Wt + static_cast<size_t>(c) * d, 1, a.dot2c, a.dot2abs);
          eb = sg != 0 ? sg > 0 : exact_bit<true>(a.X, i, d, a.Wt, c);
        }
        bit = __shfl_sync(0xFFFFFFFFu, eb ? 1 : 0, 0) != 0;
      }
    }
    if (lane == 0) {
      ++nre;
      if ((bit ? 1u : 0u) != tb) {
        const int j = c / K, k = c - j * K;
        if (mode & kStoreIds) {
          IdT* p = reinterpret_cast<IdT*>(a.ids) + static_cast<size_t>(j) * ld + i;
          if constexpr (sizeof(IdT) == 2) {
            const uintptr_t ad = reinterpret_cast<uintptr_t>(p);
            atomicXor(reinterpret_cast<unsigned int*>(ad & ~static_cast<uintptr_t>(3)),
                      (1u << k) << ((ad & 2u) * 8u));
          } else {
            atomicXor(reinterpret_cast<unsigned int*>(p), 1u << k);
          }
        }
        if (mode & kStoreIdsRowMajor) atomicXor(a.ids_rm + i * L + j, 1u << k);
      }
    }
  }
  if (lane == 0 && nre) atomicAdd(&a.st->rechecks, nre);
}

}  // namespace

int gemm_smem_bytes() { return kSmemBytes; }

cudaError_t launch_hash_gemm(const GemmArgs& a, const void* tmX, const void* tmW, int num_sms, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const long long grid = min(static_cast<long long>(num_sms), a.ntiles);
  const CUtensorMap& mx = *static_cast<const CUtensorMap*>(tmX);
  const CUtensorMap& mw = *static_cast<const CUtensorMap*>(tmW);
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = smem_limit(kern, kSmemBytes);
    if (e != cudaSuccess) return e;
    kern<<<static_cast<unsigned>(grid), kThreads, kSmemBytes, s>>>(a, mx, mw);
    return cudaGetLastError();
  };
  if (a.fp8) {
    if (a.mode & kStoreProj)
      return a.K > 16 ? go(hash_gemm_kernel<uint32_t, 0, true, true>) : go(hash_gemm_kernel<uint16_t, 0, true, true>);
    if (a.K > 16) return go(hash_gemm_kernel<uint32_t, 0, false, true>);
    if (a.K == 16) return go(hash_gemm_kernel<uint16_t, 16, false, true>);
    return go(hash_gemm_kernel<uint16_t, 0, false, true>);
  }
  if (a.mode & kStoreProj)
    return a.K > 16 ? go(hash_gemm_kernel<uint32_t, 0, true, false>) : go(hash_gemm_kernel<uint16_t, 0, true, false>);
  if (a.K > 16) return go(hash_gemm_kernel<uint32_t, 0, false, false>);
  if (a.K == 16) return go(hash_gemm_kernel<uint16_t, 16, false, false>);
  return go(hash_gemm_kernel<uint16_t, 0, false, false>);
}

cudaError_t launch_recheck_cols(const GemmArgs& a, int nseg, int num_sms, cudaStream_t s) {
  if (a.n <= 0 || nseg <= 0) return cudaSuccess;
  auto go = [&](auto kern) -> cudaError_t {
    int per_sm = 0;
    cudaError_t e = blocks_per_sm(&per_sm, kern, 256, 0);
    if (e != cudaSuccess) return e;
    const unsigned grid = static_cast<unsigned>(num_sms * max(1, per_sm));
    if (nseg > kMaxDeferSegs) return cudaErrorInvalidConfiguration;
    kern<<<grid, 256, 0, s>>>(a, nseg);
    return cudaGetLastError();
  };
  if (a.Wt16) return a.K > 16 ? go(recheck_cols_kernel<uint32_t, true>) : go(recheck_cols_kernel<uint16_t, true>);
  return a.K > 16 ? go(recheck_cols_kernel<uint32_t, false>) : go(recheck_cols_kernel<uint16_t, false>);
}

}  // namespace ace
