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
//     instruction; over S instructions at most S * 5.25 * 2^-23 * sum |x_i w'_i| (a 1.5x
//     margin is applied);
//   - normalisation: w' is w_c / ||w_c|| rounded to binary32 elementwise (2^-24);
//   - the binary64 reference itself (gamma64_d).
// A point whose |projection| is inside the bound on some column of a table is appended to a
// deferred list; recheck_kernel recomputes those bits in binary64 (index order) and inserts
// the final ids, so every id equals the binary64 definition.
//
// Roles (one CTA per SM, persistent over 128-point tiles):
//   warp 0       TMEM allocation, B image load (resident W'), MMA issue (one lane)
//   warps 1-4    converters: X tile (bulk copy into staging, or plain loads for the tail)
//                -> bf16 hi/lo operand images + per-row bound
//   warps 5-8    epilogue: tcgen05.ld, guard classification, bit packing, id store,
//                warp-merged count increments, deferral of ambiguous tables
#include "guard.cuh"
#include "tc_ptx.cuh"
#include "tc_plan.h"

namespace ace {
namespace {

using namespace tc;

constexpr int kThreads = 288;
constexpr int kConv0 = 32;    // first converter thread
constexpr int kEpi0 = 160;    // first epilogue thread
constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz

struct Smem {
  uint64_t st_full;
  uint64_t b_full;
  uint64_t drain;
  uint64_t a_full[2], a_empty[2];
  uint64_t bnd_full[2], bnd_empty[2];
  uint64_t t_full[2], t_empty[2];
  uint32_t taddr;
  int abort;
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

template <bool BF16, typename IdT>
__global__ void __launch_bounds__(kThreads, 1) hash_tc_kernel(const __grid_constant__ TcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* Bimg = smem;
  // A stage s: hi image at off_a + 2 s a_bytes, lo image right after it
  auto a_hi = [&](int st) { return smem + a.off_a + 2 * st * a.a_bytes; };
  auto a_lo = [&](int st) { return smem + a.off_a + (2 * st + 1) * a.a_bytes; };
  uint8_t* stage = smem + a.off_stage;
  float* bnd = reinterpret_cast<float*>(smem + a.off_bnd);          // [2][128]
  uint32_t* wbits = reinterpret_cast<uint32_t*>(smem + a.off_bits);  // [8][128]
  uint32_t* wamb = wbits + 8 * 128;                                  // [8][128]
  Smem* S = reinterpret_cast<Smem*>(smem + a.off_ctl);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long ntiles = a.ntiles;
  const int esz = BF16 ? 2 : 4;

  if (tid == 0) {
    S->abort = 0;
    mbar_init(&S->st_full, 1);
    mbar_init(&S->b_full, 1);
    mbar_init(&S->drain, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(&S->a_full[s], 128);
      mbar_init(&S->a_empty[s], 1);
      mbar_init(&S->bnd_full[s], 128);
      mbar_init(&S->bnd_empty[s], 128);
      mbar_init(&S->t_full[s], 1);
      mbar_init(&S->t_empty[s], 128);
    }
    mbar_fence_init();
  }
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
          const int b = static_cast<int>(item & 1);
          if (item >= 2 && !mbar_wait(&S->t_empty[b], ((item >> 1) + 1) & 1, &S->abort, kWaitCycles)) {
            ok = false;
            set_abort(S, a.st);
            break;
          }
          tc_fence_after();
          const TcChunk& ch = a.chunk[c];
          const uint32_t idesc = idesc_bf16(128, ch.N);
          const uint32_t bhi = smem_u32(Bimg) + ch.boff_hi, blo = smem_u32(Bimg) + ch.boff_lo;
          const uint32_t dt = tmem + static_cast<uint32_t>(b * 256);
          uint32_t acc = 0;
          // x_hi . w_hi, x_hi . w_lo, x_lo . w_hi
          for (int p = 0; p < 3; ++p) {
            const uint32_t as = (p == 2) ? alo : ahi;
            const uint32_t bs = (p == 1) ? blo : bhi;
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
      // drain: wait until every MMA this thread issued has completed
      // (bounded by time only: TMEM must not be released under a running MMA)
      const int never = 0;
      mma_commit(&S->drain);
      if (!mbar_wait(&S->drain, 0, &never, kWaitCycles)) set_abort(S, a.st);
    }
    __syncwarp();
  } else if (warp >= 1 && warp <= 4) {
    // ------------------------------------------------------------------ converters
    const int r = tid - kConv0;  // row of the tile
    const bool aligned = (reinterpret_cast<uintptr_t>(a.X) & 15u) == 0;
    const uint32_t tile_bytes = static_cast<uint32_t>(128) * a.d * esz;
    auto full_tile = [&](long long m) { return aligned && (m + 1) * 128 <= a.n; };
    int staged = 0;        // staging-buffer phases consumed
    bool pending = false;  // (thread r == 0) a bulk copy into the staging buffer is in flight
    if (r == 0 && blockIdx.x < ntiles && full_tile(blockIdx.x)) {
      pending = true;
      mbar_expect_tx(&S->st_full, tile_bytes);
      bulk_g2s(stage, static_cast<const uint8_t*>(a.X) + static_cast<size_t>(blockIdx.x) * tile_bytes, tile_bytes,
               &S->st_full);
    }
    int tl = 0;
    for (long long m = blockIdx.x; m < ntiles; m += gridDim.x, ++tl) {
      const int s = tl & 1;
      const bool full = full_tile(m);
      bool ok = S->abort == 0;
      if (ok && full) {
        if (mbar_wait(&S->st_full, staged & 1, &S->abort, kWaitCycles)) {
          if (r == 0) pending = false;
          ++staged;
        } else {
          ok = false;
          set_abort(S, a.st);
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
      const long long i = m * 128 + r;
      const bool valid = i < a.n;
      float q = 0.f;
      const int ngrp = a.d_pad / 8;
      const int rot = (a.d & 1) ? 0 : r;  // rotate the read order when d is even (bank spread)
      for (int gi = 0; gi < ngrp; ++gi) {
        const int g = (gi + rot) % ngrp;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int k = g * 8 + e;
          float x = 0.f;
          if (valid && k < a.d) {
            if (full) x = BF16 ? __uint_as_float(static_cast<unsigned>(reinterpret_cast<const unsigned short*>(stage)[r * a.d + k]) << 16)
                               : reinterpret_cast<const float*>(stage)[r * a.d + k];
            else x = xval<BF16>(a.X, i * a.d + k);
          }
          v[e] = x;
          q = fmaf(x, x, q);
        }
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float h0 = __bfloat162float(__float2bfloat16_rn(v[2 * e]));
          const float h1 = __bfloat162float(__float2bfloat16_rn(v[2 * e + 1]));
          hi[e] = pack_bf16x2(h0, h1);
          lo[e] = pack_bf16x2(v[2 * e] - h0, v[2 * e + 1] - h1);
        }
        const uint32_t off = kmajor_offset(r, g * 8, a.d_pad);
        *reinterpret_cast<uint4*>(a_hi(s) + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(a_lo(s) + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
      // per-row bound: tau * ||x||_up + tau_abs; +inf forces a binary64 recheck of every column
      float B;
      if (!isfinite(q) || q < a.qmin) B = __int_as_float(0x7f800000);
      else B = fmaf(a.tau, sqrtf(q * a.xfac) * 1.00000095367431640625f, a.tau_abs);
      bnd[s * 128 + r] = B;
      if (valid && !isfinite(q)) atomicAdd(&a.st->nonfinite, 1ull);
      fence_proxy_async();
      mbar_arrive(&S->a_full[s]);
      mbar_arrive(&S->bnd_full[s]);
      conv_bar_or(false);  // every converter has finished reading the staging buffer
      const long long mn = m + gridDim.x;
      if (r == 0 && mn < ntiles && full_tile(mn)) {
        pending = true;
        mbar_expect_tx(&S->st_full, tile_bytes);
        bulk_g2s(stage, static_cast<const uint8_t*>(a.X) + static_cast<size_t>(mn) * tile_bytes, tile_bytes,
                 &S->st_full);
      }
    }
    // leave no bulk copy in flight: wait (bounded, ignoring the abort flag) for an issued
    // copy that was never consumed
    if (r == 0 && pending) {
      const int never = 0;
      mbar_wait(&S->st_full, staged & 1, &never, kWaitCycles);
    }
  } else {
    // ------------------------------------------------------------------ epilogue
    const int q4 = warp & 3;
    const int r = q4 * 32 + lane;  // TMEM lane = tile row
    const int et = tid - kEpi0;    // 0..127, for the bits scratch
    (void)et;
    const unsigned lanemask_lt = (1u << lane) - 1u;
    long long item = 0;
    int tl = 0;
    bool ok = true;
    for (long long m = blockIdx.x; ok && m < ntiles; m += gridDim.x, ++tl) {
      const int s = tl & 1;
      ok = mbar_wait(&S->bnd_full[s], (tl >> 1) & 1, &S->abort, kWaitCycles);
      if (!__all_sync(0xFFFFFFFFu, ok)) {
        ok = false;
        set_abort(S, a.st);
        break;
      }
      const float B = bnd[s * 128 + r];
      mbar_arrive(&S->bnd_empty[s]);
      const long long i = m * 128 + r;
      const bool valid = i < a.n;
      for (int c = 0; c < a.nchunks; ++c, ++item) {
        const int b = static_cast<int>(item & 1);
        ok = mbar_wait(&S->t_full[b], (item >> 1) & 1, &S->abort, kWaitCycles);
        if (!__all_sync(0xFFFFFFFFu, ok)) {
          ok = false;
          set_abort(S, a.st);
          break;
        }
        tc_fence_after();
        const TcChunk& ch = a.chunk[c];
        const int ncols = ch.ntab * a.K;
        const int ng = (ncols + 31) >> 5;
        const uint32_t tbase = tmem + (static_cast<uint32_t>(q4 * 32) << 16) + static_cast<uint32_t>(b * 256);
#pragma unroll 1
        for (int g = 0; g < ng; ++g) {
          uint32_t v[32];
          tmem_ld32(tbase + 32u * g, v);
          tmem_ld_wait();
          const int left = ncols - 32 * g;
          const uint32_t vmask = left >= 32 ? 0xFFFFFFFFu : ((1u << left) - 1u);
          uint32_t neg = 0;
          bool any = false;
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            neg |= (v[k] >> 31) << k;
            any |= !(fabsf(__uint_as_float(v[k])) > B);
          }
          uint32_t am = 0;
          if (any) {
#pragma unroll
            for (int k = 0; k < 32; ++k) am |= (!(fabsf(__uint_as_float(v[k])) > B) ? 1u : 0u) << k;
            am &= vmask;
          }
          wbits[g * 128 + r] = ~neg;
          wamb[g * 128 + r] = am;
        }
        tc_fence_before();
        mbar_arrive(&S->t_empty[b]);
        // pack, resolve, store, insert
        for (int t = 0; t < ch.ntab; ++t) {
          const int cb = t * a.K;
          const int w0 = cb >> 5, sh = cb & 31;
          unsigned long long bv = wbits[w0 * 128 + r], av = wamb[w0 * 128 + r];
          if (w0 + 1 < ng) {
            bv |= static_cast<unsigned long long>(wbits[(w0 + 1) * 128 + r]) << 32;
            av |= static_cast<unsigned long long>(wamb[(w0 + 1) * 128 + r]) << 32;
          }
          const uint32_t kmask = (1u << a.K) - 1u;
          uint32_t id = static_cast<uint32_t>(bv >> sh) & kmask;
          const uint32_t amb = static_cast<uint32_t>(av >> sh) & kmask;
          const int j = ch.tab0 + t;
          bool def = valid && amb != 0;
          const uint32_t dm = __ballot_sync(0xFFFFFFFFu, def);
          if (dm) {
            const int leader = __ffs(dm) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(a.defer_count, static_cast<unsigned long long>(__popc(dm)));
            base = __shfl_sync(0xFFFFFFFFu, base, leader);
            if (def) {
              const unsigned long long idx = base + __popc(dm & lanemask_lt);
              if (idx < a.defer_cap) {
                a.defer[2 * idx] = static_cast<unsigned long long>(i);
                a.defer[2 * idx + 1] = static_cast<unsigned long long>(id) | (static_cast<unsigned long long>(amb) << 24) |
                                       (static_cast<unsigned long long>(j) << 48);
              } else {
                // list full: resolve here (slow, still exact)
                uint32_t m2 = amb;
                while (m2) {
                  const int k = __ffs(m2) - 1;
                  m2 &= m2 - 1u;
                  if (exact_bit<BF16>(a.X, i, a.d, a.Wt, j * a.K + k)) id |= 1u << k;
                  else id &= ~(1u << k);
                }
                atomicAdd(&a.st->rechecks, static_cast<unsigned long long>(__popc(amb)));
                def = false;
              }
            }
          }
          const bool fin = valid && !def;
          if (fin) {
            if (a.mode & kStoreIds) reinterpret_cast<IdT*>(a.ids)[static_cast<size_t>(j) * a.ld + i] = static_cast<IdT>(id);
            if (a.mode & kStoreIdsRowMajor) a.ids_rm[i * a.L + j] = id;
          }
          if (a.mode & kInsert) {
            const uint32_t key = fin ? id : 0xFFFFFFFFu;
            const uint32_t grp = __match_any_sync(0xFFFFFFFFu, key);
            if (fin && lane == __ffs(grp) - 1)
              atomicAdd(a.counts + (static_cast<size_t>(j) << a.K) + id, static_cast<uint32_t>(__popc(grp)));
          }
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// Resolves the deferred (point, table) pairs: binary64 bits (index order), final id, store,
// insert.
template <bool BF16, typename IdT>
__global__ void __launch_bounds__(256) recheck_kernel(const __grid_constant__ TcArgs a) {
  const unsigned long long cnt = min(*a.defer_count, a.defer_cap);
  unsigned long long nre = 0;
  for (unsigned long long e = static_cast<unsigned long long>(blockIdx.x) * blockDim.x + threadIdx.x; e < cnt;
       e += static_cast<unsigned long long>(gridDim.x) * blockDim.x) {
    const long long i = static_cast<long long>(a.defer[2 * e]);
    const unsigned long long w = a.defer[2 * e + 1];
    uint32_t id = static_cast<uint32_t>(w & 0xFFFFFFull);
    const uint32_t amb = static_cast<uint32_t>((w >> 24) & 0xFFFFFFull);
    const int j = static_cast<int>(w >> 48);
    uint32_t m = amb;
    while (m) {
      const int k = __ffs(m) - 1;
      m &= m - 1u;
      if (exact_bit<BF16>(a.X, i, a.d, a.Wt, j * a.K + k)) id |= 1u << k;
      else id &= ~(1u << k);
    }
    nre += __popc(amb);
    if (a.mode & kStoreIds) reinterpret_cast<IdT*>(a.ids)[static_cast<size_t>(j) * a.ld + i] = static_cast<IdT>(id);
    if (a.mode & kStoreIdsRowMajor) a.ids_rm[i * a.L + j] = id;
    if (a.mode & kInsert) atomicAdd(a.counts + (static_cast<size_t>(j) << a.K) + id, 1u);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) nre += __shfl_down_sync(0xFFFFFFFFu, nre, off);
  if ((threadIdx.x & 31) == 0 && nre) atomicAdd(&a.st->rechecks, nre);
}

}  // namespace

cudaError_t launch_hash_tc(const TcArgs& a, int num_sms, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const long long grid = min(static_cast<long long>(num_sms), a.ntiles);
  const bool id16 = a.K <= 16;
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, a.smem_bytes);
    if (e != cudaSuccess) return e;
    kern<<<static_cast<unsigned>(grid), kThreads, a.smem_bytes, s>>>(a);
    return cudaGetLastError();
  };
  if (a.x_bf16) return id16 ? go(hash_tc_kernel<true, uint16_t>) : go(hash_tc_kernel<true, uint32_t>);
  return id16 ? go(hash_tc_kernel<false, uint16_t>) : go(hash_tc_kernel<false, uint32_t>);
}

cudaError_t launch_recheck(const TcArgs& a, int num_sms, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const unsigned grid = static_cast<unsigned>(num_sms * 4);
  const bool id16 = a.K <= 16;
  if (a.x_bf16) {
    if (id16) recheck_kernel<true, uint16_t><<<grid, 256, 0, s>>>(a);
    else recheck_kernel<true, uint32_t><<<grid, 256, 0, s>>>(a);
  } else {
    if (id16) recheck_kernel<false, uint16_t><<<grid, 256, 0, s>>>(a);
    else recheck_kernel<false, uint32_t><<<grid, 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace ace
