// Structured SRP hashing (ACE_W_HADAMARD detectors; §2.2, the Fast-JL family): every block of
// dp projections of a point is the Walsh-Hadamard transform of the point with random signs,
// y = H D_b x, computed in O(dp log dp) additions by one warp per point.
//
// Layout: lane l holds coordinates e * 32 + l (e < E = dp / 32), so the loads of a row are
// coalesced; the stages on the slot bits run within the lane (on register pairs, with the
// paired binary32 operations); for dp <= 512 the five stages on the low index bits are
// shuffles across lanes and after the transform the ballot of slot e over the lanes is
// exactly the 32-bit sign word of columns b dp + 32 e .. + 31; for dp = 1024 a transpose
// through shared memory makes those stages in-lane too, and each lane packs one sign word.
//
// Exactness: each output is a sum of dp terms +-x_i formed by a tree of m = log2(dp) rounded
// additions, so |y^ - y| <= gamma_m sum|x_i| (Higham, Accuracy and Stability of Numerical
// Algorithms, §4.2: any summation tree of height m), and the binary64 definition (Eq. 1 with
// this W: index-order sum of x_i w_i) is within gamma64_d sum|x_i| of y.  An output with
// |y^| > cband sum|x_i| + babs (upper bounds of both, with sum|x_i| rounded upwards) has the
// sign of the definition; a point whose smallest output clears that bound needs no per-output
// test.  The others are evaluated by the definition: by the whole warp, as a binary64 sum that
// is exact in any order, when the row's coordinates span few enough binades
// (exact_tier_applies); otherwise by each lane in index order from the stored +-1 W.
#include <algorithm>

#include "f32x2.cuh"
#include "fwht_exact.cuh"
#include "fwht_plan.h"
#include "guard.cuh"
#include "launch_cache.h"

namespace ace {
namespace {

// Ids of 32 consecutive points are gathered in shared memory and stored per table with one
// point per lane (coalesced) when L * 32 ids fit kIdBufBytes; otherwise each point's ids are
// stored as it is finished.
constexpr int kIdBufBytes = 4096;

// Dynamic shared memory of one 8-warp block: per warp the sign words of its current point and
// an id buffer; the per-lane sign masks of every block of columns; for dp = 1024 a 32 x 33
// transpose tile per warp.
template <int E, int ESZ>
struct FwhtSmem {
  static constexpr size_t words = 0;                                         // uint32 [8][kFwhtMaxWords]
  static constexpr size_t idbuf = words + 8 * kFwhtMaxWords * 4;             // bytes [8][kIdBufBytes]
  static constexpr size_t smask = idbuf + 8 * kIdBufBytes;                   // uint32 [kFwhtMaxWords / E][32]
  static constexpr size_t tbuf = smask + (kFwhtMaxWords / E) * 32 * 4;       // float [8][32 * 33] (E = 32)
  static constexpr size_t xrow = tbuf + (E == 32 ? 8 * 32 * 33 * 4 : 0);     // bytes [8][2][dp * ESZ] (E >= 16)
  static constexpr size_t bytes = xrow + (E >= 16 ? 8 * 2 * (E * 32) * ESZ : 0);
};

// Asynchronous 16-byte copy global -> shared (cp.async, completion by group).
__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// The definition of a bit under privacy noise (§4.5), in binary64: the index-order sum plus
// eta exactly (a binary32 times k / 4, |k| <= 32).
template <bool BF16>
__device__ __noinline__ bool noisy_exact_bit(const FwhtArgs& a, long long i, int col) {
  const float cw = counter_w(a.nseed, static_cast<uint64_t>(a.nbase + i) * a.KL + col);
  return exact_bit_add<BF16>(a.X, i, a.d, a.Wt, col, static_cast<double>(a.nsig) * static_cast<double>(cw));
}

// Walsh-Hadamard stages on the bits of the register index e (v[e] +- v[e + h] for h = 1, 2, ..,
// E / 2): the first within adjacent registers, the others on register pairs at once.
template <int E>
__device__ __forceinline__ void inlane_stages(float (&v)[E]) {
  if constexpr (E >= 2) {
#pragma unroll
    for (int e = 0; e < E; e += 2) {
      const float lo = v[e], hi = v[e + 1];
      v[e] = __fadd_rn(lo, hi);
      v[e + 1] = __fsub_rn(lo, hi);
    }
  }
#pragma unroll
  for (int h = 2; h < E; h <<= 1) {
#pragma unroll
    for (int e = 0; e < E; e += 2) {
      if ((e & h) == 0) {
        const uint64_t lo = pk2(v[e], v[e + 1]), hi = pk2(v[e + h], v[e + h + 1]);
        unpk2(add2(lo, hi), v[e], v[e + 1]);
        unpk2(sub2(lo, hi), v[e + h], v[e + h + 1]);
      }
    }
  }
}

// Blocks per SM the register budget is sized for: short rows need few registers, and more
// resident warps hide the latency of their shuffles.
template <int E>
constexpr int kFwhtMinBlocks = E <= 4 ? 4 : (E == 8 ? 3 : 2);

// OUT: 0 ids; 1 the measurement path (the transform's binary32 outputs, no ids); 2 ids with
// privacy noise (a separate instantiation, so that the others carry none of its registers).
template <bool BF16, typename IdT, int E, int OUT>
__global__ void __launch_bounds__(256, kFwhtMinBlocks<E>) hash_fwht_kernel(const __grid_constant__ FwhtArgs a) {
  constexpr bool PROJ = OUT == 1;
  extern __shared__ __align__(16) unsigned char fsm[];
  using SM = FwhtSmem<E, BF16 ? 2 : 4>;
  uint32_t (*words)[kFwhtMaxWords] = reinterpret_cast<uint32_t (*)[kFwhtMaxWords]>(fsm + SM::words);
  unsigned char (*idbuf)[kIdBufBytes] = reinterpret_cast<unsigned char (*)[kIdBufBytes]>(fsm + SM::idbuf);
  uint32_t* const smask = reinterpret_cast<uint32_t*>(fsm + SM::smask);  // [nblk][32]: lane l's flip bits of block b
  float (*tbuf)[32 * 33] = reinterpret_cast<float (*)[32 * 33]>(fsm + SM::tbuf);
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int d = a.d, dp = a.dp, K = a.K, L = a.L, KL = a.KL, nblk = a.nblk, mode = a.mode;
  const long long n = a.n, ld = a.ld;
  const float cband = a.cband, babs = a.babs;
  // privacy noise (§4.5): eta is added to each output in place (outputs col >= KL are padding
  // and never become bits); its binary32 rounding and the addition's stay within 2^-24 (8 nsig
  // + |y|) (|eta| <= 8 nsig), allowed for with a factor 2
  constexpr bool noisy = OUT == 2;
  const float nall = __fmul_ru(8.f, a.nsig);
  uint32_t* const wrow = words[wib];
  IdT* const ibuf = reinterpret_cast<IdT*>(idbuf[wib]);  // [L][32]
  const bool gather = static_cast<long long>(L) * 32 * static_cast<long long>(sizeof(IdT)) <= kIdBufBytes &&
                      (mode & kStoreIds) && !PROJ;
  const int nwords = nblk * E;
  // per-lane sign masks, the same for every point: bit e of smask[b][l] is the sign bit of
  // coordinate 32 e + l in block b
  for (int t = threadIdx.x; t < nblk * 32; t += blockDim.x) {
    const int b = t / 32, l = t % 32;
    uint32_t mk = 0u;
    for (int e = 0; e < E; ++e) mk |= ((__ldg(a.dsign + b * E + e) >> l) & 1u) << e;
    smask[t] = mk;
  }
  __syncthreads();
  unsigned long long nre = 0;
  // each warp takes groups of 32 consecutive points
  const long long ngroups = (n + 31) / 32;
  const long long nwarps = static_cast<long long>(gridDim.x) * (blockDim.x >> 5);
  // Long rows (E >= 16) whose byte length is a multiple of 16 are staged in shared memory by
  // asynchronous copies, double-buffered per warp: the next point's row is in flight while the
  // current one is transformed.  The padding beyond d stays zero (it is never copied).
  constexpr int kEsz = BF16 ? 2 : 4;
  const bool staged = E >= 16 && (static_cast<long long>(d) * kEsz) % 16 == 0 &&
                      (reinterpret_cast<uintptr_t>(a.X) & 15u) == 0;
  unsigned char* const xr = fsm + SM::xrow + static_cast<size_t>(wib) * 2 * (E * 32) * kEsz;
  const int rbytes = d * kEsz, nchunk = rbytes / 16;
  if (E >= 16) {
    for (int t = lane; t < 2 * E * 32 * kEsz / 4; t += 32) reinterpret_cast<uint32_t*>(xr)[t] = 0u;  // zero padding
    __syncwarp();
  }
  auto stage = [&](long long ii, int buf) {  // row ii into buffer buf (one copy group)
    const unsigned char* src = static_cast<const unsigned char*>(a.X) + ii * rbytes;
    unsigned char* dst = xr + buf * (E * 32) * kEsz;
    for (int c = lane; c < nchunk; c += 32) cp16(dst + c * 16, src + c * 16);
    cp_commit();
  };
  for (long long g = static_cast<long long>(blockIdx.x) * (blockDim.x >> 5) + wib; g < ngroups; g += nwarps) {
    const long long i0 = g * 32;
    const int np = static_cast<int>(min(32LL, n - i0));
    if (staged) stage(i0, 0);
    // For short rows (E <= 8) each point's loads are issued for the next point while it is
    // transformed; for long rows the registers are better spent on resident warps.
    constexpr bool kPrefetch = E <= 8;
    float xn[E];
    if constexpr (kPrefetch) {
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int t = e * 32 + lane;
        xn[e] = t < d ? load_x<BF16>(a.X, i0 * d + t) : 0.f;
      }
    }
    for (int p = 0; p < np; ++p) {
      const long long i = i0 + p;
      float x[E];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int t = e * 32 + lane;
        if constexpr (kPrefetch) {
          x[e] = xn[e];
          if (p + 1 < np) xn[e] = t < d ? load_x<BF16>(a.X, (i + 1) * d + t) : 0.f;
        } else if (!staged) {
          x[e] = t < d ? load_x<BF16>(a.X, i * d + t) : 0.f;
        }
      }
      if (staged) {
        if (p + 1 < np) {
          stage(i + 1, (p + 1) & 1);
          cp_wait1();  // this point's group has landed
        } else {
          cp_wait0();
        }
        __syncwarp();
        const unsigned char* row = xr + (p & 1) * (E * 32) * kEsz;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const int t = e * 32 + lane;
          if constexpr (BF16) x[e] = __uint_as_float(static_cast<uint32_t>(reinterpret_cast<const uint16_t*>(row)[t]) << 16);
          else x[e] = reinterpret_cast<const float*>(row)[t];
        }
        __syncwarp();  // (the buffer is refilled two points later)
      }
      // sum|x_t| rounded upwards and the squared norm, four chains each (any order of upward
      // roundings bounds the sum from above)
      float sa4[4] = {0.f, 0.f, 0.f, 0.f}, q4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int e = 0; e < E; ++e) sa4[e & 3] = __fadd_ru(sa4[e & 3], fabsf(x[e]));
      if constexpr (E >= 4) {
        uint64_t qa = pk2(0.f, 0.f), qb = pk2(0.f, 0.f);
#pragma unroll
        for (int e = 0; e < E; e += 4) {
          const uint64_t xa = pk2(x[e], x[e + 1]), xb = pk2(x[e + 2], x[e + 3]);
          qa = fma2(xa, xa, qa);
          qb = fma2(xb, xb, qb);
        }
        unpk2(qa, q4[0], q4[1]);
        unpk2(qb, q4[2], q4[3]);
      } else {
#pragma unroll
        for (int e = 0; e < E; ++e) q4[e] = x[e] * x[e];
      }
      float sa = __fadd_ru(__fadd_ru(sa4[0], sa4[1]), __fadd_ru(sa4[2], sa4[3]));
      float q = (q4[0] + q4[1]) + (q4[2] + q4[3]);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        sa = __fadd_ru(sa, __shfl_xor_sync(0xFFFFFFFFu, sa, off));
        q += __shfl_xor_sync(0xFFFFFFFFu, q, off);
      }
      if (lane == 0 && !isfinite(q) && !PROJ) atomicAdd(&a.st->nonfinite, 1ull);
      const float B = __fmaf_ru(cband, sa, babs);  // +inf or NaN for a non-finite row: all exact
      // uniform threshold: with noise, |v| > Bt implies |v| > B + 2^-23 (nall + |v|)
      const float Bt = noisy ? __fmul_ru(__fmaf_ru(1.1920928955078125e-07f, nall, B), 1.0000002384185791f) : B;
      int exact_ok = -1;  // the cooperative exact tier applies to this row (computed when first needed)
      for (int b = 0; b < nblk; ++b) {
        // sign flips: bit e of this lane's mask for block b flips coordinate 32 e + lane
        const uint32_t fm = smask[b * 32 + lane];
        float v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = __uint_as_float(__float_as_uint(x[e]) ^ (((fm >> e) & 1u) << 31));
        // butterflies on the slot bits (bit 5.. of t = 32 e + lane), within the lane
        inlane_stages<E>(v);
        if constexpr (E == 32) {
          // dp = 1024: transpose through shared memory (lane l then holds t = 32 l .. 32 l + 31),
          // so the five stages on the low bits are within the lane too, and the lane's 32
          // outputs are the 32 columns of one sign word
          float* const tile = tbuf[wib];  // [32][33]
#pragma unroll
          for (int e = 0; e < 32; ++e) tile[e * 33 + lane] = v[e];
          __syncwarp();
#pragma unroll
          for (int e = 0; e < 32; ++e) v[e] = tile[lane * 33 + e];
          __syncwarp();
          inlane_stages<32>(v);
        } else {
          // butterflies on the lane bits: o + s v with s = -1 on the upper lane of each pair
          // (one rounded operation, the same as the sum or the difference)
#pragma unroll
          for (int h = 1; h < 32; h <<= 1) {
            const float sg = (lane & h) ? -1.f : 1.f;
            float o[E];
#pragma unroll
            for (int e = 0; e < E; ++e) o[e] = __shfl_xor_sync(0xFFFFFFFFu, v[e], h);
            if constexpr (E == 1) {
              v[0] = __fmaf_rn(sg, v[0], o[0]);
            } else {
              const uint64_t sg2 = pk2(sg, sg);
#pragma unroll
              for (int e = 0; e < E; e += 2) unpk2(fma2(sg2, pk2(v[e], v[e + 1]), pk2(o[e], o[e + 1])), v[e], v[e + 1]);
            }
          }
        }
        // output e of this lane is column b dp + cofs(e)
        auto cofs = [&](int e) { return E == 32 ? lane * 32 + e : e * 32 + lane; };
        if constexpr (PROJ) {
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int col = b * dp + cofs(e);
            if (col < KL) a.proj[i * static_cast<long long>(KL) + col] = v[e];
          }
          continue;
        }
        if constexpr (noisy) {
          const uint64_t rb = static_cast<uint64_t>(a.nbase + i) * KL + b * dp;
#pragma unroll
          for (int e = 0; e < E; ++e) v[e] = __fadd_rn(v[e], __fmul_rn(a.nsig, counter_w(a.nseed, rb + cofs(e))));
        }
        // sign words (bit = [v > 0]; the outputs inside the bound are corrected below)
        float mv = fabsf(v[0]);
#pragma unroll
        for (int e = 1; e < E; ++e) mv = fminf(mv, fabsf(v[e]));  // (a NaN output makes the row's bound NaN)
        if constexpr (E == 32) {
          // outside the bound v is neither 0 nor NaN, so [v > 0] is the complement of the sign
          // bit: the sign bits are funnelled into four bytes, one shift per output
          uint32_t c[4] = {0u, 0u, 0u, 0u};
#pragma unroll
          for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int e = 8 * k + 7; e >= 8 * k; --e) c[k] = __funnelshift_l(__float_as_uint(v[e]), c[k], 1);
          wrow[b * 32 + lane] = ~((c[0] | (c[1] << 8)) | ((c[2] << 16) | (c[3] << 24)));
        } else {
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const uint32_t wv = __ballot_sync(0xFFFFFFFFu, v[e] > 0.f);
            if (lane == 0) wrow[b * E + e] = wv;
          }
        }
        uint32_t amb = 0u;  // bit e: output e is inside the bound (or NaN), a column < KL
        if (!(mv > Bt)) {
#pragma unroll
          for (int e = 0; e < E; ++e)
            if (!(fabsf(v[e]) > Bt) && b * dp + cofs(e) < KL) amb |= 1u << e;
        }
        uint32_t any = __ballot_sync(0xFFFFFFFFu, amb != 0u);
        if (any) {
          __syncwarp();
          if (exact_ok < 0) exact_ok = exact_tier_applies<BF16, E>(x, a.m) ? 1 : 0;
          if (exact_ok) {
            // one output at a time, by the whole warp: the binary64 sum of +-x_t is exact, so
            // it is the definition's index-order sum
            while (any) {
              const int src = __ffs(any) - 1;
              const uint32_t am = __shfl_sync(0xFFFFFFFFu, amb, src);
              const int e = __ffs(am) - 1;
              const int j = E == 32 ? src * 32 + e : e * 32 + src;
              double sum = coop_sum<E>(x, fm, j, lane);
              bool bit;
              if constexpr (noisy) {
                const float cw = counter_w(a.nseed, static_cast<uint64_t>(a.nbase + i) * KL + b * dp + j);
                bit = __dadd_rn(sum, static_cast<double>(a.nsig) * static_cast<double>(cw)) > 0.0;
              } else {
                bit = sum > 0.0;
              }
              if (lane == 0) {
                const int c = b * dp + j;
                wrow[c >> 5] = (wrow[c >> 5] & ~(1u << (c & 31))) | ((bit ? 1u : 0u) << (c & 31));
                ++nre;
              }
              if (lane == src) amb &= amb - 1u;
              any = __ballot_sync(0xFFFFFFFFu, amb != 0u);
              __syncwarp();
            }
          } else {
            // rows whose exponent range is too wide (or not finite): each lane evaluates the
            // definition in index order
            while (amb) {
              const int e = __ffs(amb) - 1;
              amb &= amb - 1u;
              const int c = b * dp + cofs(e);
              bool bit;
              if constexpr (noisy) bit = noisy_exact_bit<BF16>(a, i, c);
              else bit = exact_bit<BF16>(a.X, i, d, a.Wt, c);
              if (bit) atomicOr(&wrow[c >> 5], 1u << (c & 31));
              else atomicAnd(&wrow[c >> 5], ~(1u << (c & 31)));
              ++nre;
            }
          }
        }
      }
      __syncwarp();
      if (!PROJ) {
        for (int j = lane; j < L; j += 32) {
          const uint32_t id = extract_bits(wrow, nwords, j * K, K);
          if (gather) ibuf[j * 32 + p] = static_cast<IdT>(id);
          else if (mode & kStoreIds) reinterpret_cast<IdT*>(a.ids)[static_cast<size_t>(j) * ld + i] = static_cast<IdT>(id);
          if (mode & kStoreIdsRowMajor) a.ids_rm[i * L + j] = id;
        }
      }
      __syncwarp();  // the words are rewritten for the next point
    }
    if (gather) {  // table j of the group's points: one point per lane
      for (int j = 0; j < L; ++j)
        if (lane < np) reinterpret_cast<IdT*>(a.ids)[static_cast<size_t>(j) * ld + i0 + lane] = ibuf[j * 32 + lane];
      __syncwarp();
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) nre += __shfl_xor_sync(0xFFFFFFFFu, nre, off);
  if (lane == 0 && nre) atomicAdd(&a.st->rechecks, nre);
}

}  // namespace

cudaError_t launch_hash_fwht(const FwhtArgs& a, int num_sms, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const int E = a.dp / 32;
  if (a.dp < 32 || a.dp > kFwhtMaxDp || (a.dp & (a.dp - 1)) || a.nblk * E > kFwhtMaxWords)
    return cudaErrorInvalidValue;
  const long long want = ((a.n + 31) / 32 + 7) / 8;  // groups of 32 points, 8 warps per block
  // one wave of resident blocks, each looping over groups (no tail waves, one prologue each)
  auto go = [&](auto kern, size_t smem) -> cudaError_t {
    cudaError_t e = smem_limit(kern, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = blocks_per_sm(&per_sm, kern, 256, smem);
    if (e != cudaSuccess) return e;
    const unsigned grid =
        static_cast<unsigned>(std::min<long long>(want, static_cast<long long>(num_sms) * std::max(1, per_sm)));
    kern<<<grid, 256, smem, s>>>(a);
    return cudaGetLastError();
  };
  const bool proj = (a.mode & kStoreProj) != 0;
  const bool b16 = a.x_bf16 != 0, id16 = a.K <= 16;
  const bool noisy = !proj && a.nsig != 0.f;
#define ACE_FWHT_CASE(EV)                                                                          \
  case EV:                                                                                         \
    if (proj)                                                                                      \
      return b16 ? go(hash_fwht_kernel<true, uint32_t, EV, 1>, FwhtSmem<EV, 2>::bytes)             \
                 : go(hash_fwht_kernel<false, uint32_t, EV, 1>, FwhtSmem<EV, 4>::bytes);           \
    if (noisy) {                                                                                   \
      if (b16)                                                                                     \
        return id16 ? go(hash_fwht_kernel<true, uint16_t, EV, 2>, FwhtSmem<EV, 2>::bytes)          \
                    : go(hash_fwht_kernel<true, uint32_t, EV, 2>, FwhtSmem<EV, 2>::bytes);         \
      return id16 ? go(hash_fwht_kernel<false, uint16_t, EV, 2>, FwhtSmem<EV, 4>::bytes)           \
                  : go(hash_fwht_kernel<false, uint32_t, EV, 2>, FwhtSmem<EV, 4>::bytes);          \
    }                                                                                              \
    if (b16)                                                                                       \
      return id16 ? go(hash_fwht_kernel<true, uint16_t, EV, 0>, FwhtSmem<EV, 2>::bytes)            \
                  : go(hash_fwht_kernel<true, uint32_t, EV, 0>, FwhtSmem<EV, 2>::bytes);           \
    return id16 ? go(hash_fwht_kernel<false, uint16_t, EV, 0>, FwhtSmem<EV, 4>::bytes)             \
                : go(hash_fwht_kernel<false, uint32_t, EV, 0>, FwhtSmem<EV, 4>::bytes);
  switch (E) {
    ACE_FWHT_CASE(1)
    ACE_FWHT_CASE(2)
    ACE_FWHT_CASE(4)
    ACE_FWHT_CASE(8)
    ACE_FWHT_CASE(16)
    ACE_FWHT_CASE(32)
    default:
      return cudaErrorInvalidValue;
  }
#undef ACE_FWHT_CASE
}

}  // namespace ace
