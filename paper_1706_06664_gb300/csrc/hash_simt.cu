// SRP hashing on the SIMT cores in binary32 ("plain FP32 GPU path").
//
// One CTA projects a tile of 128 points onto the columns of `tpb` whole tables
// (tpb = floor(128 / K), so a table never straddles two CTAs), packs each table's K sign
// bits into its bucket id (Eq. 2) and then, per mode, writes the ids and/or increments the
// count arrays (Algorithm 1 counting phase).
//
// Exactness (Eq. 1 as defined in guard.cuh): every accumulator is one sequential binary32
// FMA chain over i = 0..d-1 (zero padding adds exact zeros), so
//   |s32 - s| <= gamma_d sum_i |x_i w_i| + d 2^-150,  gamma_d = d 2^-24 / (1 - d 2^-24),
// and the binary64 reference satisfies |s64 - s| <= gamma64_d sum_i |x_i w_i|.  With
// sum |x_i w_i| <= ||x|| ||w_c||, the host folds both gammas, ||w_c|| and a 2% margin into
// cB[c]; when |s32| > cB[c] * ||x||_up + babs the sign of s32 is the sign of s64 (and s64
// is non-zero); otherwise the Dot2 filter (guard.cuh) decides the bit, and the binary64
// definition only what Dot2 cannot (exact ties, NaN, overflow).  At d = 1024 about 1.6
// columns per point land inside the binary32 bound; a binary64 chain of 1024 dependent FMAs
// per such column cost four times the projection itself on GB300.
//
// Staging: d is walked in chunks of DK coordinates; each chunk of X (k-major) and of the
// block's W columns is double-buffered in shared memory and filled by asynchronous copies
// while the previous chunk is multiplied.
#include "flag_wait.cuh"
#include "guard.cuh"
#include "score_block.cuh"
#include "launch_cache.h"

namespace ace {
namespace {

constexpr int DK = 32;   // d per staged chunk
constexpr int NT = 256;  // threads: 16 column groups x 16 point groups

// Tile variants: RM points x NC columns per thread (RM, NC in {4, 8}); a block covers
// BM = 16 RM points and BN = 16 NC columns (whole tables: floor(BN / K) of them).  The point
// rows of a thread are groups of four, 64 apart; its columns likewise.
template <int RM, int NC>
struct SimtTile {
  static constexpr int BM = 16 * RM, BN = 16 * NC, NW = BN / 32 > 0 ? BN / 32 : 1;
  // shared-memory layout (bytes), carved from one dynamic buffer; the W and X chunks are
  // double-buffered (the next chunk's copies are in flight while this one is multiplied)
  static constexpr int XLD = BM + 4;  // X chunk stored k-major: 16-byte rows of four points per load
  static constexpr size_t ws_bytes = sizeof(float) * DK * BN, xs_bytes = sizeof(float) * DK * XLD;
  static constexpr size_t off_ws = 0;                                         // float [2][DK][BN]
  static constexpr size_t off_xs = off_ws + 2 * ws_bytes;                     // float [2][DK][XLD]
  static constexpr size_t off_bits = off_xs + 2 * xs_bytes;                   // uint32 [BM][NW]
  static constexpr size_t off_amb = off_bits + sizeof(uint32_t) * BM * NW;    // uint32 [BM][NW]
  static constexpr size_t off_xn = off_amb + sizeof(uint32_t) * BM * NW;      // float [BM]
  static constexpr size_t bytes = off_xn + sizeof(float) * BM;
};
constexpr size_t kSimtSmemMax = SimtTile<8, 8>::bytes;
static_assert(SimtTile<8, 4>::bytes <= kSimtSmemMax && SimtTile<4, 8>::bytes <= kSimtSmemMax, "smem");

// Asynchronous 4-byte copy global -> shared (cp.async, completion by group).
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Block `blk` of one detector's hash: tile blk / ntb of BM points, table block blk % ntb.
// NOISY: the variant that can add privacy noise (used when a detector of the launch has it on;
// a separate instantiation, so that the noise-free kernel carries none of its registers).
template <bool BF16, typename IdT, int RM, int NC, bool NOISY>
__device__ __forceinline__ void hash_simt_block(const HashArgs& a, int tpb, int ntb, long long blk, uint8_t* sbuf) {
  using T = SimtTile<RM, NC>;
  constexpr int BM = T::BM, BN = T::BN, NW = T::NW;
  auto Wbuf = [&](int b) { return reinterpret_cast<float (*)[BN]>(sbuf + T::off_ws + b * T::ws_bytes); };
  constexpr int XLD = T::XLD;
  auto Xbuf = [&](int b) { return reinterpret_cast<float (*)[XLD]>(sbuf + T::off_xs + b * T::xs_bytes); };
  uint32_t (*bits)[NW] = reinterpret_cast<uint32_t (*)[NW]>(sbuf + T::off_bits);
  uint32_t (*amb)[NW] = reinterpret_cast<uint32_t (*)[NW]>(sbuf + T::off_amb);
  float* xn = reinterpret_cast<float*>(sbuf + T::off_xn);

  const long long tile = blk / ntb;
  const int tb = static_cast<int>(blk % ntb);
  const int j0 = tb * tpb;
  const int ntab = min(tpb, a.L - j0);
  const int c0 = j0 * a.K;
  const int ncol = ntab * a.K;
  const long long i0 = tile * BM;
  const int npt = static_cast<int>(min(static_cast<long long>(BM), a.n - i0));
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  auto prow = [&](int r) { return (r >> 2) * 64 + ty * 4 + (r & 3); };  // point of register row r
  auto pcol = [&](int c) { return (c >> 2) * 64 + tx * 4 + (c & 3); };  // column of register column c

  float acc[RM][NC];
#pragma unroll
  for (int r = 0; r < RM; ++r)
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[r][c] = 0.f;
  float q = 0.f;

  // Chunk kc of X and W into buffer b: binary32 elements by asynchronous 4-byte copies (one
  // group per chunk), zeros and bfloat16 or regenerated values by plain stores.
  auto stage = [&](int kc, int b) {
    float (*Xs)[XLD] = Xbuf(b);
    float (*Ws)[BN] = Wbuf(b);
    for (int e = threadIdx.x; e < BM * DK; e += NT) {
      const int p = e / DK, k = e % DK;
      const bool in = p < npt && kc + k < a.d;
      if constexpr (BF16) {
        Xs[k][p] = in ? load_x<true>(a.X, (i0 + p) * a.d + kc + k) : 0.f;
      } else {
        if (in) cp_async4(&Xs[k][p], static_cast<const float*>(a.X) + (i0 + p) * a.d + kc + k);
        else Xs[k][p] = 0.f;
      }
    }
    if (a.wgen) {  // ACE_W_COUNTER: the tile is regenerated from the seed
      for (int e = threadIdx.x; e < DK * BN; e += NT) {
        const int k = e / BN, c = e % BN;
        Ws[k][c] = (c < ncol && kc + k < a.d) ? counter_w(a.wseed, static_cast<size_t>(kc + k) * a.KL + c0 + c) : 0.f;
      }
    } else {
      for (int e = threadIdx.x; e < DK * BN; e += NT) {
        const int k = e / BN, c = e % BN;
        if (c < ncol && kc + k < a.d) cp_async4(&Ws[k][c], a.W + static_cast<size_t>(kc + k) * a.KL + c0 + c);
        else Ws[k][c] = 0.f;
      }
    }
    cp_async_commit();
  };
  stage(0, 0);
  for (int kc = 0, b = 0; kc < a.d; kc += DK, b ^= 1) {
    if (kc + DK < a.d) {
      stage(kc + DK, b ^ 1);  // its buffer was last read before the previous chunk's closing barrier
      cp_async_wait1();       // this chunk's copies (the older group) have landed
    } else {
      cp_async_wait0();
    }
    __syncthreads();
    float (*Xs)[XLD] = Xbuf(b);
    float (*Ws)[BN] = Wbuf(b);
    // the chunk's coordinates below d only (the zero padding of the last chunk would add exact
    // zeros: skipping it changes no sum)
    const int kn = min(DK, a.d - kc);
    if (threadIdx.x < BM) {
#pragma unroll 8
      for (int k = 0; k < kn; ++k) q = fmaf(Xs[k][threadIdx.x], Xs[k][threadIdx.x], q);
    }
#pragma unroll 4
    for (int k = 0; k < kn; ++k) {
      float xa[RM], wb[NC];
#pragma unroll
      for (int g = 0; g < RM / 4; ++g) {  // rows 4 g .. 4 g + 3 are points g 64 + 4 ty .. + 3
        const float4 x4 = *reinterpret_cast<const float4*>(&Xs[k][g * 64 + ty * 4]);
        xa[4 * g] = x4.x;
        xa[4 * g + 1] = x4.y;
        xa[4 * g + 2] = x4.z;
        xa[4 * g + 3] = x4.w;
      }
#pragma unroll
      for (int g = 0; g < NC / 4; ++g) {
        const float4 w = *reinterpret_cast<const float4*>(&Ws[k][g * 64 + tx * 4]);
        wb[4 * g] = w.x;
        wb[4 * g + 1] = w.y;
        wb[4 * g + 2] = w.z;
        wb[4 * g + 3] = w.w;
      }
#pragma unroll
      for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[r][c] = fmaf(xa[r], wb[c], acc[r][c]);
    }
    __syncthreads();
  }

  // ---- guard classification ------------------------------------------------------------
  if (threadIdx.x < BM) {
    xn[threadIdx.x] = norm_upper(q, a.xfac, a.xabs);
    if (!isfinite(q) && tb == 0 && static_cast<int>(threadIdx.x) < npt && !(a.mode & kStoreProj))
      atomicAdd(&a.st->nonfinite, 1ull);
  }
  for (int e = threadIdx.x; e < BM * NW; e += NT) {
    (&bits[0][0])[e] = 0u;
    (&amb[0][0])[e] = 0u;
  }
  if (a.mode & kStoreProj) {  // measurement path: the binary32 estimates themselves
#pragma unroll
    for (int r = 0; r < RM; ++r) {
      const int p = prow(r);
      if (p < npt) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int col = pcol(c);
          if (col < ncol) a.proj[(i0 + p) * a.KL + c0 + col] = acc[r][c];
        }
      }
    }
    return;  // nothing else in this mode (the whole block takes this branch)
  }
  float cb[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const int col = pcol(c);
    cb[c] = col < ncol ? __ldg(a.cB + c0 + col) : 0.f;
  }
  __syncthreads();
  // privacy noise (§4.5): the sign of x.w_c + eta is taken.  eta is added in place; its
  // binary32 rounding and the addition's add at most 2^-24 (|eta| + |sum|) <= 2^-24 (8 nsig +
  // |sum|) to the distance from the definition (|eta| <= 8 nsig), allowed for with a factor 2.
  const bool noisy = NOISY && a.nsig != 0.f;
  float nall = 0.f;
  if (noisy) {
    nall = __fmul_ru(8.f, a.nsig);
#pragma unroll
    for (int r = 0; r < RM; ++r) {
      const uint64_t rb = static_cast<uint64_t>(a.nbase + i0 + prow(r)) * a.KL + c0;
#pragma unroll
      for (int c = 0; c < NC; ++c)
        acc[r][c] = __fadd_rn(acc[r][c], __fmul_rn(a.nsig, counter_w(a.nseed, rb + pcol(c))));
    }
  }
#pragma unroll
  for (int r = 0; r < RM; ++r) {
    const int p = prow(r);
    const float xu = xn[p];
#pragma unroll
    for (int g = 0; g < NC / 4; ++g) {
      uint32_t sb = 0u, ab = 0u;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int col = g * 64 + tx * 4 + c;
        if (col < ncol) {
          const float sv = acc[r][g * 4 + c];
          float B = fmaf(cb[g * 4 + c], xu, a.babs);
          if (noisy) B = __fmaf_ru(1.1920928955078125e-07f, __fadd_ru(nall, fabsf(sv)), B);
          if (fabsf(sv) > B) sb |= (sv > 0.f ? 1u : 0u) << c;
          else ab |= 1u << c;
        }
      }
      const int col0 = g * 64 + tx * 4;
      if (sb) atomicOr(&bits[p][col0 >> 5], sb << (col0 & 31));
      if (ab) atomicOr(&amb[p][col0 >> 5], ab << (col0 & 31));
    }
  }
  __syncthreads();

  // ---- warp recheck of the columns inside the bound ----------------------------------------
  // Each non-zero word of the ambiguity bitmap goes to one warp (a ballot over 32 words at a
  // time finds them).  For each (point, column) in it, the warp splits the dot product over
  // its 32 lanes (lane l: coordinates l, l + 32, ...; binary32 FMA chains), joins the lanes'
  // sums by a butterfly of shuffles and keeps, alongside, the sum R of the magnitudes of every
  // rounded partial result.  u R / (1 - u), inflated for R's own rounding, plus the binary64
  // sum's error bounds the distance of the result from the definition whatever the summation
  // tree, and near zero it is far tighter than the a priori bound: a decided bit leaves the
  // bitmap.  Every lane computes the same values (addition is commutative), so the loop stays
  // uniform.
  const int lane = threadIdx.x & 31;
  for (int base = (threadIdx.x >> 5) * 32; base < BM * NW; base += NT) {
    const uint32_t mw = base + lane < BM * NW ? (&amb[0][0])[base + lane] : 0u;
    uint32_t nz = __ballot_sync(0xFFFFFFFFu, mw != 0u && (base + lane) / NW < npt);
    while (nz) {
      const int q = __ffs(nz) - 1;
      nz &= nz - 1u;
      const int p = (base + q) / NW, wi = (base + q) % NW;
      uint32_t m = __shfl_sync(0xFFFFFFFFu, mw, q);
      const long long xb = (i0 + p) * static_cast<long long>(a.d);
      const float xu = xn[p];
      uint32_t done = 0u, set = 0u;
      while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1u;
        const int col = c0 + wi * 32 + b;
        const float* w = a.Wt + static_cast<size_t>(col) * a.d;
        float s = 0.f, r = 0.f;
        for (int t = lane; t < a.d; t += 32) {
          s = fmaf(load_x<BF16>(a.X, xb + t), __ldg(w + t), s);
          r = __fadd_rn(r, fabsf(s));
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          const float so = __shfl_xor_sync(0xFFFFFFFFu, s, off);
          const float ro = __shfl_xor_sync(0xFFFFFFFFu, r, off);
          s = __fadd_rn(s, so);
          r = __fadd_rn(__fadd_rn(r, ro), fabsf(s));
        }
        float bound = __fmaf_ru(a.runc, r, __fmaf_ru(__fmul_ru(a.run64, __ldg(a.cB + col)), xu, a.runabs));
        if (noisy) {
          const float eta = __fmul_rn(a.nsig, counter_w(a.nseed, static_cast<uint64_t>(a.nbase + i0 + p) * a.KL + col));
          s = __fadd_rn(s, eta);
          bound = __fmaf_ru(1.1920928955078125e-07f, __fadd_ru(fabsf(eta), fabsf(s)), bound);
        }
        if (fabsf(s) > bound) {
          done |= 1u << b;
          if (s > 0.f) set |= 1u << b;
        }
      }
      if (lane == 0 && done) {
        bits[p][wi] |= set;
        amb[p][wi] &= ~done;
      }
    }
  }
  __syncthreads();

  // ---- pack, recheck, store / insert -----------------------------------------------------
  const int K = a.K;
  for (int e = threadIdx.x; e < ntab * BM; e += NT) {
    const int t = e / BM, p = e % BM;
    const bool valid = p < npt;
    const int cbit = t * K;
    uint32_t id = extract_bits(bits[p], NW, cbit, K);
    const uint32_t am = extract_bits(amb[p], NW, cbit, K);
    if (valid && am) {
      const long long i = i0 + p;
      uint32_t m = am;
      unsigned long long nre = 0;
      while (m) {
        const int k = __ffs(m) - 1;
        m &= m - 1u;
        const int col = c0 + cbit + k;
        const float* wc = a.Wt + static_cast<size_t>(col) * a.d;
        if (noisy) {  // eta in binary32 for Dot2; exactly in binary64 (a binary32 times k/4, |k| <= 32)
          const float cw = counter_w(a.nseed, static_cast<uint64_t>(a.nbase + i) * a.KL + col);
          const int sg = dot2_sign_add<BF16>(a.X, i, a.d, wc, 1, a.dot2c, a.dot2abs, __fmul_rn(a.nsig, cw));
          if (sg != 0 ? sg > 0
                      : exact_bit_add<BF16>(a.X, i, a.d, a.Wt, col, static_cast<double>(a.nsig) * static_cast<double>(cw)))
            id |= 1u << k;
        } else {
          const int sg = dot2_sign<BF16>(a.X, i, a.d, wc, 1, a.dot2c, a.dot2abs);
          if (sg != 0 ? sg > 0 : exact_bit<BF16>(a.X, i, a.d, a.Wt, col)) id |= 1u << k;
        }
        ++nre;
      }
      atomicAdd(&a.st->rechecks, nre);
    }
    const int j = j0 + t;
    if (valid) {
      if (a.mode & kStoreIds) reinterpret_cast<IdT*>(a.ids)[static_cast<size_t>(j) * a.ld + i0 + p] = static_cast<IdT>(id);
      if (a.mode & kStoreIdsRowMajor) a.ids_rm[(i0 + p) * a.L + j] = id;
    }
    if (a.mode & kInsert) {
      const uint32_t key = valid ? id : 0xFFFFFFFFu;
      const uint32_t grp = __match_any_sync(0xFFFFFFFFu, key);
      if (valid && lane == __ffs(grp) - 1)
        atomicAdd(a.counts + (static_cast<size_t>(j) << K) + id, static_cast<uint32_t>(__popc(grp)));
    }
  }
}

// The SIMT tile variants (RM, NC): 0 = (8, 8), 1 = (8, 4), 2 = (4, 8), 3 = (4, 4).
__host__ __device__ constexpr int tile_rows(int t) { return (t & 2) ? 4 : 8; }
__host__ __device__ constexpr int tile_cols(int t) { return (t & 1) ? 4 : 8; }

// Tables per block and table blocks of a detector for tile variant t.
__host__ __device__ inline void tile_blocks(const HashArgs& a, int t, int& tpb, int& ntb) {
  tpb = 16 * tile_cols(t) / a.K;  // K <= 24, so tpb >= 2
  ntb = (a.L + tpb - 1) / tpb;
}

template <bool BF16, typename IdT, bool NOISY>
__device__ __forceinline__ void hash_block_any(const HashArgs& a, long long blk, uint8_t* sbuf) {
  int tpb, ntb;
  tile_blocks(a, a.tile, tpb, ntb);
  switch (a.tile) {
    case 1: hash_simt_block<BF16, IdT, 8, 4, NOISY>(a, tpb, ntb, blk, sbuf); break;
    case 2: hash_simt_block<BF16, IdT, 4, 8, NOISY>(a, tpb, ntb, blk, sbuf); break;
    case 3: hash_simt_block<BF16, IdT, 4, 4, NOISY>(a, tpb, ntb, blk, sbuf); break;
    default: hash_simt_block<BF16, IdT, 8, 8, NOISY>(a, tpb, ntb, blk, sbuf); break;
  }
}

template <bool BF16, typename IdT, bool NOISY>
__global__ void __launch_bounds__(NT, 2) hash_simt_kernel(HashArgs a) {
  extern __shared__ __align__(16) uint8_t sbuf[];
  hash_block_any<BF16, IdT, NOISY>(a, blockIdx.x, sbuf);
}

// Every detector's insert_score in one persistent launch.  Work items are dispensed in order
// from one counter: the hash blocks of all detectors (binary32 engine, counts incremented),
// then their query-phase blocks, then their score and flag blocks.  A query block of detector
// g waits until every hash block of g is done (hdone[g]), and a flag block until g's last
// query block has derived mu, sigma and the threshold (sready[g]).  An item only ever waits
// for items dispensed before it, all of which are held by running blocks, so every wait ends.
constexpr int kBatchSmemDets = 2048;  // item prefixes kept in shared memory up to this many detectors

// The detector of item b: binary search of the prefixes (in shared memory when they fit).
template <typename T>
__device__ __forceinline__ int find_det(const T* start, int ndet, long long b) {
  int lo = 0, hi = ndet;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (static_cast<long long>(start[mid]) <= b) lo = mid;
    else hi = mid;
  }
  return lo;
}

template <bool BF16, typename IdT, bool NOISY>
__global__ void __launch_bounds__(NT, 2)
    batch_kernel(const HashArgs* __restrict__ args, const ScoreJob* __restrict__ jobs,
                 const long long* __restrict__ hstart, const long long* __restrict__ sstart, int ndet,
                 unsigned long long* next, unsigned int* hdone, unsigned int* sready) {
  extern __shared__ __align__(16) uint8_t sbuf[];
  __shared__ long long item_s;
  const long long H = hstart[ndet], S = sstart[ndet];
  // item prefixes as 32-bit offsets in shared memory (after the hash tile), when they fit
  const bool pre_smem = ndet <= kBatchSmemDets && H + 2 * S < 0x7FFFFFFFLL;
  unsigned int* const hs32 = reinterpret_cast<unsigned int*>(sbuf + kSimtSmemMax);
  unsigned int* const ss32 = hs32 + kBatchSmemDets + 1;
  if (pre_smem) {
    for (int g = threadIdx.x; g <= ndet; g += NT) {
      hs32[g] = static_cast<unsigned int>(hstart[g]);
      ss32[g] = static_cast<unsigned int>(sstart[g]);
    }
  }
  __syncthreads();
  auto hdet = [&](long long b) { return pre_smem ? find_det(hs32, ndet, b) : find_det(hstart, ndet, b); };
  auto sdet = [&](long long b) { return pre_smem ? find_det(ss32, ndet, b) : find_det(sstart, ndet, b); };
  const long long total = H + 2 * S;
  for (;;) {
    if (threadIdx.x == 0) item_s = static_cast<long long>(atomicAdd(next, 1ull));
    __syncthreads();
    const long long it = item_s;
    __syncthreads();
    if (it >= total) break;
    if (it < H) {
      const int g = hdet(it);
      const HashArgs a = args[g];  // a copy: the block's loops read these fields many times
      hash_block_any<BF16, IdT, NOISY>(a, it - (pre_smem ? static_cast<long long>(hs32[g]) : hstart[g]), sbuf);
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(hdone + g, 1u);
      }
    } else if (it < H + S) {
      const long long b = it - H;
      const int g = sdet(b);
      const ScoreJob j = jobs[g];
      if (threadIdx.x == 0) wait_at_least(hdone + g, static_cast<unsigned int>(hstart[g + 1] - hstart[g]), j.st);
      __syncthreads();
      const bool last = score_block<IdT, false>(static_cast<const IdT*>(j.ids), j.ld, j.n, j.K, j.L, j.alpha, j.counts,
                                                j.sums, j.st, b - sstart[g], sstart[g + 1] - sstart[g]);
      if (last) {  // thread 0 of the block that derived mu, sigma and t
        __threadfence();
        atomicExch(sready + g, 1u);
      }
    } else {
      const long long b = it - H - S;
      const int g = sdet(b);
      const ScoreJob j = jobs[g];
      if (threadIdx.x == 0) wait_at_least(sready + g, 1u, j.st);
      __syncthreads();
      flags_block(j, b - sstart[g]);
    }
    __syncthreads();  // shared memory is reused by the next item
  }
}

}  // namespace

int simt_tile_rows(int t) { return tile_rows(t); }
int simt_tile_cols(int t) { return tile_cols(t); }

long long hash_simt_blocks(const HashArgs& a) {
  if (a.n <= 0) return 0;
  int tpb, ntb;
  tile_blocks(a, a.tile, tpb, ntb);
  return (a.n + 16 * tile_rows(a.tile) - 1) / (16 * tile_rows(a.tile)) * ntb;
}

cudaError_t launch_batch(const HashArgs* args_dev, const ScoreJob* jobs_dev, const long long* hstart_dev,
                         const long long* sstart_dev, int ndet, unsigned long long* next, unsigned int* hdone,
                         unsigned int* sready, bool bf16, bool id16, bool noisy, int num_sms, cudaStream_t s) {
  const size_t smem = kSimtSmemMax + 2 * sizeof(unsigned int) * (kBatchSmemDets + 1);
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = smem_limit(kern, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = blocks_per_sm(&per_sm, kern, NT, smem);
    if (e != cudaSuccess) return e;
    kern<<<static_cast<unsigned>(num_sms * max(1, per_sm)), NT, smem, s>>>(args_dev, jobs_dev, hstart_dev, sstart_dev,
                                                                          ndet, next, hdone, sready);
    return cudaGetLastError();
  };
  if (noisy) {
    if (bf16) return id16 ? go(batch_kernel<true, uint16_t, true>) : go(batch_kernel<true, uint32_t, true>);
    return id16 ? go(batch_kernel<false, uint16_t, true>) : go(batch_kernel<false, uint32_t, true>);
  }
  if (bf16) return id16 ? go(batch_kernel<true, uint16_t, false>) : go(batch_kernel<true, uint32_t, false>);
  return id16 ? go(batch_kernel<false, uint16_t, false>) : go(batch_kernel<false, uint32_t, false>);
}

cudaError_t launch_hash_simt(const HashArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const long long blocks = hash_simt_blocks(a);
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  const dim3 grid(static_cast<unsigned>(blocks));
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = smem_limit(kern, static_cast<int>(kSimtSmemMax));
    if (e != cudaSuccess) return e;
    kern<<<grid, NT, kSimtSmemMax, s>>>(a);
    return cudaGetLastError();
  };
  const bool id16 = a.K <= 16;
  if (a.nsig != 0.f) {
    if (a.x_bf16) return id16 ? go(hash_simt_kernel<true, uint16_t, true>) : go(hash_simt_kernel<true, uint32_t, true>);
    return id16 ? go(hash_simt_kernel<false, uint16_t, true>) : go(hash_simt_kernel<false, uint32_t, true>);
  }
  if (a.x_bf16) return id16 ? go(hash_simt_kernel<true, uint16_t, false>) : go(hash_simt_kernel<true, uint32_t, false>);
  return id16 ? go(hash_simt_kernel<false, uint16_t, false>) : go(hash_simt_kernel<false, uint32_t, false>);
}

}  // namespace ace
