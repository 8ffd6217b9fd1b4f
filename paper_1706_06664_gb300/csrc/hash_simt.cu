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
#include "guard.cuh"

namespace ace {
namespace {

constexpr int BM = 128;  // points per CTA
constexpr int BN = 128;  // columns per CTA (at most)
constexpr int DK = 32;   // d per staged chunk
constexpr int NT = 256;  // threads: 16 column groups x 16 point groups, 8 x 8 outputs each

// Block `blk` of one detector's hash: tile blk / ntb of 128 points, table block blk % ntb.
template <bool BF16, typename IdT>
__device__ __forceinline__ void hash_simt_block(const HashArgs& a, int tpb, int ntb, long long blk) {
  __shared__ float Xs[BM][DK + 1];
  __shared__ __align__(16) float Ws[DK][BN];
  __shared__ uint32_t bits[BM][BN / 32];
  __shared__ uint32_t amb[BM][BN / 32];
  __shared__ float xn[BM];

  const long long tile = blk / ntb;
  const int tb = static_cast<int>(blk % ntb);
  const int j0 = tb * tpb;
  const int ntab = min(tpb, a.L - j0);
  const int c0 = j0 * a.K;
  const int ncol = ntab * a.K;
  const long long i0 = tile * BM;
  const int npt = static_cast<int>(min(static_cast<long long>(BM), a.n - i0));
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;

  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
  float q = 0.f;

  for (int kc = 0; kc < a.d; kc += DK) {
    for (int e = threadIdx.x; e < BM * DK; e += NT) {
      const int p = e / DK, k = e % DK;
      float v = 0.f;
      if (p < npt && kc + k < a.d) v = load_x<BF16>(a.X, (i0 + p) * a.d + kc + k);
      Xs[p][k] = v;
    }
    for (int e = threadIdx.x; e < DK * BN; e += NT) {
      const int k = e / BN, c = e % BN;
      float v = 0.f;
      if (c < ncol && kc + k < a.d) v = __ldg(a.W + static_cast<size_t>(kc + k) * a.KL + c0 + c);
      Ws[k][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < BM) {
#pragma unroll 8
      for (int k = 0; k < DK; ++k) q = fmaf(Xs[threadIdx.x][k], Xs[threadIdx.x][k], q);
    }
#pragma unroll 4
    for (int k = 0; k < DK; ++k) {
      float xa[8], wb[8];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        xa[r] = Xs[ty * 4 + r][k];
        xa[4 + r] = Xs[64 + ty * 4 + r][k];
      }
      const float4 w0 = *reinterpret_cast<const float4*>(&Ws[k][tx * 4]);
      const float4 w1 = *reinterpret_cast<const float4*>(&Ws[k][64 + tx * 4]);
      wb[0] = w0.x; wb[1] = w0.y; wb[2] = w0.z; wb[3] = w0.w;
      wb[4] = w1.x; wb[5] = w1.y; wb[6] = w1.z; wb[7] = w1.w;
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(xa[r], wb[c], acc[r][c]);
    }
    __syncthreads();
  }

  // ---- guard classification ------------------------------------------------------------
  if (threadIdx.x < BM) {
    xn[threadIdx.x] = norm_upper(q, a.xfac, a.xabs);
    if (!isfinite(q) && tb == 0 && static_cast<int>(threadIdx.x) < npt && !(a.mode & kStoreProj))
      atomicAdd(&a.st->nonfinite, 1ull);
  }
  for (int e = threadIdx.x; e < BM * (BN / 32); e += NT) {
    (&bits[0][0])[e] = 0u;
    (&amb[0][0])[e] = 0u;
  }
  if (a.mode & kStoreProj) {  // measurement path: the binary32 estimates themselves
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int p = (r < 4) ? ty * 4 + r : 64 + ty * 4 + (r - 4);
      if (p < npt) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int col = (c >> 2) * 64 + tx * 4 + (c & 3);
          if (col < ncol) a.proj[(i0 + p) * a.KL + c0 + col] = acc[r][c];
        }
      }
    }
    return;  // nothing else in this mode (the whole block takes this branch)
  }
  float cb[8];
#pragma unroll
  for (int g = 0; g < 2; ++g)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int col = g * 64 + tx * 4 + c;
      cb[g * 4 + c] = col < ncol ? __ldg(a.cB + c0 + col) : 0.f;
    }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int p = (r < 4) ? ty * 4 + r : 64 + ty * 4 + (r - 4);
    const float xu = xn[p];
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      uint32_t sb = 0u, ab = 0u;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int col = g * 64 + tx * 4 + c;
        if (col < ncol) {
          const float s = acc[r][g * 4 + c];
          const float B = fmaf(cb[g * 4 + c], xu, a.babs);
          if (fabsf(s) > B) sb |= (s > 0.f ? 1u : 0u) << c;
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
  for (int base = (threadIdx.x >> 5) * 32; base < BM * (BN / 32); base += NT) {
    const uint32_t mw = (&amb[0][0])[base + lane];
    uint32_t nz = __ballot_sync(0xFFFFFFFFu, mw != 0u && (base + lane) / (BN / 32) < npt);
    while (nz) {
      const int q = __ffs(nz) - 1;
      nz &= nz - 1u;
      const int p = (base + q) / (BN / 32), wi = (base + q) % (BN / 32);
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
        const float bound = __fmaf_ru(a.runc, r, __fmaf_ru(__fmul_ru(a.run64, __ldg(a.cB + col)), xu, a.runabs));
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
    uint32_t id = extract_bits(bits[p], BN / 32, cbit, K);
    const uint32_t am = extract_bits(amb[p], BN / 32, cbit, K);
    if (valid && am) {
      const long long i = i0 + p;
      uint32_t m = am;
      unsigned long long nre = 0;
      while (m) {
        const int k = __ffs(m) - 1;
        m &= m - 1u;
        const int col = c0 + cbit + k;
        const int sg = dot2_sign<BF16>(a.X, i, a.d, a.Wt + static_cast<size_t>(col) * a.d, 1, a.dot2c, a.dot2abs);
        if (sg != 0 ? sg > 0 : exact_bit<BF16>(a.X, i, a.d, a.Wt, col)) id |= 1u << k;
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

template <bool BF16, typename IdT>
__global__ void __launch_bounds__(NT, 2) hash_simt_kernel(HashArgs a, int tpb, int ntb) {
  hash_simt_block<BF16, IdT>(a, tpb, ntb, blockIdx.x);
}

// Many detectors in one launch: block index b of the whole batch belongs to detector g with
// start[g] <= b < start[g + 1]; each detector's blocks run exactly as in its own launch.
template <bool BF16, typename IdT>
__global__ void __launch_bounds__(NT, 2) hash_simt_batched_kernel(const HashArgs* __restrict__ args,
                                                                  const long long* __restrict__ start, int ndet) {
  const long long total = start[ndet];
  for (long long b = blockIdx.x; b < total; b += gridDim.x) {
    int lo = 0, hi = ndet;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (start[mid] <= b) lo = mid;
      else hi = mid;
    }
    const HashArgs a = args[lo];
    const int tpb = BN / a.K;
    const int ntb = (a.L + tpb - 1) / tpb;
    hash_simt_block<BF16, IdT>(a, tpb, ntb, b - start[lo]);
    __syncthreads();  // shared memory is reused by the next block
  }
}

}  // namespace

long long hash_simt_blocks(const HashArgs& a) {
  if (a.n <= 0) return 0;
  const int tpb = BN / a.K;
  const int ntb = (a.L + tpb - 1) / tpb;
  return (a.n + BM - 1) / BM * ntb;
}

cudaError_t launch_hash_simt_batched(const HashArgs* args_dev, const long long* start_dev, int ndet, bool bf16,
                                     bool id16, int num_sms, cudaStream_t s) {
  const unsigned grid = static_cast<unsigned>(num_sms * 2);  // two blocks per SM (registers)
  if (bf16) {
    if (id16) hash_simt_batched_kernel<true, uint16_t><<<grid, NT, 0, s>>>(args_dev, start_dev, ndet);
    else hash_simt_batched_kernel<true, uint32_t><<<grid, NT, 0, s>>>(args_dev, start_dev, ndet);
  } else {
    if (id16) hash_simt_batched_kernel<false, uint16_t><<<grid, NT, 0, s>>>(args_dev, start_dev, ndet);
    else hash_simt_batched_kernel<false, uint32_t><<<grid, NT, 0, s>>>(args_dev, start_dev, ndet);
  }
  return cudaGetLastError();
}

cudaError_t launch_hash_simt(const HashArgs& a, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const int tpb = BN / a.K;  // K <= 24, so tpb >= 5
  const int ntb = (a.L + tpb - 1) / tpb;
  const long long tiles = (a.n + BM - 1) / BM;
  const long long blocks = tiles * ntb;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  const dim3 grid(static_cast<unsigned>(blocks));
  const bool id16 = a.K <= 16;
  if (a.x_bf16) {
    if (id16) hash_simt_kernel<true, uint16_t><<<grid, NT, 0, s>>>(a, tpb, ntb);
    else hash_simt_kernel<true, uint32_t><<<grid, NT, 0, s>>>(a, tpb, ntb);
  } else {
    if (id16) hash_simt_kernel<false, uint16_t><<<grid, NT, 0, s>>>(a, tpb, ntb);
    else hash_simt_kernel<false, uint32_t><<<grid, NT, 0, s>>>(a, tpb, ntb);
  }
  return cudaGetLastError();
}

}  // namespace ace
