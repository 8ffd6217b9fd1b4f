// Resolution of the (point, table) pairs that the tensor-core hash kernel deferred: their
// K bits recomputed exactly, binary32 first, then the Dot2 filter, then the binary64
// definition of Eq. 1 for what neither can decide.
#include "guard.cuh"
#include "tc_plan.h"

namespace ace {
namespace {

// Resolves the deferred (point, table) pairs: lane k of an entry's lane group recomputes
// column j K + k as a binary32 FMA chain in index order and decides its bit with the smaller
// of two rigorous bounds on its distance from the binary64 definition: the SIMT engine's a
// priori bound (gamma_d sum|x_i w_i| + d 2^-150, folded into cB32[c] ||x||_up + babs32) and the
// chain's running error bound (u / (1 - u) times the sum of the partial sums' magnitudes,
// accumulated alongside, plus the binary64 sum's own error), which is several times tighter
// where the sum crosses zero -- exactly the deferred columns.  A bit inside both goes to the
// Dot2 filter, and only what Dot2 cannot decide is evaluated in binary64, index order (the
// definition).  GB300 issues binary64 FMAs at a small fraction of the binary32 rate, so the
// filters keep that path to exact ties.  The id is the ballot of the lanes' bits.
template <bool BF16, typename IdT>
__global__ void __launch_bounds__(256) recheck_kernel(const __grid_constant__ TcArgs a, int nseg) {
  // Entries live in nseg per-CTA segments of the deferred list; warp gw works on segment
  // gw % nseg with the other warps of that segment.  Each half warp takes one entry (K <= 16;
  // else a whole warp): lane k recomputes column j K + k.
  __shared__ __align__(16) float xsm[8][2][kMaxD];  // per warp, per half-warp entry
  const int d = a.d, K = a.K, L = a.L, mode = a.mode, dp = a.dp;
  const long long ld = a.ld;
  const void* const X = a.X;
  const float* const Wt = a.Wt;
  const float* const Wp = a.Wp;
  const float* const cB32 = a.cB32;
  const float xfac32 = a.xfac32, xabs32 = a.xabs32, babs32 = a.babs32;
  const float dot2c = a.dot2c, dot2abs = a.dot2abs;
  const float runc = a.runc, run64 = a.run64, runabs = a.runabs;
  IdT* const ids = reinterpret_cast<IdT*>(a.ids);
  uint32_t* const ids_rm = a.ids_rm;
  const uint32_t kmask = (1u << K) - 1u;
  const int lane = threadIdx.x & 31;
  const int width = K <= 16 ? 16 : 32;  // lanes per entry
  const int sub = lane / width, sl = lane % width;
  const unsigned per_warp = 32 / width;
  const unsigned nwarps = gridDim.x * (blockDim.x >> 5);
  const unsigned gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (gw >= nwarps - nwarps % static_cast<unsigned>(nseg) && nwarps >= static_cast<unsigned>(nseg)) return;
  const int seg = static_cast<int>(gw % static_cast<unsigned>(nseg));
  const unsigned lw = gw / static_cast<unsigned>(nseg);             // this warp's rank in the segment
  const unsigned nw = max(1u, nwarps / static_cast<unsigned>(nseg));  // warps per segment
  const unsigned long long cnt = a.defer_counts[seg];
  const unsigned long long* const list = a.defer + a.seg_cap * static_cast<unsigned long long>(seg);
  float* const xe = xsm[threadIdx.x >> 5][sub];  // this entry's x, read as a shared-memory broadcast
  const unsigned long long stride = static_cast<unsigned long long>(nw) * per_warp;
  auto word_at = [&](unsigned long long e) -> unsigned long long { return e < cnt ? list[e] : 0ull; };
  // lane sl's coordinates sl + width m of point i
  auto load_row = [&](bool has, long long i, float (&xv)[4]) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int t = sl + width * m;
      xv[m] = (has && t < d && t < kMaxD) ? load_x<BF16>(X, i * d + t) : 0.f;
    }
  };
  // Software pipeline over this warp's rounds: while round r is computed, the x row of round
  // r + 1 and the entry word of round r + 2 are in flight (each depends on the one before).
  const unsigned long long e0 = static_cast<unsigned long long>(lw) * per_warp + sub;
  unsigned long long w_cur = word_at(e0);
  float xv[4];
  load_row(e0 < cnt, static_cast<long long>(w_cur >> 24), xv);
  unsigned long long w_nxt = word_at(e0 + stride);
  unsigned long long nre = 0;
  for (unsigned long long base = static_cast<unsigned long long>(lw) * per_warp; base < cnt; base += stride) {
    const unsigned long long e = base + sub;
    const bool has = e < cnt;
    const long long i = static_cast<long long>(w_cur >> 24);
    const int j = static_cast<int>(w_cur & 0xFFFFFFull);
    float xn[4];
    load_row(e + stride < cnt, static_cast<long long>(w_nxt >> 24), xn);
    const unsigned long long w_nn = word_at(e + 2 * stride);
    // stage x (zero beyond d) and its squared norm
    float q = 0.f;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int t = sl + width * m;
      if (t < kMaxD) {
        xe[t] = xv[m];
        q = fmaf(xv[m], xv[m], q);
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
      if (off < width) q += __shfl_xor_sync(0xFFFFFFFFu, q, off);
    __syncwarp();
    const float xu = norm_upper(q, xfac32, xabs32);
    const int col = j * K + (sl < K ? sl : 0);
    // binary32 FMA chain in index order (the zero padding adds exact zeros): x from shared
    // memory and the column of W with 16-byte loads
    const float4* wq = reinterpret_cast<const float4*>(Wp + static_cast<size_t>(col) * dp);
    const float4* xq = reinterpret_cast<const float4*>(xe);
    float s32 = 0.f, run = 0.f;  // run: binary32 sum of |partial sums|
#pragma unroll 4
    for (int t4 = 0; t4 < dp / 4; ++t4) {
      const float4 w = __ldg(wq + t4);
      const float4 x = xq[t4];
      s32 = fmaf(x.x, w.x, s32);
      run = __fadd_rn(run, fabsf(s32));
      s32 = fmaf(x.y, w.y, s32);
      run = __fadd_rn(run, fabsf(s32));
      s32 = fmaf(x.z, w.z, s32);
      run = __fadd_rn(run, fabsf(s32));
      s32 = fmaf(x.w, w.w, s32);
      run = __fadd_rn(run, fabsf(s32));
    }
    bool bit = false;
    if (has && sl < K) {
      const float cb = __ldg(cB32 + col);
      const float brun = __fmaf_ru(runc, run, __fmaf_ru(__fmul_ru(run64, cb), xu, runabs));
      if (fabsf(s32) > fminf(fmaf(cb, xu, babs32), brun)) {
        bit = s32 > 0.f;
      } else {
        const int sg = dot2_sign<BF16>(X, i, d, Wp + static_cast<size_t>(col) * dp, 1, dot2c, dot2abs);
        bit = sg != 0 ? sg > 0 : exact_bit<BF16>(X, i, d, Wt, col);
      }
    }
    const uint32_t bal = __ballot_sync(0xFFFFFFFFu, bit);
    const uint32_t id = (bal >> (sub * width)) & kmask;
    if (has && sl == 0) {
      if (mode & kTagDeferred) {  // the insert pass skips this table: count it here
        ids[static_cast<size_t>(j) * ld + i] = static_cast<IdT>(id | 0x8000u);
        atomicAdd(a.counts + (static_cast<size_t>(j) << K) + id, 1u);
      } else if (mode & kStoreIds) {
        ids[static_cast<size_t>(j) * ld + i] = static_cast<IdT>(id);
      }
      if (mode & kStoreIdsRowMajor) ids_rm[i * L + j] = id;
      nre += static_cast<unsigned long long>(K);
    }
    __syncwarp();  // xe is rewritten by the next entry
    w_cur = w_nxt;
    w_nxt = w_nn;
#pragma unroll
    for (int m = 0; m < 4; ++m) xv[m] = xn[m];
  }
  if (nre) atomicAdd(&a.st->rechecks, nre);
}

}  // namespace

cudaError_t launch_recheck(const TcArgs& a, int num_sms, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const int nseg = static_cast<int>(min(static_cast<long long>(num_sms), a.ntiles));  // one segment per CTA
  // one wave: as many 256-thread blocks per SM as its registers and threads allow
  auto go = [&](auto kern) -> cudaError_t {
    // a small shared-memory carveout leaves most of the SM's L1 to cache W (d x KL binary32,
    // read row by row for every entry)
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 25);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0);
    if (e != cudaSuccess) return e;
    const unsigned grid = static_cast<unsigned>(num_sms * max(1, per_sm));
    if (grid * 8u < static_cast<unsigned>(nseg)) return cudaErrorInvalidConfiguration;  // a warp per segment at least
    kern<<<grid, 256, 0, s>>>(a, nseg);
    return cudaGetLastError();
  };
  const bool id16 = a.K <= 16;
  if (a.x_bf16) return id16 ? go(recheck_kernel<true, uint16_t>) : go(recheck_kernel<true, uint32_t>);
  return id16 ? go(recheck_kernel<false, uint16_t>) : go(recheck_kernel<false, uint32_t>);
}

}  // namespace ace
