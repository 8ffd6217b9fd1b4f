// The score family ACE estimates, computed exactly: S(q, D) = sum_i p(q, x_i)^K (Eq. 3) with
// SRP's collision probability p(q, x) = 1 - acos(q.x / (||q|| ||x||)) / pi (§3), for a set of
// queries against a dataset.  Theorem 1 states that ACE's score (1/L) sum_j A_j[H_j(q)] is an
// unbiased estimator of it; the estimator-accuracy workload compares the two (and the random
// sampling estimator RSE, Eq. 10, which is this same sum over a sample scaled by n / L).
//
// One thread per (point, query) pair: binary64 dot product and squared norm of the point in
// index order, the query's squared norm once per block, cos clamped to [-1, 1], acos, and the
// K-th power by repeated squaring; each block writes the sum of its points' terms for its query
// (a fixed-order tree), and a second pass adds the blocks' sums in block order, so the result
// does not depend on scheduling.  A zero vector has no angle: its bits are all 0 (sign(0) = 0),
// while each bit of a non-zero point is 1 with probability 1/2, so p = 1/2 (and p = 1 for two
// zero vectors).  GB300's binary64 rate bounds this pass (2 d + 2 flop per pair and dimension).
#include "ace_internal.h"

namespace ace {
namespace {

template <bool BF16>
__device__ __forceinline__ double ld_elem(const void* p, long long idx) {
  if constexpr (BF16) {
    const unsigned short h = __ldg(reinterpret_cast<const unsigned short*>(p) + idx);
    return static_cast<double>(__uint_as_float(static_cast<unsigned>(h) << 16));
  } else {
    return static_cast<double>(__ldg(reinterpret_cast<const float*>(p) + idx));
  }
}

__device__ __forceinline__ double ipow(double p, int K) {
  double r = 1.0;
  while (K) {
    if (K & 1) r *= p;
    p *= p;
    K >>= 1;
  }
  return r;
}

template <bool BF16>
__global__ void __launch_bounds__(256) exact_score_kernel(const void* __restrict__ Q, const void* __restrict__ D,
                                                          long long nd, int d, int K, double* __restrict__ part) {
  __shared__ double red[256];
  const int q = blockIdx.y;
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  // ||q||^2, index order, by thread 0 (broadcast through shared memory)
  if (threadIdx.x == 0) {
    double qq = 0.0;
    for (int k = 0; k < d; ++k) {
      const double v = ld_elem<BF16>(Q, static_cast<long long>(q) * d + k);
      qq = fma(v, v, qq);
    }
    red[0] = qq;
  }
  __syncthreads();
  const double qq = red[0];
  __syncthreads();
  double term = 0.0;
  if (i < nd) {
    double dot = 0.0, xx = 0.0;
    for (int k = 0; k < d; ++k) {
      const double x = ld_elem<BF16>(D, i * d + k);
      const double y = ld_elem<BF16>(Q, static_cast<long long>(q) * d + k);
      dot = fma(x, y, dot);
      xx = fma(x, x, xx);
    }
    double p;
    if (xx == 0.0 || qq == 0.0) {
      p = (xx == 0.0 && qq == 0.0) ? 1.0 : 0.5;
    } else {
      double c = dot / sqrt(xx * qq);
      c = fmin(1.0, fmax(-1.0, c));
      p = 1.0 - acos(c) / 3.141592653589793;
    }
    term = ipow(p, K);
  }
  red[threadIdx.x] = term;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (static_cast<int>(threadIdx.x) < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[static_cast<size_t>(q) * gridDim.x + blockIdx.x] = red[0];
}

// S[q] = sum of the blocks' sums of query q, in block order (one thread per query).
__global__ void __launch_bounds__(128) exact_score_fold(const double* __restrict__ part, long long nq, int nblk,
                                                        double* __restrict__ S) {
  const long long q = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[static_cast<size_t>(q) * nblk + b];
  S[q] = s;
}

}  // namespace

size_t exact_score_scratch(long long nq, long long nd) {
  const long long nblk = (nd + 255) / 256;
  return static_cast<size_t>(nq) * static_cast<size_t>(nblk) * sizeof(double);
}

cudaError_t launch_exact_score(const void* Q, long long nq, const void* D, long long nd, int d, int bf16, int K,
                               double* part, double* S, cudaStream_t s) {
  if (nq <= 0) return cudaSuccess;
  const long long nblk = (nd + 255) / 256;
  if (nblk > 0) {
    const dim3 grid(static_cast<unsigned>(nblk), static_cast<unsigned>(nq));
    if (bf16) exact_score_kernel<true><<<grid, 256, 0, s>>>(Q, D, nd, d, K, part);
    else exact_score_kernel<false><<<grid, 256, 0, s>>>(Q, D, nd, d, K, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  exact_score_fold<<<static_cast<unsigned>((nq + 127) / 128), 128, 0, s>>>(part, nq, static_cast<int>(nblk), S);
  return cudaGetLastError();
}

}  // namespace ace
