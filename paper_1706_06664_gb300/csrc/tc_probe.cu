// Measurement hook: one chain of tcgen05 MMAs on caller-chosen operands.
//
// The tensor-core guard bands (hash_tc.cu, hash_gemm.cu) rest on a model of how one MMA
// instruction accumulates its products and the accumulator in binary32.  This kernel runs
// D = A . B^T (A 128 x kd, B N x kd, K-major) into one TMEM accumulator, exactly like the hash
// kernels do, and returns D, so that a test can feed chosen sums and check the model against
// the hardware: bfloat16 operands as kd/16 kind::f16 MMAs of 128 x N x 16, or E4M3 operands
// as kd/32 kind::f8f6f4 MMAs of 128 x N x 32.
#include "ace_internal.h"
#include "flag_wait.cuh"
#include "tc_ptx.cuh"

namespace ace {
namespace {

using namespace tc;

constexpr long long kProbeWait = 2000000000LL;  // about 1 s at 2 GHz

// FP8: A and B hold E4M3 bytes (kd a multiple of 32); else bfloat16 bit patterns (kd a
// multiple of 16).
template <bool FP8>
__global__ void __launch_bounds__(128, 1)
    tc_probe_kernel(const void* __restrict__ Av, const void* __restrict__ Bv, int kd, int N,
                    float* __restrict__ D, int* __restrict__ status) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ uint64_t bar;
  __shared__ uint32_t taddr;
  constexpr int kEb = FP8 ? 1 : 2;  // bytes per element
  uint8_t* const sa = sm;
  uint8_t* const sb = sm + 128 * kd * kEb;
  const int tid = threadIdx.x, warp = tid >> 5;
  // operands in the K-major, no-swizzle canonical layout (core matrices of 8 rows x 16 bytes)
  if constexpr (FP8) {
    const uint8_t* A = static_cast<const uint8_t*>(Av);
    const uint8_t* B = static_cast<const uint8_t*>(Bv);
    for (int e = tid; e < 128 * kd; e += 128) sa[kmajor_offset8(e / kd, e % kd, kd)] = A[e];
    for (int e = tid; e < N * kd; e += 128) sb[kmajor_offset8(e / kd, e % kd, kd)] = B[e];
  } else {
    const uint16_t* A = static_cast<const uint16_t*>(Av);
    const uint16_t* B = static_cast<const uint16_t*>(Bv);
    for (int e = tid; e < 128 * kd; e += 128)
      *reinterpret_cast<uint16_t*>(sa + kmajor_offset(e / kd, e % kd, kd)) = A[e];
    for (int e = tid; e < N * kd; e += 128)
      *reinterpret_cast<uint16_t*>(sb + kmajor_offset(e / kd, e % kd, kd)) = B[e];
  }
  fence_proxy_async();
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  if (warp == 0) {
    tmem_alloc(&taddr, 256);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = taddr;
  if (tid == 0) {
    // one instruction spans two K-adjacent core matrices (32 bytes of each row)
    const uint32_t sbo = static_cast<uint32_t>(kd) * 8u * kEb;
    const int nk = kd / (32 / kEb);
    for (int ks = 0; ks < nk; ++ks) {
      const uint64_t ad = smem_desc(smem_u32(sa) + 256u * ks, 128, sbo);
      const uint64_t bd = smem_desc(smem_u32(sb) + 256u * ks, 128, sbo);
      if constexpr (FP8) mma_e4m3(tmem, ad, bd, idesc_e4m3(128, N), ks > 0 ? 1u : 0u);
      else mma_bf16(tmem, ad, bd, idesc_bf16(128, N), ks > 0 ? 1u : 0u);
    }
    mma_commit(&bar);
  }
  __syncwarp();
  const int never = 0;
  const bool ok = mbar_wait(&bar, 0, &never, kProbeWait);
  if (!ok && tid == 0) *status = 1;
  tc_fence_after();
  if (ok) {
    uint32_t v[64];
    const int row = warp * 32 + (tid & 31);
    for (int c = 0; c < N; c += 64) {
      tmem_ld64(tmem + (static_cast<uint32_t>(warp * 32) << 16) + static_cast<uint32_t>(c), v);
      tmem_ld_wait(v);
#pragma unroll
      for (int j = 0; j < 64; ++j)
        if (c + j < N) D[static_cast<size_t>(row) * N + c + j] = __uint_as_float(v[j]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, 256);
  }
}

// Failure-detection probe: the library's bounded waits, made to run out on events that never
// happen, with nothing in flight.  kind 0 (the tensor-core kernels' wait): the CTA holds TMEM
// as the hash kernels do, waits for a barrier phase that expects two arrivals and gets one,
// gives up after `limit` cycles (raising ACE_STATUS_TIMEOUT), then waits once more with the
// abort flag already set (which returns at once), frees its TMEM and returns.  kind 1 (the
// batched launch's wait): thread 0 waits for a device flag that nothing sets.  cycles[0]: the
// cycles the first wait took; cycles[1]: those of the aborted wait (kind 0).
__global__ void __launch_bounds__(128, 1)
    wait_probe_kernel(int kind, long long limit, const unsigned int* flag, DevStats* st, long long* cycles) {
  __shared__ uint64_t bar;
  __shared__ uint32_t taddr;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (kind == 1) {
    if (tid == 0) {
      const long long t0 = clock64();
      wait_at_least(flag, 1u, st, limit);
      cycles[0] = clock64() - t0;
      cycles[1] = 0;
    }
    return;
  }
  if (tid == 0) {
    mbar_init(&bar, 2);
    mbar_fence_init();
    abort_flag = 0;
  }
  if (warp == 0) {
    tmem_alloc(&taddr, 32);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0) {
    mbar_arrive(&bar);  // one of the two arrivals the phase needs
    long long t0 = clock64();
    if (!mbar_wait(&bar, 0, &abort_flag, limit)) {
      atomicOr(&st->status, static_cast<unsigned>(ACE_STATUS_TIMEOUT));
      abort_flag = 1;
    }
    cycles[0] = clock64() - t0;
    t0 = clock64();
    mbar_wait(&bar, 0, &abort_flag, limit);  // returns at once: the abort flag is set
    cycles[1] = clock64() - t0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(taddr, 32);
}

}  // namespace

cudaError_t launch_wait_probe(int kind, long long limit, const unsigned int* flag, DevStats* st, long long* cycles,
                              cudaStream_t s) {
  wait_probe_kernel<<<1, 128, 0, s>>>(kind, limit, flag, st, cycles);
  return cudaGetLastError();
}

cudaError_t launch_tc_probe(const void* A, const void* B, int kd, int N, bool fp8, float* D, int* status,
                            cudaStream_t s) {
  const int smem = (128 + N) * kd * (fp8 ? 1 : 2);
  auto go = [&](auto kern) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<1, 128, smem, s>>>(A, B, kd, N, D, status);
    return cudaGetLastError();
  };
  return fp8 ? go(tc_probe_kernel<true>) : go(tc_probe_kernel<false>);
}

}  // namespace ace
