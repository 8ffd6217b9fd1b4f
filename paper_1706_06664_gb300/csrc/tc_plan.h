// Launch description of the tensor-core hash kernel (shared by the runtime and the kernel).
#pragma once

#include <cstdint>

#include "ace_internal.h"

namespace ace {

constexpr int kTcMaxChunks = 16;
constexpr int kTcBufs = 2;       // TMEM accumulator buffers (and epilogue warp groups)
constexpr int kTcBufCols = 256;  // columns of one buffer: a chunk has N <= kTcBufCols
constexpr int kMaxD = 64;  // largest d of the resident design (staging and recheck registers)

// One chunk: whole tables [tab0, tab0 + ntab), N = ntab*K rounded up to 16 MMA columns,
// and the byte offsets of its hi and lo operand images inside the resident B image.
struct TcChunk {
  int tab0, ntab, N;
  uint32_t boff_hi, boff_lo;
};

struct TcArgs {
  const void* X;
  int x_bf16;
  long long n, ntiles;
  int d, d_pad, K, L;
  const uint8_t* bimg;  // K-major no-swizzle images of W' (unit columns), hi and lo per chunk
  int bimg_bytes;
  int nchunks;
  TcChunk chunk[kTcMaxChunks];
  float tau, tau_abs, xfac, qmin;  // row bound = tau * ||x||_up + tau_abs (or +inf if q < qmin)
  int mode;
  void* ids;
  long long ld;
  uint32_t* ids_rm;
  uint32_t* counts;
  DevStats* st;
  const float* Wt;  // [KL][d] original W, columns contiguous (binary64 recheck)
  const float* W;   // [d][KL] original W, rows contiguous
  const float* Wp;  // [KL][dp] original W, columns contiguous and zero-padded to dp = d rounded up to 4
  int dp;
  const float* cB32;                // SIMT-engine guard coefficients per column
  float xfac32, xabs32, babs32;     // SIMT-engine norm inflation and absolute allowances
  float dot2c, dot2abs;             // Dot2 filter: bound = dot2c * sum|x_i w_i|^ + dot2abs
  float runc, run64, runabs;        // recheck running bound: runc * R^ + run64 * cB32[c] * ||x||^ + runabs
  float* proj;                      // [n][KL] estimates x.w_c (measurement path, kStoreProj)
  const float* wnorm;               // [KL] ||w_c|| (binary32), to scale x.w'_c back to x.w_c
  unsigned long long* defer;         // (point << 24 | table) per deferred pair; one segment per CTA
  unsigned int* defer_counts;        // entries per segment, written by each CTA at exit
  unsigned long long seg_cap;        // entries per segment
  // dynamic shared-memory layout (bytes)
  int off_a, a_bytes, off_stage, off_bnd, off_bits, off_ctl, smem_bytes;
};

cudaError_t launch_hash_tc(const TcArgs& a, int num_sms, cudaStream_t s);
cudaError_t launch_recheck(const TcArgs& a, int num_sms, cudaStream_t s);

}  // namespace ace
