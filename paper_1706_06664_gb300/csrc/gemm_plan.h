// Launch description of the streaming tensor-core hash kernel (hash_gemm.cu), shared by the
// runtime and the kernels.  The streaming engine covers large d: the bfloat16 input X and the
// projection image both stream through shared memory in 64-wide k-blocks, instead of the
// resident design of hash_tc.cu whose whole W' image sits in shared memory (d <= 64).
#pragma once

#include <cstdint>

#include "ace_internal.h"

namespace ace {

constexpr int kGemmBM = 128;     // points per tile = MMA M (one TMEM lane per point)
constexpr int kGemmBN = 256;     // image columns per unit = MMA N
constexpr int kGemmBK = 64;      // d per k-block: one 128-byte swizzle atom of bfloat16
constexpr int kGemmStages = 4;   // shared-memory ring of (X k-block, image k-block) pairs
constexpr int kGemmStagesF8 = 3; // the E4M3 ring: X k-block, two image planes, two X planes

// Deferred (point, column) entry: point << 17 | column << 1 | the bit the tensor cores stored.
constexpr int kGemmEntryShift = 17;

struct GemmArgs {
  const void* X;              // n x d bfloat16 bits, row-major (the tensor map covers it)
  long long n, ntiles;        // points, 128-point tiles
  int d, dp, nkb;             // dp = d rounded up to 64; nkb = dp / 64 k-blocks
  int K, L, KL;
  int tpu, nunits;            // whole tables per 256-column unit; units per tile
  int nprod;                  // 2: x.w'_lo then x.w'_hi (binary32 W split in two); 1: x.w'_hi only;
                              // E4M3 (fp8): 2 passes, the three small products then X1.W1
  int fp8;                    // E4M3 operands: X = X1 + X2 (+ X3) per row, w' = W1 + W2 (+ W3)
  const uint8_t* img8;        // E4M3 image: [unit][k-block][W1, W2][256 rows x 64 bytes], each
                              // block in the K-major no-swizzle canonical layout (16 KB)
  int klp;                    // image rows of one part (nunits * 256); the lo part follows the hi part
  // Row bound B = ca * E + cx * ||x||_up + tau_abs (every column when q < qmin or q is not
  // finite), E bounding the sum over the hi-pass MMA instructions t of
  // ||x_<16t|| WP_t + ||x_Bt|| WB_t, with WP_t, WB_t the largest norms over the columns of
  // w'_hi's prefix [0, 16t) and block [16t, 16t + 16); see hash_gemm.cu.
  float ca, cx, tau_abs, xfac, qmin;
  // E4M3 only: B += ksw (||X2|| + ||X3||) + kt0 T0 + c3 ||X3||, with
  // T0 = ||X2|| (w1m + w2m) + ||X1|| w2m bounding the magnitudes of the three small products
  float ksw, kt0, c3, w1m, w2m;
  int S;                      // MMA instructions per pass (dp / 16)
  const float* wprof;         // [2][nkb] per k-block: sum of its four WP_t, then sqrt of the
                              // sum of its four WB_t^2 (rounded up)
  const float* colf;          // [nunits][256] per image column: its norm (rounded up) when the
                              // columns are not unit vectors (the bound of column c is B colf[c],
                              // WP and WB then being those of the normalised columns); else null
  int mode;                   // HashMode bits (kStoreIds, kStoreIdsRowMajor, kStoreProj)
  void* ids;                  // table-major ids [L][ld] (uint16 for K <= 16, else uint32)
  long long ld;
  uint32_t* ids_rm;           // [n][L] uint32 (kStoreIdsRowMajor)
  float* proj;                // [n][KL] estimates (kStoreProj)
  const float* wnorm;         // [KL] ||w_c||, to scale x.w'_c back to x.w_c (kStoreProj)
  DevStats* st;
  // exact resolution of the deferred columns (binary32 running bound, Dot2, binary64)
  const float* Wt;            // [KL][d] binary32 W, columns contiguous
  const uint16_t* Wt16;       // [KL][d] the same as bfloat16 bits when every entry is a
                              // bfloat16 value (half the recheck's W traffic), else null
  const float* cB32;          // [KL] the SIMT engine's a priori coefficient per column
  float xfac32, xabs32, babs32, dot2c, dot2abs, runc, run64, runabs;
  unsigned long long* defer;  // one segment of seg_cap entries per CTA
  unsigned int* defer_counts; // entries per segment (written by each CTA at exit)
  unsigned long long seg_cap;
  int smem_bytes;
};

// Launches the hash kernel; tmX and tmW are CUtensorMap objects (128-byte aligned, 128 bytes)
// describing X and the image.
cudaError_t launch_hash_gemm(const GemmArgs& a, const void* tmX, const void* tmW, int num_sms, cudaStream_t s);
cudaError_t launch_recheck_cols(const GemmArgs& a, int nseg, int num_sms, cudaStream_t s);
int gemm_smem_bytes();

}  // namespace ace
