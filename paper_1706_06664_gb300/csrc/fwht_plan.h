// Launch description of the structured-projection engine (hash_fwht.cu), shared by the runtime
// and the kernel.
//
// A detector created with ACE_W_HADAMARD has the projection W[i][c] = D_b[i] H[j][i] for
// column c = b * dp + j (c < K L, i < d): dp = the power of two >= max(d, 32), H the
// Sylvester-Hadamard matrix of order dp (H[j][i] = (-1)^popcount(i & j), unnormalised), and D_b
// a diagonal of random signs per block b of dp columns (D_b[i] = -1 when the SplitMix64 draw of
// index b * dp + i has its lowest bit set).  All of x.w_c for one block are then the fast
// Walsh-Hadamard transform of the sign-flipped x: O(dp log dp) additions instead of d dp
// multiply-adds (§2.2: the Fast-JL family of projections).  The entries are +-1, so the
// binary64 definition of every bit is the usual one (Eq. 1 with this W), and the other engines
// compute the same ids from the stored W.
#pragma once

#include <cstdint>

#include "ace_internal.h"

namespace ace {

constexpr int kFwhtMaxDp = 1024;   // the transform of a row lives in one warp's registers
constexpr int kFwhtMaxWords = 160; // sign words per point (K L <= 4096 + one block's padding)

struct FwhtArgs {
  const void* X;
  int x_bf16;
  long long n;
  int d, dp, m;               // m = log2(dp)
  int K, L, KL, nblk;         // nblk = ceil(K L / dp) blocks of dp columns
  const uint32_t* dsign;      // [nblk][dp / 32] bit i of word (b, i / 32): D_b[i] = -1
  const float* Wt;            // [KL][d] the explicit +-1 W, columns contiguous (binary64 recheck)
  float cband;                // bound = cband * sum|x_i| + babs (the transform's and binary64's errors)
  float babs;
  int mode;                   // HashMode bits (kStoreIds, kStoreIdsRowMajor, kStoreProj)
  void* ids;                  // table-major ids [L][ld]
  long long ld;
  uint32_t* ids_rm;           // [n][L] (kStoreIdsRowMajor)
  float* proj;                // [n][KL] (kStoreProj)
  DevStats* st;
  // privacy noise (§4.5): output c of point p is y_c + nsig * counter_w(nseed, (nbase + p) KL + c);
  // nsig = 0: no noise
  float nsig;
  unsigned long long nseed;
  long long nbase;
};

cudaError_t launch_hash_fwht(const FwhtArgs& a, int num_sms, cudaStream_t s);

// The order dp of the transform for dimension d (the power of two >= max(d, 32)).
inline int fwht_order(int d) {
  int dp = 32;
  while (dp < d) dp *= 2;
  return dp;
}

// Host generator of the structured W (projection_gen.cpp): W [d][KL] and the sign words
// dsign [ceil(KL / dp)][dp / 32] (bit set: D_b[i] = -1).
void generate_projection_hadamard(int d, int K, int L, uint64_t seed, float* W, uint32_t* dsign);

}  // namespace ace
