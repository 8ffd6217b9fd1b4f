// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "ace.h"
#include "exact_div.h"

namespace ace {

// Device-resident running state of one detector.  All sums are exact integers; the three
// doubles are the statistics of the last score call (for ace_stats).
struct DevStats {
  unsigned long long n_scored;   // N
  unsigned long long S1[2];      // lo, hi
  unsigned long long S2[2];      // lo, hi
  unsigned long long Q[2];       // scratch for ace_stats: sum of count^2
  unsigned long long rechecks;   // binary64 recomputations
  unsigned long long nonfinite;  // points with a non-finite squared norm
  unsigned long long deferred;   // (point, table) pairs the tensor-core engine deferred
  unsigned int status;           // ACE_STATUS_* bits
  unsigned int done;             // blocks of the running score kernel that have folded (reset by its last)
  double mu, sigma, threshold;
};

enum HashMode : int {
  kStoreIds = 1,      // write ids to the table-major scratch [L][ld]
  kInsert = 2,        // increment the count arrays
  kStoreIdsRowMajor = 4,  // write uint32 ids point-major [n][L] (ace_hash)
  kStoreProj = 8,         // write the engine's binary32 projection estimates [n][KL] (ace_project)
  // Tensor-core engine, 16-bit ids, K <= 15: a deferred table's id is stored with bit 15 set
  // (a value no count range holds, so the insert pass skips it), and the recheck kernel stores
  // the resolved id, still tagged, and increments its count itself.  The insert pass can then
  // run while the deferred tables are resolved; the score gather masks the tag off.
  kTagDeferred = 16
};

// The integer-only projection entry of ACE_W_COUNTER detectors (§3.4 regenerates projections
// from stored seeds instead of storing them): W.flat[f] = (popcount(z_f) - 32) / 4, z_f the
// SplitMix64 draw t = f of the detector's seed (the same counter-mode definition as the
// Box-Muller generator: finaliser of seed + (f + 1) * 0x9E3779B97F4A7C15).  popcount of 64
// fair bits is Binomial(64, 1/2): the entry has mean 0 and variance exactly 1, takes the 65
// values k/4, |k| <= 32 (all bfloat16 values), and is computed exactly on host and device
// alike, so kernels can regenerate W tiles instead of reading them.
__host__ __device__ inline float counter_w(uint64_t seed, uint64_t f) {
  uint64_t z = seed + (f + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
#ifdef __CUDA_ARCH__
  const int pc = __popcll(z);
#else
  const int pc = __builtin_popcountll(z);
#endif
  return static_cast<float>(pc - 32) * 0.25f;
}

// Everything a hash kernel needs.  Columns c = j*K + k; W is d x KL row-major.
struct HashArgs {
  const void* X;        // n x d, binary32 or bfloat16 bits
  int x_bf16;           // 0: binary32, 1: bfloat16
  long long n;
  int d, K, L, KL;
  const float* W;       // [d][KL] binary32 (null when wgen: the tiles are regenerated)
  unsigned long long wseed;  // ACE_W_COUNTER: the seed of counter_w
  int wgen;             // 1: W tiles are regenerated from wseed (counter_w) instead of read
  const float* Wt;      // [KL][d] binary32 (columns contiguous, for the binary64 recheck)
  const float* cB;      // [KL] guard coefficient: margin * gamma * ||w_c|| (rounded up)
  float xfac;           // squared-norm inflation (1 + 2 gamma_d + slack)
  float xabs;           // squared-norm underflow allowance
  float babs;           // absolute allowance in the projection bound
  float dot2c, dot2abs; // Dot2 filter (before binary64): bound = dot2c * sum|x_i w_i|^ + dot2abs
  float runc, run64, runabs;  // warp recheck: bound = runc * R^ + run64 * cB[c] * ||x||^ + runabs
  int mode;             // HashMode bits
  void* ids;            // scratch ids (uint16 when K <= 16, else uint32), [L][ld]
  long long ld;         // leading dimension of the scratch ids (>= n)
  uint32_t* ids_rm;     // [n][L] uint32 (kStoreIdsRowMajor)
  uint32_t* counts;     // [L][2^K]
  DevStats* st;
  float* proj;          // [n][KL] (kStoreProj)
  int tile;             // SIMT tile variant (0: 128 points x 128 columns per block; 1: 128 x 64;
                        // 2: 64 x 128; 3: 64 x 64)
  // privacy noise (§4.5; ace_set_privacy): projection c of point p is x.w_c + eta with
  // eta = nsig * counter_w(nseed, (nbase + p) * KL + c); nsig = 0: no noise
  float nsig;
  unsigned long long nseed;
  long long nbase;
};

// One detector's share of a batched query phase and flags pass.
struct ScoreJob {
  const void* ids;  // table-major ids [L][ld]
  long long ld, n;
  int K, L;
  double alpha;
  const uint32_t* counts;
  uint32_t* sums;
  DevStats* st;
  DivConst div;
  double* scores;   // may be null
  uint8_t* flags;   // may be null
};

// Kernels launched from the runtime (each returns the launch error).
cudaError_t launch_hash_simt(const HashArgs& a, cudaStream_t s);
cudaError_t launch_score_gather(const void* ids, int ids16, long long ld, long long n, int K, int L, double alpha,
                                const uint32_t* counts, uint32_t* sums, DevStats* st, cudaStream_t s);
cudaError_t launch_flags(const uint32_t* sums, long long n, const DivConst& div, const DevStats* st,
                         double* scores, uint8_t* flags, cudaStream_t s);
cudaError_t launch_insert_from_ids(const void* ids, int ids16, long long ld, long long n, int K, int L,
                                   uint32_t* counts, int num_sms, cudaStream_t s);
cudaError_t launch_sum_squares(const uint32_t* counts, long long total, DevStats* st, cudaStream_t s);
long long hash_simt_blocks(const HashArgs& a);
int simt_tile_rows(int tile);
int simt_tile_cols(int tile);
// Every detector's hash + insert, query phase and flags in one persistent launch (hash_simt.cu).
cudaError_t launch_batch(const HashArgs* args_dev, const ScoreJob* jobs_dev, const long long* hstart_dev,
                         const long long* sstart_dev, int ndet, unsigned long long* next, unsigned int* hdone,
                         unsigned int* sready, bool bf16, bool id16, bool noisy, int num_sms, cudaStream_t s);
cudaError_t launch_delete_check(const uint32_t* hist, const uint32_t* counts, long long total, unsigned int* flag,
                                int num_sms, cudaStream_t s);
cudaError_t launch_window_evict(const void* ring, int ids16, long long cap, long long start, long long m, int K, int L,
                                uint32_t* counts, int num_sms, cudaStream_t s);
cudaError_t launch_delete_apply(const uint32_t* hist, uint32_t* counts, long long total, int num_sms, cudaStream_t s);

// Measurement hook: D = A . B^T as kd/16 tcgen05 MMAs of 128 x N x 16 (tc_probe.cu).
cudaError_t launch_tc_probe(const void* A, const void* B, int kd, int N, bool fp8, float* D, int* status,
                            cudaStream_t s);
cudaError_t launch_wait_probe(int kind, long long limit, const unsigned int* flag, DevStats* st, long long* cycles,
                              cudaStream_t s);

// Host-side generator of the projection matrix (SplitMix64 counter mode + Box-Muller).
// Exact S(q, D) = sum_i p(q, x_i)^K for nq queries (exact_score.cu); part holds
// exact_score_scratch(nq, nd) bytes.
size_t exact_score_scratch(long long nq, long long nd);
cudaError_t launch_exact_score(const void* Q, long long nq, const void* D, long long nd, int d, int bf16, int K,
                               double* part, double* S, cudaStream_t s);

void generate_projection(int d, int K, int L, uint64_t seed, float* W);
void generate_projection_counter(int d, int K, int L, uint64_t seed, float* W);
// Rounds every entry to bfloat16 (round to nearest even), keeping binary32 storage.
void round_projection_bf16(float* W, uint64_t total);

}  // namespace ace
