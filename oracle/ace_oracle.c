/*
 * ace_oracle.c — plain, slow, obviously correct CPU reference for the ACE hot path
 * (Luo & Shrivastava, "Arrays of (locality-sensitive) Count Estimators").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load this file.  It shares no code, header, table or helper
 * with the CUDA library; neither includes nor links the other.
 *
 * Every floating-point step is IEEE binary64 and is compiled with -ffp-contract=off and
 * without fast-math, so each operation is one correctly rounded IEEE operation in the
 * order written here.  Integer work (bucket ids, counts, sums) is exact.
 *
 * Paper map:
 *   oracle_projection_from_seed  Algorithm 1's hash initialisation: K*L independent Gaussian
 *                                projection vectors, w_i ~ N(0,1) (§2.1).  Generator:
 *                                SplitMix64 in counter mode + Box-Muller (see below).
 *   oracle_projection_counter    the integer-only projection (§3.4 regenerates projections
 *                                from stored seeds): W.flat[f] = (popcount(draw_f) - 32) / 4
 *                                with the same SplitMix64 counter-mode draws.
 *   oracle_projection_hadamard   the structured +-1 projection (Fast-JL family, §2.2): rows of
 *                                a Sylvester-Hadamard matrix with random signs per block.
 *   oracle_hash                  Eq. 1 (SRP bit h_w(x) = sign(w^T x)) and Eq. 2
 *                                (K bits concatenated into the meta-hash H_j), §3.2.
 *   oracle_insert                Algorithm 1 pre-processing phase; §3.2 (counting phase).
 *   oracle_mu_incremental        Eq. 11 (mean update on insertion, §3.4.1), point by point.
 *   oracle_delete                §3.4.1 deletion: A_j[H_j(x)] -= 1 for every point of a batch.
 *   oracle_mu_decremental        Eq. 12 (mean update on deletion, §3.4.1), point by point.
 *   oracle_gather / oracle_score Algorithm 1 query phase; §3.2 (query phase):
 *                                S^(q) = (1/L) sum_j A_j[H_j(q)].
 *   oracle_stats_*               §5.3 threshold rule: report a point whose score is below
 *                                mu - alpha*sigma of the scores (alpha = 1 is the paper's
 *                                mu - sigma).
 *
 * Readings of the paper taken here (each is listed in the design notes):
 *   - sign(0): the bit is 1 iff the projection is strictly positive (Eq. 1 leaves 0 open).
 *   - bit order: h_{j,1} is the least significant bit of H_j; column c = j*K + k.
 *   - the projection is the binary64 sum, in index order, of the exact products
 *     (double)x_i * (double)w_i of the stored inputs.
 *   - counts are uint32 (the paper's 16-bit shorts are a memory choice, §3.4); a count
 *     that would pass 2^32-1 is an overflow error, never a wrap.
 *   - Eq. 11 is applied with the counts read BEFORE the point's own increment, and Eq. 12
 *     with the counts read BEFORE the point's own decrement.
 *   - deleting a batch that would take a count below zero (a point that was never inserted)
 *     is an error that leaves the arrays unchanged.
 *   - sigma is the population standard deviation of every score returned for the
 *     detector so far, the current batch included; the flag is score < mu - alpha*sigma.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ---------------------------------------------------------------------------------- */
/* Projection matrix from a seed.                                                      */
/*                                                                                     */
/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014), used in counter mode: draw number t   */
/* of a seed s is the SplitMix64 output for the state s + (t+1)*0x9E3779B97F4A7C15.     */
/* Box-Muller (1958): for pair p, u1 = (top 53 bits of draw 2p, plus 1) * 2^-53 in     */
/* (0,1], u2 = (top 53 bits of draw 2p+1) * 2^-53 in [0,1), r = sqrt(-2 ln u1),        */
/* g0 = r cos(2 pi u2) fills flat index 2p, g1 = r sin(2 pi u2) fills flat index 2p+1. */
/* Flat index f = i*KL + c for the d x KL row-major matrix; each value is rounded to   */
/* binary32.                                                                           */
/* ---------------------------------------------------------------------------------- */
static uint64_t splitmix64_draw(uint64_t seed, uint64_t t) {
  uint64_t z = seed + (t + 1u) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

uint64_t oracle_splitmix64_draw(uint64_t seed, uint64_t t) { return splitmix64_draw(seed, t); }

void oracle_projection_from_seed(int d, int K, int L, uint64_t seed, float* W) {
  const uint64_t total = (uint64_t)d * (uint64_t)K * (uint64_t)L;
  const double two_pi = 2.0 * 3.14159265358979323846;
  for (uint64_t f = 0; f < total; ++f) {
    uint64_t p = f / 2u;
    uint64_t a = splitmix64_draw(seed, 2u * p);
    uint64_t b = splitmix64_draw(seed, 2u * p + 1u);
    double u1 = (double)((a >> 11) + 1u) * 0x1.0p-53;
    double u2 = (double)(b >> 11) * 0x1.0p-53;
    double r = sqrt(-2.0 * log(u1));
    double ang = two_pi * u2;
    double g = (f % 2u == 0u) ? r * cos(ang) : r * sin(ang);
    W[f] = (float)g;
  }
}

/* Number of one bits of v, one bit cleared per step (v & (v - 1) drops the lowest one).    */
static int ones64(uint64_t v) {
  int c = 0;
  while (v) {
    v &= v - 1u;
    ++c;
  }
  return c;
}

/* Integer-only projection: entry f is (ones(draw_f) - 32) / 4, draw_f the f-th SplitMix64  */
/* draw of the seed.  The number of ones of 64 fair bits is Binomial(64, 1/2): mean 0,      */
/* variance 16/16 = 1 after the shift and the division (exact in binary32).                 */
void oracle_projection_counter(int d, int K, int L, uint64_t seed, float* W) {
  const uint64_t total = (uint64_t)d * (uint64_t)K * (uint64_t)L;
  for (uint64_t f = 0; f < total; ++f) {
    int k = ones64(splitmix64_draw(seed, f)) - 32;
    W[f] = (float)k / 4.0f;
  }
}

/* Structured projection (ACE_W_HADAMARD; the Fast-JL family of §2.2): dp = the power of    */
/* two >= max(d, 32); column c = b dp + j has W[i][c] = D_b[i] * H[j][i] with the Sylvester  */
/* Hadamard entry H[j][i] = (-1)^(number of ones of i AND j) and D_b[i] = -1 when draw        */
/* b dp + i of the seed is odd, +1 otherwise.                                                  */
void oracle_projection_hadamard(int d, int K, int L, uint64_t seed, float* W) {
  const int KL = K * L;
  int dp = 32;
  while (dp < d) dp *= 2;
  for (int i = 0; i < d; ++i) {
    for (int c = 0; c < KL; ++c) {
      const int b = c / dp, j = c % dp;
      const int dneg = (int)(splitmix64_draw(seed, (uint64_t)b * (uint64_t)dp + (uint64_t)i) & 1u);
      const int hneg = ones64((uint64_t)(i & j)) & 1;
      W[(size_t)i * KL + c] = (dneg ^ hneg) ? -1.0f : 1.0f;
    }
  }
}

/* The same matrix with every binary32 value then rounded to bfloat16 (the upper 16 bits  */
/* of a binary32 pattern), round to nearest, ties to an even last bit; values are finite.   */
/* Kept as binary32 values.                                                                */
void oracle_projection_from_seed_bf16(int d, int K, int L, uint64_t seed, float* W) {
  oracle_projection_from_seed(d, K, L, seed, W);
  const uint64_t total = (uint64_t)d * (uint64_t)K * (uint64_t)L;
  for (uint64_t f = 0; f < total; ++f) {
    uint32_t bits;
    memcpy(&bits, &W[f], sizeof bits);
    uint32_t keep = bits >> 16, rest = bits & 0xFFFFu;
    if (rest > 0x8000u || (rest == 0x8000u && (keep & 1u))) keep += 1u;
    bits = keep << 16;
    memcpy(&W[f], &bits, sizeof bits);
  }
}

/* ---------------------------------------------------------------------------------- */
/* Eq. 1 and Eq. 2.                                                                    */
/* ---------------------------------------------------------------------------------- */
static double bf16_bits_to_double(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, sizeof f);
  return (double)f;
}

/* One SRP bit: [ sum_i x_i * w_{i,c} > 0 ], the sum taken in binary64, in index order. */
static int srp_bit(const double* x, int d, const float* W, int KL, int c) {
  double s = 0.0;
  for (int i = 0; i < d; ++i) s += x[i] * (double)W[(size_t)i * KL + c];
  return s > 0.0;
}

/*
 * ids[i*L + j] = H_j(x_i) = sum_{k<K} h_{j,k}(x_i) * 2^k, with h_{j,k} the SRP bit of
 * column c = j*K + k.  X is n x d row-major; x_dtype 0 = binary32, 1 = bfloat16 bits.
 */
void oracle_hash(const void* X, int x_dtype, int64_t n, int d, const float* W, int K, int L,
                 uint32_t* ids) {
  const int KL = K * L;
#pragma omp parallel
  {
    double* x = (double*)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      for (int t = 0; t < d; ++t) {
        size_t at = (size_t)i * (size_t)d + (size_t)t;
        x[t] = x_dtype == 0 ? (double)((const float*)X)[at] : bf16_bits_to_double(((const uint16_t*)X)[at]);
      }
      for (int j = 0; j < L; ++j) {
        uint32_t h = 0;
        for (int k = 0; k < K; ++k) h |= (uint32_t)srp_bit(x, d, W, KL, j * K + k) << k;
        ids[(size_t)i * L + j] = h;
      }
    }
    free(x);
  }
}

/*
 * §4.5, privacy-preserving SRP: the sign is taken of the projection plus noise,
 * bit = [ s + eta > 0 ] with s the binary64 index-order sum of Eq. 1 and
 * eta = sigma * (ones(draw t of noise_seed) - 32) / 4, t = (nbase + i) * KL + c: centred,
 * scaled Binomial(64, 1/2) noise of variance sigma^2 (the library's Gaussian stand-in),
 * exact in binary64 (sigma has 24 significant bits, (ones - 32) / 4 at most 6).
 */
void oracle_hash_noisy(const void* X, int x_dtype, int64_t n, int d, const float* W, int K, int L,
                       float sigma, uint64_t noise_seed, uint64_t nbase, uint32_t* ids) {
  const int KL = K * L;
#pragma omp parallel
  {
    double* x = (double*)malloc(sizeof(double) * (size_t)(d > 0 ? d : 1));
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      for (int t = 0; t < d; ++t) {
        size_t at = (size_t)i * (size_t)d + (size_t)t;
        x[t] = x_dtype == 0 ? (double)((const float*)X)[at] : bf16_bits_to_double(((const uint16_t*)X)[at]);
      }
      for (int j = 0; j < L; ++j) {
        uint32_t h = 0;
        for (int k = 0; k < K; ++k) {
          const int c = j * K + k;
          double s = 0.0;
          for (int t = 0; t < d; ++t) s += x[t] * (double)W[(size_t)t * KL + c];
          const uint64_t idx = (nbase + (uint64_t)i) * (uint64_t)KL + (uint64_t)c;
          const double g = (double)(ones64(splitmix64_draw(noise_seed, idx)) - 32) / 4.0;
          const double eta = (double)sigma * g;
          h |= (uint32_t)(s + eta > 0.0) << k;
        }
        ids[(size_t)i * L + j] = h;
      }
    }
    free(x);
  }
}

/* Raw projections s[i*KL + c] (binary64, index order) for tests that look at margins. */
void oracle_project(const void* X, int x_dtype, int64_t n, int d, const float* W, int KL, double* s) {
  for (int64_t i = 0; i < n; ++i)
    for (int c = 0; c < KL; ++c) {
      double acc = 0.0;
      for (int t = 0; t < d; ++t) {
        size_t at = (size_t)i * (size_t)d + (size_t)t;
        double xv = x_dtype == 0 ? (double)((const float*)X)[at] : bf16_bits_to_double(((const uint16_t*)X)[at]);
        acc += xv * (double)W[(size_t)t * KL + c];
      }
      s[(size_t)i * KL + c] = acc;
    }
}

/* ---------------------------------------------------------------------------------- */
/* Counting phase (Algorithm 1 pre-processing; §3.2).                                  */
/* counts is L x 2^K, row j = array A_j.  Returns 0, or 1 if a count would overflow    */
/* (the arrays are then left as they were).                                            */
/* ---------------------------------------------------------------------------------- */
int oracle_insert(const uint32_t* ids, int64_t n, int K, int L, uint32_t* counts) {
  const size_t B = (size_t)1 << K;
  /* overflow check first, so a failing batch leaves the arrays untouched */
  uint32_t* scratch = (uint32_t*)malloc(sizeof(uint32_t) * B * (size_t)L);
  memcpy(scratch, counts, sizeof(uint32_t) * B * (size_t)L);
  for (int64_t i = 0; i < n; ++i)
    for (int j = 0; j < L; ++j) {
      uint32_t* a = &scratch[(size_t)j * B + ids[(size_t)i * L + j]];
      if (*a == UINT32_MAX) { free(scratch); return 1; }
      *a += 1u;
    }
  memcpy(counts, scratch, sizeof(uint32_t) * B * (size_t)L);
  free(scratch);
  return 0;
}

/* ---------------------------------------------------------------------------------- */
/* Deletion (§3.4.1): A_j[H_j(x)] -= 1 for every point.  Returns 0, or 1 if a count     */
/* would go below zero (the arrays are then left as they were).                        */
/* ---------------------------------------------------------------------------------- */
int oracle_delete(const uint32_t* ids, int64_t n, int K, int L, uint32_t* counts) {
  const size_t B = (size_t)1 << K;
  uint32_t* scratch = (uint32_t*)malloc(sizeof(uint32_t) * B * (size_t)L);
  memcpy(scratch, counts, sizeof(uint32_t) * B * (size_t)L);
  for (int64_t i = 0; i < n; ++i)
    for (int j = 0; j < L; ++j) {
      uint32_t* a = &scratch[(size_t)j * B + ids[(size_t)i * L + j]];
      if (*a == 0u) { free(scratch); return 1; }
      *a -= 1u;
    }
  memcpy(counts, scratch, sizeof(uint32_t) * B * (size_t)L);
  free(scratch);
  return 0;
}

/*
 * Eq. 12, applied literally point by point: before x's decrements,
 *   mu' = ( n*mu - sum_j (2*A_j[H_j(x)] - 1)/L ) / (n-1),
 * with A_j read before x's own decrement.  counts is updated as it goes (the caller makes
 * sure every count stays >= 0).  mu_trace[i] receives mu after point i (0 once the last
 * point is gone).  Returns the final mu.
 */
double oracle_mu_decremental(const uint32_t* ids, int64_t n, int K, int L, uint32_t* counts,
                             int64_t n_before, double mu_before, double* mu_trace) {
  const size_t B = (size_t)1 << K;
  double mu = mu_before;
  int64_t m = n_before;
  for (int64_t i = 0; i < n; ++i) {
    double decre = 0.0;
    for (int j = 0; j < L; ++j) {
      uint32_t* a = &counts[(size_t)j * B + ids[(size_t)i * L + j]];
      decre += (2.0 * (double)(*a) - 1.0) / (double)L;
      *a -= 1u;
    }
    mu = m > 1 ? ((double)m * mu - decre) / (double)(m - 1) : 0.0;
    m -= 1;
    if (mu_trace) mu_trace[i] = mu;
  }
  return mu;
}

/* Q = sum_j sum_b A_j[b]^2 as two 64-bit halves (lo, hi). */
void oracle_sum_squares(const uint32_t* counts, int K, int L, uint64_t* q_lo_hi) {
  const size_t total = ((size_t)1 << K) * (size_t)L;
  u128 q = 0;
  for (size_t t = 0; t < total; ++t) q += (u128)counts[t] * (u128)counts[t];
  q_lo_hi[0] = (uint64_t)q;
  q_lo_hi[1] = (uint64_t)(q >> 64);
}

/*
 * Eq. 11, applied literally point by point: before x's increments,
 *   mu' = ( n*mu + sum_j (2*A_j[H_j(x)] + 1)/L ) / (n+1),
 * with A_j read before x's own increment.  counts is updated as it goes.
 * mu_trace[i] receives mu after point i.  Returns the final mu.
 */
double oracle_mu_incremental(const uint32_t* ids, int64_t n, int K, int L, uint32_t* counts,
                             int64_t n_before, double mu_before, double* mu_trace) {
  const size_t B = (size_t)1 << K;
  double mu = mu_before;
  int64_t m = n_before;
  for (int64_t i = 0; i < n; ++i) {
    double incre = 0.0;
    for (int j = 0; j < L; ++j) {
      uint32_t* a = &counts[(size_t)j * B + ids[(size_t)i * L + j]];
      incre += (2.0 * (double)(*a) + 1.0) / (double)L;
      *a += 1u;
    }
    mu = ((double)m * mu + incre) / (double)(m + 1);
    m += 1;
    if (mu_trace) mu_trace[i] = mu;
  }
  return mu;
}

/* ---------------------------------------------------------------------------------- */
/* Query phase (Algorithm 1; §3.2): c_i = sum_j A_j[H_j(q_i)], score_i = c_i / L.      */
/* Returns 0, or 1 if some c_i does not fit in 32 bits.                                */
/* ---------------------------------------------------------------------------------- */
int oracle_gather(const uint32_t* ids, int64_t n, int K, int L, const uint32_t* counts,
                  uint32_t* sums) {
  const size_t B = (size_t)1 << K;
  int err = 0;
  for (int64_t i = 0; i < n; ++i) {
    uint64_t c = 0;
    for (int j = 0; j < L; ++j) c += counts[(size_t)j * B + ids[(size_t)i * L + j]];
    if (c > UINT32_MAX) err = 1;
    sums[i] = (uint32_t)c;
  }
  return err;
}

/* ---------------------------------------------------------------------------------- */
/* Score statistics (§5.3): N scores so far, S1 = sum c, S2 = sum c^2 (exact, 128-bit). */
/* ---------------------------------------------------------------------------------- */
typedef struct {
  uint64_t N;
  u128 S1, S2;
} oracle_running;

/* Folds a batch of sums into (N, S1, S2), given as 5 words: N, S1 lo/hi, S2 lo/hi. */
void oracle_stats_fold(uint64_t* st, const uint32_t* sums, int64_t n) {
  u128 S1 = ((u128)st[2] << 64) | st[1];
  u128 S2 = ((u128)st[4] << 64) | st[3];
  for (int64_t i = 0; i < n; ++i) {
    S1 += (u128)sums[i];
    S2 += (u128)sums[i] * (u128)sums[i];
  }
  st[0] += (uint64_t)n;
  st[1] = (uint64_t)S1; st[2] = (uint64_t)(S1 >> 64);
  st[3] = (uint64_t)S2; st[4] = (uint64_t)(S2 >> 64);
}

/*
 * mu = S1 / (N L); sigma = sqrt(N S2 - S1^2) / (N L) (population standard deviation of
 * the scores c/L; the radicand is an exact non-negative integer); t = mu - alpha*sigma.
 * out = {mu, sigma, t}.  Returns 0, 1 if N = 0, 2 if N*S2 does not fit in 128 bits.
 */
int oracle_stats_threshold(const uint64_t* st, int L, double alpha, double* out) {
  uint64_t N = st[0];
  u128 S1 = ((u128)st[2] << 64) | st[1];
  u128 S2 = ((u128)st[4] << 64) | st[3];
  if (N == 0) { out[0] = out[1] = out[2] = 0.0; return 1; }
  if (S2 != 0 && (u128)N > (~(u128)0) / S2) return 2;
  u128 var_num = (u128)N * S2 - S1 * S1;
  double NL = (double)N * (double)L;
  double mu = (double)S1 / NL;
  double sigma = sqrt((double)var_num) / NL;
  double as = alpha * sigma;
  out[0] = mu;
  out[1] = sigma;
  out[2] = mu - as;
  return 0;
}

/* score_i = c_i / L (binary64) and flag_i = [score_i < t]. */
void oracle_score_flags(const uint32_t* sums, int64_t n, int L, double t, double* scores,
                        uint8_t* flags) {
  for (int64_t i = 0; i < n; ++i) {
    double s = (double)sums[i] / (double)L;
    if (scores) scores[i] = s;
    if (flags) flags[i] = (uint8_t)(s < t);
  }
}

/* mu of the inserted set from Q (closed form of Eq. 11 summed over the inserts). */
double oracle_mu_from_q(const uint64_t* q_lo_hi, uint64_t n_ins, int L) {
  u128 q = ((u128)q_lo_hi[1] << 64) | q_lo_hi[0];
  return (double)q / ((double)n_ins * (double)L);
}

#ifdef _OPENMP
#include <omp.h>
int oracle_num_threads(void) { return omp_get_max_threads(); }
void oracle_set_num_threads(int t) { if (t > 0) omp_set_num_threads(t); }
#else
int oracle_num_threads(void) { return 1; }
void oracle_set_num_threads(int t) { (void)t; }
#endif
