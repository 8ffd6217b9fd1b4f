/*
 * ace.h — C ABI of the GB300 (sm_103a) ACE hot path.
 *
 * ACE (Arrays of locality-sensitive Count Estimators; Luo & Shrivastava) keeps L arrays
 * A_1..A_L of 2^K counters.  A point x is hashed by K*L signed random projections
 * (Eq. 1: h_w(x) = sign(w^T x), w ~ N(0, I)); each group of K bits forms a bucket id
 * H_j(x) (Eq. 2).  Inserting x increments A_j[H_j(x)] for every j (Algorithm 1,
 * pre-processing phase, §3.2); the score of a query q is (1/L) sum_j A_j[H_j(q)]
 * (Algorithm 1, query phase, §3.2); a point is reported when its score is below
 * mu - alpha*sigma of the scores (§5.3 uses alpha = 1).
 *
 * Definitions this library computes exactly (the same as the project's CPU reference):
 *   - SRP bit of column c for point x:  [ s > 0 ], s = the binary64 sum, in index order
 *     i = 0..d-1, of (double)x_i * (double)W[i][c].  A zero projection gives bit 0.
 *   - bucket id  H_j(x) = sum_{k<K} bit(c = j*K + k) * 2^k   (first bit is the LSB).
 *   - counts are uint32; sums c = sum_j A_j[H_j(q)] are uint32; scores are c / L (binary64).
 *   - mu = S1/(N L), sigma = sqrt(N S2 - S1^2)/(N L), threshold = mu - alpha*sigma, where
 *     N, S1 = sum c, S2 = sum c^2 run over every point scored by this detector, the
 *     current call included; flag = score < threshold.  Each is one correctly rounded
 *     binary64 operation on exact integers, so the values are bit-reproducible.
 * The projection itself runs in binary32 (SIMT) or bfloat16 (tensor cores) with a
 * rigorous error bound; every projection whose magnitude is inside the bound is recomputed
 * in binary64 in index order, so bucket ids never depend on the fast path.
 *
 * Conventions
 *   - Every device pointer is a CUDA global-memory address on the detector's device,
 *     row-major and contiguous, aligned to its element size; the caller owns it.
 *   - X is n x d: binary32 (ACE_F32) or bfloat16 bit patterns (ACE_BF16).
 *   - Calls that take a stream are asynchronous on it (a cudaStream_t; NULL = legacy
 *     default stream).  Only ace_stats, ace_get_counts, ace_get_projection and the *_host
 *     entry points block, and they block on that stream only.
 *   - A handle may be used from one host thread at a time; calls on one handle must be
 *     ordered (same stream, or the caller orders the streams).
 *   - Every function returns ACE_OK or an error code; ace_last_error() gives this
 *     thread's last message.  No C++ exception crosses the ABI.  On any error other than
 *     ACE_ERR_CUDA the detector's state is unchanged.
 */
#ifndef ACE_GB300_H
#define ACE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ace_detector* ace_handle;

enum {
  ACE_OK = 0,
  ACE_ERR_ARG = 1,      /* invalid argument (sizes, null pointer, dtype)                */
  ACE_ERR_OOM = 2,      /* a device or host allocation failed                           */
  ACE_ERR_OVERFLOW = 3, /* a count, a per-point sum or N*S2 would not fit its width     */
  ACE_ERR_TIMEOUT = 4,  /* a bounded device-side wait gave up                           */
  ACE_ERR_CUDA = 5,     /* a CUDA runtime call failed (message in ace_last_error)       */
  ACE_ERR_UNSUPPORTED = 6 /* the requested path is not available for this shape/device  */
};

enum { ACE_F32 = 0, ACE_BF16 = 1 };

/* Projection precision (the sign bits are exact on every path; this picks the engine). */
enum {
  ACE_PROJ_AUTO = -1, /* fastest available path for the detector's shape (default)       */
  ACE_PROJ_FP32 = 0,  /* binary32 FMA on the SIMT cores                                   */
  ACE_PROJ_BF16 = 1,  /* bfloat16 split operands on tcgen05 tensor cores, binary32 accum.  */
  ACE_PROJ_FWHT = 3,  /* structured engine of ACE_W_HADAMARD detectors: fast Walsh-Hadamard
                         transforms, O(dp log dp) additions per block of dp projections     */
  ACE_PROJ_FP8 = 2    /* E4M3 split operands (X = X1 + X2 per row with a power-of-two row
                         scale, W = W1 + W2 per column), four kind::f8f6f4 products in binary32:
                         streaming engine and bfloat16-valued W (ACE_W_BF16) only          */
};

/* Device-status bits reported by ace_stats (sticky until ace_reset). */
enum {
  ACE_STATUS_SUM_OVERFLOW = 1u, /* some per-point sum c did not fit in uint32            */
  ACE_STATUS_TIMEOUT = 2u       /* a bounded device wait gave up                          */
};

typedef struct {
  uint64_t n_ins;           /* points inserted                                          */
  uint64_t n_scored;        /* N: points scored (every score / insert_score call)       */
  uint64_t Q_lo, Q_hi;      /* Q = sum_j sum_b A_j[b]^2 (128-bit)                       */
  uint64_t S1_lo, S1_hi;    /* S1 = sum of per-point sums c over scored points           */
  uint64_t S2_lo, S2_hi;    /* S2 = sum of c^2                                           */
  double mu_ins;            /* mean score of the inserted set: Q / (n_ins L) (Eq. 11)    */
  double mu;                /* S1 / (N L)                                                */
  double sigma;             /* sqrt(N S2 - S1^2) / (N L), population                     */
  uint64_t rechecks;        /* projections recomputed in binary64 (inside the bound)     */
  uint64_t nonfinite_points;/* points with a NaN/Inf coordinate or an overflowing norm   */
  uint32_t status;          /* ACE_STATUS_* bits                                         */
  int32_t precision;        /* ACE_PROJ_* path used by the last hash                     */
  uint64_t deferred;        /* entries the tensor-core engines left to exact resolution  */
                            /* (inside their error bound): (point, table) pairs for the   */
                            /* resident engine (d <= 64), (point, column) pairs for the   */
                            /* streaming one (larger d); 0 on the SIMT engine             */
  int32_t tc_products;      /* products per tensor-core accumulation in the last hash:   */
                            /* 3 (resident engine, x and W split in bfloat16), 2          */
                            /* (streaming, W split), 1 (streaming, bfloat16-valued W),    */
                            /* 4 (streaming E4M3: X1 W1, X1 W2, X2 W1, X2 W2), 0 (SIMT)   */
} ace_stats_t;

/* Creation flags (ace_create_ex). */
enum {
  ACE_W_BF16 = 1u,   /* round every drawn W entry to bfloat16 (nearest even), kept as binary32 */
  ACE_W_COUNTER = 2u, /* integer-only entries regenerated from the seed inside the kernels  */
  ACE_W_HADAMARD = 4u /* structured +-1 projections: Walsh-Hadamard rows with random signs  */
};

/*
 * ace_create — Algorithm 1's hash initialisation (§3.2) and array allocation.
 * Draws the d x (K*L) projection matrix W, w ~ N(0,1) (§2.1), from `seed` with SplitMix64
 * in counter mode (draw t = SplitMix64 output for state seed + (t+1)*0x9E3779B97F4A7C15)
 * and Box-Muller on pairs of draws (u1 = (draw_2p >> 11) + 1) * 2^-53, u2 = (draw_2p+1 >> 11)
 * * 2^-53, r = sqrt(-2 ln u1), W.flat[2p] = r cos(2 pi u2), W.flat[2p+1] = r sin(2 pi u2),
 * each rounded to binary32; W.flat[i*K*L + c] = W[i][c]), and zeroes L arrays of 2^K
 * uint32 counters on the current CUDA device.
 * Limits: d >= 1, 1 <= K <= 24, L >= 1, K*L <= 65536.  *out receives the handle.
 * Errors: ACE_ERR_ARG, ACE_ERR_OOM, ACE_ERR_CUDA.
 */
int ace_create(int d, int K, int L, uint64_t seed, ace_handle* out);

/*
 * ace_create_ex — ace_create with creation flags.  ACE_W_BF16: each drawn W entry (binary32,
 * as ace_create) is rounded to bfloat16, round to nearest even.  The paper fixes neither the
 * precision of W nor how it is stored, only w ~ N(0,1) (§2.1; §3.4 regenerates projections
 * from stored seeds); with bfloat16-valued W the streaming tensor-core engine forms every
 * product x_i w_i exactly in one bfloat16 MMA instead of two, and every id stays the binary64
 * definition's for that W.  An explicit W whose entries are all bfloat16 values
 * (ace_create_with_projection) gets the same single-product path.
 * Errors: as ace_create; ACE_ERR_ARG for unknown flags.
 */
int ace_create_ex(int d, int K, int L, uint64_t seed, unsigned flags, ace_handle* out);
/*
 * ACE_W_COUNTER (ace_create_ex; §3.4 keeps the seeds of the projections and regenerates them
 * instead of storing them): W.flat[i*K*L + c] = (popcount(draw_f) - 32) / 4 with draw_f the
 * SplitMix64 draw of index f = i*K*L + c in the counter mode above: an integer-only
 * generator whose entries have mean 0 and variance 1 (Binomial(64, 1/2) - 32, over 4) and are
 * bfloat16 values.  SRP's collision probability 1 - theta/pi holds for such a W approximately
 * (exactly for Gaussian entries).  The binary32 engine (single calls and batches) regenerates
 * its W tiles from the seed inside the kernel instead of reading a stored W; the exact recheck
 * tiers and the tensor-core images still use a materialised copy.  Ids, counts and scores are
 * the binary64 definition's for this W.  Takes precedence over ACE_W_BF16 (its entries are
 * bfloat16 values already).  A checkpoint of such a detector (ace_save) loads as a detector
 * with the same W stored (ace_load): the results are the same.
 *
 * ACE_W_HADAMARD (§2.2: Fast-JL projections, O(d log d + m) hashes): W[i][c] = D_b[i] H[j][i]
 * for column c = b dp + j, with dp the power of two >= max(d, 32), H the Sylvester-Hadamard
 * matrix of order dp (H[j][i] = (-1)^popcount(i & j)), and D_b[i] = -1 when the SplitMix64
 * draw of index b dp + i (the counter mode above) has its lowest bit set, +1 otherwise.  Each
 * block of dp projections of a point is then one Walsh-Hadamard transform of the point with
 * random signs; the structured engine (ACE_PROJ_FWHT, chosen by ACE_PROJ_AUTO when d <= 1024
 * and ceil(K*L / dp) dp <= 5120) computes it with O(dp log dp) additions per block and resolves every
 * sign inside its rounding bound by the binary64 definition.  The entries are +-1 (bfloat16
 * values), so every other engine computes the same ids from the stored W.  SRP's collision
 * probability 1 - theta/pi holds for one column; columns of one block are orthogonal rather
 * than independent.  Excludes ACE_W_COUNTER.
 */

/* As ace_create, with an explicit host d x (K*L) row-major binary32 W (copied). */
int ace_create_with_projection(int d, int K, int L, const float* W_host, ace_handle* out);

/* Frees the handle and its device memory (synchronises the device first).  NULL is ok. */
int ace_destroy(ace_handle h);

/* Zeroes the arrays and every running statistic; keeps W.  Asynchronous on `stream`. */
int ace_reset(ace_handle h, void* stream);

/*
 * ace_set_graph — graph replay for repeated calls (small batches are bound by launch
 * latency): with enable = 1, an ace_score or ace_insert_score call whose arguments (X pointer,
 * n, dtype, alpha, output pointers, stream, engine) equal the previous call's reuses a CUDA
 * graph of that call's kernels: the first call with new arguments runs directly, the second
 * captures its launches, later ones replay them.  Results are those of direct calls (the
 * graph reads X and writes the outputs at replay time; n_ins and the overflow check are kept
 * on the host per call).  Calls run directly (no graph) on the legacy or per-thread default
 * stream (which cannot be captured), on a stream the caller is capturing already, while the
 * timing hook is on, and with a window set; if a capture fails, graph replay turns itself off
 * for the handle and the call runs directly.  No counterpart in the paper (an execution
 * detail).  Errors: ACE_ERR_ARG.
 */
int ace_set_graph(ace_handle h, int enable);

/* Selects the projection engine (ACE_PROJ_*).  Results do not depend on it.  ACE_PROJ_BF16
 * and ACE_PROJ_FP8 fail with ACE_ERR_UNSUPPORTED where their engine does not apply (FP8: an
 * sm_103 device, d > 64 and a multiple of 8, a detector whose W entries are all bfloat16
 * values, and bfloat16 input at a 16-byte-aligned address when hashing). */
int ace_set_precision(ace_handle h, int precision);

/*
 * ace_set_privacy — privacy-preserving hashing (§4.5): the bits of a point are the signs of
 * its projections with noise added after the projection and before the sign, so the data
 * never leaves the hashing step (the ids carry the noise; everything after them is
 * unchanged).  From this call on, bit c of a point hashed by ace_insert, ace_score,
 * ace_insert_score or ace_hash (and the host-buffer, batched, serving and allocation-free
 * forms) is [x.w_c + eta > 0] (the binary64 sum of Eq. 1 plus eta, exactly; ties are 0),
 * with
 *   eta = sigma * g,  g = (number of one bits of SplitMix64 draw t of noise_seed - 32) / 4,
 *   t = (m + i) * K L + c,
 * m the number of points this detector hashed with noise before the call and i the point's
 * row in the batch.  g is Binomial(64, 1/2) centred and scaled: mean 0, variance 1, values
 * k / 4 for |k| <= 32 — a stand-in for the paper's N(0, 1) that is exactly representable, so
 * every bit has one binary64 definition that the engines reproduce.  A point gets fresh
 * noise each time it is hashed (an insert_score call hashes once for both).  sigma = 0 turns
 * the noise off.  Each call restarts m at 0.  While the noise is on: the engines are the
 * binary32 SIMT one and, for ACE_W_HADAMARD detectors, the structured one (ACE_PROJ_AUTO
 * picks between them; ACE_PROJ_BF16 and ACE_PROJ_FP8 are refused); ace_delete returns
 * ACE_ERR_UNSUPPORTED (a point does not hash to the ids it was inserted with; a window
 * removes points by their stored ids and stays exact); graph replay is not used; ace_project
 * returns the noise-free projections.  ace_save keeps sigma, the seed and m.
 * Errors: ACE_ERR_ARG (sigma not 0 and outside [2^-60, 2^60] or not a number; noise_seed
 * equal to the seed the detector was created from), ACE_ERR_UNSUPPORTED (precision set to
 * ACE_PROJ_BF16 or ACE_PROJ_FP8).
 */
int ace_set_privacy(ace_handle h, float sigma, uint64_t noise_seed);

/* The privacy settings: sigma (0: off), the noise seed and m, the noise index of the next
 * point (any pointer may be NULL). */
int ace_get_privacy(ace_handle h, float* sigma, uint64_t* noise_seed, uint64_t* next_index);

/*
 * ace_insert — counting phase (Algorithm 1 pre-processing; §3.2, counting phase):
 * for every point x of X (n x d), A_j[H_j(x)] += 1 for j = 1..L.  The result does not
 * depend on the order of the points.  n = 0 is a no-op.
 * Errors: ACE_ERR_ARG; ACE_ERR_OVERFLOW if n_ins + n would exceed 2^32 - 1 (a count could
 * then overflow; nothing is inserted); ACE_ERR_CUDA.
 */
int ace_insert(ace_handle h, const void* X_dev, int64_t n, int dtype, void* stream);

/*
 * ace_score — query phase (Algorithm 1; §3.2, query phase) and the §5.3
 * threshold rule, against the arrays as they stand at the start of the call (scoring
 * never inserts).  For each point: sums_dev[i] = c_i = sum_j A_j[H_j(x_i)] (uint32),
 * scores_dev[i] = c_i / L (binary64), flags_dev[i] = 1 if scores_dev[i] < mu - alpha*sigma
 * else 0, with mu and sigma over every point scored so far including this call.
 * Any of the three outputs may be NULL.  Errors: ACE_ERR_ARG, ACE_ERR_OOM, ACE_ERR_CUDA.
 */
int ace_score(ace_handle h, const void* X_dev, int64_t n, int dtype, double alpha,
              double* scores_dev, uint32_t* sums_dev, uint8_t* flags_dev, void* stream);

/* Inserts the whole batch, then scores it against the updated arrays (same outputs). */
int ace_insert_score(ace_handle h, const void* X_dev, int64_t n, int dtype, double alpha,
                     double* scores_dev, uint32_t* sums_dev, uint8_t* flags_dev, void* stream);

/*
 * ace_insert_score_host — ace_insert_score on HOST buffers: X_host (n x d, pinned or
 * pageable) is copied to the device, processed, and the outputs copied back to host
 * (any of them may be NULL).  Blocks until the outputs are in host memory.
 */
int ace_insert_score_host(ace_handle h, const void* X_host, int64_t n, int dtype, double alpha,
                          double* scores_host, uint32_t* sums_host, uint8_t* flags_host,
                          void* stream);

/*
 * ace_delete — §3.4.1 deletion: removes the points of X_dev (n x d, device, as ace_insert)
 * from the count arrays, A_j[H_j(x)] -= 1 for every point, so that mu_ins follows Eq. 12
 * (ace_stats reports it as Q / (n_ins L), Q = sum of count^2, which Eq. 12 keeps in closed
 * form).  All or nothing: if some bucket would go below zero (a point of the batch was never
 * inserted), or n exceeds the points inserted, nothing changes and ACE_ERR_ARG is returned.
 * The statistics of returned scores (N, S1, S2, mu, sigma) are not changed.  Synchronises
 * `stream` once (to read the check).
 */
int ace_delete(ace_handle h, const void* X_dev, int64_t n, int dtype, void* stream);

/*
 * ace_window_enable — sliding window over the inserted points, for drifting streams (§3.4.1:
 * removing points by decrementing their counts keeps the mean of Eq. 11 / Eq. 12 exact).
 * After ace_window_enable(h, W), h's arrays count only the last W points inserted (in call
 * order, rows of a batch in order): before a batch of n points is inserted (ace_insert,
 * ace_insert_score, the host-buffer and server paths), the oldest max(0, held + n - W) points
 * are removed, their counts decremented on the device.  The ids of the held points are kept
 * in a device ring of W * L ids (2 bytes each for K <= 16, else 4).  A batch larger than W
 * is refused with ACE_ERR_ARG.  ace_stats' n_ins and mu_ins then describe the held points;
 * the score statistics (N, S1, S2) keep running over every score returned.  W = 0 turns the
 * window off.  The window can be set only while the detector holds no points (new, or after
 * ace_reset, which empties it).  ace_delete, ace_batch_insert_score, the allocation-free
 * entry point and ace_save refuse a windowed detector (ACE_ERR_ARG).  Synchronises the device.
 * Errors: ACE_ERR_ARG, ACE_ERR_OOM, ACE_ERR_CUDA.
 */
int ace_window_enable(ace_handle h, int64_t window_points);

/*
 * ace_batch_insert_score — ace_insert_score on `count` distinct detectors at once, each with
 * its own X_dev[g] (n[g] x d_g, device; one dtype for the whole batch) and optional outputs
 * (scores_dev, sums_dev, flags_dev: arrays of `count` device pointers, or NULL; an entry may
 * be NULL).  Every detector's results are exactly those of its own ace_insert_score call
 * (Algorithm 1 counting and query phases, §5.3 rule on its own statistics); the work of all
 * detectors runs as one persistent launch on the binary32 engine (every detector's hash +
 * insert blocks, then its query blocks once its hash is done, then its score/flag blocks once
 * its statistics are derived), so many small detectors fill the GPU together.  The engine's
 * tile (points x columns per block) is picked per detector shape by an autotuner that times
 * the variants on the first batch meeting the shape and keeps the fastest for the process
 * (ace_batch_tile reports it).  The K of all detectors is <= 16, or > 16
 * for all.  All or nothing on argument errors; asynchronous on `stream`.  (The paper states
 * the method for one dataset; running many detectors together is this library's.)
 */
int ace_batch_insert_score(const ace_handle* dets, int count, const void* const* X_dev, const int64_t* n, int dtype,
                           double alpha, double* const* scores_dev, uint32_t* const* sums_dev,
                           uint8_t* const* flags_dev, void* stream);

/*
 * ace_batch_tile — the tile the batched engine's autotuner chose for detectors of this shape
 * (d rounded up to a power of two, K, L, dtype): points and columns per block, or 0 and 0 if
 * no batch has met the shape yet.  Measurement and test hook.  Errors: ACE_ERR_ARG.
 */
int ace_batch_tile(int d, int K, int L, int dtype, int* points, int* columns);

/* Operations of a host-buffer request (ace_server_submit). */
enum { ACE_OP_INSERT = 0, ACE_OP_SCORE = 1, ACE_OP_INSERT_SCORE = 2 };

/*
 * Request server: continuous batching of host-buffer requests over several detectors (the
 * paper states the method for one dataset; serving many detectors is this library's).
 * ace_server_create takes n_dets detector handles (the server owns their use until it is
 * destroyed: make no other call on them meanwhile) and a device-memory budget for the staged
 * bytes of requests in flight (a request larger than the budget still runs, alone).
 * ace_server_submit queues one request — op ACE_OP_INSERT (Algorithm 1 counting phase),
 * ACE_OP_SCORE (query phase and §5.3 rule) or ACE_OP_INSERT_SCORE — on detector `det` with
 * X_host (n x d, pinned for asynchrony) and optional output buffers (ignored for inserts),
 * and returns a ticket at once; X_host and the outputs must stay valid until the ticket is
 * waited for.  One scheduler thread (the environment variable ACE_SERVER_THREADS, 1 to 4, sets
 * more; detector i then belongs to thread i mod their number) admits queued requests, the
 * earliest first, as slots (two per detector) and memory free up; each detector's
 * requests run in submission order on its own stream, so every result is the same as in a
 * run of that detector's requests alone, while different detectors overlap on the device.
 * Inserts that follow one another in a detector's order (no other request of it between them;
 * not on a windowed detector) are admitted together as one launch set of up to 65,536 points,
 * which leaves the same counts as inserting them one by one.  A detector may appear only once.
 * ace_server_wait blocks until the ticket's request has completed and returns its latency from
 * submission to completion in seconds (or its error code); each ticket is waited for once.
 * ace_server_drain waits for everything submitted; ace_server_destroy drains, stops the
 * scheduler threads and releases the server (not the detectors).  ace_server_info reports the
 * number of scheduler threads and how many requests were admitted inside another's launch
 * set (either pointer may be NULL).
 */
typedef struct ace_server_s* ace_server;
int ace_server_create(const ace_handle* dets, int n_dets, size_t mem_budget_bytes, ace_server* out);
int ace_server_submit(ace_server s, int det, int op, const void* X_host, int64_t n, int dtype, double alpha,
                      double* scores_host, uint32_t* sums_host, uint8_t* flags_host, uint64_t* ticket);
int ace_server_wait(ace_server s, uint64_t ticket, double* latency_s);
int ace_server_drain(ace_server s);
int ace_server_destroy(ace_server s);
int ace_server_info(ace_server s, int* threads, uint64_t* coalesced);

/*
 * ace_insert_score_host_async — ace_insert_score_host without the wait: enqueues the copy
 * of X_host (in chunks, each hashed as soon as it has arrived; in one copy when an earlier
 * batch is still in flight, whose work then overlaps it), the insert, the query phase and
 * the copies of the outputs back to the host buffers on `stream`, and returns.  Batches
 * are processed in call order with the same results as synchronous calls.  Until
 * ace_host_wait returns, X_host must not change and the outputs are not valid.  At most two
 * batches are in flight per detector (a third call first waits for the oldest); the copy of
 * one batch overlaps the computation of the previous one.  A call on a different stream
 * first waits for the batches in flight.  Device-path calls (ace_insert, ace_score, ...) on
 * another stream must not overlap batches in flight.  Outputs may be NULL.  Error codes as
 * ace_insert_score_host; an error reported here leaves earlier batches enqueued.
 */
int ace_insert_score_host_async(ace_handle h, const void* X_host, int64_t n, int dtype, double alpha,
                                double* scores_host, uint32_t* sums_host, uint8_t* flags_host,
                                void* stream);

/* Blocks until every batch enqueued by ace_insert_score_host_async has completed; returns
 * ACE_ERR_CUDA if one of them failed on the device. */
int ace_host_wait(ace_handle h);

/*
 * ace_hash — Eq. 1 + Eq. 2 only: ids_dev[i*L + j] = H_j(x_i) (uint32, n x L).  No state
 * changes except the recheck counter.
 */
int ace_hash(ace_handle h, const void* X_dev, int64_t n, int dtype, uint32_t* ids_dev,
             void* stream);

/*
 * ace_project — measurement of the engines' error: proj_dev[i*KL + c] = the active engine's
 * binary32 estimate of x_i.w_c (Eq. 1 before the sign): the SIMT engine's FMA chain, or the
 * tensor-core engine's accumulator of x.(w_c/||w_c||) multiplied by ||w_c|| (one more binary32
 * rounding).  proj_dev is n x KL float, device, caller-owned.  No state changes (no ids, no
 * counts, no counters).  Asynchronous on `stream`.
 */
int ace_project(ace_handle h, const void* X_dev, int64_t n, int dtype, float* proj_dev, void* stream);

/* Synchronises `stream`, then fills *out (Q is computed from the arrays here). */
int ace_stats(ace_handle h, void* stream, ace_stats_t* out);

/* Copies the L x 2^K counts (row j = A_j) to host memory.  Synchronises `stream`. */
int ace_get_counts(ace_handle h, uint32_t* counts_host, void* stream);

/* Copies the d x (K*L) binary32 W to host memory. */
int ace_get_projection(ace_handle h, float* W_host);

/*
 * Checkpoint of a detector (the paper keeps its arrays in memory; saving and restoring them
 * lets a long stream be scored across process restarts).  The blob holds everything that
 * determines later results: the shape, W, the L x 2^K counts, n_ins, the running score
 * statistics N, S1, S2 (and the recheck/status counters) and the privacy settings
 * (ace_set_privacy), with a checksum.  ace_load also reads the earlier layout without the
 * privacy settings.
 *   ace_save_size — bytes of the blob for this detector.
 *   ace_save — writes the blob to host memory buf (cap bytes, at least ace_save_size);
 *              synchronises `stream` (to read the counts as of all work enqueued on it).
 *   ace_load — creates a new detector on the current CUDA device from a blob; every later
 *              call on it gives exactly the results the saved detector would have given.
 *              The engine selection starts at ACE_PROJ_AUTO.
 * Errors: ACE_ERR_ARG (NULL, short buffer, bad magic, version, shape, size or checksum),
 * ACE_ERR_OOM, ACE_ERR_CUDA.
 */
int ace_save_size(ace_handle h, size_t* bytes);
int ace_save(ace_handle h, void* buf, size_t cap, void* stream);
int ace_load(const void* buf, size_t bytes, ace_handle* out);

/* Detector shape. */
int ace_get_shape(ace_handle h, int* d, int* K, int* L);

/* This thread's last error message ("" if none).  The pointer stays valid until the
 * next call on this thread. */
const char* ace_last_error(void);

/*
 * Per-phase timing hook.  While enabled, the library brackets each kernel it launches with
 * a pair of CUDA events on the caller's stream; ace_profile_read() waits for them and
 * returns the summed durations per phase (and clears them).  The launch counters count
 * every kernel the library launched on this handle since creation or the last read.
 */
enum { ACE_PHASE_HASH = 0, ACE_PHASE_SCORE = 1, ACE_PHASE_FLAGS = 2, ACE_PHASE_OTHER = 3, ACE_PHASE_RECHECK = 4,
       ACE_PHASE_INSERT = 5, ACE_NPHASE = 6 };
typedef struct {
  uint64_t launches[ACE_NPHASE]; /* kernels launched per phase                           */
  double ms[ACE_NPHASE];         /* summed event time per phase (enabled periods only)   */
  uint64_t timed[ACE_NPHASE];    /* launches that were timed                              */
} ace_profile_t;
int ace_profile_enable(ace_handle h, int enable);
/*
 * ace_profile_phases — restricts the events of the timing hook to the phases whose bit is set
 * in mask (bit p = ACE_PHASE p; 0 restores all phases, the default), so that a timed run can
 * bracket one kernel without paying for events around the others.  No counterpart in the
 * paper (measurement only).  Errors: ACE_ERR_ARG (NULL handle).
 */
int ace_profile_phases(ace_handle h, unsigned mask);
int ace_profile_read(ace_handle h, ace_profile_t* out);

/*
 * ace_insert_score_noalloc — ace_insert_score for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is an engineering entry point.  Some callers
 * cannot call cudaMalloc: a process whose device memory is entirely reserved by another
 * allocator (a framework's caching pool), or a latency-bound loop that must never block
 * (cudaFree synchronises the whole device, and ace_insert_score may grow its scratch).
 * This variant allocates nothing.  Its scratch (the cached bucket ids, and the per-point
 * sums when sums_dev is NULL) lives in one static device array of
 * ACE_NOALLOC_SCRATCH_BYTES (32 MiB) inside the library, which every GPU that loads the
 * library holds until the process exits.
 *   - A batch must fit: n*L*(2 if K <= 16 else 4) bytes of ids, rounded up to 256, plus
 *     4*n bytes when sums_dev is NULL, must not exceed ACE_NOALLOC_SCRATCH_BYTES; larger
 *     batches fail with ACE_ERR_ARG and change nothing.
 *   - The first call on each device looks up the array's device address (with that device
 *     current); make that first call before any stream capture begins.
 *   - Every call, on every handle of the process, shares the one array, and a call
 *     overwrites what the previous call left there.  Calls whose kernels overlap on the GPU
 *     (different streams, or different handles without ordering) race on it: order them.
 * Outputs, semantics and the other errors are those of ace_insert_score.
 */
#define ACE_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int ace_insert_score_noalloc(ace_handle h, const void* X_dev, int64_t n, int dtype, double alpha,
                             double* scores_dev, uint32_t* sums_dev, uint8_t* flags_dev, void* stream);

/*
 * ace_exact_score — the score family ACE estimates, computed exactly (Eq. 3 with SRP's
 * collision probability, §3): S_dev[q] = sum_i p(q, x_i)^K, p(q, x) = 1 - acos(q.x / (||q||
 * ||x||)) / pi, for nq queries Q_dev (nq x d) against nd points D_dev (nd x d), both binary32
 * or both bfloat16 (dtype).  Theorem 1 makes ACE's score (1/L) sum_j A_j[H_j(q)] of a detector
 * holding D an unbiased estimator of S(q, D); the random sampling estimator RSE (Eq. 10) is this
 * sum over a sample of D scaled by nd / (sample size).  Binary64 arithmetic throughout (dot
 * products and norms in index order, cos clamped to [-1, 1]); a zero vector has p = 1/2 against
 * a non-zero one (its SRP bits are all 0) and p = 1 against another zero vector.  The sum over
 * the points is taken in a fixed order, so the result does not depend on scheduling.
 * nq <= 65535, 1 <= K <= 64.  Synchronous on `stream` (it allocates and frees a scratch of
 * 8 nq ceil(nd / 256) bytes).  Errors: ACE_ERR_ARG, ACE_ERR_OOM, ACE_ERR_CUDA.
 */
int ace_exact_score(const void* Q_dev, int64_t nq, const void* D_dev, int64_t nd, int d, int dtype, int K,
                    double* S_dev, void* stream);

/*
 * ace_wait_probe — failure detection without a GPU fault: runs one of the library's bounded
 * device waits on an event that never happens, with nothing in flight, and reports how it
 * gave up.  kind 0: the tensor-core kernels' barrier wait, in a CTA that holds tensor memory
 * as the hash kernels do (it frees it after giving up; a second wait, with the abort flag
 * already set, returns at once); kind 1: the batched launch's wait on a device flag.
 * limit_cycles in [1e5, 1e9] SM cycles.  *status = ACE_STATUS_TIMEOUT when the wait gave up;
 * cycles_out (2 entries, may be NULL): the cycles the wait took and, for kind 0, those of the
 * aborted wait.  Synchronises the device; the context stays usable.  No counterpart in the
 * paper (an execution detail).  Errors: ACE_ERR_ARG, ACE_ERR_UNSUPPORTED (kind 0 needs an
 * sm_103 device), ACE_ERR_CUDA.
 */
int ace_wait_probe(int kind, int64_t limit_cycles, uint32_t* status, int64_t* cycles_out);

/*
 * ace_tc_probe — measurement hook for the tensor-core engines' error model.  Computes
 * D = A . B^T (A: 128 x kdim, B: ncols x kdim, bfloat16 bit patterns, row-major, host; D:
 * 128 x ncols binary32, host) on the tcgen05 tensor cores as kdim/16 MMA instructions of
 * 128 x ncols x 16 accumulating into one TMEM accumulator in k order, the way the hash kernels
 * accumulate Eq. 1's projections.  The guard bands of the tensor-core engines assume that one
 * such instruction adds its 16 products and the accumulator with an error of at most
 * 5.25 * 2^-23 times the sum of their magnitudes; a test feeds chosen sums through this hook to
 * check that assumption on the device at hand.  (The paper has no counterpart: it computes
 * Eq. 1 in one precision.)  kdim and ncols are multiples of 16 in [16, 256].  Synchronous
 * (it allocates and frees its own device buffers).
 * Errors: ACE_ERR_ARG, ACE_ERR_UNSUPPORTED (not an sm_103 device), ACE_ERR_TIMEOUT, ACE_ERR_CUDA.
 */
int ace_tc_probe(const uint16_t* A_host, const uint16_t* B_host, int kdim, int ncols, float* D_host);

/*
 * ace_tc_probe_fp8 — the same hook for E4M3 operands: A (128 x kdim) and B (ncols x kdim) hold
 * E4M3 bytes (row-major, host), and D = A . B^T is computed as kdim/32 kind::f8f6f4 MMA
 * instructions of 128 x ncols x 32 accumulating into one binary32 TMEM accumulator in k
 * order, the way the FP8 projection (ACE_PROJ_FP8) accumulates.  kdim is a multiple of 32 and
 * ncols a multiple of 16, both in [32, 256] and [16, 256].  Synchronous.  Errors as
 * ace_tc_probe.
 */
int ace_tc_probe_fp8(const uint8_t* A_host, const uint8_t* B_host, int kdim, int ncols, float* D_host);

/* Library version string. */
const char* ace_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ACE_GB300_H */
