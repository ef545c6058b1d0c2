/*
 * tfstat.h -- C ABI of the GB300 library for the semi-coherent time-frequency
 * track statistic of arXiv:2510.20891 ("Ab uno disce omnes: single-harmonic
 * search for extreme mass-ratio inspirals").
 *
 * The method (paper Sec. II.B-II.D):
 *   1. Cut the strain into non-overlapping segments of duration T_SFT, window
 *      each and Fourier transform it (the SFTs d~_{alpha,k}, Delta f = 1/T_SFT).
 *   2. Normalise the power by the known PSD: P[alpha,k] = 4 Delta f |d~|^2 / S_n,
 *      generalised here for a window (see tfs_build_sfts).
 *   3. Model a frequency track with an SVD basis, f_alpha = f_ref + sum_k c_k U_{k,alpha}
 *      (Sec. II.C), evaluated at the segment midpoints t_alpha = (alpha + 1/2) T_SFT.
 *   4. Sum the normalised power along the track, nearest bin b = floor(f T_SFT + 1/2)
 *      plus +-m neighbours: S = sum_alpha sum_{|j|<=m} P[alpha, b_alpha + j]
 *      (Eq. det_stat in its nearest-bin, non-chirping reading).
 *   5. Keep the k best tracks (Sec. II.D keeps the best 512 of 1024 walkers).
 *
 * Conventions for every entry point:
 *   - Return value: TFS_OK (0) or a negative TFS_ERR_* code; tfs_last_error()
 *     then gives a human-readable reason (thread-local string).
 *   - Nothing is written to caller buffers when a call fails validation.
 *   - Ownership: the caller owns every buffer it passes; the library owns the
 *     handles (tfs_table, tfs_basis) it returns, released with *_free.
 *   - mem = TFS_MEM_HOST: all array arguments are host pointers; the call copies
 *     inputs to the device, computes, copies results back and returns only
 *     when they are in place.  mem = TFS_MEM_DEVICE: all array arguments are
 *     device pointers of the current device; work is enqueued on `stream`
 *     (a cudaStream_t, NULL = legacy default stream) and the call returns
 *     without waiting, except where an entry point says otherwise.
 *   - Handles are bound to the device that was current when they were made.
 *   - Row-major layouts throughout; indices are 0-based.
 */
#ifndef TFSTAT_H_
#define TFSTAT_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define TFS_OK 0
#define TFS_ERR_INVALID_ARG (-1) /* shape, pointer, enum or range violation */
#define TFS_ERR_OOM (-2)         /* device or host allocation failed, or over budget */
#define TFS_ERR_CUDA (-3)        /* a CUDA runtime call or kernel failed */
#define TFS_ERR_TIMEOUT (-4)     /* a bounded device wait gave up; the context stays usable */
#define TFS_ERR_BUSY (-5)        /* resource in use (e.g. server queue full) */
#define TFS_ERR_NOT_FOUND (-6)   /* unknown id or ticket */

/* ---- enums ------------------------------------------------------------- */
#define TFS_F32 0    /* table storage: IEEE binary32 */
#define TFS_BF16 1   /* bfloat16, round to nearest even */
#define TFS_F16 2    /* IEEE binary16, round to nearest even (overflow -> inf) */
#define TFS_F8E4M3 3 /* FP8 E4M3 with a per-segment FP32 scale s_alpha: with e* the lower median of
                        floor(log2 P) over the row's positive entries, s_alpha = fl32(min(max_k P,
                        256 * 2^e*) / 448); stored codes saturate at 448 (outliers clip) */

#define TFS_WINDOW_RECT 0 /* w[n] = 1 */
#define TFS_WINDOW_HANN 1 /* periodic Hann, w[n] = sin^2(pi n / L) */

#define TFS_MEM_HOST 0
#define TFS_MEM_DEVICE 1

typedef struct tfs_table tfs_table; /* device-resident normalised power table */
typedef struct tfs_basis tfs_basis; /* device-resident track basis U [K][n_seg] (FP64) */

/* Ties of the track->bin rounding (|frac(x) - 1/2| <= 1e-9, x = f T_SFT).
 * The caller sets `capacity` and the two host arrays (or NULL with capacity 0);
 * the library writes `count` (total ties) and `n_stored` = min(count, capacity)
 * entries (track index, segment index) in unspecified order. */
typedef struct {
  int64_t count;
  int32_t n_stored;
  int32_t capacity;
  int64_t* track;
  int32_t* seg;
} tfs_tie_report;

/* ---- housekeeping ------------------------------------------------------ */
/* Version of this ABI (major * 10000 + minor * 100 + patch). */
int tfs_version(void);
/* Reason for the last failing call on this thread ("" if none). Never NULL. */
const char* tfs_last_error(void);

/* ---- step 1-2: strain -> normalised power table (paper Sec. II.B, II.E) --
 * strain [n] FP64 samples at spacing dt seconds.  L = T_sft/dt must be an
 * even integer >= 4 with prime factors 2, 3, 5 only and L <= 2^20
 * (else INVALID_ARG); n_seg = floor(n / L) segments (the ragged tail is
 * dropped; 1 <= n_seg <= 65535 required); n_bin = L/2 + 1 bins at frequencies k / T_sft.
 * psd [n_bin] FP64: the one-sided PSD S_n(k / T_sft) in Hz^-1.
 * Output P[alpha][k] = 4 |d~_{alpha,k}|^2 / (dt * sum_n w[n]^2 * S_n(k/T_sft)),
 * d~_{alpha,k} = dt sum_n w[n] x[alpha L + n] exp(-2 pi i n k / L), which is
 * the paper's 4 Delta f |d~|^2 / S_n for the rectangular window and gives
 * chi^2_2 (mean 2) noise power for any window.  P[alpha][0] = 0 and P = 0
 * wherever S_n is not finite and positive.  Computed in FP64, stored in
 * `dtype` (TFS_F32 / BF16 / F16 / F8E4M3).  mem refers to strain and psd.
 * Synchronous: returns when the table is complete. */
int tfs_build_sfts(const double* strain, int64_t n, double dt, double T_sft, int window, const double* psd,
                   int dtype, int mem, void* stream, tfs_table** out);

/* Recompute an existing table (made by tfs_build_sfts) from new strain of
 * the same length in segments, with the dt, T_sft, window, PSD and dtype
 * given at build time.  Allocates only stream-ordered scratch.  Enqueued on
 * `stream`; with stream NULL the call returns when the table is complete.
 * Otherwise mem = DEVICE returns without waiting and mem = HOST returns once
 * the strain has been copied (the host buffer may then be reused), the
 * transform still running on `stream`.  INVALID_ARG if n / L differs from
 * n_seg or the table was not built from strain. */
int tfs_table_rebuild(tfs_table* t, const double* strain, int64_t n, int mem, void* stream);

/* Wrap an existing FP64 power table P [n_seg][n_bin] (e.g. computed elsewhere)
 * as a table stored in `dtype`, quantised exactly as tfs_build_sfts does.
 * Synchronous. */
int tfs_table_from_power(const double* P, int64_t n_seg, int64_t n_bin, double T_sft, int dtype, int mem,
                         void* stream, tfs_table** out);

/* Shape and storage of a table. Any output pointer may be NULL. row_stride is
 * the element pitch of a row on the device (>= n_bin, a multiple of 32). */
int tfs_table_info(const tfs_table* t, int64_t* n_seg, int64_t* n_bin, int* dtype, double* T_sft,
                   int64_t* row_stride);

/* Copy the table out to host memory as FP64 dequantised values P [n_seg][n_bin]
 * (FP8: q * s_alpha in FP32, widened) and, for FP8, the scales [n_seg] (may be NULL). */
int tfs_table_to_host(const tfs_table* t, double* P, float* scales);

/* Device bytes held by the table: its stored values plus the window sums kept
 * for the neighbour half-widths m it has been evaluated with (the statistic
 * reads W_m[alpha][c] = sum_{|j|<=m} P[alpha][c+j], FP32, one row of n_bin + 2m
 * centres rounded up to 32 per segment, built on the first evaluation with that
 * m, recomputed with the table by tfs_table_rebuild and released with it). */
int64_t tfs_table_bytes(const tfs_table* t);

int tfs_table_free(tfs_table* t);

/* ---- track basis (paper Sec. II.C) --------------------------------------
 * tracks [M][n_seg] FP64: training frequency tracks (Hz) at t_alpha.
 * Uncentred truncated SVD F = U S V^T; the basis is the first K rows of V^T
 * (orthonormal rows, the paper's V_{p,alpha}), sign-fixed so the entry of
 * largest magnitude of each row is positive.  K = 0 chooses the smallest K
 * (<= min(M, n_seg, 32)) for which every training track reconstructs with
 * max_alpha |F - F V^T V| / max_alpha |F| <= tol.  Also records the singular
 * values and the box [cmin_k, cmax_k] of the training projections C = F V^T.
 * Computed with FP64 kernels (randomised range finder with power iterations)
 * plus host Gram-Schmidt and one-sided Jacobi on the thin factors.
 * 0 <= K <= min(M, n_seg, 32).  Synchronous. */
int tfs_build_basis(const double* tracks, int64_t M, int64_t n_seg, int K, double tol, int mem, void* stream,
                    tfs_basis** out);

/* Wrap a given basis U [K][n_seg] (host FP64, rows need not be orthonormal). */
int tfs_basis_from_host(const double* U, int K, int64_t n_seg, tfs_basis** out);

int tfs_basis_info(const tfs_basis* b, int* K, int64_t* n_seg);

/* Copy out U [K][n_seg], sigma [K], cmin [K], cmax [K] (host; any may be NULL;
 * sigma/cmin/cmax are zeros for a basis made by tfs_basis_from_host). */
int tfs_basis_to_host(const tfs_basis* b, double* U, double* sigma, double* cmin, double* cmax);

int tfs_basis_free(tfs_basis* b);

/* ---- steps 3-5: the statistic over a batch of tracks --------------------
 * coeffs [N][K] FP64 (K of the basis), f_ref [N] FP64 (Hz) or NULL for zeros.
 * Track t: f_{t,alpha} = f_ref[t] + sum_k coeffs[t][k] U[k][alpha], x = f T_sft,
 * b = floor(x + 1/2).  The bin equals the one FP64 arithmetic gives when
 * the sum is formed left to right with each product and sum rounded
 * separately (the GPU resolves every case that FP32 cannot decide in that
 * FP64 order).  stat[t] = sum_alpha sum_{j=-m..m} P[alpha][b+j] with bins
 * outside [0, n_bin) contributing 0 and non-finite x contributing 0,
 * accumulated in FP32 from the stored (dequantised) values.  0 <= m <= 64.
 * topk in [0, 1024]: if > 0, top_idx/top_val [min(topk, N)] receive the
 * largest stat values in descending order (ties: lower index first; NaN
 * lowest).  ties may be NULL; if given, the call waits for completion to
 * fill it (even with mem = DEVICE).  The basis must have n_seg equal to the
 * table's.  N may be 0.  stat may be NULL only if topk > 0 (then the
 * per-track values are kept in library scratch).  mem = HOST without a tie
 * report: the inputs go up in chunks (whole rounds of full tiles over the SMs,
 * at least 64 MB of coefficients each, at most 6 chunks) on a library stream,
 * each chunk evaluated by its own launch as soon as it has arrived (the
 * launches alternate between `stream` and a library stream that first waits
 * for the work enqueued on `stream`; `stream` waits for both before the top-k)
 * and its values read back while the next one runs; the bins are unchanged and
 * the statistic agrees with the one-launch result within FP32 rounding (which
 * pairs the FP32 filter leaves to the FP64 fix-up depends on the tiling).  Host
 * buffers should be pinned for the copies to overlap. */
int tfs_eval_stat(const tfs_table* table, const tfs_basis* basis, const double* coeffs, const double* f_ref,
                  int64_t N, int m, int topk, float* stat, int64_t* top_idx, float* top_val, tfs_tie_report* ties,
                  int mem, void* stream);

/* ---- step 4 alone, for verification: the bin of every (track, segment) ----
 * Runs the same fused kernel as tfs_eval_stat and writes bins [N][n_seg]
 * (int32): the bin b = floor(f T_sft + 1/2) whenever the window b-m..b+m
 * overlaps [0, n_bin); INT32_MIN if it lies wholly below bin 0, INT32_MAX if
 * wholly above the table or x is not finite.  N * n_seg < 2^34.  Synchronous. */
int tfs_eval_bins(const tfs_table* table, const tfs_basis* basis, const double* coeffs, const double* f_ref,
                  int64_t N, int m, int32_t* bins, int mem, void* stream);

/* ---- steps 3-5 for many datasets in one launch ------------------------------
 * The paper evaluates one dataset at a time; this entry point serves a batch
 * of independent searches (different tables, bases, track counts, m) with a
 * single persistent kernel launch per table dtype, so that small searches fill
 * the GPU together.  Each job's bins are those of tfs_eval_stat on the same
 * job; its statistic agrees with tfs_eval_stat's within FP32 rounding of the
 * sum (how tracks are grouped into tiles decides which pairs take the FP64
 * path, so the last bits may differ), and the same call repeated gives
 * bit-identical results.  All pointers inside the jobs are device
 * pointers of the current device; `jobs` itself is a host array of n_jobs
 * (1 <= n_jobs <= 4096) entries, read during the call only.  Per job: table
 * and basis with equal n_seg, 0 <= N < 2^31, 0 <= m <= 64, 0 <= topk <= 1024,
 * stat [N] or NULL (then topk > 0), top_idx/top_val [min(topk, N)] when
 * topk > 0.  Ties are not reported.
 * flags: 0, or TFS_JOB_SEGMENT_CUTS to apply the paper's segment exclusions
 * (second-order cut Sec. II.B; low frequency and low fdot Sec. II.D): segment alpha of a track contributes 0 when, with the track's
 * derivatives taken by finite differences at the segment midpoints
 * (fdot = central difference / (2 T_sft) inside, one-sided at the two ends;
 * fddot T_sft^3 / 6 = ((f[a+1] - 2 f[a]) + f[a-1]) T_sft / 6 inside, the
 * nearest inner value at the ends), the second-order term exceeds 1, or
 * f < 10^-3.5 Hz, or fdot < 1e-13 Hz/s.  Every exclusion is decided as the
 * FP64 evaluation in that operation order decides it.  reserved must be 0.
 * dev_status: a device int, or NULL.  Given, the call is fully asynchronous
 * and enqueues only stream-ordered work (cudaMallocAsync scratch, kernels,
 * memsets), so it can be captured into a CUDA graph: it zeroes *dev_status,
 * and a kernel sets it to 1 if a bounded device wait gave up.  NULL: the call
 * waits for completion and returns TFS_ERR_TIMEOUT in that case.  The first
 * call for a (basis, T_sft, coefficient slot count) builds cached per-segment
 * data and synchronises `stream` once: make it before any capture. */
typedef struct tfs_job {
  const tfs_table* table;
  const tfs_basis* basis;
  const double* coeffs; /* [N][K] */
  const double* f_ref;  /* [N] or NULL */
  int64_t N;
  int32_t m;
  int32_t topk;
  float* stat;          /* [N] or NULL */
  int64_t* top_idx;     /* [min(topk, N)] */
  float* top_val;       /* [min(topk, N)] */
  int32_t flags;        /* 0 or TFS_JOB_SEGMENT_CUTS */
  int32_t reserved;     /* 0 */
} tfs_job;

#define TFS_JOB_SEGMENT_CUTS 1

int tfs_eval_batch(const tfs_job* jobs, int n_jobs, int* dev_status, void* stream);

/* ---- launch-shape autotuning ---------------------------------------------
 * Not part of the paper's method: it picks how the statistic kernel is laid
 * out for a kind of workload, along four axes.  group (1..32) is the largest
 * number of consecutive segments one staging slot carries (a slot never
 * crosses a multiple of 32 segments), i.e. how many segments the consumers
 * take per hand-off; slots (2..8) is the depth of the staging ring;
 * pcap is the number of window sums of one segment's band staged per tile
 * (wider bands are cut to it and their pairs outside it take the slower exact
 * path); tile_div (1, 2, 4 or 8) divides the tracks per tile (smaller tiles:
 * more of them, better balance for small jobs); tile_class picks the tracks
 * each consumer thread carries (1: the large class, 12 for K <= 6; 2: the small
 * class, 4 for K <= 8, whose tiles are a third as large; 0: automatic, the
 * small class when a launch has fewer tracks than one round of large tiles
 * over the SMs).  Zeros select the defaults (group 32, slots 2, pcap 2048,
 * tile_div 1, automatic tile class).  tfs_autotune_batch evaluates
 * `jobs` (as tfs_eval_batch, overwriting their outputs) under candidate shapes,
 * `reps` times each, by coordinate descent from the default shape (each of the
 * five axes in turn, two passes, a move must gain 0.5%), and keeps the fastest for every
 * launch of this kind (coefficient slots, widest row and longest job in powers
 * of two, single job or batch); later tfs_eval_stat / tfs_eval_batch calls of
 * that kind use it.  best_ms and default_ms (either may be NULL) receive the
 * time per call of the chosen and of the default shape.  Synchronous.  The
 * choices live in the process; save and load them as a small JSON object
 * {"key": [pcap, tile_div, slots, group, tile_class], ...}. */
typedef struct tfs_tuning {
  int32_t pcap;
  int32_t tile_div;
  int32_t slots;
  int32_t group;
  int32_t tile_class;
} tfs_tuning;

int tfs_autotune_batch(const tfs_job* jobs, int n_jobs, int reps, tfs_tuning* best, double* best_ms,
                       double* default_ms, void* stream);
int tfs_tuning_save(const char* path);
int tfs_tuning_load(const char* path);
int tfs_tuning_clear(void);

/* ---- serving: many resident datasets, requests batched as they arrive -------
 * The paper evaluates walker populations in batches (Sec. II.D); serving many
 * independent searches at once has no counterpart in the paper.  A server keeps
 * datasets' tables on the current device under a byte budget and evaluates
 * submitted requests (a dataset, a batch of tracks) with continuous batching:
 * one worker thread keeps up to two tfs_eval_batch launches in flight on two
 * streams and admits queued requests (first come, first served) as soon as
 * their buffers, plus their table if it was evicted, fit under the budget.
 * Idle tables are evicted least recently used first; their bytes stay in host
 * memory and return on the next use (an eviction waits for the device).
 * Thread-safe: submit and wait may be called from any threads. */
typedef struct tfs_server tfs_server;

typedef struct tfs_server_stats {
  int64_t submitted, completed, failed, tracks_completed;
  int64_t evictions, loads, batches;
  int64_t used_bytes, resident_bytes, budget_bytes;
  double mean_jobs_per_batch;
  double p50_ms, p99_ms, mean_ms; /* latency: submit to the return of tfs_server_wait */
} tfs_server_stats;

/* budget_bytes > 0 bounds resident tables plus admitted requests' device
 * buffers (approximately: per-call scratch of tfs_eval_batch is not counted);
 * 1 <= max_batch_jobs <= 4096 requests per launch.  Binds the current device. */
int tfs_server_create(int64_t budget_bytes, int max_batch_jobs, tfs_server** out);

/* The server takes ownership of `table` (freed by tfs_server_free; do not free
 * it yourself) and borrows `basis` (it must outlive the server).  ds_id
 * receives the dataset's id (0, 1, ...). */
int tfs_server_add_dataset(tfs_server* s, tfs_table* table, const tfs_basis* basis, int* ds_id);

/* Queue a request: coeffs [N][K] and f_ref [N] (or NULL) are HOST arrays that
 * must stay valid until tfs_server_wait returns for the ticket (they are read
 * when the request is admitted).  1 <= N < 2^31, 0 <= m <= 64, 0 <= topk <= 1024.
 * Returns TFS_ERR_OOM if the request and its table alone exceed the budget,
 * TFS_ERR_NOT_FOUND for an unknown dataset.  Does not wait. */
int tfs_server_submit(tfs_server* s, int ds_id, const double* coeffs, const double* f_ref, int64_t N, int m,
                      int topk, int64_t* ticket);

/* Wait for a ticket (timeout_ms < 0: no limit) and copy its results to host
 * stat [N], top_idx / top_val [min(topk, N)] (any may be NULL).  The statistic
 * is the one tfs_eval_stat gives within FP32 rounding (the bins are identical).
 * The copies run on a stream of the server (one per concurrent waiter, kept
 * until tfs_server_free) straight into the destinations, pageable or pinned;
 * stat's pages are written (zeros) on the host first, so that the device does
 * not take page faults on memory that was never touched.
 * TFS_ERR_TIMEOUT leaves the ticket valid; any other return consumes it. */
int tfs_server_wait(tfs_server* s, int64_t ticket, int timeout_ms, float* stat, int64_t* top_idx, float* top_val);

int tfs_server_get_stats(tfs_server* s, tfs_server_stats* out);

/* Stops the worker after the queued requests ran, frees the server's tables
 * and buffers.  Tickets not yet waited for are dropped. */
int tfs_server_free(tfs_server* s);

/* ---- saving and restoring a table (not part of the paper's method) ---------
 * tfs_table_export copies the stored table exactly as it is held, row-major
 * [n_seg][row_stride] elements of the storage dtype (row_stride from
 * tfs_table_info; elements beyond n_bin are 0), into host `data`
 * (n_seg * row_stride * element size bytes), and the FP8 scales [n_seg] into
 * host `scales` (may be NULL for other dtypes).  tfs_table_import builds a
 * table from those bytes: the round trip is exact (the same stored values, so
 * the same statistic bit for bit), and a search can resume from saved tables.
 * Synchronous.  The importer's row_stride is that of tfs_table_from_power for
 * the same n_bin (a multiple of 32 elements). */
int tfs_table_export(const tfs_table* t, void* data, float* scales);
int tfs_table_import(const void* data, const float* scales, int64_t n_seg, int64_t n_bin, double T_sft, int dtype,
                     tfs_table** out);

/* ---- data chunks and shifted bases (the T_pl search of Sec. II.D) ----------
 * The paper searches data of growing duration T_obs (0.1 yr, then 12 SFTs more
 * per chunk, 48 chunks) for a plunge at the end of each chunk, aligning one
 * precomputed basis (plunge at the end of the year) by an integer time shift.
 * tfs_table_view: the rows seg0 .. seg0 + n_seg - 1 of a table as a table of
 * their own, sharing the device memory (no copy; valid while t lives; freeing
 * the view with tfs_table_free leaves t intact; a view cannot be rebuilt from
 * strain or handed to a server).  tfs_basis_view: the columns seg0 .. seg0 +
 * n_seg - 1 of every basis row as a new basis (a device copy of the K x n_seg
 * slice, with the training statistics copied); for a chunk of n_obs segments
 * of a year of n_seg, seg0 = n_seg - n_obs puts the basis's plunge at the
 * chunk's end.  Synchronous.  0 <= seg0, 1 <= n_seg, seg0 + n_seg within the
 * parent, else INVALID_ARG. */
int tfs_table_view(const tfs_table* t, int64_t seg0, int64_t n_seg, tfs_table** out);
int tfs_basis_view(const tfs_basis* b, int64_t seg0, int64_t n_seg, tfs_basis** out);

/* ---- differential evolution of a walker population (Sec. II.D, Eq. de_step) --
 * The paper's track-space DE without crossover: for every walker t,
 * f_trial = f_t + F_t (f_r1[t] - f_r2[t]), projected back to coefficients by the
 * basis pseudo-inverse and kept when it lies in the prior and raises the
 * statistic.  Tracks are linear in the coefficients, so the projection of the
 * proposal is exactly c_t + F_t (c_r1 - c_r2); both calls work on coefficients.
 * tfs_de_propose: c [N][K] (FP64), r1, r2 [N] (int32 walker indices into c),
 * F [N] (float, the paper draws it from U[0.3, 1.5]), lo, hi [K] (the prior
 * box) -> c_trial [N][K] and in_prior [N] (1 when every coefficient lies in
 * [lo, hi]).  tfs_de_accept: where in_prior[t] and s_trial[t] > s[t], copies
 * c_trial[t] into c[t] and s_trial[t] into s[t].  All pointers device pointers
 * of the current device; random draws are the caller's; stream-ordered and
 * asynchronous.  N in [0, 2^31), K in [1, 32]. */
int tfs_de_propose(const double* c, int64_t N, int K, const int32_t* r1, const int32_t* r2, const float* F,
                   const double* lo, const double* hi, double* c_trial, int32_t* in_prior, void* stream);
int tfs_de_accept(double* c, float* s, const double* c_trial, const float* s_trial, const int32_t* in_prior,
                  int64_t N, int K, void* stream);

/* The random draws of one DE iteration (Sec. II.D: for walker t of a chunk of W,
 * two distinct partners r1, r2 other than t from the same chunk, and F_DE
 * uniform in [f_lo, f_hi)), from the counter-based SplitMix64 generator (Steele,
 * Lea and Flood 2014): s(k) = mix(seed + k * 0x9E3779B97F4A7C15 mod 2^64) with
 * its 64-bit finaliser.  Walker g = c W + t of iteration i = *iter takes
 * z_j = s(3 (i n + g) + j), j = 1, 2, 3 (n = n_chunks W); a = 1 + ((z_1 >> 32)
 * (W - 1) >> 32), b = 1 + ((z_2 >> 32) (W - 2) >> 32), b += (b >= a);
 * r1 = c W + (t + a) mod W, r2 = c W + (t + b) mod W; F = f_lo + (f_hi - f_lo)
 * u with u = (z_3 >> 40) 2^-24, each FP32 operation rounded to nearest.
 * iter: a device int32, read and then incremented by the call (so a captured
 * graph draws afresh on every replay).  r1, r2 (int32) and F (float) [n]
 * device arrays.  W >= 3, n < 2^31, f_lo <= f_hi.  Stream-ordered, asynchronous. */
int tfs_de_draw(uint64_t seed, int32_t* iter, int64_t n_chunks, int W, float f_lo, float f_hi, int32_t* r1,
                int32_t* r2, float* F, void* stream);

/* ---- the paper's linear-chirp statistic (Sec. II.B, Eq. det_stat) ----------
 * The full per-segment statistic of the paper: the local waveform of segment
 * alpha is the chirping sinusoid exp(i [2 pi f_a (t - t_a) + pi fdot_a (t - t_a)^2])
 * (t_a the segment midpoint, f_a = f_ref + sum_k c_k U_k,alpha, fdot_a its
 * finite difference: (f_{a+1} - f_{a-1}) / (2 T_sft) inside, one-sided at the
 * ends, 0 for one segment), maximised over amplitude and phase:
 *   S_alpha = 4 / (dt sum w^2) |sum_k d~*_{alpha,k} h~_{alpha,k} / S_k|^2 / sum_k |h~_{alpha,k}|^2 / S_k
 * over the 2P + 1 bins k = b - P .. b + P around the nearest bin
 * b = floor(f_a T_sft + 1/2) that lie in the table (the DC bin and bins whose
 * S_n is not finite and positive left out); S_alpha = 0 when b itself lies
 * outside the table or no bin is left.
 * d~ is the Hann-windowed SFT of the strain (Sec. II.B); h~ the template's SFT,
 * evaluated as the Fourier integral of the windowed chirp at TFS_CHIRP_M = 256
 * points (equal to the sampled SFT within about 1e-6 of its peak for P <= 111
 * and |fdot| T_sft^2 <= 100: the aliasing of the Hann-windowed template's
 * tails).  The paper uses P = 100 (TFS_CHIRP_P).
 *
 * tfs_build_chirp_table: strain [n] (host or device per mem, FP64), dt,
 * T_sft (L = T_sft/dt an even 2,3,5-smooth integer in [512, 2^20]), psd [L/2+1]
 * one-sided S_n(k/T_sft).  Builds the device table z [n_seg][n_bin] (complex
 * FP32: sqrt(4 dt / (sum w^2 S_ref)) X_k S_ref / S_k with X the windowed DFT
 * and S_ref the median usable S_n) and wt [n_bin] = S_ref / S_k (0 where
 * unusable).  Synchronous; the handle is freed with tfs_ctable_free.
 * tfs_ctable_to_host copies z ([n_seg][n_bin][2] floats) and/or wt to host.
 *
 * tfs_eval_chirp_stat: coeffs [N][K] (FP64), f_ref [N] or NULL, stat [N]
 * (FP32) or NULL with topk > 0, top_idx / top_val [min(topk, N)]: device
 * pointers of the current device.  0 <= N < 2^31, 0 <= P <= 111, flags 0 or
 * TFS_JOB_SEGMENT_CUTS (the exclusions of tfs_job; an excluded segment
 * contributes 0), 0 <= topk <= 1024.  The bins b are those of the FP64
 * oracle, bit for bit.  Stream-ordered and asynchronous on `stream`
 * (scratch by cudaMallocAsync). */
typedef struct tfs_ctable tfs_ctable; /* device-resident linear-chirp table */
#define TFS_CHIRP_P 100
#define TFS_CHIRP_M 256
int tfs_build_chirp_table(const double* strain, int64_t n, double dt, double T_sft, const double* psd, int mem,
                          void* stream, tfs_ctable** out);
int tfs_ctable_info(const tfs_ctable* t, int64_t* n_seg, int64_t* n_bin, double* T_sft, double* dt, double* s_ref);
int tfs_ctable_to_host(const tfs_ctable* t, float* z, float* wt);
int tfs_ctable_free(tfs_ctable* t);
int tfs_eval_chirp_stat(const tfs_ctable* ct, const tfs_basis* basis, const double* coeffs, const double* f_ref,
                        int64_t N, int P, int flags, float* stat, int topk, int64_t* top_idx, float* top_val,
                        void* stream);

/* Linear-chirp statistic of many jobs in one launch (up to 64 per launch;
 * larger batches are split): each job as tfs_eval_chirp_stat without top-k
 * (coeffs [N][K], f_ref [N] or NULL, stat [N]: device pointers; 0 <= P <= 111;
 * flags 0 or TFS_JOB_SEGMENT_CUTS).  1 <= n_jobs <= 4096; stream-ordered and
 * asynchronous.  tfs_ctable_view: rows seg0 .. seg0 + n_seg - 1 of a chirp
 * table sharing its memory (as tfs_table_view; freed with tfs_ctable_free). */
typedef struct tfs_chirp_job {
  const tfs_ctable* table;
  const tfs_basis* basis;
  const double* coeffs; /* [N][K] */
  const double* f_ref;  /* [N] or NULL */
  int64_t N;
  int32_t P;
  int32_t flags;
  float* stat;          /* [N] */
} tfs_chirp_job;
int tfs_eval_chirp_batch(const tfs_chirp_job* jobs, int n_jobs, void* stream);
int tfs_ctable_view(const tfs_ctable* t, int64_t seg0, int64_t n_seg, tfs_ctable** out);

/* Measurement support, not part of the paper's method: the current device's L2
 * read bandwidth in GB/s (a buffer of buffer_bytes, 1 MB .. 1 GB, read `reps`
 * times, 1..1000, after one warm-up pass, with 16-byte L1-bypassing loads).
 * Allocates and frees its buffer; synchronous on the default stream. */
int tfs_measure_l2_read(int64_t buffer_bytes, int reps, double* gbs);

/* Number of kernels this library has launched in this process (all devices). */
long long tfs_kernel_launches(void);

/* Failure-detection control (not part of the paper's method).  Every wait of
 * the statistic kernel on one of its pipeline barriers gives up after
 * limit_ns nanoseconds (limit_ns <= 0 restores the default, 2 s); the kernel
 * then leaves its loops, lets every copy still in flight land and reports a
 * timeout, so that the call returns TFS_ERR_TIMEOUT (or sets dev_status) and
 * the context stays usable.  hold = 1 makes the kernel's staging warp first
 * wait for a signal that nothing sends, so that the next statistic launches
 * time out after limit_ns: a deterministic way for tests to exercise that
 * path without a fault.  hold = 0 is normal operation.  Process-wide; read
 * when a launch is enqueued. */
int tfs_set_wait_limit(int64_t limit_ns, int hold);

/* ---- step 5 alone: top-k of a float array ---------------------------------
 * k in [1, 1024], 1 <= N < 2^31.  Writes min(k, N) entries of idx (int64) and
 * val in descending order of val; equal values keep the lower index first,
 * -0.0 equals +0.0, NaN ranks below every number.  Device scratch (about
 * 8 KB plus 4 bytes per 4096 elements) is allocated stream-ordered per call. */
int tfs_topk(const float* val_in, int64_t N, int k, int64_t* idx, float* val, int mem, void* stream);

/* ---- step 5 over many arrays at once ---------------------------------------
 * The top-k of n independent arrays (paper Sec. II.D keeps the best walkers of
 * every data chunk): vals[i] [Ns[i]] device floats, ks[i] in [0, 1024] (0 or
 * Ns[i] = 0 skips array i), idx[i] / val[i] device outputs of min(ks[i], Ns[i])
 * entries, each exactly what tfs_topk gives for that array alone (same order,
 * ties, -0 and NaN rules).  The host arrays vals, Ns, ks, idx, val (n entries)
 * are read during the call.  One set of 9 kernel launches covers up to 64
 * arrays (more take one set per 64), instead of 9 per array.  Device scratch
 * (about 600 KB plus 4 bytes per 4096 elements) is stream-ordered; the call
 * returns without waiting unless stream is NULL. */
int tfs_topk_batch(const float* const* vals, const int64_t* Ns, const int* ks, int n, int64_t* const* idx,
                   float* const* val, void* stream);

/* ---- top-k that allocates nothing -----------------------------------------
 * The paper has no counterpart; this is a service for callers that must not
 * allocate device memory themselves or through the library: for example a
 * serving loop that reserved all of its device memory up front under a
 * budget, code that runs while another framework's allocator owns the
 * device's free memory, or a latency-critical loop that cannot afford
 * cudaMalloc / cudaFree, which may synchronise the device.
 * Same result as tfs_topk (mem = DEVICE): val_in [N], idx [min(k, N)] and
 * val [min(k, N)] are device pointers of the current device; work is enqueued
 * on `stream` and the call returns without waiting.  The scratch is a fixed
 * file-scope device array (about 74 KB, held by every device that loads the
 * library until the process exits) for 1 <= N <= 2^26; larger N returns
 * INVALID_ARG.  The call makes no allocation of any kind.  The first call on
 * a device looks up the array's device address with that device current
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call shares the one array and reinitialises what must start at zero,
 * so calls whose work overlaps on the device (on different streams, or from
 * different threads) race and give wrong results: order them. */
int tfs_topk_noalloc(const float* val_in, int64_t N, int k, int64_t* idx, float* val, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TFSTAT_H_ */
