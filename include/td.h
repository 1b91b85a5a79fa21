/*
 * td.h -- C ABI of the B300-native time-domain Gaussian likelihood.
 *
 * Method (arXiv 2603.06010, Sec. II): for residuals r = d - h(theta) on the
 * kept samples t_0 < ... < t_{N'-1} of a segment,
 *
 *     logL = -1/2 r^T C^{-1} r - 1/2 log det C - (N'/2) log 2 pi,
 *
 * where C_ij = rho(|t_i - t_j|) is the stationary-noise covariance built from
 * the autocovariance rho (Sec. II, the Toeplitz covariance; Sec. II.B items
 * 1-2, segments and gaps: gap samples are deleted, leaving the kept x kept
 * principal submatrix).  C = L L^T is factored once (Sec. II.A); every
 * evaluation whitens r with W = L^{-1} (Sec. II.A, Eq. eq:td_like_whitened)
 * and reduces chi2 = |W r|^2.
 *
 * Conventions shared by every call:
 *   - Every pointer argument documented "device" must point to memory of the
 *     device that was current when the segment was created; "host" pointers
 *     are ordinary CPU memory.
 *   - Residual batches are float32, column-major N' x K with leading
 *     dimension ldr >= N' (column k = residual k, kept samples only).
 *   - Outputs logL / chi2 are float64 arrays of K entries.
 *   - Calls taking a stream are asynchronous and stream-ordered unless stated
 *     otherwise; the caller keeps inputs alive and unmodified until the work
 *     on that stream has completed.
 *   - Errors are returned as td_status, never trapped; td_last_error()
 *     gives a thread-local message for the last failing call on the thread.
 *   - A segment is used by one host thread at a time, and its evaluation
 *     calls are ordered with each other on the device (one stream, or
 *     streams ordered by events): they share the segment's scratch buffers
 *     and cached work lists.  Different segments may run concurrently from
 *     different threads and streams (the server keeps at most one batch per
 *     segment in flight for this reason).
 *   - No device kernel spins without a bound: every wait inside a kernel
 *     gives up after a time limit (td_options.wait_limit_ns) and the call
 *     reports TD_ERR_TIMEOUT on the next synchronising call.
 */
#ifndef TD_H
#define TD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct td_segment td_segment;   /* opaque: owns device copies and factors */

typedef enum {
  TD_OK = 0,
  TD_ERR_INVALID = 1,       /* bad argument (null pointer, size, ldr < N', ...) */
  TD_ERR_NOT_PD = 2,        /* covariance not positive definite; see td_last_pivot */
  TD_ERR_OOM = 3,           /* device allocation failed */
  TD_ERR_CUDA = 4,          /* a CUDA runtime/driver call failed */
  TD_ERR_TIMEOUT = 5,       /* a bounded in-kernel wait ran out */
  TD_ERR_NOT_FACTORED = 6,  /* td_factor has not succeeded on this segment */
  TD_ERR_UNSUPPORTED = 7,   /* precision/size combination not built */
  TD_ERR_BUSY = 8           /* server admission refused (capacity) or request already running */
} td_status;

typedef enum {
  TD_PREC_FP64 = 0,    /* plain FP64 blocked forward substitution (CUDA cores) */
  TD_PREC_BF16X6 = 1,  /* L^{-1} and R as 3 bf16 slices each -- a fixed-point hi
                          slice (|.| <= 255 times a per-row / per-column power-of-two
                          quantum) and 2 floating remainder slices; 6 tensor-core
                          products; the hi*hi sum accumulates exactly in one FP32
                          accumulator, the 5 others in a second; combined in
                          double-float.  chi2 ~2e-8 relative to FP64 when many rows
                          share the sum; up to ~1.2e-7 for a column of a few rows
                          whose chi2 rests on one row (N' below a few hundred). */
  TD_PREC_BF16X3 = 2,  /* hi + 1 remainder slice, 3 products: ~1e-5 relative, below
                          the accuracy bar (kept to show why more products are needed) */
  TD_PREC_AUTO = 3,    /* default: TD_PREC_BF16X6 for 2048 <= N' <= 32768, TD_PREC_BF16X10
                          beyond (the 6-product |dlogL| grows as ~N' x 1e-8: 3.4e-4
                          measured at N' = 32257) and below (the 6-product chi2 error
                          grows as fewer rows carry a column's chi2: 2e-8 relative at
                          N' = 8192, 1.03e-7 measured on a gapped N' = 739 segment,
                          1.15e-7 at N' = 47).  A grouped launch gives each segment
                          the count td_loglike_batch would (one product launch per
                          count present). */
  TD_PREC_BF16X10 = 4  /* 4 slices each, the 10 products a+b <= 3: chi2 ~1e-9 relative */
} td_precision;

typedef enum {
  TD_PATH_AUTO = 0,
  TD_PATH_TENSOR = 1,   /* tcgen05 split-product GEMM, 256-row operator tiles over whole
                           rows, chi2 in the epilogue (large K) */
  TD_PATH_STREAM = 2,   /* the same kernel with long rows cut into k-chunks of a length
                           fixed by N' (more work items; the operator streams from HBM),
                           chunk results added in double-float by a reduce kernel */
  TD_PATH_FP64 = 3,     /* plain FP64 forward substitution */
  TD_PATH_STREAM64 = 4, /* as TD_PATH_STREAM with 64-row operator tiles */
  TD_PATH_SMALLK = 5,   /* K <= 256: operator rows as the MMA M dimension and the residual
                           columns as N (16, 32, 64, 128 or 256), so the MMA is not padded
                           to 128 columns and every operator tile is read once; default
                           for K <= 32, and for 64 < K <= 256 while N' < 24576 */
  TD_PATH_TENSOR128 = 6, /* as TD_PATH_TENSOR with 128-row operator tiles (two accumulator
                            pairs in TMEM: a tile's epilogue overlaps the next tile's MMAs) */
  TD_PATH_STREAM128 = 7, /* as TD_PATH_STREAM with 128-row operator tiles */
  TD_PATH_GSCE = 8      /* gap-free segments prepared by td_gs_prepare: chi2 by the
                           Gohberg-Semencul formula with circulant-embedded FFTs
                           (Sec. III.A), O(N log N) per column, FP32 FFTs with
                           double-float sums, one 8-CTA thread-block cluster per
                           column pair; `precision` is not used.  A column is
                           transformed together with its neighbour (columns 2j, 2j+1
                           share one complex FFT), so results agree across batches
                           within rounding, not bitwise.  TD_PATH_AUTO takes this path
                           too on a prepared segment where it measured faster than the
                           dense product (K <= 256, or N >= 24576), or when the
                           segment has no dense operator (prepared only), except with
                           refinement or TD_PREC_FP64. */
} td_path;

typedef struct {
  int precision;        /* td_precision; default TD_PREC_AUTO */
  int path;             /* td_path; default TD_PATH_AUTO */
  int refine;           /* 1 (or any nonzero value but 2): one refinement step (Sec. III.C precision scheme).
                           w~ = L^{-1} r at `precision`; s = r - L w~ from bf16 slices of
                           L with ten products (exact hi*hi, ~1e-9 of |L||w~|); delta =
                           L^{-1} s at `precision`; chi2 = |w~ + delta|^2.  Brings
                           any precision (BF16X3 included) to about 1e-8 in chi2 at
                           about three passes' cost.  128-row tiles: whole rows with
                           element-wise epilogues when they fill the GPU, else split-k
                           through the chunk reduction; TD_PATH_TENSOR* / TD_PATH_STREAM*
                           fix that choice (and so a column's bits across batches).
                           Needs the FP64 factor L: TD_ERR_UNSUPPORTED on
                           segments built by td_factor_many(TD_FACTOR_NO_FP64) or after
                           td_segment_release_fp64; TD_ERR_INVALID with TD_PREC_FP64 or
                           TD_PATH_FP64; grouped launches: TD_ERR_UNSUPPORTED.  The
                           slices of L (as large as the operator's) are made on the
                           first refined call, with two FP32 N'p x K buffers.
                           2: the same step with s = r - L w~ formed to FP64
                           accuracy: split products of six exact bf16 slices of L
                           and of w~ on the tensor cores, one 128-column chunk of L
                           at a time, accumulated in FP64 (one more N'p x K FP64
                           buffer), and delta computed with at least six products;
                           chi2 then agrees with the FP64 oracle to ~1e-12 from any
                           first-pass precision, at about three to six passes' cost. */
  int reserved0;
  int64_t wait_limit_ns;/* bound on any in-kernel wait; <= 0 -> 1 s */
} td_options;

/* Fill *opt with the defaults (TD_PREC_AUTO, auto path, no refinement, 1 s waits). */
void td_options_default(td_options* opt);

/*
 * td_segment_create -- one analysis segment of one detector.
 *   acf  : host, float64[n]; acf[k] = rho(k), lags 0..n-1 (Sec. II.B item 1:
 *          the ACF truncated to the segment).  Copied.
 *   n    : samples in the segment, n >= 1.
 *   mask : host, uint8[n], 1 = kept, 0 = gap sample (Sec. II.B item 2);
 *          NULL = no gaps.  At least one sample must be kept.  Copied.
 *   stream: CUDA stream (cudaStream_t) for the device copies; 0 = legacy.
 *   out  : receives the new segment.  The caller releases it with
 *          td_segment_destroy.
 * Validation: acf[0] > 0 and finite, n >= 1, >= 1 kept sample.
 * The call synchronises `stream` before returning.
 */
td_status td_segment_create(const double* acf, int64_t n, const uint8_t* mask,
                            void* stream, td_segment** out);

/*
 * td_factor -- C_kept = L L^T (Sec. II.A; Sec. III.A "Factorization of the
 * covariance matrix": once per segment, cached).  Blocked right-looking
 * Cholesky in blocks of 128 that carries the identity along, so the same
 * eliminations give the whitening operator L^{-1}; each block's factor and
 * inverse are FP64 on the CUDA cores, and the O(N'^3) panel and trailing
 * updates are FP64-accurate split products on the bf16 tensor cores (six
 * exact bf16 slices per FP64 operand row, about 2^-46 of sum |a||b| per
 * product; TD_FACTOR_FP64_CORES in td_factor_many selects the all-FP64
 * CUDA-core route instead).  Then log det C = 2 sum log L_ii (FP64) and the
 * operator's bf16 slices for the per-evaluation paths.  All results stay
 * resident on the device and are owned by the segment.  Synchronises `stream`.
 * Returns TD_ERR_NOT_PD if a pivot is <= 0 or not finite; td_last_pivot
 * then gives the 0-based kept-sample index of the first failing pivot.
 * TD_ERR_TIMEOUT if a bounded in-kernel wait ran out (2 s).
 */
td_status td_factor(td_segment* s, void* stream);

/*
 * Free the segment's FP64 factor (L and its diagonal-tile inverses), and the
 * refinement's slices of L if a refined call made them, keeping the whitening
 * operator slices and log det: the tensor-core paths keep working, the FP64
 * path and refinement then return TD_ERR_UNSUPPORTED.  Saves 8 N'^2 bytes of
 * device memory (more with the refinement state).  Synchronises the device.
 */
td_status td_segment_release_fp64(td_segment* s);

/*
 * Factor checkpoint and resume.  The factor is the O(N'^3) step of the
 * method (Sec. II.A; Sec. III.A: computed once and cached); these calls keep
 * it across device evictions and process restarts.
 * td_segment_save -- write the segment's evaluation state to the file `path`:
 *   the ACF and kept indices, and whichever of these are resident: the
 *   whitening operator slices and log det (after td_factor or
 *   td_factor_many), the FP64 factor L with its diagonal-tile inverses
 *   (unless released), the Gohberg-Semencul spectra (after td_gs_prepare).
 *   The file is written as "<path>.tmp" and renamed onto `path`, so a failed
 *   save leaves no partial file.  Device reads are ordered on `stream` and the
 *   call synchronises it.  TD_ERR_NOT_FACTORED when there is nothing to save;
 *   TD_ERR_INVALID when the file cannot be written.
 * td_segment_load -- create a new segment on the current device from such a
 *   file, with the same resident state; its results are bit-identical to the
 *   saved segment's.  The header (magic, version, sizes) is checked against
 *   the file size before any device work, and a 64-bit FNV-1a checksum of
 *   the payload after it has been read: a wrong, truncated or corrupted file
 *   returns TD_ERR_INVALID and *out = NULL.  The caller owns *out
 *   (td_segment_destroy).  Synchronises `stream`.
 */
td_status td_segment_save(const td_segment* s, const char* path, void* stream);
td_status td_segment_load(const char* path, void* stream, td_segment** out);

/*
 * td_factor_many -- factor several segments.  flags = 0: td_factor on each.
 * flags = TD_FACTOR_NO_FP64: keep only what the tensor-core paths need; every
 * gap-free segment then gets its whitening operator in O(N^2) by the
 * Levinson-Durbin recursion (rows of L^{-1} are the normalised
 * prediction-error filters; Sec. II.B item 6 names Levinson and Durbin):
 * one CTA per segment runs the recursion in FP64 and writes the rows, many
 * segments per launch (batched so their temporary N'^2 FP64 rows fit a
 * share of free memory), and log det C = sum log v_t; segments with gaps use
 * td_factor and then release their FP64 factor.  Segments longer than 2^20
 * samples also take td_factor.
 * The FP64 path of such segments returns TD_ERR_UNSUPPORTED.  Synchronises
 * `stream`; TD_ERR_NOT_PD as td_factor (td_last_pivot gives the order).
 */
#define TD_FACTOR_NO_FP64 1
#define TD_FACTOR_FP64_CORES 2   /* factor segments that take the Cholesky on the FP64 CUDA cores
                                    (64-wide blocks, L^{-1} by forward substitution; several times
                                    slower than the default tensor-core route; FP64 arithmetic throughout) */
td_status td_factor_many(td_segment* const* segs, int nseg, int flags, void* stream);

/*
 * td_gs_prepare -- Gohberg-Semencul form of a gap-free segment's inverse
 * covariance (Sec. III.A, the GS formula and Eq. eq:toeplitz_fft), for
 * td_loglike_batch with path TD_PATH_GSCE.  x = C^{-1} e_1 by the
 * Levinson-Durbin recursion in FP64 (O(N^2) once; no N^2 storage), log det C
 * = sum log v_t, then the spectra of the two circulant embeddings (length M
 * = the power of two >= 2N) by an FP64 FFT, rounded to FP32.  Keeps
 * 9 M / 4 x 8 bytes on the device (M = 16384 at N = 8192: 288 KB).  chi2
 * from FP32 FFTs is ~1.5e-8 rms relative at N = 1024 (below: too few terms
 * to average the rounding, so N >= 1024).
 * Independent of td_factor: a segment may have both.  Synchronises `stream`.
 * Errors: TD_ERR_UNSUPPORTED for a segment with gaps, N < 1024 or N > 32768;
 * TD_ERR_NOT_PD (td_last_pivot gives the order); TD_ERR_OOM.
 */
td_status td_gs_prepare(td_segment* s, void* stream);

/* log det C_kept (host scalar).  Requires a successful td_factor (or, for a
   segment only prepared by td_gs_prepare, gives the recursion's value). */
td_status td_logdet(const td_segment* s, double* out);

/* N' (kept sample count); -1 for a NULL segment. */
int64_t td_kept(const td_segment* s);

/* 0-based failing pivot of the last td_factor that returned TD_ERR_NOT_PD, else -1. */
int64_t td_last_pivot(const td_segment* s);

/*
 * td_loglike_batch -- per-evaluation hot path (Sec. II.A, Eq.
 * eq:td_like_whitened; Sec. III.A, the CDO whitening of cached operators):
 *   W = L^{-1} R,  chi2_k = sum_i W_ik^2 (FP64 reduction),
 *   logL_k = -chi2_k/2 - logdet/2 - (N'/2) log 2 pi.
 *   R    : device, float32, column-major N' x K, leading dimension ldr >= N'.
 *          Read only; caller-owned.
 *   K    : number of residual columns, 0 <= K <= 2^30; K = 0 is a no-op.
 *   logL : device, float64[K], caller-owned, overwritten.
 *   opt  : NULL = defaults.
 *   chi2 : optional device float64[K] (NULL = not written).
 *   stream: CUDA stream; asynchronous.  The segment's scratch space grows on
 *          first use for a given K (that call may allocate); later calls with
 *          K no larger do not allocate (call td_reserve before graph capture).
 * With a fixed path (opt->path other than TD_PATH_AUTO) the results for one
 * column do not depend on the other columns of the batch (fixed reduction
 * order), so a column evaluated alone or in any batch gives the same bits.
 * TD_PATH_AUTO picks the tile shape by (N', K), so a different K may change
 * the last bits (within the accuracy bar, never beyond it).
 */
td_status td_loglike_batch(td_segment* s, const float* R, int64_t ldr, int64_t K,
                           double* logL, const td_options* opt, double* chi2,
                           void* stream);

/*
 * td_loglike_batch_gather -- td_loglike_batch for residuals given at every
 * sample of the segment (gaps included): R is device float32, column-major
 * n x K, leading dimension ldr >= n; the kept rows (Sec. II.B items 1-2: gap
 * samples are deleted) are gathered on the device into a buffer the segment
 * owns (it grows on first use for a given K and is freed with the segment),
 * then evaluated exactly as td_loglike_batch on them (same results, bit for
 * bit).  K <= 65535 per call.  Asynchronous on `stream`.
 */
td_status td_loglike_batch_gather(td_segment* s, const float* R, int64_t ldr, int64_t K,
                                  double* logL, const td_options* opt, double* chi2,
                                  void* stream);

/*
 * td_loglike_batch_host -- the same evaluation with HOST buffers (the
 * batched evaluation of Sec. III.A fed from CPU memory).
 *   R    : host, float32, column-major N' x K, leading dimension ldr >= N'.
 *          Pinned memory (cudaHostAlloc / cudaHostRegister) lets the copies
 *          overlap the evaluation; pageable memory works, serialised.
 *   logL : host, float64[K], overwritten.  chi2: optional host float64[K].
 *   opt  : as for td_loglike_batch.
 *   stream: the evaluation runs on it; the host -> device copies run on a
 *          stream of the segment.  The call returns after the results are in
 *          host memory (it synchronises `stream`).
 * The batch is cut into chunks of 512 columns, double-buffered: chunk j+1 is
 * copied while chunk j is evaluated.  The segment keeps two staging buffers
 * of 512 N' floats and K-entry result buffers (allocated on first use, grown
 * when a larger K arrives, freed by td_segment_destroy).  Each chunk goes
 * through td_loglike_batch, so the results equal that call's bit for bit.
 * Not for use during stream capture.
 */
td_status td_loglike_batch_host(td_segment* s, const float* R, int64_t ldr, int64_t K,
                                double* logL, const td_options* opt, double* chi2,
                                void* stream);

/*
 * Template-input form (Sec. III.A: the data vector is fixed and whitened
 * once, every evaluation brings a template h) and the SNRs of Sec. II.B
 * item 7, with <a, b> = a^T C^{-1} b (Eq. eqn:ip):
 *   chi2 = <d - h, d - h>,  logL as td_loglike_batch,
 *   rho_mf = <d, h> / sqrt(<h, h>),  rho_eff^2 = <d, d> - <d - h, d - h>.
 *
 * td_set_data -- store the data vector d (float64, N' kept samples, host or
 *   device memory: copied) and compute <d, d> (d rounded once to float32 and
 *   whitened with `opt`).  Synchronises `stream`.  Requires a factored segment.
 * td_data_inner -- <d, d> of the stored data vector (host scalar).
 * td_template_batch -- K templates H (device, float32, column-major N' x K,
 *   leading dimension ldh >= N'): r_k = fl32(d - h_k) goes through
 *   td_loglike_batch; when out->hh, out->dh or out->rho_mf is requested the
 *   templates are whitened in the same batch (2K columns) and
 *   <d, h> = (<d, d> + <h, h> - chi2) / 2.  Outputs (device float64[K], NULL
 *   = not written; logL required) in td_template_out.  Asynchronous on
 *   `stream`; the segment's template buffers grow on first use (they may
 *   allocate).  K <= 65535 per call.  TD_ERR_INVALID without td_set_data.
 */
typedef struct td_template_out {
  double* logL;      /* required */
  double* chi2;      /* <d - h, d - h> */
  double* hh;        /* <h, h> */
  double* dh;        /* <d, h> */
  double* rho_mf;    /* <d, h> / sqrt(<h, h>) (0 when <h, h> = 0) */
  double* rho_eff2;  /* <d, d> - chi2 */
} td_template_out;
td_status td_set_data(td_segment* s, const double* d, const td_options* opt, void* stream);
td_status td_data_inner(const td_segment* s, double* dd);
td_status td_template_batch(td_segment* s, const float* H, int64_t ldh, int64_t K,
                            const td_template_out* out, const td_options* opt, void* stream);

/*
 * td_project_batch -- the template form with the detector projection and the
 * placement of each template done on the device, ahead of the same path
 * (Sec. II.B, waveform conditioning: zeros around the waveform place its
 * peak at the requested time; Sec. III.A, data projection and conditioning:
 * h = F_plus h_plus + F_cross h_cross).  For template k and segment sample t
 * (0 <= t < n; only kept samples are used):
 *   u = t - offset[k];
 *   h_k(t) = fl32(fl32(fp[k] hp[k ldw + u]) + fl32(fc[k] hc[k ldw + u]))   if 0 <= u < lw, else 0,
 * with fp[k], fc[k] rounded to float32 first (float32 products and sum, no
 * fused multiply-add); the residual is fl32(d - h_k) at the kept samples (d
 * from td_set_data), so the results equal td_template_batch on those
 * templates bit for bit.  Outputs as for td_template_batch.  The polarizations of a network's detectors are the same
 * arrays: one upload of hp, hc serves every detector's segment.
 *   hp, hc : device float32, template k's waveform at hp + k ldw (lw samples at
 *            the segment's rate); hc = NULL: no cross polarization (fc unused).
 *   ldw    : >= max(lw, 1).   lw >= 0 (lw = 0: h = 0).
 *   fp, fc : device float64[K] antenna factors.
 *   offset : device int64[K], the segment sample of waveform sample 0 (any
 *            value; waveform samples outside the segment or in a gap drop out).
 * Asynchronous on `stream`; buffers as td_template_batch (K <= 65535).
 * TD_ERR_INVALID for NULL or inconsistent arguments or without td_set_data.
 */
td_status td_project_batch(td_segment* s, const float* hp, const float* hc, int64_t ldw, int64_t lw,
                           int64_t K, const double* fp, const double* fc, const int64_t* offset,
                           const td_template_out* out, const td_options* opt, void* stream);

/*
 * td_loglike_batch_noalloc -- the evaluation td_loglike_batch makes with the
 * default precision (TD_PREC_AUTO: six split products, ten below 2048 and above
 * 32768 kept samples) on one fixed tile shape (64 operator rows per tile), so
 * results agree with td_loglike_batch within rounding, not bit for bit; for
 * callers that cannot allocate device memory while they
 * run: an application whose device memory is all reserved by its own caching
 * pool, a process under a hard device-memory cap, or a latency-critical loop
 * that must not enter cudaMalloc (which can synchronise the device).  This call
 * allocates nothing: its scratch (residual slices and chi2 partials) is one
 * fixed device array of TD_NOALLOC_SCRATCH_BYTES inside this library, which
 * every GPU that loads the library holds until the process exits.  The paper
 * has no counterpart; it is a property of this library's interface.
 *   Arguments as for td_loglike_batch (R, ldr, K, logL, chi2 caller-owned,
 *   device memory).  The segment must be factored (td_factor allocates) with
 *   its operator resident (else TD_ERR_NOT_FACTORED).
 *   Size limit: 8 K N8 + 8 K ceil(N'/256) * 4 bytes must fit (N8 = N' rounded
 *   up to 8, the slices' row rounded to 256 bytes), e.g. N' = 8192 with K up
 *   to 504;
 *   larger batches return TD_ERR_INVALID before any device work.
 *   The first call on a device looks up the array's device address (once per
 *   device, with that device current); make that first call before any stream
 *   capture.  Every call shares the one array, so calls whose kernels overlap
 *   on the GPU (other streams, other segments at the same time) race on it;
 *   serialise them.  Nothing in the array needs clearing: a call writes every
 *   scratch byte it reads.
 */
#define TD_NOALLOC_SCRATCH_BYTES (32ll << 20)
td_status td_loglike_batch_noalloc(td_segment* s, const float* R, int64_t ldr, int64_t K,
                                   double* logL, double* chi2, void* stream);

/* Pre-size the segment's scratch for batches of up to K columns (allocates). */
td_status td_reserve(td_segment* s, int64_t K, const td_options* opt);

/*
 * Grouped evaluation -- many segments (uneven N', own K each) in one
 * persistent tensor-core launch (the covariance of disjoint segments and
 * detectors is block-diagonal, Sec. II.B items 1 and 3).  Arrays have nseg
 * entries; R[i], ldr[i], K[i], logL[i] as for td_loglike_batch on segs[i];
 * chi2 may be NULL (or an array of per-segment device pointers, each may be
 * NULL).  All segments must be factored on the current device.
 *
 * td_group_create builds a plan: device work lists, segment descriptors and
 * scratch (this call allocates and synchronises).  The plan keeps the
 * pointers it was given: later launches read R[i] and write logL[i] there.
 * td_group_launch enqueues the evaluation on `stream` (four kernels whatever
 * nseg, two more for each further slice count its segments take, one more
 * with a joint sum, and before each product kernel of the main orientation a
 * 4-byte memset of its work counter: the product takes its items, segment by
 * segment, as its CTAs become free; no allocation; capturable in a CUDA
 * graph).  td_group_graph_launch
 * captures the launch into a CUDA graph on first use and replays it.
 * td_group_tune times the candidate tile shapes and chunk sizes on the plan's
 * own inputs, keeps the fastest, and records it for later plans of the same
 * kind in this process (synchronises; writes logL).  td_group_check reports a
 * device-side error (bounded-wait timeout).  td_group_shape reports the
 * chosen operator tile height, chunk multiplier and work-item count.
 */
typedef struct td_group td_group;
td_status td_group_create(td_segment* const* segs, const float* const* R, const int64_t* ldr,
                          const int64_t* K, double* const* logL, double* const* chi2, int nseg,
                          const td_options* opt, void* stream, td_group** out);
td_status td_group_launch(td_group* g, void* stream);
td_status td_group_graph_launch(td_group* g, void* stream);
td_status td_group_tune(td_group* g, void* stream, double* best_ms);
td_status td_group_check(td_group* g, void* stream);
int td_group_shape(const td_group* g, int* bn, int* s_factor, int* n_items);
void td_group_destroy(td_group* g);

/*
 * td_group_set_joint -- multi-detector likelihood (Sec. II.B item 3: the
 * detectors' log-likelihoods add): every later launch of the group also
 * writes joint[k] = sum over the group's segments (in their order) of
 * logL_i[k].  All segments must have the same K; joint is device float64[K],
 * caller-owned; NULL turns the sum off.  Drops a captured graph (the next
 * td_group_graph_launch captures again).
 */
td_status td_group_set_joint(td_group* g, double* joint);

/*
 * td_group_clock -- as td_profile_clock, for the product launches of this
 * group (direct, graph or autotuner launches) since the previous call or
 * td_group_create.
 */
td_status td_group_clock(td_group* g, void* stream, double* mhz);

/* One-shot grouped evaluation: create, launch, check, destroy (synchronises). */
td_status td_loglike_grouped(td_segment* const* segs, const float* const* R,
                             const int64_t* ldr, const int64_t* K, double* const* logL,
                             int nseg, const td_options* opt, void* stream);

/*
 * td_check -- synchronise `stream` and report any error a kernel of this
 * segment recorded on the device since the last check (TD_ERR_TIMEOUT when a
 * bounded wait ran out).  Clears the recorded error.
 */
td_status td_check(td_segment* s, void* stream);

/*
 * Instrumentation.  td_profile_enable(s, 1) makes every later hot-path call
 * on s bracket its dominant kernel (the tensor-core product, or the FP64
 * forward substitution) with CUDA events recorded on the call's own stream,
 * and count every kernel the call launches.  td_profile_read synchronises
 * those events and returns the summed dominant-kernel time (ms), the number
 * of dominant-kernel launches and the total kernels launched since enabling,
 * then resets the counters.  At most 4096 bracketed launches are kept.
 */
td_status td_profile_enable(td_segment* s, int enable);
td_status td_profile_read(td_segment* s, double* ms_total, int64_t* dominant_launches,
                          int64_t* kernels_launched);

/*
 * td_profile_clock -- the SM clock (MHz) the split-product kernel (the
 * 256/128/64-row tensor-core kernel, single or list mode, refinement
 * included) actually ran at on this segment's work since the previous read
 * or td_profile_enable: each CTA's MMA-issuing thread counts SM cycles
 * (clock64) and global-timer nanoseconds from its start until its last MMA
 * retired, the sums over CTAs and launches are kept in the segment's device
 * status word, and *mhz = 1000 x cycles / ns.  A reading below the nominal
 * clock under load is the power or thermal limit at work.  Synchronises
 * `stream`, then clears the sums.  TD_ERR_INVALID when no such kernel ran
 * since the last read (the small-batch kernel does not record).
 */
td_status td_profile_clock(td_segment* s, void* stream, double* mhz);

/* Release a segment and all device memory it owns (synchronises its work). */
void td_segment_destroy(td_segment* s);

/*
 * Serving runtime -- many concurrent likelihood requests on many resident
 * segments (the paper's pool of concurrent proposal evaluations, Sec. III.B
 * "CPU acceleration", as requests).  A scheduler thread packs the pending
 * columns of one segment into one batch whenever one of n_streams streams is
 * free (continuous batching: requests arriving while other batches run join
 * the next batch of their segment); batches of different segments run
 * concurrently.  Whitening operators stay resident in HBM under
 * resident_bytes_budget with LRU eviction; an evicted operator is kept in
 * pinned host memory and copied back on its next use.  Operators live in the
 * server's stream-ordered device pool and their spill copies in a pinned
 * host pool reserved at creation (host_spill_bytes), so eviction (an
 * asynchronous copy out, the first time, and a release to the pool) and
 * reload (an asynchronous copy in) synchronise neither the host nor the
 * device while serving.  All calls are thread-safe.  Results of a request are within the
 * library's accuracy bar of the same request evaluated alone; bit-identical
 * with `deterministic` set.
 *   add_segment: host acf/mask as td_segment_create; the factor is computed on
 *     first use or by td_server_prefetch (synchronous; also reserves scratch
 *     and builds the work lists for batches up to max_batch_cols, so serving
 *     allocates nothing).  The FP64 factor is released after factoring.
 *   submit: R (device, float32, N' x K column-major, leading dimension ldr) and
 *     logL (device, float64[K]) are caller-owned and must stay valid until the
 *     request completes; 1 <= K <= max_batch_cols.  Returns TD_ERR_BUSY when
 *     the pending-column capacity would be exceeded (admission refused).
 *   poll: state 0 pending, 1 running, 2 done, 3 cancelled, 4 failed.
 *   wait: blocks up to timeout_us (TD_ERR_TIMEOUT after).
 *   cancel: only before the request is batched (TD_ERR_BUSY after).
 *   pause: stops batching new work (for tests and draining).
 *   replay: submits n requests at t_submit_s[i] seconds after the call
 *     (open-loop load from a native thread); tickets[i] = -1 if refused.
 *   get_stats: latency percentiles from submission to completion, evaluations per
 *     second between the first submission and the last completion, LRU
 *     counters; reset != 0 clears them.
 */
typedef struct td_server td_server;
typedef struct {
  int64_t max_batch_cols;        /* widest batch the scheduler packs (and largest request) */
  int64_t max_pending_cols;      /* admission capacity: queued + running columns */
  int64_t resident_bytes_budget; /* HBM budget for resident operators; 0 = unlimited */
  int n_streams;                 /* concurrent batches, 1..16 */
  int precision;                 /* td_precision of the tensor-core path; default TD_PREC_AUTO */
  int64_t max_kept;              /* largest N' a segment may have (sizes batch buffers) */
  int gs_gapfree;                /* nonzero: gap-free segments with 1024 <= N <= 32768 also get
                                    the Gohberg-Semencul form (td_gs_prepare) on first use;
                                    batches that TD_PATH_AUTO sends to GSCE (K <= 256, or
                                    N >= 24576) then run without loading the dense operator
                                    (O(N) device memory for such segments).  Default 0. */
  int deterministic;             /* nonzero: every batch takes one fixed path per segment (the
                                    small-batch kernel in chunks of at most 256 columns; no GSCE),
                                    so a request's logL is bit-identical alone and in any mix of
                                    other requests (a column's arithmetic then depends on its own
                                    values and its segment only).  Default 0: the automatic path,
                                    whose tile shape follows the batch width (results agree within
                                    the accuracy bar, not bit for bit). */
  int64_t host_spill_bytes;      /* pinned host memory reserved at creation for the spill copies of
                                    evicted operators (carved per segment at its first eviction);
                                    beyond it each copy is pinned on its own (cudaMallocHost, which
                                    blocks the scheduler).  Default 0. */
} td_server_config;
typedef struct {
  double p50_us, p99_us, max_us, evals_per_s;
  int64_t requests_done, evals, batches, hits, misses, evictions, refused, failed, resident_bytes;
  int64_t reloads;               /* misses served by copying a spilled operator back from pinned host memory */
} td_server_stats;
void td_server_config_default(td_server_config* c);
td_status td_server_create(const td_server_config* cfg, td_server** out);
td_status td_server_add_segment(td_server* srv, const double* acf, int64_t n, const uint8_t* mask,
                                int64_t* seg_id);
td_status td_server_prefetch(td_server* srv, int64_t seg_id);
/* Change the HBM budget for resident operators (0 = unlimited): idle
 * segments are evicted at once, least recently used first, until it holds
 * (synchronises); later misses evict as they need room. */
td_status td_server_set_budget(td_server* srv, int64_t resident_bytes_budget);
td_status td_server_submit(td_server* srv, int64_t seg_id, const float* R, int64_t ldr, int64_t K,
                           double* logL, int64_t* ticket);
td_status td_server_poll(td_server* srv, int64_t ticket, int* state);
/* Latency of a finished request (submission to completion, microseconds);
 * TD_ERR_BUSY while it is not done. */
td_status td_server_latency(td_server* srv, int64_t ticket, double* us);
td_status td_server_wait(td_server* srv, int64_t ticket, int64_t timeout_us);
td_status td_server_cancel(td_server* srv, int64_t ticket);
td_status td_server_pause(td_server* srv, int paused);
td_status td_server_drain(td_server* srv, int64_t timeout_us);
td_status td_server_replay(td_server* srv, const double* t_submit_s, const int64_t* seg,
                           const float* const* R, const int64_t* ldr, const int64_t* K,
                           double* const* logL, int64_t n, int64_t* tickets);
td_status td_server_get_stats(td_server* srv, td_server_stats* out, int reset);
void td_server_destroy(td_server* srv);

/* Thread-local message for the last failing call on this thread ("" if none). */
const char* td_last_error(void);

/* Bytes of device memory the segment holds resident (factor + operators). */
int64_t td_resident_bytes(const td_segment* s);

/*
 * td_debug_bounded_wait -- runs one tiny kernel whose wait is on a flag that
 * nothing sets, bounded by limit_ns; returns TD_ERR_TIMEOUT when the bound
 * ran out (the expected outcome) and leaves the context usable.  Exists to
 * test the bounded-wait machinery without faulting a GPU.  Synchronous.
 */
td_status td_debug_bounded_wait(int64_t limit_ns, void* stream);

/*
 * td_debug_plan -- the work list the grouped launch of the main orientation
 * would build (host code only; no device is touched).  For nseg segments of
 * nk[i] kept samples and K[i] columns, operator tiles of bn rows (256, 128 or
 * 64) and k-chunks of S k-blocks (32 kept samples each), writes one record of
 * six ints per work item to out: segment, row tile, column tile (128
 * columns), first k-block, k-blocks, chunk slot (-1 for a whole row), in
 * launch order: segment by segment (by_segment != 0, the order the dynamic
 * schedule takes) or longest first.  Returns the item count, or -count when
 * cap (in records) is too small (nothing written), or -1 on bad arguments.
 * Exists to test the planning logic on a machine without a GPU.
 */
int td_debug_plan(const int64_t* nk, const int64_t* K, int nseg, int bn, int S, int by_segment, int* out,
                  int cap);

#ifdef __cplusplus
}
#endif
#endif /* TD_H */
