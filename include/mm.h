/*
 * mm.h -- C ABI of the GB300 Malliavin-Mancino Fourier covariance library.
 *
 * The library computes, for D assets observed at asynchronous event times,
 *   (1) the Fourier coefficients F(dp_i)(k), |k| <= N, of each asset's
 *       log-price returns (Eq. (4), Sec. 2.2) with a type-1 NUFFT (Sec. 2.2.5:
 *       spreading Eq. (12), FFT Eq. (13), deconvolution Eq. (14));
 *   (2) the D x D integrated covariance Sigma under the Dirichlet (Eq. (2)) or
 *       Fejer (Eq. (3)) basis and the correlation R (Algorithm 3).
 * Citations name the paper: Chang, Pienaar & Gebbie, "Malliavin-Mancino
 * estimators implemented with non-uniform fast Fourier transforms",
 * arXiv:2003.02842. Equations are numbered in display order; algorithms in
 * appendix order (Algorithm 2 Nyquist, 3 MM estimators, 4 time rescaling,
 * 8-10 NUFFT with Gaussian, Kaiser-Bessel and ES kernels).
 *
 * Conventions shared by every call:
 *  - Event data is CSR: offsets[D+1] (int64, non-decreasing, offsets[0] = 0,
 *    offsets[D] <= desc.max_events); t[offsets[D]] event times (float64, any
 *    unit, strictly increasing within an asset); logp[offsets[D]] log-prices
 *    (float64). Asset i owns events offsets[i] .. offsets[i+1]-1. Its returns
 *    delta_h = logp[h+1] - logp[h] sit at the left end point t[h] (Sec. 2.1);
 *    an asset with fewer than two events has no returns and zero coefficients.
 *  - Pointers named d_* are device pointers on the current device; h_* are
 *    host pointers (pinned memory makes the copies asynchronous). The caller
 *    owns every input and output buffer; the plan owns only its workspace.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Device-side calls are asynchronous on it unless stated otherwise.
 *  - Coefficients are Hermitian-half, F-convention (the 1/(2 pi) of Eq. (4)
 *    included): d_coeffs[i * (N+1) + k] = F(dp_i)(k), k = 0..N; complex128
 *    (interleaved double re, im) for MM_PREC_FP64, complex64 otherwise.
 *    F(dp_i)(-k) = conj(F(dp_i)(k)).
 *  - Sigma and R are D x D row-major, float64 for MM_PREC_FP64 and float32
 *    otherwise. R_ii = 1 exactly; a zero-variance asset gives NaN in its row
 *    and column of R and the non-fatal status MM_ERR_ZERO_VARIANCE at the
 *    next mm_plan_sync.
 *  - Errors found on the host are returned at once and nothing is launched.
 *    Errors that need the data (unsorted or repeated times, non-finite
 *    values, a bounded device wait that gave up) are recorded in a device
 *    status word; mm_plan_sync returns and clears the first of them. All
 *    device indexing is bounds-checked, so bad data gives bad numbers and a
 *    status, never an out-of-bounds access.
 *  - A plan is used by one host thread at a time. Calls that overlap on the
 *    GPU through different streams must use different plans (they share the
 *    plan's workspace).
 */
#ifndef MM_GB300_H
#define MM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MM_OK = 0,
  MM_ERR_INVALID_ARG = 1,     /* bad pointer, size or enum; bad offsets array */
  MM_ERR_UNSORTED = 2,        /* event times decrease within an asset */
  MM_ERR_DUPLICATE_TIME = 3,  /* two events of an asset share a time (Delta t0 = 0, Algorithm 2) */
  MM_ERR_DEGENERATE_SPAN = 4, /* t_max <= t_min or non-finite bounds (Algorithm 4) */
  MM_ERR_CUTOFF = 5,          /* N > N_max, N < 1 under Fejer, or no Nyquist cutoff */
  MM_ERR_OOM = 6,             /* workspace allocation failed at plan creation */
  MM_ERR_CUDA = 7,            /* a CUDA runtime call or launch failed */
  MM_ERR_TIMEOUT = 8,         /* a bounded device-side wait gave up */
  MM_ERR_ZERO_VARIANCE = 9,   /* non-fatal: Sigma_ii = 0 for some asset, R has NaN */
  MM_ERR_NONFINITE = 10,      /* NaN or Inf time or log-price in the input */
  MM_ERR_UNSUPPORTED = 11     /* request outside what this build supports */
} mm_status;

/* Basis kernel of the contraction: Dirichlet Eq. (2) / Algorithm 3 C.1,
 * weights 1/(2N+1); Fejer Eq. (3) / Algorithm 3 C.2, weights
 * (1 - |k|/N)/(N+1), taken literally (so Sigma_Fejer carries N/(N+1)). */
typedef enum { MM_BASIS_DIRICHLET = 0, MM_BASIS_FEJER = 1 } mm_basis;

/* Averaging kernel of the NUFFT (Sec. 2.2.5): Gaussian with the fast Gaussian
 * gridding split (Eqs. (5)-(6), (17), Algorithm 8), Kaiser-Bessel
 * (Eqs. (7)-(8), Algorithm 9), exponential of semicircle (Eqs. (9)-(10),
 * Algorithm 10). The spreading half-width M_sp(tol) follows the rules of
 * Sec. 2.2.5. */
typedef enum { MM_KERNEL_GAUSS = 0, MM_KERNEL_KB = 1, MM_KERNEL_ES = 2 } mm_kernel;

/* MM_PREC_FP64: every stage in float64. MM_PREC_MIXED_*: rescaling, phase
 * reduction to grid offsets, differencing into returns and the diagonal
 * normalisation in float64; spreading, FFT and deconvolution in float32; the
 * contraction on the tensor cores as split bf16 (hi*hi + hi*lo + lo*hi) or
 * split tf32 products with float32 accumulation. */
typedef enum {
  MM_PREC_FP64 = 0,
  MM_PREC_MIXED_BF16X3 = 1,
  MM_PREC_MIXED_3XTF32 = 2
} mm_precision;

typedef struct {
  int32_t D;            /* number of assets, >= 1 */
  int32_t N_max;        /* largest cutoff any call will use, >= 0 */
  int64_t max_events;   /* upper bound on offsets[D]; sizes the host-staging buffers */
  double tol;           /* NUFFT tolerance eps in (0, 0.5) (Sec. 2.2.5) */
  mm_kernel kernel;
  mm_basis basis;
  mm_precision prec;
  int32_t spread_tile;  /* grid cells per spreading block; 0 = library default */
  int32_t spread_algo;  /* 0 library default (= 1 unless mm_autotune chose otherwise);
                           1 separate prep / scatter-into-tile / FFT kernels (the mixed
                           path evaluates the kernel as per-tap polynomials and
                           accumulates exactly in integers); 2 as 1 with a gather per
                           grid cell (no atomics: the FP64 path's sums then come out
                           in a fixed order); 3 stages (a2)-(c) in one launch with
                           each asset's grid row resident in shared memory (one CTA
                           per row, or a cluster of two for rows too large for one;
                           the mixed path with polynomial taps, after the prep
                           kernel), or, where that does not apply, stages (a)-(c)
                           in one CTA per asset for a single problem whose grid fits
                           in shared memory; else 1. All compute Eq. (12). */
  int32_t fft_algo;     /* stages (b)-(c) in the mixed precisions: 0 library default
                           (the grid in shared memory when it fits: as 2 when one
                           asset's row fits one CTA, else as 4; otherwise 1);
                           1 two-pass FFT through global memory; 2 one CTA per
                           asset; 4 a cluster of two CTAs per asset (decimation in
                           time by 2, halves joined through distributed shared
                           memory); 5 as 2 with the polynomial scatter storing the
                           grid in the FFT's digit-reversed input order (one bulk
                           copy per row). 3 and 6 (two or three CTAs per asset with
                           a radix-2 or radix-3 step on load) are not built: they
                           measured slower on every workload. The FP64 path always
                           uses 1. All compute Eqs. (13)-(14). */
  int32_t gram_algo;    /* stage (d) in the mixed precisions: 0 library default (2 from
                           192 assets up, else 1); 1 each CTA converts its
                           tiles of the weighted coefficients to split precision in
                           registers; 2 a streaming pass writes the weighted operand once
                           as hi and lo planes and the contraction loads them by TMA
                           (warp-specialised producer / MMA / epilogue). Both compute
                           Eqs. (2)/(3) with the same split products. */
  int32_t reserved[3];  /* must be zero */
} mm_plan_desc;

typedef struct mm_plan_s* mm_plan;

/* Per-stage timing and launch counters (device time from CUDA events on the
 * launching stream, summed since the last reset). */
enum { MM_STAGE_PREP = 0, MM_STAGE_SPREAD = 1, MM_STAGE_FFT_COLS = 2, MM_STAGE_FFT_ROWS = 3,
       MM_STAGE_GRAM = 4, MM_STAGE_REDUCE = 5, MM_STAGE_SETUP = 6, MM_STAGE_FUSED = 7, MM_STAGE_FFT = 8,
       MM_STAGE_SPLIT = 9, /* the contraction operand's pre-split pass */
       MM_NUM_STAGES = 10 };

typedef struct {
  int32_t msp;           /* spreading half-width M_sp */
  int32_t N;             /* cutoff of the last call */
  int64_t Mr;            /* oversampled grid size of the last call */
  int64_t fft_P, fft_Q;  /* Mr/2 = P * Q factorisation of the last call */
  int64_t workspace_bytes;
  int64_t launches;      /* kernels launched by this plan since creation */
  int32_t gram_splits;   /* split-K factor of the last contraction */
  int32_t spread_algo;   /* stage (a)-(c) variant in use: 1 scatter, 2 gather, 3 fused
                            (the resident row when res_sub > 0) */
  int32_t spread_tile;   /* grid cells per spreading block in use */
  int32_t fft_lg_cols;   /* FFT pass 1: log2 of the columns per block */
  int32_t fft_rowblk;    /* FFT pass 2: lower rows per block */
  float tuned_ms;        /* mm_coeffs time of the configuration mm_autotune chose (0 if untuned) */
  int32_t fft_algo;      /* stages (b)-(c) in use: 0 per-asset shared-memory FFT, 1 two-pass */
  int32_t fft_passes;    /* per-asset FFT: number of radix passes (0 when not in use) */
  int32_t fft_radix[4];  /* per-asset FFT: radix of each pass */
  int32_t fft_split;     /* per-asset FFT: 1 one CTA per asset, 3 a cluster of two CTAs joined
                            through distributed shared memory; 0 when not in use */
  int32_t spread_poly;   /* 1: float32 spreading evaluates the kernel as per-tap polynomials
                            (error <= max(3e-7, tol/10)) and accumulates exactly in integers */
  int32_t graphs;        /* 1: steady mm_estimate calls replay a captured CUDA graph */
  int64_t graph_launches; /* mm_estimate calls served by a graph replay since creation */
  int32_t gram_algo;     /* stage (d) of the last contraction: 1 in-register conversion,
                            2 pre-split operand by TMA, 3 FP64 path; 0 before the first */
  int32_t res_sub;       /* spread_algo 3 with the grid row resident after the prep kernel:
                            cells per sub-range of the row; 0 when not in use */
} mm_plan_info;

/* Create a plan: validates desc, allocates the workspace on the current
 * device (grid, FFT tables, contraction partials, staging for the host-buffer
 * entry point). Returns MM_ERR_INVALID_ARG for a bad desc, MM_ERR_OOM when an
 * allocation fails. *out is NULL on failure. */
mm_status mm_plan_create(const mm_plan_desc* desc, mm_plan* out);

/* Release the plan and its workspace (synchronises the device first). */
mm_status mm_destroy(mm_plan plan);

/* Fourier coefficients F(dp_i)(k), k = 0..N, of every asset (Eq. (4)) by the
 * type-1 NUFFT of Sec. 2.2.5.
 *  N > 0: the cutoff (N <= N_max). N <= 0: the Nyquist cutoff of Algorithm 2,
 *         N = min_i floor(span / (2 min-gap_i)); this form synchronises the
 *         stream to read N back.
 *  t0 < t1: rescale with that window, t~ = 2 pi (t - t0)/(t1 - t0) (events
 *         must lie in [t0, t1]); otherwise t0, t1 are taken as the minimum
 *         and maximum time over all assets (Algorithm 4).
 *  d_coeffs: D * (N+1) complex elements (see conventions).
 *  N_used: optional host pointer receiving the cutoff used. */
mm_status mm_coeffs(mm_plan plan, const int64_t* d_offsets, const double* d_t,
                    const double* d_logp, int32_t N, double t0, double t1,
                    void* d_coeffs, int32_t* N_used, void* stream);

/* Covariance from coefficients (Algorithm 3 step C, Eqs. (2)/(3)):
 * Sigma_ij = sum_{|k|<=N} w_k (2 pi)^2 conj(F_i(k)) F_j(k), computed as a
 * split-K Hermitian rank-(2N+1) update (tensor cores in the mixed
 * precisions). d_coeffs as written by mm_coeffs for the same N. */
mm_status mm_cov(mm_plan plan, const void* d_coeffs, int32_t N, void* d_sigma, void* stream);

/* Covariance and correlation R_ij = Sigma_ij / (sqrt(Sigma_ii) sqrt(Sigma_jj))
 * (Algorithm 3, last step), the normalisation in float64. d_sigma may be
 * NULL when only R is wanted. */
mm_status mm_corr(mm_plan plan, const void* d_coeffs, int32_t N, void* d_sigma_or_null,
                  void* d_R, void* stream);

/* Covariance with a cutoff per pair of assets (Sec. 3.1: assets with their
 * own cutoffs, e.g. their own Nyquist cutoffs in the arrival-time
 * representation, give D(D-1)/2 pairwise estimates): Sigma_ij is Eq. (2)
 * (Dirichlet) or Eq. (3) (Fejer), the plan's basis, at
 * N_ij = min(h_N[i], h_N[j]), from d_coeffs as mm_coeffs writes them at
 * N_coeffs ([D][N_coeffs + 1], the plan's precision); R_ij = Sigma_ij /
 * sqrt(Sigma_ii Sigma_jj), R_ii = 1. Such a matrix need not be positive
 * semi-definite; psd_repair = 1 replaces Sigma (before R is formed) by the
 * positive semi-definite matrix closest to it in the Frobenius norm,
 * V max(Lambda, 0) V^T from its eigendecomposition (a cyclic Jacobi
 * iteration, in float64 for FP64 plans and float32 for the mixed precisions:
 * in one CTA while the matrix and its eigenvectors fit its shared memory,
 * else over every SM under a cooperative launch; D <= 4000, else
 * MM_ERR_UNSUPPORTED), leaving it unchanged when
 * no eigenvalue is negative; *d_clipped_or_null (device int) receives the
 * number of negative eigenvalues clipped (0 without repair).
 * h_N: host array of D cutoffs, each in [0, N_coeffs] ([1, N_coeffs] for
 * Fejer), else MM_ERR_CUTOFF; read before the call returns. Outputs D x D
 * row-major float32 (mixed plans) or float64 (FP64 plans), caller owned; a
 * non-positive variance gives NaN entries and MM_ERR_ZERO_VARIANCE at the
 * next mm_plan_sync. Asynchronous on stream; not available on batch plans. */
mm_status mm_corr_pairwise(mm_plan plan, const void* d_coeffs, int32_t N_coeffs, const int32_t* h_N,
                           int32_t psd_repair, void* d_sigma_or_null, void* d_R, int32_t* d_clipped_or_null,
                           void* stream);

/* mm_corr without a plan and without allocating anything, for callers that
 * cannot call cudaMalloc (their device memory is owned by a pool or an
 * allocator they must not bypass, or an allocation may not fail at that
 * point). The paper has no counterpart; this is a deployment convenience.
 * It runs the same contraction as mm_corr on coefficients laid out as
 * mm_coeffs writes them (D x (N+1), complex128 for MM_PREC_FP64, complex64
 * otherwise) and writes Sigma (optional) and R as mm_corr does. Its scratch
 * (weights, split-K partial tiles, a status word) is one file-scope device
 * array of about 2 MB that every GPU loading the library keeps until the
 * process exits. Limits: 1 <= D <= 128 and 0 <= N <= 65535; larger sizes
 * return MM_ERR_UNSUPPORTED. The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture. All calls share the array, and the array keeps the
 * last call's contents, so calls that overlap on the GPU race: order them
 * (one stream, or explicit synchronisation). The call synchronises the
 * stream and returns the contraction's device status (MM_OK,
 * MM_ERR_ZERO_VARIANCE or MM_ERR_TIMEOUT); on a stream that is being
 * captured into a graph it launches nothing and returns MM_ERR_INVALID_ARG. */
mm_status mm_corr_noalloc(int32_t D, int32_t N, mm_basis basis, mm_precision prec, const void* d_coeffs,
                          void* d_sigma_or_null, void* d_R, void* stream);

/* Whole Algorithm 3 on device buffers: mm_coeffs followed by mm_corr.
 * d_coeffs receives the coefficients (it is also the contraction's input). */
mm_status mm_estimate(mm_plan plan, const int64_t* d_offsets, const double* d_t,
                      const double* d_logp, int32_t N, double t0, double t1, void* d_coeffs,
                      void* d_sigma_or_null, void* d_R, int32_t* N_used, void* stream);

/* Whole Algorithm 3 from host buffers: copies h_offsets (D+1) to the plan's
 * device staging buffer; h_t and h_logp (h_offsets[D] each, <= max_events)
 * are read by the kernels in place when both are pinned, mapped host memory
 * (cudaHostAlloc / cudaMallocHost, or cudaHostRegister) and are copied to
 * staging buffers otherwise; runs mm_estimate; Sigma and R are written in
 * place when their buffers are pinned and mapped, else copied back (the
 * coefficients, when h_coeffs is not NULL, are always copied back); and
 * synchronises the stream before returning. The host buffers must not
 * change (inputs) or be read (outputs) until the call returns.
 * Returns the device status word as mm_plan_sync would. */
mm_status mm_estimate_host(mm_plan plan, const int64_t* h_offsets, const double* h_t,
                           const double* h_logp, int32_t N, double t0, double t1,
                           void* h_coeffs_or_null, void* h_sigma_or_null, void* h_R,
                           int32_t* N_used, void* stream);

/* Autotuner: times mm_coeffs on the caller's data for every candidate
 * configuration of stages (a)-(c) (spreading variant scatter / gather /
 * fused, cells per spreading block, FFT column and row blocking), reps calls
 * each after one warm-up call, and keeps the fastest in the plan for all
 * later calls (mm_plan_get_info reports it). d_coeffs is scratch of
 * D * (N+1) complex elements. Synchronises the stream; allocates nothing. */
mm_status mm_autotune(mm_plan plan, const int64_t* d_offsets, const double* d_t, const double* d_logp,
                      int32_t N, double t0, double t1, void* d_coeffs, int32_t reps, void* stream);

/* Nyquist cutoff of Algorithm 2 on device data (synchronises the stream).
 * Window as for mm_coeffs. Returns MM_ERR_CUTOFF when no asset has two
 * events, MM_ERR_DUPLICATE_TIME when some gap is zero. */
mm_status mm_nyquist(mm_plan plan, const int64_t* d_offsets, const double* d_t, double t0,
                     double t1, int32_t* N_out, void* stream);

/* Wait for the plan's work on its last stream and return (and clear) the
 * first device-side status recorded since the last call (MM_OK if none). */
mm_status mm_plan_sync(mm_plan plan);

/* Plan facts for inspection and tests. */
mm_status mm_plan_get_info(mm_plan plan, mm_plan_info* info);

/* Stage timing: enable (1) / disable (0) CUDA-event timing of every stage;
 * read the summed milliseconds and launch counts per stage (MM_NUM_STAGES
 * entries each, either pointer may be NULL); reset clears them. Reading
 * synchronises the events it reads. */
mm_status mm_profile_enable(mm_plan plan, int32_t on);
mm_status mm_profile_read(mm_plan plan, double* ms, int64_t* launches, int32_t reset);

/* CUDA graph replay of mm_estimate (and of the compute of mm_estimate_host),
 * on (1, the default) or off (0). A call is steady when the plan's tables,
 * contraction weights and configuration are already built for its N > 0 and
 * stage timing is off; the first steady call with a given set of device
 * pointers, N, window and configuration captures its launches (one graph for
 * each of the two FP32 accumulators the contraction alternates between) and
 * later ones replay them with one launch. The results are those of the eager
 * launches; the graph reads the inputs' current contents. Other calls, and
 * every call with graphs off, launch eagerly. */
mm_status mm_plan_set_graphs(mm_plan plan, int32_t on);

/* Limit, in nanoseconds, of the tensor-core contraction's device-side waits
 * on its own MMA completions (mm_cov, mm_corr, mm_estimate on the mixed
 * precisions); ns = 0 makes each wait a single non-blocking test, ns < 0
 * restores the default of one second. A diagnostic of the bounded-wait path
 * (failure detection without a GPU fault): a limit shorter than the MMAs
 * take (0 always is) makes the contraction give up, leave the
 * accumulator unwritten, let the MMAs it issued finish, free its tensor
 * memory and record MM_ERR_TIMEOUT, which the next mm_plan_sync (or the
 * synchronous call) returns; Sigma and R of that call are then undefined.
 * Later calls with the default limit are unaffected. Graphs captured with
 * the old limit are re-captured. Not part of the paper's method. */
mm_status mm_plan_set_wait_limit(mm_plan plan, int64_t ns);

/* Static text for a status code. */
const char* mm_status_string(mm_status s);

/* Library version as major*10000 + minor*100 + patch. */
int32_t mm_version(void);

/* ------------------------------------------------------------------------
 * Batched form: many independent problems of one shape (Monte Carlo
 * replications of D assets), each with its own events and its own rescaling
 * (Algorithm 4 per problem), and for each problem the covariance and
 * correlation at every cutoff of an ascending list N_1 < ... < N_J (an
 * Epps-effect sweep, Sec. 3.3), all from one set of coefficients at N_J:
 * the sweep is a prefix-weighted contraction (segment sums of the per-mode
 * products over (N_{j-1}, N_j], then prefix sums and the weights of
 * Eq. (2) or (3) per cutoff), not J separate contractions.
 *
 * Events are CSR over all reps * D assets in problem-major order (asset i
 * of problem r is entry r * D + i). Outputs are float32, layout
 * [reps][J][D][D], row-major per matrix. The first call with a given set of
 * inputs runs eagerly and captures the whole launch sequence (stages (a)-(c)
 * for every problem and the sweep) into a CUDA graph; later calls with the
 * same pointers and cutoffs replay it with a single graph launch.
 * ------------------------------------------------------------------------ */
typedef struct {
  int32_t reps;          /* problems in the batch, >= 1 */
  int32_t D;             /* assets per problem, 1 .. 12 */
  int32_t N_max;         /* largest cutoff of any sweep, >= 1 */
  int32_t reserved0;     /* must be zero */
  int64_t max_events;    /* upper bound on the batch's total event count */
  double tol;            /* NUFFT tolerance (Sec. 2.2.5) */
  mm_kernel kernel;
  mm_basis basis;
  mm_precision prec;     /* MM_PREC_MIXED_*: stages (a)-(c) in float32; the sweep
                            contraction accumulates in float32 on the CUDA cores
                            (D <= 12 makes it memory-bound), normalised in float64.
                            MM_PREC_FP64: the same form in float64 throughout
                            (complex128 coefficients, float64 Sigma and R): the
                            mixed form's comparator */
  int32_t spread_algo;   /* stages (a)-(c) as mm_plan_desc.spread_algo (0 .. 3) */
  int32_t reserved[4];   /* must be zero */
} mm_batch_desc;

typedef struct mm_batch_s* mm_batch;

typedef struct {
  int64_t graph_launches;  /* calls served by one CUDA graph launch */
  int64_t launches;        /* kernels launched by the batch (graph replays included) */
  int64_t Mr;              /* oversampled grid size of the last call */
  int32_t graph_captures;  /* graphs captured so far */
  int32_t graph_kernels;   /* kernels in the captured graph */
  int32_t spread_tile;
  int32_t fft_algo;
  int32_t fft_split;
  int32_t fft_passes;
  float tuned_ms;
} mm_batch_info;

/* Create a batch: validates desc and allocates the workspace of reps * D
 * assets (grids, coefficients at N_max, tables) on the current device.
 * MM_ERR_UNSUPPORTED for D > 12. */
mm_status mm_batch_create(const mm_batch_desc* desc, mm_batch* out);
mm_status mm_batch_destroy(mm_batch batch);

/* Sweep: h_cutoffs (host, n_cutoffs <= 128, strictly increasing, each in
 * [0 or 1 (Fejer), N_max]); d_R and d_sigma_or_null receive
 * reps * n_cutoffs * D * D floats (doubles for MM_PREC_FP64). Asynchronous on stream (a change of
 * cutoffs synchronises it once); device-side errors are reported by
 * mm_batch_sync. */
mm_status mm_batch_epps(mm_batch batch, const int64_t* d_offsets, const double* d_t, const double* d_logp,
                        const int32_t* h_cutoffs, int32_t n_cutoffs, void* d_sigma_or_null, void* d_R,
                        void* stream);

/* mm_autotune for stages (a)-(c) on this batch's data at cutoff N; later
 * sweeps re-capture their graph with the chosen configuration. */
mm_status mm_batch_autotune(mm_batch batch, const int64_t* d_offsets, const double* d_t, const double* d_logp,
                            int32_t N, int32_t reps, void* stream);

/* Device pointer to the coefficients of the last sweep (complex64, or
 * complex128 for MM_PREC_FP64; [reps * D][*ld], F-convention, k = 0..N_J)
 * and their row stride. Valid until the next call; owned by the batch. */
mm_status mm_batch_coeffs(mm_batch batch, const void** d_coeffs, int32_t* ld);

/* Copy those coefficients (reps * D * ld complex64 or complex128) into d_dst on stream. */
mm_status mm_batch_copy_coeffs(mm_batch batch, void* d_dst, void* stream);

/* Per-stage timing of the batch's launches, as mm_profile_enable /
 * mm_profile_read (the sweep is counted as the contraction stage). While
 * profiling is on, mm_batch_epps launches eagerly instead of replaying its
 * graph, so that every stage can be timed. */
mm_status mm_batch_profile_enable(mm_batch batch, int32_t on);
mm_status mm_batch_profile_read(mm_batch batch, double* ms, int64_t* launches, int32_t reset);

/* Synchronise the last call's stream and return its device status as
 * mm_plan_sync does. */
mm_status mm_batch_sync(mm_batch batch);
mm_status mm_batch_get_info(mm_batch batch, mm_batch_info* info);

/* ------------------------------------------------------------------------
 * Serving form: a request loop over one day's events kept resident on the
 * device (per-asset sorted CSR, loaded once). A request asks for Sigma and
 * R (Algorithm 3) of an asset subset over a window [t0, t1] at a cutoff N:
 * given, from Eq. (19) for a sampling interval dt_equiv, or (N = 0 and
 * dt_equiv = 0) the window's Nyquist cutoff (Algorithm 2, capped at N_max).
 * Times are rescaled with the window (Algorithm 4 over [t0, t1]), so an
 * asset's coefficients do not depend on the other requested assets.
 *
 * Continuous batching: a native scheduler thread admits queued requests into
 * execution slots as slots free up; each slot runs on its own CUDA stream, so
 * requests in flight overlap on the GPU. The slot count is the number of
 * slots (each sized for the largest admissible request: D assets,
 * request_max_events events in the window, N_max) that fit in hbm_budget,
 * at least one and at most max_slots. Results are written to the caller's
 * host buffers; completions are polled, out of order, with host timestamps.
 *
 * Resident coefficients (cache_rows > 0): the coefficients of each requested
 * asset over the request's window at its cutoff stay on the device (rows of
 * N_max + 1, least recently used evicted first), and a later request with
 * the same window and cutoff computes only its other assets. Requests whose
 * cutoff is the window's Nyquist cutoff (known only on the device) are not
 * cached; neither are rows of a request that failed. mm_server_load empties
 * the cache.
 * ------------------------------------------------------------------------ */
typedef struct {
  int32_t D;                   /* assets in the resident store, 1 .. 4096 */
  int32_t N_max;               /* largest cutoff served */
  int64_t max_events;          /* events in the resident store (upper bound) */
  int64_t request_max_events;  /* events a request's window may hold (0 = max_events) */
  int64_t hbm_budget;          /* bytes for the slots' workspace (0 = max_slots slots) */
  int32_t max_slots;           /* 1 .. 64 */
  int32_t cache_rows;          /* >= 0: coefficient rows kept resident across requests, each
                                  N_max + 1 coefficients of one (asset, window, cutoff); 0 = none */
  double tol;
  mm_kernel kernel;
  mm_basis basis;
  mm_precision prec;
  int32_t reserved[4];         /* must be zero */
} mm_server_desc;

typedef struct {
  double t0, t1;               /* window, t0 < t1, in the store's time unit */
  int32_t n_assets;            /* 1 .. D */
  int32_t N;                   /* > 0: cutoff; 0: from dt_equiv, or Nyquist when dt_equiv = 0 */
  const int32_t* assets;       /* host, n_assets distinct asset ids (copied at submit) */
  double dt_equiv;             /* > 0 with N = 0: N = floor((T/dt - 1)/2), T = t1 - t0 (Eq. (19)) */
  void* h_R;                   /* host, n_assets^2 elements (float32, float64 for FP64) */
  void* h_sigma_or_null;       /* host, same layout, or NULL */
} mm_request;

typedef struct {
  int64_t ticket;
  int32_t status;              /* mm_status of the request */
  int32_t n_assets;
  int32_t N;                   /* cutoff used */
  int32_t reserved;
  double t_submit, t_start, t_done;  /* seconds on the server's clock */
} mm_completion;

typedef struct {
  int64_t submitted, completed;
  int64_t slot_bytes;          /* device workspace per slot */
  int64_t resident_bytes;      /* the resident event store */
  int32_t slots, inflight, peak_inflight, queued;
  int64_t launches;            /* kernels launched for requests since creation (the window
                                  gather and the slot plans' own, graph replays included) */
  int64_t cache_hits;          /* requested assets served from resident coefficient rows */
  int64_t cache_misses;        /* requested assets whose coefficients were computed (cached requests) */
} mm_server_stats;

typedef struct mm_server_s* mm_server;

mm_status mm_server_create(const mm_server_desc* desc, mm_server* out);
/* Upload the store: h_offsets[D+1], h_t and h_logp (h_offsets[D] each),
 * strictly increasing times per asset (checked on the host). Only while no
 * request is queued or in flight. */
mm_status mm_server_load(mm_server server, const int64_t* h_offsets, const double* h_t, const double* h_logp);
/* Queue a request; returns at once with its ticket. */
mm_status mm_server_submit(mm_server server, const mm_request* request, int64_t* ticket);
/* Up to max completions (waiting up to wait_s seconds for the first). The
 * request's h_R / h_sigma hold its result once its completion is returned. */
mm_status mm_server_poll(mm_server server, mm_completion* out, int32_t max, int32_t* n_out, double wait_s);
mm_status mm_server_get_stats(mm_server server, mm_server_stats* stats);
/* Finish queued and in-flight requests, stop the scheduler, free everything. */
mm_status mm_server_destroy(mm_server server);

#ifdef __cplusplus
}
#endif

#endif /* MM_GB300_H */
