// mm_common.cuh -- shared device types, parameters and launch declarations of
// the GB300 Malliavin-Mancino NUFFT library (internal; not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mm.h"

namespace mmgpu {

// Device status bits, OR-ed by kernels into the plan's status word; the host
// maps the lowest set bit to an mm_status.
enum : int {
  ST_BAD_OFFSETS = 1 << 0,
  ST_UNSORTED = 1 << 1,
  ST_DUPLICATE = 1 << 2,
  ST_SPAN = 1 << 3,
  ST_NONFINITE = 1 << 4,
  ST_TIMEOUT = 1 << 5,
  ST_ZERO_VAR = 1 << 6,
  ST_CUTOFF = 1 << 7,
  ST_OUT_OF_WINDOW = 1 << 8,
};

// Device-side waits give up after this long (unless a plan sets its own
// limit for the contraction) and report ST_TIMEOUT.
constexpr uint64_t kDefaultWaitNs = 1000000000ull;  // 1 s

template <typename T>
struct __align__(2 * sizeof(T)) Cplx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ Cplx<T> cmul(Cplx<T> a, Cplx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ Cplx<T> cadd(Cplx<T> a, Cplx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
__device__ __forceinline__ Cplx<T> csub(Cplx<T> a, Cplx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T>
__device__ __forceinline__ Cplx<T> cconj(Cplx<T> a) { return {a.x, -a.y}; }
// multiply by -i
template <typename T>
__device__ __forceinline__ Cplx<T> cmul_mi(Cplx<T> a) { return {a.y, -a.x}; }

constexpr int kMaxRadices = 12;
constexpr int kMaxFftLen = 1024;   // largest P or Q of the two-pass FFT
constexpr double kPi = 3.14159265358979323846264338327950288;

// Spreading parameters (Sec. 2.2.5 and Algorithms 8-10), all derived on the
// host from (kernel, tol, N, M_r).
struct SpreadParams {
  int D;
  int64_t Mr;        // grid size
  int tile;          // cells per block
  int ntiles;        // blocks per asset
  int msp;           // M_sp
  int klo, khi;      // stencil offsets k in [klo, khi] around b0
  int kernel;        // mm_kernel
  int single_tile;   // 1: one block covers the whole (small) grid
  int algo;          // 0: scatter into a shared-memory tile, 1: gather per cell
  int fused;         // 1: stages (a)-(c) in one CTA per asset (grid in shared memory)
  // grid layout for the per-asset FFT: with perm_np > 0 the complex point m
  // of an asset's grid row (cells 2m, 2m+1) is stored at its mixed-radix
  // digit reversal sum_p q_p perm_stride[p], m = q_0 + rad_0 (q_1 + ...)
  int perm_np;
  int perm_rad[4];
  int perm_stride[4];
  unsigned perm_magic[4];  // exact-division multipliers of perm_rad
  // kernel constants
  double es_beta;    // ES: beta
  double es_inv_w;   // ES: 1 / M_sp  (support half-width in cells)
  double g_t1;       // Gaussian: t1 of Algorithm 8 (exponent per cell^2)
  double kb_b;       // KB: b = pi (2 - 1/sigma)
  double kb_inv_phi0;// KB: 1 / phi(0) (kernel normalised to peak 1)
  int64_t max_events;
  // spreading tiles are dispatched asset by asset in this order (the assets
  // ranked by event count, heaviest first, written by k_bounds), or in index
  // order when null
  const int* order;
};

constexpr int kOrderMaxAssets = 256;  // k_bounds ranks the assets of a single problem up to this D

// Averaging kernel of the float32 path as one polynomial per stencil tap:
// phi(k - d) ~ sum_i c[j][i] (d - 1/2)^i for tap k = klo + j and d in [0, 1),
// fitted on the host (Chebyshev interpolation, float64) for the plan's
// kernel, M_sp and sigma; evaluated by Horner's rule on the FMA pipe.
constexpr int kPolyDeg = 8;
constexpr int kPolyMaxTaps = 32;
struct KernelPoly {
  float c[kPolyMaxTaps][kPolyDeg + 1];
};

// Rescaling of Algorithm 4 in exact fixed point, written by k_bounds for the
// current call: t_fix = trunc(t * 2^F) (int64, |t| < 2^(62-F)); the cell
// coordinate u = (t - t0) M_r / span is u_fix = ((t_fix - t0_fix) * S) >> sh
// = floor(u * 2^40), so b0 = u_fix >> 40 and d = (u_fix mod 2^40) / 2^40.
struct Rescale {
  double t0, t1;             // window used (data minimum / maximum or caller's)
  long long t0_fix;          // t0 in units of 2^-F
  unsigned long long S;      // cell scale of grid scale_Mr: 64-bit multiplier, in [2^63, 2^64)
  int F;                     // fractional bits of the time fixed point
  int sh;                    // right shift of the 128-bit product, 0..127
  float s_hi, s_lo;          // the float-pair cell scale of the same grid
  long long scale_Mr;        // grid size the cell scales belong to (0: not computed)
};
constexpr int kUFrac = 40;   // fractional bits of u_fix

struct FftParams {
  int64_t n;         // complex length = Mr / 2
  int P, Q;          // n = P * Q
  int nrad_p, nrad_q;
  int rad_p[kMaxRadices], rad_q[kMaxRadices];
  int lg_cols;       // pass 1: log2 of the columns (j2 values) per block
  int rowblk;        // pass 2: lower rows per block
  int lg_rowcols;    // pass 2: log2 of the rows held per block (>= 2 rowblk, padded)
  int H;             // pass 2: number of lower rows = P/2 + 1
  int N;             // cutoff
};

// Per-asset shared-memory FFT (mm_fft_asset.cu): an asset's n-point complex
// transform is split over `split` CTAs (1 or 2), each transforming nl =
// n / split points as nl = rad[0] * ... * rad[npass-1]; pass p works on
// blocks of length rad[p] * stride[p]; its twiddle anchor rows (w^1..w^4 of
// w = w_{L_p}^j, one row per j < stride[p]) start at row tw_off[p].
constexpr int kMaxAssetPasses = 4;
struct AssetFft {
  int n;
  int nl;
  int split;    // CTAs per asset: 1, or 2 as a cluster (pair)
  int pair;     // split 2: a cluster of two CTAs (decimation in time by 2)
  int pre_perm; // split 1: the spread kernel stored the grid in digit-reversed order
  int dif;      // decimation in frequency (natural-order input); else in time
  int N;
  int npass;
  int tw_rows;  // anchor rows over all passes
  int rev_lo;   // decimation in frequency: rev(k) = T_lo[k mod rev_lo] + T_hi[k / rev_lo]
  int rev_hi;   // (tables of rev_lo and rev_hi ints after the anchors; rev_lo * rev_hi = nl)
  int rad[kMaxAssetPasses];
  int stride[kMaxAssetPasses];
  int tw_off[kMaxAssetPasses];
};

struct GramParams {
  int D;
  int N;             // modes k = 0..N
  int ld;            // leading dimension (complex elements) of the coefficients
  int tile;          // output tile edge (128 tensor path, 64 fp64 path)
  int ntiles;        // ceil(D / tile)
  int npairs;        // ntiles (ntiles+1) / 2
  int splits;        // split-K factor
  int chunk;         // complex modes per K-chunk
  int nchunks;       // ceil((N+1) / chunk)
  int chunks_per_split;
  int Dp;            // row stride of the FP32 accumulator (D rounded up to 4)
  unsigned long long wait_ns;  // limit of the tensor-core kernel's progress waits
};

struct GroupScale;  // per-problem fixed-point scales (mm_spread_dev.cuh)

// Batched cutoff sweep (mm_epps.cu).
constexpr int kMaxCutoffs = 128;
constexpr int kMaxEppsAssets = 12;

// ---------------------------------------------------------------- launchers
// Each returns cudaGetLastError() of its launch.
// Mr > 0: also the cell scales of grid Mr (so later kernels do no float64
// arithmetic for them); 0 when the grid is not known yet.
// order != NULL (a single problem of D <= kOrderMaxAssets): also ranks the
// assets by event count, heaviest first, into order[0..D-1].
cudaError_t launch_bounds(const int64_t* off, const double* t, int D, int gsize, int64_t max_events,
                          double w0, double w1, int64_t Mr, Rescale* rs, int* status, int* order, cudaStream_t s);
cudaError_t launch_group_scales(const Rescale* rs, int G, int64_t Mr, GroupScale* out, const int* status,
                                cudaStream_t s);
size_t group_scale_bytes();
cudaError_t launch_min_gap(const int64_t* off, const double* t, int D, const Rescale* rs,
                           unsigned long long* gapbits, int* nyq, int* status, cudaStream_t s);
cudaError_t launch_prep_f32(const int64_t* off, const double* t, const double* logp, const Rescale* rs,
                            const GroupScale* gsc, int gsize, int D, int64_t Mr, int64_t max_events, int* rb0,
                            void* rd, void* rv, int* status, cudaStream_t s);
cudaError_t launch_prep_f64(const int64_t* off, const double* t, const double* logp, const Rescale* rs,
                            const GroupScale* gsc, int gsize, int D, int64_t Mr, int64_t max_events, int* rb0,
                            void* rd, void* rv, int* status, cudaStream_t s);
cudaError_t launch_spread_f32(const int64_t* off, const int* rb0, const void* rd, const void* rv,
                              const SpreadParams& p, float* grid, const int* status, cudaStream_t s);
// float32 scatter with the polynomial taps and int32 fixed-point shared
// accumulation (per-tile power-of-two scale); false if the tap count has no
// instantiation
bool spread_poly_supported(int ntaps);
cudaError_t launch_spread_poly(const int64_t* off, const int* rb0, const void* rd, const void* rv,
                               const SpreadParams& p, const KernelPoly& poly, float* grid, const int* status,
                               cudaStream_t s);
cudaError_t launch_spread_f64(const int64_t* off, const int* rb0, const void* rd, const void* rv,
                              const SpreadParams& p, double* grid, const int* status, cudaStream_t s);

cudaError_t launch_gl_nodes(int nq, double* x, double* w, cudaStream_t s);
cudaError_t launch_setup_tables(int kernel, int msp, int64_t Mr, int N, int64_t n,
                                const SpreadParams& sp, double tau, const double* glx,
                                const double* glw, int nq, void* W, void* U, void* decon,
                                bool fp64, cudaStream_t s);
cudaError_t launch_fft_cols_f32(float* grid, const FftParams& f, int D, const void* W, const int* status, cudaStream_t s);
cudaError_t launch_fft_cols_f64(double* grid, const FftParams& f, int D, const void* W, const int* status, cudaStream_t s);
cudaError_t launch_fft_rows_f32(const float* grid, const FftParams& f, int D, const void* W,
                                const void* U, const void* decon, void* coeffs, const int* status, cudaStream_t s);
cudaError_t launch_fft_rows_f64(const double* grid, const FftParams& f, int D, const void* W,
                                const void* U, const void* decon, void* coeffs, const int* status, cudaStream_t s);
int spread_max_tile(bool fp64);
size_t fused_smem(const FftParams& f, int64_t Mr, bool fp64);
cudaError_t launch_coeff_fused(bool fp64, const int64_t* off, const double* t, const double* logp, const Rescale* rs,
                               const SpreadParams& sp, const FftParams& f, const void* W, const void* U,
                               const void* decon, void* coeffs, int* status, cudaStream_t s);
size_t fft_cols_smem(const FftParams& f, bool fp64);
bool asset_fft_radix_ok(int R);
size_t asset_fft_smem(const AssetFft& f);
cudaError_t launch_asset_twiddles(const AssetFft& f, void* tw, cudaStream_t s);
cudaError_t launch_fft_asset(const float* grid, const AssetFft& f, int D, const void* W, const void* tw,
                             const void* U, const void* decon, void* coeffs, int* status, cudaStream_t s);
// Stages (a2)-(c) in one launch with the grid row resident in shared
// memory (one CTA per asset, or the cluster pair for f.pair): records in,
// coefficients out. sub = cells per sub-range from spread_fft_sub (0: the
// row does not fit with the staging area within smem_limit).
constexpr int kResStaticSmem = 4096;  // static shared memory of those kernels, rounded up
int spread_fft_sub(const AssetFft& f, int64_t Mr, size_t smem_limit);
size_t spread_fft_smem(const AssetFft& f, int sub);
cudaError_t launch_spread_fft(const int64_t* off, const int* rb0, const void* rd, const void* rv,
                              const SpreadParams& sp, const KernelPoly& poly, int sub, const AssetFft& f, int D,
                              const void* W, const void* tw, const void* U, const void* decon, void* coeffs,
                              const int* status, cudaStream_t s);
size_t fft_rows_smem(const FftParams& f, bool fp64);

cudaError_t launch_gram_weights(int basis, int N, bool fp64, void* wsq, cudaStream_t s);
cudaError_t launch_gram_f64(const void* coeffs, const GramParams& g, const double* wsq,
                            double* partial, cudaStream_t s);
cudaError_t launch_gram_tc(int mode, const void* coeffs, const GramParams& g, const float* wsq,
                           float* acc, int* status, int* done, float* sigma, float* R, float* zero_next,
                           cudaStream_t s);  // done != NULL: the last CTA writes Sigma and R (D <= 256)
cudaError_t launch_corr_acc(const float* acc, const GramParams& g, float* sigma, float* R, float* zero_next,
                            int* status, cudaStream_t s);
cudaError_t launch_reduce_corr(bool fp64, const void* partial, const GramParams& g,
                               void* sigma, void* R, int* status, cudaStream_t s);
size_t gram_tc_smem(int mode, bool two_tiles);
// Pre-split contraction (mm_gram_tma.cu): the operand's hi and lo planes
// (gram_tma_plane_bytes each, for D assets up to N_max), the split pass, and
// the TMA-fed contraction into the FP32 accumulator.
size_t gram_tma_plane_bytes(int mode, int D, int N_max, int chunk);
cudaError_t launch_gram_split(int mode, const void* coeffs, const GramParams& g, const float* wsq, void* hi,
                              void* lo, cudaStream_t s);
cudaError_t launch_gram_tma(int mode, const GramParams& g, void* hi, void* lo, float* acc, int* status,
                            cudaStream_t s);
int epps_max_assets();

// Plan internals used by the serving engine (mm_server.cu).
mm_status plan_create_no_staging(const mm_plan_desc* desc, mm_plan* out);  // no host-buffer entry staging
mm_status plan_set_active_assets(mm_plan p, int D);
int* plan_status_word(mm_plan p);
mm_status plan_flags_to_status(int flags);
cudaError_t launch_epps(int Dg, bool fejer, bool fp64, const void* coef, int ld, const int* cut, int ncut, int G,
                        void* sigma, void* R, int* status, int grid, cudaStream_t s);

// Pairwise-cutoff covariance (float64 D x D into sig) and its repair to the
// nearest positive semi-definite matrix (D <= pairwise_psd_max_assets(): one CTA while the
// matrix and eigenvectors fit its shared memory, else every SM under a cooperative launch).
int pairwise_psd_max_assets();
cudaError_t launch_pairwise(bool fp64, bool fejer, const void* coeffs, int ld, const int* Nv, int D,
                            double* sig, cudaStream_t s);
cudaError_t launch_psd_repair(bool fp64, double* sig, double* A, double* V, int D, int* clipped, void* sync,
                              int* status, cudaStream_t s);
size_t psd_sync_bytes();  // the multi-CTA repair's barrier and reduction words
cudaError_t launch_pairwise_out(bool fp64, const double* sig, int D, void* sigma, void* R, int* status,
                                cudaStream_t s);

// ------------------------------------------------- programmatic launches
// The hot path's kernels are launched with programmatic stream
// serialization: a kernel may be scheduled before its predecessor in the
// stream has finished, runs only set-up that touches neither global memory
// written by earlier kernels nor memory they read, then waits at pdl_wait()
// until the predecessor has completed and its writes are visible (a no-op
// when launched normally). pdl_trigger() lets the successor be scheduled.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace mmgpu
