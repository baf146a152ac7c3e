// mm_api.cu -- the C ABI of include/mm.h: plans, per-cutoff configuration and
// the stream-ordered launch sequence of the hot path
//   bounds (Algorithm 4) -> spread (Eq. (12)) -> FFT pass 1 -> FFT pass 2 with
//   unpack + deconvolution (Eqs. (13)-(14)) -> split-K Gram (Algorithm 3
//   step C) -> FP64 reduce + correlation (Algorithm 3, last step).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <vector>

#include "mm_common.cuh"

using namespace mmgpu;

namespace {

constexpr int kSMs = 152;           // GB300: 2 dies x 76 SMs
constexpr int kGlNodes = 128;       // Gauss-Legendre nodes for the ES transform
constexpr int kMaxGramCtas = 2 * kSMs;
constexpr int kGramTmaMinAssets = 192;  // default switch to the pre-split contraction

struct Prof {
  int stage;
  cudaEvent_t a, b;
};

bool smooth235(int64_t x) {
  for (int p : {2, 3, 5})
    while (x % p == 0) x /= p;
  return x == 1;
}

// Radix plan of an L-point FFT (L 5-smooth): radix 8 first, then 4, 2, 5, 3.
int radix_plan(int L, int* rad) {
  int n = 0;
  while (L % 8 == 0) { rad[n++] = 8; L /= 8; }
  while (L % 4 == 0) { rad[n++] = 4; L /= 4; }
  while (L % 2 == 0) { rad[n++] = 2; L /= 2; }
  while (L % 5 == 0) { rad[n++] = 5; L /= 5; }
  while (L % 3 == 0) { rad[n++] = 3; L /= 3; }
  return n;
}

// Smallest even 5-smooth n >= nmin that splits as P * Q with P, Q <= kMaxFftLen;
// P is the divisor closest to sqrt(n). Returns false when none exists.
bool choose_fft(int64_t nmin, int64_t* n_out, int* P_out, int* Q_out) {
  const int64_t cap = (int64_t)kMaxFftLen * kMaxFftLen;
  for (int64_t n = std::max<int64_t>(nmin, 2); n <= cap; ++n) {
    if ((n & 1) || !smooth235(n)) continue;  // even n: rows of M_r = 2n floats stay 16-byte aligned
    int bestP = -1;
    double best = 1e300;
    for (int64_t P = 1; P <= kMaxFftLen && P <= n; ++P) {
      if (n % P) continue;
      int64_t Q = n / P;
      if (Q > kMaxFftLen) continue;
      double d = fabs(log((double)P) - log((double)Q));
      if (d < best) { best = d; bestP = (int)P; }
    }
    if (bestP > 0) {
      *n_out = n;
      *P_out = bestP;
      *Q_out = (int)(n / bestP);
      return true;
    }
  }
  return false;
}

// Plan of the per-asset FFT of n points split over `split` CTAs: the local
// length nl = n / split factored into the fewest radices from the compiled
// set up to maxr (largest smallest factor on ties). Entry p has stride
// nl / (R_0 ... R_p); the last entry (unit stride, butterflies contiguous in
// shared memory) gets an odd radix where one exists. Returns false when nl
// needs more than kMaxAssetPasses factors.
bool plan_asset_fft(int64_t n, int split, int N, int maxr, AssetFft* out) {
  static const int kRad[] = {32, 30, 27, 25, 24, 20, 18, 16, 15, 12, 10, 9, 8, 6, 5, 4, 3, 2};
  if (split < 1 || n % split) return false;
  const int64_t nl = n / split;
  std::vector<int> best, cur;
  std::function<void(int64_t, int)> rec = [&](int64_t rest, int maxr) {
    if (rest == 1) {
      auto key = [](const std::vector<int>& v) {
        return std::make_pair((int)v.size(), -*std::min_element(v.begin(), v.end()));
      };
      if (best.empty() || key(cur) < key(best)) best = cur;
      return;
    }
    if ((int)cur.size() >= kMaxAssetPasses) return;
    if (!best.empty() && (int)cur.size() + 1 > (int)best.size()) return;
    for (int r : kRad) {
      if (r > maxr || rest % r) continue;
      cur.push_back(r);
      rec(rest / r, r);
      cur.pop_back();
    }
  };
  if (nl < 2 || nl > (1 << 15)) return false;
  rec(nl, maxr);
  if (best.empty()) return false;
  // descending, so that the pass of largest stride (entry 0, which needs
  // stride rows of twiddle anchors) has the largest radix; the last entry is
  // the unit-stride pass, where an odd radix keeps the 8-byte shared-memory
  // accesses of a warp free of bank conflicts: the smallest odd radix goes
  // there
  std::sort(best.begin(), best.end(), [](int a, int b) { return a > b; });
  for (int q = (int)best.size() - 1; q >= 0; --q)
    if (best[q] & 1) {
      const int r = best[q];
      best.erase(best.begin() + q);
      best.push_back(r);
      break;
    }
  AssetFft f{};
  f.n = (int)n;
  f.nl = (int)nl;
  f.split = split;
  f.N = N;
  f.npass = (int)best.size();
  int64_t L = nl;
  int off = 0;
  for (int q = 0; q < f.npass; ++q) {
    f.rad[q] = best[q];
    f.stride[q] = (int)(L / best[q]);
    f.tw_off[q] = off;
    if (f.stride[q] > 1) off += f.stride[q];
    L /= best[q];
  }
  for (int q = f.npass; q < kMaxAssetPasses; ++q) {
    f.rad[q] = 1;
    f.stride[q] = 1;
    f.tw_off[q] = off;
  }
  f.tw_rows = off;
  // digit-reversal tables: the two largest radices' digits and the rest
  f.rev_lo = f.npass >= 2 ? f.rad[0] * f.rad[1] : f.rad[0];
  f.rev_hi = (int)(nl / f.rev_lo);
  f.dif = 1;  // decimation in frequency unless the caller's input order says otherwise
  *out = f;
  return true;
}

// Twiddle entries (complex) of an asset FFT plan: four anchors per row.
int64_t asset_twiddle_count(const AssetFft& f) { return 4 * (int64_t)f.tw_rows; }

// The averaging kernel at signed distance x (grid cells) as the device
// evaluates it (Eqs. (5), (7), (9) with the plan's constants), in float64.
double kernel_at(const SpreadParams& s, double x) {
  if (s.kernel == MM_KERNEL_GAUSS) return exp(-s.g_t1 * x * x);
  if (s.kernel == MM_KERNEL_ES) {
    const double y = x * s.es_inv_w, v = 1.0 - y * y;
    return v >= 0.0 ? exp(s.es_beta * (sqrt(v) - 1.0)) : 0.0;
  }
  const double b = s.kb_b, ck = s.kb_inv_phi0 / kPi;
  const double s2 = (double)s.msp * s.msp - x * x;
  if (s2 > 0.0) return sinh(b * sqrt(s2)) / sqrt(s2) * ck;
  if (s2 < 0.0) return sin(b * sqrt(-s2)) / sqrt(-s2) * ck;
  return b * ck;
}

// Per-tap polynomials of the float32 spreading kernel: Chebyshev
// interpolation of phi(k - d), d in [0, 1], at kPolyDeg + 1 nodes, rewritten
// in powers of z = d - 1/2 and rounded to float32. Returns the largest error
// of the float32 Horner evaluation over a fine sample of d.
double fit_kernel_poly(const SpreadParams& s, KernelPoly* out) {
  constexpr int n = kPolyDeg + 1;
  memset(out, 0, sizeof(*out));
  const int nt = s.khi - s.klo + 1;
  if (nt > kPolyMaxTaps) return 1e300;
  double tn[n], T[n][n];  // nodes; monomial coefficients of T_i in t
  for (int m = 0; m < n; ++m) tn[m] = cos(kPi * (m + 0.5) / n);
  memset(T, 0, sizeof(T));
  T[0][0] = 1.0;
  if (n > 1) T[1][1] = 1.0;
  for (int i = 2; i < n; ++i)
    for (int q = 0; q < n; ++q) T[i][q] = (q > 0 ? 2.0 * T[i - 1][q - 1] : 0.0) - T[i - 2][q];
  double worst = 0.0;
  for (int j = 0; j < nt; ++j) {
    const int k = s.klo + j;
    double y[n], a[n], mono[n];
    for (int m = 0; m < n; ++m) y[m] = kernel_at(s, (double)k - (0.5 * tn[m] + 0.5));
    for (int i = 0; i < n; ++i) {
      double acc = 0.0;
      for (int m = 0; m < n; ++m) acc += y[m] * cos(kPi * i * (m + 0.5) / n);
      a[i] = (i == 0 ? 1.0 : 2.0) * acc / n;
    }
    for (int q = 0; q < n; ++q) {
      mono[q] = 0.0;
      for (int i = 0; i < n; ++i) mono[q] += a[i] * T[i][q];
      out->c[j][q] = (float)(mono[q] * ldexp(1.0, q));  // t = 2z
    }
    for (int q = 0; q <= 128; ++q) {
      const double d = q / 128.0;
      const float z = (float)(d - 0.5);
      float acc = out->c[j][n - 1];
      for (int i = n - 2; i >= 0; --i) acc = fmaf(acc, z, out->c[j][i]);
      worst = std::max(worst, fabs((double)acc - kernel_at(s, (double)k - d)));
    }
  }
  return worst;
}

// M_sp rules of Sec. 2.2.5 (sigma = 2).
int msp_rule(mm_kernel k, double eps) {
  const double sigma = 2.0;
  if (k == MM_KERNEL_GAUSS) return (int)floor(-log(eps) * (sigma - 0.5) / (kPi * (sigma - 1.0)) + 0.5);
  const int digits = (int)ceil(log10(1.0 / eps) - 1e-9);
  const int m = (int)floor(0.5 * (double)(digits + 2));
  return k == MM_KERNEL_ES ? m + 2 : m;
}

mm_status flags_to_status(int f) {
  if (f & (ST_BAD_OFFSETS | ST_OUT_OF_WINDOW)) return MM_ERR_INVALID_ARG;
  if (f & ST_SPAN) return MM_ERR_DEGENERATE_SPAN;
  if (f & ST_UNSORTED) return MM_ERR_UNSORTED;
  if (f & ST_DUPLICATE) return MM_ERR_DUPLICATE_TIME;
  if (f & ST_NONFINITE) return MM_ERR_NONFINITE;
  if (f & ST_CUTOFF) return MM_ERR_CUTOFF;
  if (f & ST_TIMEOUT) return MM_ERR_TIMEOUT;
  if (f & ST_ZERO_VAR) return MM_ERR_ZERO_VARIANCE;
  return MM_OK;
}

}  // namespace

struct mm_plan_s {
  mm_plan_desc desc{};
  int dev = 0;
  int smem_optin = 0;  // largest dynamic shared memory per block on this device
  bool fp64 = false;
  size_t cs = 8;   // bytes per complex coefficient
  size_t rs = 4;   // bytes per real grid cell / output element
  int msp = 0, klo = 0, khi = 0;
  int64_t n_max = 0;
  int D = 0;                      // assets of the current call (<= desc.D; a server slot varies it)
  int cfg_D = -1;                 // D of the cached configuration
  int gsize = 0;                  // assets per problem (D for a single problem)
  int G = 1;                      // problems (a batch has G > 1)
  bool batch = false;             // created for a batch: no contraction or host-staging workspace
  // workspace
  void* grid = nullptr;
  int* rec_b0 = nullptr;          // per-event records of the prep kernel
  void* rec_d = nullptr;
  void* rec_v = nullptr;
  void* W = nullptr;
  void* atw = nullptr;            // per-asset FFT pass twiddles (mixed path)
  int64_t atw_cap = 0;            // entries allocated
  int atw_n = -1, atw_npass = -1;  // plan the twiddles were built for
  int atw_rad[kMaxAssetPasses] = {};
  void* U = nullptr;
  void* decon = nullptr;
  double* glx = nullptr;
  double* glw = nullptr;
  Rescale* bounds = nullptr;       // one per problem
  void* gscale = nullptr;          // per-problem cell scales (batched form)
  int* status = nullptr;  // [0] sticky flags, [1] gate, [2] Nyquist N
  unsigned long long* gapbits = nullptr;
  void* wsq = nullptr;
  void* partial = nullptr;        // FP64 path: per-split partial tiles
  size_t partial_bytes = 0;
  float* acc[2] = {nullptr, nullptr};  // mixed path: FP32 accumulators, used alternately
  void* tma_hi = nullptr;         // mixed path, pre-split contraction: operand hi and lo planes
  void* tma_lo = nullptr;         // (Dpad x kpc complex modes, pad rows zero)
  int gram_used = 0;              // contraction variant of the last call (mm_plan_info.gram_algo)
  int* gram_done = nullptr;       // contraction CTAs finished (the last one runs the epilogue)
  int* pw_N = nullptr;            // pairwise-cutoff covariance: per-asset cutoffs,
  double* pw_sig = nullptr;       // the float64 estimate,
  double* pw_A = nullptr;         // the repair's working matrix and eigenvectors
  double* pw_V = nullptr;         // (allocated on first use)
  int* pw_clip = nullptr;
  void* pw_sync = nullptr;        // the multi-CTA repair's barrier words
  int acc_sel = 0;
  bool acc_dirty = true;          // clear both before the next contraction
  int acc_D = -1;                 // D whose D x Dp region the last epilogue cleared
  int64_t* s_off = nullptr;
  double* s_t = nullptr;
  double* s_p = nullptr;
  void* s_coef = nullptr;
  void* s_sigma = nullptr;
  void* s_R = nullptr;
  int* h_status = nullptr;        // pinned: the host-buffer entry point's status read-back
  int* asset_order = nullptr;     // spreading dispatch order (single problems of D <= kOrderMaxAssets)
  int64_t workspace = 0;
  // per-cutoff configuration
  int cfg_N = -1;
  int tab_N = -1;
  // autotuned choices (-1 = library default); applied by configure()
  int tune_algo = -1;     // 0 scatter, 1 gather, 2 fused
  int tune_tile = -1;     // spreading cells per block
  int tune_lgcols = -1;   // FFT pass 1: log2 columns per block
  int tune_rowblk = -1;   // FFT pass 2: lower rows per block
  float tune_ms = 0.f;    // time of the chosen configuration
  int tune_fft = -1;      // 0 per-asset shared-memory FFT, 1 two-pass FFT
  int tune_split = -1;    // per-asset FFT: 1 one CTA per asset, 3 the cluster pair
  int tune_maxr = -1;     // per-asset FFT: largest radix (16 or 32)
  int tune_perm = -1;     // 1: the scatter stores the grid in the FFT's input order (split 1)
  int res_sub = 0;        // > 0: stages (a2)-(c) in one launch, grid row resident (cells per sub-range)
  int64_t Mr = 0;
  FftParams fft{};
  AssetFft afft{};
  bool use_afft = false;  // stages (b)-(c) by the per-asset FFT kernel
  SpreadParams sp{};
  double tau = 0;
  int w_N = -1, w_basis = -1;
  GramParams gram{};
  KernelPoly poly{};
  bool poly_ok = false;   // float32 spreading with polynomial taps and integer accumulation
  int tune_poly = -1;     // autotuner override: 0 off
  cudaStream_t last = nullptr;
  // replay of mm_estimate's launch sequence: one graph per accumulator in use
  // (the sequence differs only in which accumulator it fills and clears)
  struct EstGraph {
    cudaGraphExec_t exec = nullptr;
    const void* key[6] = {};  // inputs and outputs it was captured with
    int N = -1, D = -1, cfg = -1;
    double t0 = 0.0, t1 = 0.0;
    int kernels = 0;
  } eg[2];
  cudaStream_t cap = nullptr;  // capture stream
  int cfg_gen = 0;             // configuration generation (a graph holds one)
  uint64_t wait_ns = kDefaultWaitNs;  // limit of the contraction's device waits
  bool graphs = true;
  int64_t graph_launches = 0;
  // instrumentation
  bool prof = false;
  std::vector<Prof> pending;
  std::vector<cudaEvent_t> pool;  // reusable timing events
  double ms[MM_NUM_STAGES] = {};
  int64_t nl[MM_NUM_STAGES] = {};
  int64_t launches = 0;
};

namespace {

#define MM_CUDA(call)                                 \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return MM_ERR_CUDA;        \
  } while (0)

mm_status dalloc(mm_plan p, void** ptr, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return MM_ERR_OOM;
  }
  p->workspace += (int64_t)bytes;
  return MM_OK;
}

void free_all(mm_plan p) {
  void* ptrs[] = {p->grid, p->rec_b0, p->rec_d, p->rec_v, p->W, p->atw, p->U, p->decon, p->glx, p->glw, p->bounds, p->gscale, p->status, p->gapbits, p->wsq,
                  p->partial, p->acc[0], p->acc[1], p->gram_done, p->pw_N, p->pw_sig, p->pw_A,
                  p->pw_V, p->pw_clip, p->s_off, p->s_t, p->s_p, p->s_coef,
                  p->s_sigma, p->s_R, p->asset_order, p->tma_hi, p->tma_lo, p->pw_sync};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (p->h_status) cudaFreeHost(p->h_status);
  for (auto& e : p->eg)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  if (p->cap) cudaStreamDestroy(p->cap);
  for (auto& e : p->pending) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  p->pending.clear();
  for (cudaEvent_t e : p->pool) cudaEventDestroy(e);
  p->pool.clear();
}

cudaEvent_t take_event(mm_plan p) {
  if (!p->pool.empty()) {
    cudaEvent_t e = p->pool.back();
    p->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Stage timing helpers: when profiling is on, every launch is bracketed by a
// pair of events on the launching stream.
struct StageScope {
  mm_plan p;
  int stage;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  int count;
  StageScope(mm_plan p_, int stage_, cudaStream_t s_, int count_ = 1) : p(p_), stage(stage_), s(s_), count(count_) {
    if (p->prof) {
      a = take_event(p);
      b = take_event(p);
      cudaEventRecord(a, s);
    }
  }
  ~StageScope() {
    p->launches += count;
    p->nl[stage] += count;
    if (p->prof) {
      cudaEventRecord(b, s);
      p->pending.push_back({stage, a, b});
    }
  }
};

// Per-cutoff configuration: grid size, FFT factorisation, tiles and the
// kernel constants of Sec. 2.2.5 with sigma = M_r / M.
mm_status configure(mm_plan p, int N) {
  if (p->cfg_N == N && p->cfg_D == p->D) return MM_OK;
  const int64_t M = 2 * (int64_t)N + 1;
  int64_t n;
  int P, Q;
  if (!choose_fft(std::max<int64_t>(M, p->msp + 1), &n, &P, &Q)) return MM_ERR_UNSUPPORTED;
  if (n > p->n_max) return MM_ERR_CUTOFF;
  const int64_t Mr = 2 * n;
  const double sigma = (double)Mr / (double)M;
  FftParams f{};
  f.n = n;
  f.P = P;
  f.Q = Q;
  f.nrad_p = radix_plan(P, f.rad_p);
  f.nrad_q = radix_plan(Q, f.rad_q);
  const size_t cs = p->cs;
  const size_t budget = 48 * 1024;  // about four blocks per SM
  const int max_elems = 256 * 16;   // the FFT kernels batch at most 16 elements per thread
  int lg = 4;                       // pass 1: up to 16 adjacent columns (128 B per row in FP32)
  while (lg > 0 && (((size_t)2 * P * ((size_t)1 << lg) + P) * cs > budget || (P << lg) > max_elems)) --lg;
  while (lg > 0 && (1 << (lg - 1)) >= Q) --lg;
  f.lg_cols = lg;
  f.H = P / 2 + 1;
  f.rowblk = 8;
  auto rows_lg = [](int rb) { int l = 0; while ((1 << l) < 2 * rb) ++l; return l; };
  while (f.rowblk > 1 && (((size_t)2 * ((size_t)1 << rows_lg(f.rowblk)) * Q + Q) * cs > budget ||
                          ((1 << rows_lg(f.rowblk)) * Q) > max_elems))
    f.rowblk >>= 1;
  while (f.rowblk > 1 && f.rowblk / 2 >= f.H) f.rowblk >>= 1;
  f.lg_rowcols = rows_lg(f.rowblk);
  if (p->tune_lgcols >= 0 && p->tune_lgcols <= 5 && (1 << p->tune_lgcols) <= 2 * Q &&
      (P << p->tune_lgcols) <= max_elems && ((size_t)2 * P * ((size_t)1 << p->tune_lgcols) + P) * cs <= 100 * 1024)
    f.lg_cols = p->tune_lgcols;
  if (p->tune_rowblk >= 1 && p->tune_rowblk <= 32 && p->tune_rowblk / 2 < f.H &&
      ((1 << rows_lg(p->tune_rowblk)) * Q) <= max_elems &&
      ((size_t)2 * ((size_t)1 << rows_lg(p->tune_rowblk)) * Q + Q) * cs <= 100 * 1024) {
    f.rowblk = p->tune_rowblk;
    f.lg_rowcols = rows_lg(f.rowblk);
  }
  f.N = N;

  SpreadParams s{};
  s.D = p->D;
  s.Mr = Mr;
  s.msp = p->msp;
  s.klo = p->klo;
  s.khi = p->khi;
  s.kernel = p->desc.kernel;
  s.max_events = p->desc.max_events;
  const int tmax = spread_max_tile(p->fp64);
  // default tile: the largest (measured on GB300 with the polynomial scatter:
  // 4096 cells beat 2048 on both the block and the batched workloads)
  int tile = p->desc.spread_tile > 0 ? std::min(p->desc.spread_tile, tmax) : tmax;
  if (p->tune_tile > 0) tile = std::min(p->tune_tile, tmax);
  if (Mr <= (int64_t)tile) {
    tile = (int)Mr;
    s.single_tile = 1;
  }
  const bool fits = fused_smem(f, Mr, p->fp64) + 2048 <= (size_t)p->smem_optin;
  int algo = p->desc.spread_algo == 2 ? 1 : (p->desc.spread_algo == 3 ? 2 : 0);
  if (p->tune_algo >= 0) algo = p->tune_algo;
  // fused stages: the float32 path keeps the grid row resident after the
  // prep kernel (below, when the row and its sub-range tiles fit); the FP64
  // path and rows without the polynomial taps use the one-CTA kernel that also
  // rescales (a single problem whose grid fits)
  const bool want_fused = algo == 2;
  if (algo == 2) algo = 0;
  s.algo = algo == 1 ? 1 : 0;
  s.fused = 0;
  s.tile = tile;
  s.ntiles = (int)((Mr + tile - 1) / tile);
  s.es_beta = 2.3 * 2.0 * p->msp;
  s.es_inv_w = 1.0 / p->msp;
  const double lam = sigma * p->msp / (sigma - 0.5);
  s.g_t1 = kPi / lam;
  s.kb_b = kPi * (2.0 - 1.0 / sigma);
  s.kb_inv_phi0 = kPi * p->msp / sinh(s.kb_b * p->msp);
  p->tau = kPi * lam / ((double)Mr * (double)Mr);
  p->poly_ok = false;
  if (!p->fp64 && s.algo == 0 && p->tune_poly != 0 && spread_poly_supported(s.khi - s.klo + 1)) {
    // the fit must stay far below the NUFFT tolerance and near float32 rounding
    const double err = fit_kernel_poly(s, &p->poly);
    p->poly_ok = err <= std::max(3.0e-7, 0.1 * p->desc.tol);
  }
  // per-asset FFT: mixed path, the complex grid fits in shared memory and n
  // factors into at most kMaxAssetPasses compiled radices
  AssetFft af{};
  // one CTA per asset (its grid row lands in shared memory by bulk copies)
  // whenever the row fits, whatever the number of assets: each CTA's time is
  // set by latency (a CTA alone on an SM takes as long as two sharing one),
  // so splitting an asset over more SMs does not pay for its extra loads.
  // Larger rows: two CTAs per asset as a cluster (decimation in time by 2,
  // joined through distributed shared memory), also on request.
  int split = 1;
  int pair = 0;
  const bool caller_split = p->desc.fft_algo >= 2 && p->tune_split < 1;
  if (caller_split && p->desc.fft_algo == 4) {  // the caller's choice: the cluster pair
    split = 2;
    pair = 1;
  }
  if (p->tune_split == 1) {
    split = 1;
    pair = 0;
  } else if (p->tune_split == 3) {
    split = 2;
    pair = 1;
  }
  // radices up to 16 by default: the fully unrolled codelets of 25 to 32
  // points stall on instruction fetch, so four small passes beat three large
  // ones; radices up to 32 where the small ones need too many passes or
  // twiddle rows. The cluster pair (decimation in time, 512 threads per CTA)
  // measured the other way round: up to 32 first.
  auto fits_split = [&](int sp_) {
    const bool pair_first = sp_ == 2 && pair;
    for (int maxr : {pair_first ? 32 : 16, pair_first ? 16 : 32}) {
      if (p->tune_maxr > 0 && maxr != p->tune_maxr) continue;
      if (plan_asset_fft(n, sp_, N, maxr, &af) && asset_fft_smem(af) + 2048 <= (size_t)p->smem_optin &&
          asset_twiddle_count(af) <= p->atw_cap)
        return true;
    }
    return false;
  };
  bool afft = !p->fp64 && fits_split(split);
  if (!p->fp64 && !afft && p->tune_split < 1 && p->desc.fft_algo < 2) {
    // the other form (a large grid fits in shared memory only as two halves)
    split = split == 1 ? 2 : 1;
    pair = split == 2 ? 1 : 0;
    afft = fits_split(split);
  }
  af.pair = afft && split == 2 ? pair : 0;
  int fft_algo = p->desc.fft_algo == 1 ? 1 : 0;
  if (p->tune_fft >= 0) fft_algo = p->tune_fft == 0 ? 0 : 1;
  if (fft_algo == 1) afft = false;
  // one CTA per asset after the polynomial scatter: the scatter stores the
  // grid in the FFT's digit-reversed input order, so the FFT loads the row
  // with one bulk copy
  s.perm_np = 0;
  af.pre_perm = 0;
  const bool want_perm = p->tune_perm == 1 || (p->tune_perm < 0 && p->desc.fft_algo == 5);
  if (afft && !s.fused && split == 1 && p->poly_ok && want_perm) {
    af.pre_perm = 1;
    s.perm_np = af.npass;
    for (int q = 0; q < 4; ++q) {
      const int R = q < af.npass ? af.rad[q] : 1;
      s.perm_rad[q] = R;
      s.perm_stride[q] = q < af.npass ? af.stride[q] : 0;
      s.perm_magic[q] = R <= 1 ? 0u : 0xFFFFFFFFu / (unsigned)R + 1u;
    }
  }
  // decimation in frequency (natural-order input) except where the input
  // arrives digit-reversed (the scatter's permuted grid) and for the cluster
  // pair, whose joining step reads half its values from the partner's shared
  // memory: those reads must be contiguous (natural output order)
  af.dif = !af.pre_perm && !af.pair;
  // the resident form: decimation in time (the sub-ranges' points go straight
  // to their digit reversals, the unpacking reads natural order)
  p->res_sub = 0;
  if (want_fused && afft && p->poly_ok) {
    AssetFft rf = af;
    rf.pre_perm = 0;
    rf.dif = 0;
    const int sub = spread_fft_sub(rf, Mr, (size_t)p->smem_optin - kResStaticSmem);
    if (sub > 0) {
      p->res_sub = sub;
      af = rf;
      s.perm_np = 0;
    }
  }
  if (want_fused && !p->res_sub && fits && p->G == 1) s.fused = 1;
  p->afft = af;
  p->use_afft = afft && !s.fused;
  p->fft = f;
  p->sp = s;
  p->Mr = Mr;
  p->cfg_N = N;
  p->cfg_D = p->D;
  p->cfg_gen += 1;
  return MM_OK;
}

mm_status ensure_tables(mm_plan p, int N, cudaStream_t st) {
  if (p->tab_N == N) return MM_OK;
  StageScope sc(p, MM_STAGE_SETUP, st);
  MM_CUDA(launch_setup_tables(p->desc.kernel, p->msp, p->Mr, N, p->fft.n, p->sp, p->tau, p->glx, p->glw, kGlNodes,
                              p->W, p->U, p->decon, p->fp64, st));
  p->tab_N = N;
  return MM_OK;
}

// Pass twiddles of the per-asset FFT plan in use (rebuilt when the plan changes).
mm_status ensure_asset_twiddles(mm_plan p, cudaStream_t st) {
  const AssetFft& f = p->afft;
  if (p->fp64 || f.npass == 0 || asset_twiddle_count(f) > p->atw_cap) return MM_OK;
  const bool same = p->atw_n == f.nl && p->atw_npass == f.npass &&
                    std::equal(f.rad, f.rad + kMaxAssetPasses, p->atw_rad);
  if (same) return MM_OK;
  StageScope sc(p, MM_STAGE_SETUP, st);
  MM_CUDA(launch_asset_twiddles(f, p->atw, st));
  p->atw_n = f.nl;
  p->atw_npass = f.npass;
  std::copy(f.rad, f.rad + kMaxAssetPasses, p->atw_rad);
  return MM_OK;
}

mm_status check_plan(mm_plan p) {
  if (!p) return MM_ERR_INVALID_ARG;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return MM_ERR_CUDA;
  if (cur != p->dev && cudaSetDevice(p->dev) != cudaSuccess) return MM_ERR_CUDA;
  return MM_OK;
}

// Stage (d) by the pre-split operand and TMA (mixed precisions, single
// problems): on request, or by default from kGramTmaMinAssets assets up.
bool gram_uses_tma(mm_plan p) {
  if (p->fp64 || p->batch) return false;
  if (p->desc.gram_algo != 0) return p->desc.gram_algo == 2;
  return p->D >= kGramTmaMinAssets;
}

GramParams gram_params(mm_plan p, int N) {
  GramParams g{};
  g.wait_ns = p->wait_ns;
  g.D = p->D;
  g.N = N;
  g.ld = N + 1;
  g.Dp = (g.D + 3) / 4 * 4;
  g.tile = p->fp64 ? 64 : 128;
  g.ntiles = (g.D + g.tile - 1) / g.tile;
  g.npairs = g.ntiles * (g.ntiles + 1) / 2;
  g.chunk = p->fp64 ? 16 : (p->desc.prec == MM_PREC_MIXED_BF16X3 ? 32 : 16);
  g.nchunks = (N + 1 + g.chunk - 1) / g.chunk;
  int S;
  if (p->fp64) {
    // split K so that all SMs get work while the partial tiles stay a small
    // fraction of the operand bytes
    const double a_bytes = (double)g.D * 2.0 * (N + 1) * 8.0;
    const double tile_bytes = (double)g.tile * g.tile * 8.0;
    const int s_traffic = (int)std::max(1.0, ceil(a_bytes / (4.0 * g.npairs * tile_bytes)));
    S = std::max(1, std::min({g.nchunks, std::max(1, kMaxGramCtas / g.npairs), s_traffic}));
  } else if (gram_uses_tma(p)) {
    // one CTA per SM (its stage ring fills the shared memory): one wave
    S = std::max(1, std::min((g.nchunks + 1) / 2, std::max(1, kSMs / g.npairs)));
  } else {
    // about two CTAs per SM, at least two K-chunks each (the partial sums meet
    // in L2 through vector reductions, so more splits cost little traffic)
    S = std::max(1, std::min((g.nchunks + 1) / 2, std::max(1, kMaxGramCtas / g.npairs)));
  }
  g.chunks_per_split = (g.nchunks + S - 1) / S;
  g.splits = (g.nchunks + g.chunks_per_split - 1) / g.chunks_per_split;
  return g;
}

mm_status coeffs_impl(mm_plan p, const int64_t* off, const double* t, const double* logp, int N, double t0,
                      double t1, void* coeffs, int32_t* N_used, cudaStream_t st) {
  const int D = p->D;
  p->last = st;
  // with a given cutoff the grid is configured first, so that k_bounds also
  // computes the call's cell scales
  int64_t Mr_known = 0;
  if (N > 0) {
    if (N > p->desc.N_max) return MM_ERR_CUTOFF;
    if (p->desc.basis == MM_BASIS_FEJER && N < 1) return MM_ERR_CUTOFF;
    const mm_status rc = configure(p, N);
    if (rc != MM_OK) return rc;
    Mr_known = p->Mr;
  }
  // one condition for both sides: k_bounds writes the order the spreading
  // kernel then reads
  const bool use_order = p->asset_order && p->G == 1 && D <= kOrderMaxAssets;
  {
    StageScope sc(p, MM_STAGE_PREP, st);
    MM_CUDA(launch_bounds(off, t, D, p->gsize, p->desc.max_events, t0, t1, Mr_known, p->bounds, p->status,
                          use_order ? p->asset_order : nullptr, st));
  }
  if (N <= 0 && p->G > 1) return MM_ERR_CUTOFF;  // a batch sweeps given cutoffs
  if (N <= 0) {
    {
      StageScope sc(p, MM_STAGE_PREP, st, 2);
      MM_CUDA(launch_min_gap(off, t, D, p->bounds, p->gapbits, p->status + 2, p->status, st));
    }
    int hv[3];
    MM_CUDA(cudaMemcpyAsync(hv, p->status, sizeof(hv), cudaMemcpyDeviceToHost, st));
    MM_CUDA(cudaStreamSynchronize(st));
    if (hv[1]) return hv[0] ? flags_to_status(hv[0]) : MM_ERR_INVALID_ARG;
    if (hv[2] < 0) return MM_ERR_CUTOFF;
    N = hv[2];
  }
  if (N > p->desc.N_max) return MM_ERR_CUTOFF;
  if (p->desc.basis == MM_BASIS_FEJER && N < 1) return MM_ERR_CUTOFF;
  mm_status r = configure(p, N);
  if (r != MM_OK) return r;
  r = ensure_tables(p, N, st);
  if (r != MM_OK) return r;
  r = ensure_asset_twiddles(p, st);
  if (r != MM_OK) return r;
  if (p->sp.fused) {
    StageScope sc(p, MM_STAGE_FUSED, st);
    MM_CUDA(launch_coeff_fused(p->fp64, off, t, logp, p->bounds, p->sp, p->fft, p->W, p->U, p->decon, coeffs,
                               p->status, st));
  } else {
    const GroupScale* gsc = p->G > 1 ? (const GroupScale*)p->gscale : nullptr;
    if (gsc) {
      StageScope sc(p, MM_STAGE_PREP, st);
      MM_CUDA(launch_group_scales(p->bounds, p->G, p->Mr, (GroupScale*)p->gscale, p->status, st));
    }
    {
      StageScope sc(p, MM_STAGE_PREP, st);
      if (p->fp64)
        MM_CUDA(launch_prep_f64(off, t, logp, p->bounds, gsc, p->gsize, D, p->Mr, p->desc.max_events, p->rec_b0,
                                p->rec_d, p->rec_v, p->status, st));
      else
        MM_CUDA(launch_prep_f32(off, t, logp, p->bounds, gsc, p->gsize, D, p->Mr, p->desc.max_events, p->rec_b0,
                                p->rec_d, p->rec_v, p->status, st));
    }
    if (p->res_sub > 0) {
      StageScope sc(p, MM_STAGE_FUSED, st);
      MM_CUDA(launch_spread_fft(off, p->rec_b0, p->rec_d, p->rec_v, p->sp, p->poly, p->res_sub, p->afft, D, p->W,
                                p->atw, p->U, p->decon, coeffs, p->status, st));
      if (N_used) *N_used = N;
      return MM_OK;
    }
    {
      StageScope sc(p, MM_STAGE_SPREAD, st);
      p->sp.order = use_order ? p->asset_order : nullptr;
      if (p->fp64)
        MM_CUDA(launch_spread_f64(off, p->rec_b0, p->rec_d, p->rec_v, p->sp, (double*)p->grid, p->status, st));
      else if (p->poly_ok)
        MM_CUDA(launch_spread_poly(off, p->rec_b0, p->rec_d, p->rec_v, p->sp, p->poly, (float*)p->grid, p->status,
                                   st));
      else
        MM_CUDA(launch_spread_f32(off, p->rec_b0, p->rec_d, p->rec_v, p->sp, (float*)p->grid, p->status, st));
    }
    if (p->use_afft) {
      StageScope sc(p, MM_STAGE_FFT, st);
      MM_CUDA(launch_fft_asset((const float*)p->grid, p->afft, D, p->W, p->atw, p->U, p->decon, coeffs, p->status,
                               st));
    } else {
    {
      StageScope sc(p, MM_STAGE_FFT_COLS, st);
      if (p->fp64) MM_CUDA(launch_fft_cols_f64((double*)p->grid, p->fft, D, p->W, p->status, st));
      else MM_CUDA(launch_fft_cols_f32((float*)p->grid, p->fft, D, p->W, p->status, st));
    }
    {
      StageScope sc(p, MM_STAGE_FFT_ROWS, st);
      if (p->fp64)
        MM_CUDA(launch_fft_rows_f64((const double*)p->grid, p->fft, D, p->W, p->U, p->decon, coeffs, p->status, st));
      else
        MM_CUDA(launch_fft_rows_f32((const float*)p->grid, p->fft, D, p->W, p->U, p->decon, coeffs, p->status, st));
    }
    }
  }
  if (N_used) *N_used = N;
  return MM_OK;
}

mm_status corr_impl(mm_plan p, const void* coeffs, int N, void* sigma, void* R, cudaStream_t st) {
  if (p->batch) return MM_ERR_UNSUPPORTED;
  if (N < 0 || N > p->desc.N_max) return MM_ERR_CUTOFF;
  if (p->desc.basis == MM_BASIS_FEJER && N < 1) return MM_ERR_CUTOFF;
  p->last = st;
  GramParams g = gram_params(p, N);
  if (p->fp64 && (size_t)g.npairs * g.splits * g.tile * g.tile * p->rs > p->partial_bytes) return MM_ERR_UNSUPPORTED;
  if (p->w_N != N || p->w_basis != (int)p->desc.basis) {
    StageScope sc(p, MM_STAGE_SETUP, st);
    MM_CUDA(launch_gram_weights(p->desc.basis, N, p->fp64, p->wsq, st));
    p->w_N = N;
    p->w_basis = p->desc.basis;
  }
  if (p->fp64) {
    p->gram_used = 3;
    {
      StageScope sc(p, MM_STAGE_GRAM, st);
      MM_CUDA(launch_gram_f64(coeffs, g, (const double*)p->wsq, (double*)p->partial, st));
    }
    StageScope sc(p, MM_STAGE_REDUCE, st);
    MM_CUDA(launch_reduce_corr(true, p->partial, g, sigma, R, p->status, st));
  } else {
    const size_t acc_bytes = (size_t)g.D * g.Dp * sizeof(float);
    if (p->acc_D != g.D) p->acc_dirty = true;  // the cleared region was sized for another D
    if (p->acc_dirty) {
      MM_CUDA(cudaMemsetAsync(p->acc[0], 0, acc_bytes, st));
      MM_CUDA(cudaMemsetAsync(p->acc[1], 0, acc_bytes, st));
      p->acc_dirty = false;
    }
    float* cur = p->acc[p->acc_sel];
    float* next = p->acc[p->acc_sel ^ 1];
    p->acc_dirty = true;  // until both launches below are queued
    const int mode = p->desc.prec == MM_PREC_MIXED_BF16X3 ? 0 : 1;
    // few assets: the last contraction CTA writes Sigma and R itself (one
    // launch less); beyond that the separate epilogue's parallelism wins
    const bool tma = gram_uses_tma(p);
    const bool fuse = !tma && g.D <= 32 && R;
    if (tma) {
      {
        StageScope sc(p, MM_STAGE_SPLIT, st);
        MM_CUDA(launch_gram_split(mode, coeffs, g, (const float*)p->wsq, p->tma_hi, p->tma_lo, st));
      }
      StageScope sc(p, MM_STAGE_GRAM, st);
      MM_CUDA(launch_gram_tma(mode, g, p->tma_hi, p->tma_lo, cur, p->status, st));
    } else {
      StageScope sc(p, MM_STAGE_GRAM, st);
      MM_CUDA(launch_gram_tc(mode, coeffs, g, (const float*)p->wsq, cur, p->status, fuse ? p->gram_done : nullptr,
                             (float*)sigma, (float*)R, next, st));
    }
    p->gram_used = tma ? 2 : 1;
    if (!fuse) {
      StageScope sc(p, MM_STAGE_REDUCE, st);
      MM_CUDA(launch_corr_acc(cur, g, (float*)sigma, (float*)R, next, p->status, st));
    }
    p->acc_sel ^= 1;
    p->acc_dirty = false;
    p->acc_D = g.D;
  }
  p->gram = g;
  return MM_OK;
}

mm_status estimate_eager(mm_plan p, const int64_t* off, const double* t, const double* logp, int N, double t0,
                         double t1, void* coeffs, void* sigma, void* R, int32_t* N_used, cudaStream_t st) {
  int32_t Nu = 0;
  mm_status r = coeffs_impl(p, off, t, logp, N, t0, t1, coeffs, &Nu, st);
  if (r != MM_OK) return r;
  if (N_used) *N_used = Nu;
  return corr_impl(p, coeffs, Nu, sigma, R, st);
}

// Coefficients, Sigma and R with the launches of a steady call (tables,
// weights and configuration already built for N; no per-stage timing)
// replayed from a CUDA graph: one launch instead of six to eight, and no
// launch gaps between the kernels. The first steady call with a given set of
// inputs, outputs, cutoff, window and configuration captures the sequence
// (for the accumulator it fills), later ones replay it. Anything else runs
// eagerly.
mm_status estimate_impl(mm_plan p, const int64_t* off, const double* t, const double* logp, int N, double t0,
                        double t1, void* coeffs, void* sigma, void* R, int32_t* N_used, cudaStream_t st) {
  const bool steady = p->graphs && !p->prof && N > 0 && p->G == 1 && p->cfg_N == N && p->cfg_D == p->D &&
                      p->tab_N == N && p->w_N == N && p->w_basis == (int)p->desc.basis &&
                      (p->fp64 || (!p->acc_dirty && p->acc_D == p->D));
  if (!steady) return estimate_eager(p, off, t, logp, N, t0, t1, coeffs, sigma, R, N_used, st);
  mm_plan_s::EstGraph& G = p->eg[p->fp64 ? 0 : p->acc_sel];
  const void* key[6] = {off, t, logp, coeffs, sigma, R};
  bool same = G.exec && G.N == N && G.D == p->D && G.cfg == p->cfg_gen && G.t0 == t0 && G.t1 == t1;
  for (int i = 0; i < 6 && same; ++i) same = key[i] == G.key[i];
  if (!same) {
    if (G.exec) cudaGraphExecDestroy(G.exec);
    G.exec = nullptr;
    if (!p->cap && cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return estimate_eager(p, off, t, logp, N, t0, t1, coeffs, sigma, R, N_used, st);
    }
    // capture from the current host state, which is then put back: the
    // launches run when the graph does
    const int acc_sel = p->acc_sel, acc_D = p->acc_D;
    const bool acc_dirty = p->acc_dirty;
    const int64_t l0 = p->launches;
    cudaGraph_t g = nullptr;
    mm_status r = MM_ERR_CUDA;
    if (cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
      r = estimate_eager(p, off, t, logp, N, t0, t1, coeffs, sigma, R, nullptr, p->cap);
      if (cudaStreamEndCapture(p->cap, &g) != cudaSuccess) r = MM_ERR_CUDA;
    }
    const int kernels = (int)(p->launches - l0);
    p->launches = l0;
    p->acc_sel = acc_sel;
    p->acc_D = acc_D;
    p->acc_dirty = acc_dirty;
    cudaGraphExec_t ex = nullptr;
    if (r == MM_OK && g && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) ex = nullptr;
    if (g) cudaGraphDestroy(g);
    if (!ex) {
      cudaGetLastError();
      return estimate_eager(p, off, t, logp, N, t0, t1, coeffs, sigma, R, N_used, st);
    }
    G.exec = ex;
    for (int i = 0; i < 6; ++i) G.key[i] = key[i];
    G.N = N;
    G.D = p->D;
    G.cfg = p->cfg_gen;
    G.t0 = t0;
    G.t1 = t1;
    G.kernels = kernels;
  }
  MM_CUDA(cudaGraphLaunch(G.exec, st));
  p->graph_launches += 1;
  p->launches += G.kernels;
  p->last = st;
  // the host state the eager sequence leaves behind
  if (!p->fp64) {
    p->acc_sel ^= 1;
    p->acc_dirty = false;
    p->acc_D = p->D;
  }
  if (N_used) *N_used = N;
  return MM_OK;
}

}  // namespace

extern "C" {

int32_t mm_version(void) { return 101; }

const char* mm_status_string(mm_status s) {
  switch (s) {
    case MM_OK: return "ok";
    case MM_ERR_INVALID_ARG: return "invalid argument";
    case MM_ERR_UNSORTED: return "event times not increasing within an asset";
    case MM_ERR_DUPLICATE_TIME: return "repeated event time within an asset";
    case MM_ERR_DEGENERATE_SPAN: return "empty or degenerate time span";
    case MM_ERR_CUTOFF: return "cutoff N out of range";
    case MM_ERR_OOM: return "device allocation failed";
    case MM_ERR_CUDA: return "CUDA error";
    case MM_ERR_TIMEOUT: return "bounded device wait timed out";
    case MM_ERR_ZERO_VARIANCE: return "zero-variance asset (NaN correlations)";
    case MM_ERR_NONFINITE: return "non-finite time or log-price";
    case MM_ERR_UNSUPPORTED: return "unsupported request";
  }
  return "unknown status";
}

}  // extern "C"

namespace {

// Plan for D = G * gsize assets in G independent problems of gsize assets
// each (G = 1: the single-problem plan of mm_plan_create). A batch plan
// allocates no contraction or host-staging workspace.
mm_status plan_create_impl(const mm_plan_desc* desc, int gsize, bool batch, mm_plan* out, bool staging = true) {
  if (!out) return MM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc) return MM_ERR_INVALID_ARG;
  const mm_plan_desc& d = *desc;
  if (gsize < 1 || d.D % gsize) return MM_ERR_INVALID_ARG;
  if (d.D < 1 || d.N_max < 0 || d.max_events < 0) return MM_ERR_INVALID_ARG;
  if (!(d.tol > 0.0 && d.tol < 0.5)) return MM_ERR_INVALID_ARG;
  if (d.kernel < MM_KERNEL_GAUSS || d.kernel > MM_KERNEL_ES) return MM_ERR_INVALID_ARG;
  if (d.basis < MM_BASIS_DIRICHLET || d.basis > MM_BASIS_FEJER) return MM_ERR_INVALID_ARG;
  if (d.prec < MM_PREC_FP64 || d.prec > MM_PREC_MIXED_3XTF32) return MM_ERR_INVALID_ARG;
  if (d.spread_tile < 0 || d.spread_tile > 50000) return MM_ERR_INVALID_ARG;
  if (d.spread_algo < 0 || d.spread_algo > 3) return MM_ERR_INVALID_ARG;
  if (d.fft_algo < 0 || d.fft_algo > 5 || d.fft_algo == 3) return MM_ERR_INVALID_ARG;
  if (d.gram_algo < 0 || d.gram_algo > 2) return MM_ERR_INVALID_ARG;
  for (int i = 0; i < 3; ++i)
    if (d.reserved[i] != 0) return MM_ERR_INVALID_ARG;
  const int msp = msp_rule(d.kernel, d.tol);
  if (msp < 1 || msp > 30) return MM_ERR_UNSUPPORTED;

  mm_plan p = new mm_plan_s();
  p->desc = d;
  p->gsize = gsize;
  p->G = d.D / gsize;
  p->D = d.D;
  p->batch = batch;
  p->fp64 = d.prec == MM_PREC_FP64;
  p->cs = p->fp64 ? 16 : 8;
  p->rs = p->fp64 ? 8 : 4;
  p->msp = msp;
  p->khi = msp;
  p->klo = d.kernel == MM_KERNEL_GAUSS ? -msp + 1 : -msp;
  int64_t n;
  int P, Q;
  if (!choose_fft(std::max<int64_t>(2 * (int64_t)d.N_max + 1, msp + 1), &n, &P, &Q)) {
    delete p;
    return MM_ERR_UNSUPPORTED;
  }
  p->n_max = n;
  if (cudaGetDevice(&p->dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&p->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->dev) != cudaSuccess) {
    delete p;
    return MM_ERR_CUDA;
  }
  const size_t D = (size_t)d.D;
  const size_t Np1 = (size_t)d.N_max + 1;
  mm_status r = MM_OK;
  auto A = [&](void** ptr, size_t bytes) {
    if (r == MM_OK) r = dalloc(p, ptr, bytes);
  };
  A(&p->grid, D * 2 * (size_t)n * p->rs);
  A((void**)&p->rec_b0, (size_t)std::max<int64_t>(d.max_events, 1) * sizeof(int));
  A(&p->rec_d, (size_t)std::max<int64_t>(d.max_events, 1) * p->rs);
  A(&p->rec_v, (size_t)std::max<int64_t>(d.max_events, 1) * p->rs);
  A(&p->W, (size_t)n * p->cs);
  if (!p->fp64) {
    p->atw_cap = 2 * n;  // sum_p m_p (R_p - 1) < n (1 + 1/R_1 + ...) < 2n
    A(&p->atw, (size_t)p->atw_cap * p->cs);
  }
  A(&p->U, Np1 * p->cs);
  A(&p->decon, Np1 * p->rs);
  A((void**)&p->glx, kGlNodes * sizeof(double));
  A((void**)&p->glw, kGlNodes * sizeof(double));
  A((void**)&p->bounds, (size_t)p->G * sizeof(Rescale));
  if (!batch && D <= (size_t)kOrderMaxAssets) A((void**)&p->asset_order, std::max<size_t>(D, 1) * sizeof(int));
  if (p->G > 1) A(&p->gscale, (size_t)p->G * group_scale_bytes());
  A((void**)&p->status, 4 * sizeof(int));
  A((void**)&p->gapbits, sizeof(unsigned long long));
  A(&p->wsq, Np1 * p->rs);
  if (!batch) {
    GramParams g = gram_params(p, d.N_max);
    size_t ctas = std::max<size_t>((size_t)kMaxGramCtas, (size_t)g.npairs);
    if (p->fp64) {
      p->partial_bytes = ctas * g.tile * g.tile * p->rs;
      A(&p->partial, p->partial_bytes);
    } else {
      A((void**)&p->acc[0], D * (size_t)g.Dp * sizeof(float));
      A((void**)&p->acc[1], D * (size_t)g.Dp * sizeof(float));
      A((void**)&p->gram_done, sizeof(int));
      if (gram_uses_tma(p)) {
        const size_t pb = gram_tma_plane_bytes(d.prec == MM_PREC_MIXED_BF16X3 ? 0 : 1, d.D, d.N_max, g.chunk);
        A(&p->tma_hi, pb);
        A(&p->tma_lo, pb);
        if (r == MM_OK && (cudaMemset(p->tma_hi, 0, pb) != cudaSuccess || cudaMemset(p->tma_lo, 0, pb) != cudaSuccess))
          r = MM_ERR_CUDA;
      }
    }
  }
  if (d.max_events > 0 && !batch && staging) {
    A((void**)&p->s_off, (D + 1) * sizeof(int64_t));
    A((void**)&p->s_t, (size_t)d.max_events * sizeof(double));
    A((void**)&p->s_p, (size_t)d.max_events * sizeof(double));
    A(&p->s_coef, D * Np1 * p->cs);
    A(&p->s_sigma, D * D * p->rs);
    A(&p->s_R, D * D * p->rs);
    if (r == MM_OK && cudaMallocHost((void**)&p->h_status, sizeof(int)) != cudaSuccess) r = MM_ERR_OOM;
  }
  if (r == MM_OK) {
    if (cudaMemset(p->status, 0, 4 * sizeof(int)) != cudaSuccess) r = MM_ERR_CUDA;
    if (p->gram_done && cudaMemset(p->gram_done, 0, sizeof(int)) != cudaSuccess) r = MM_ERR_CUDA;
  }
  if (r == MM_OK) {
    if (launch_gl_nodes(kGlNodes, p->glx, p->glw, 0) != cudaSuccess) r = MM_ERR_CUDA;
    p->launches += 1;
    p->nl[MM_STAGE_SETUP] += 1;
  }
  if (r == MM_OK && cudaDeviceSynchronize() != cudaSuccess) r = MM_ERR_CUDA;
  if (r != MM_OK) {
    free_all(p);
    delete p;
    cudaGetLastError();
    return r;
  }
  *out = p;
  return MM_OK;
}

}  // namespace

extern "C" {

mm_status mm_plan_create(const mm_plan_desc* desc, mm_plan* out) {
  if (!desc) {
    if (out) *out = nullptr;
    return MM_ERR_INVALID_ARG;
  }
  return plan_create_impl(desc, desc->D > 0 ? desc->D : 1, false, out);
}

mm_status mm_destroy(mm_plan p) {
  if (!p) return MM_ERR_INVALID_ARG;
  int cur = -1;
  const int dev = p->dev;
  cudaGetDevice(&cur);
  if (cur != dev) cudaSetDevice(dev);
  cudaDeviceSynchronize();
  free_all(p);
  delete p;
  if (cur >= 0 && cur != dev) cudaSetDevice(cur);
  return MM_OK;
}

mm_status mm_coeffs(mm_plan p, const int64_t* d_offsets, const double* d_t, const double* d_logp, int32_t N,
                    double t0, double t1, void* d_coeffs, int32_t* N_used, void* stream) {
  mm_status r = check_plan(p);
  if (r != MM_OK) return r;
  if (!d_offsets || !d_t || !d_logp || !d_coeffs) return MM_ERR_INVALID_ARG;
  if (!(isfinite(t0) && isfinite(t1))) return MM_ERR_INVALID_ARG;
  return coeffs_impl(p, d_offsets, d_t, d_logp, N, t0, t1, d_coeffs, N_used, (cudaStream_t)stream);
}

mm_status mm_corr_pairwise(mm_plan p, const void* d_coeffs, int32_t N_coeffs, const int32_t* h_N,
                           int32_t psd_repair, void* d_sigma_or_null, void* d_R, int32_t* d_clipped_or_null,
                           void* stream) {
  mm_status r = check_plan(p);
  if (r != MM_OK) return r;
  if (p->batch) return MM_ERR_UNSUPPORTED;
  if (!d_coeffs || !h_N || !d_R || (psd_repair != 0 && psd_repair != 1)) return MM_ERR_INVALID_ARG;
  if (N_coeffs < 0 || N_coeffs > p->desc.N_max) return MM_ERR_CUTOFF;
  const int D = p->D;
  if (psd_repair && D > pairwise_psd_max_assets()) return MM_ERR_UNSUPPORTED;
  const int lo = p->desc.basis == MM_BASIS_FEJER ? 1 : 0;
  for (int i = 0; i < D; ++i)
    if (h_N[i] < lo || h_N[i] > N_coeffs) return MM_ERR_CUTOFF;
  if (!p->pw_N) {
    const size_t dd = (size_t)p->desc.D * p->desc.D * sizeof(double);
    mm_status a = dalloc(p, (void**)&p->pw_N, (size_t)p->desc.D * sizeof(int));
    if (a == MM_OK) a = dalloc(p, (void**)&p->pw_sig, dd);
    if (a == MM_OK && p->desc.D <= pairwise_psd_max_assets()) a = dalloc(p, (void**)&p->pw_A, dd);
    if (a == MM_OK && p->desc.D <= pairwise_psd_max_assets()) a = dalloc(p, (void**)&p->pw_V, dd);
    if (a == MM_OK) a = dalloc(p, (void**)&p->pw_clip, sizeof(int));
    if (a == MM_OK) a = dalloc(p, &p->pw_sync, psd_sync_bytes());
    if (a != MM_OK) return a;
  }
  cudaStream_t st = (cudaStream_t)stream;
  p->last = st;
  MM_CUDA(cudaMemcpyAsync(p->pw_N, h_N, (size_t)D * sizeof(int), cudaMemcpyHostToDevice, st));
  {
    StageScope sc(p, MM_STAGE_GRAM, st);
    MM_CUDA(launch_pairwise(p->fp64, p->desc.basis == MM_BASIS_FEJER, d_coeffs, N_coeffs + 1, p->pw_N, D,
                            p->pw_sig, st));
  }
  StageScope sc(p, MM_STAGE_REDUCE, st, psd_repair ? 2 : 1);
  int* clip = d_clipped_or_null ? (int*)d_clipped_or_null : p->pw_clip;
  if (psd_repair) MM_CUDA(launch_psd_repair(p->fp64, p->pw_sig, p->pw_A, p->pw_V, D, clip, p->pw_sync, p->status, st));
  else MM_CUDA(cudaMemsetAsync(clip, 0, sizeof(int), st));
  MM_CUDA(launch_pairwise_out(p->fp64, p->pw_sig, D, d_sigma_or_null, d_R, p->status, st));
  return MM_OK;
}

mm_status mm_cov(mm_plan p, const void* d_coeffs, int32_t N, void* d_sigma, void* stream) {
  mm_status r = check_plan(p);
  if (r != MM_OK) return r;
  if (!d_coeffs || !d_sigma) return MM_ERR_INVALID_ARG;
  return corr_impl(p, d_coeffs, N, d_sigma, nullptr, (cudaStream_t)stream);
}

mm_status mm_corr(mm_plan p, const void* d_coeffs, int32_t N, void* d_sigma_or_null, void* d_R, void* stream) {
  mm_status r = check_plan(p);
  if (r != MM_OK) return r;
  if (!d_coeffs || !d_R) return MM_ERR_INVALID_ARG;
  return corr_impl(p, d_coeffs, N, d_sigma_or_null, d_R, (cudaStream_t)stream);
}

mm_status mm_estimate(mm_plan p, const int64_t* d_offsets, const double* d_t, const double* d_logp, int32_t N,
                      double t0, double t1, void* d_coeffs, void* d_sigma_or_null, void* d_R, int32_t* N_used,
                      void* stream) {
  mm_status r = check_plan(p);
  if (r != MM_OK) return r;
  if (!d_offsets || !d_t || !d_logp || !d_coeffs || !d_R) return MM_ERR_INVALID_ARG;
  if (!(isfinite(t0) && isfinite(t1))) return MM_ERR_INVALID_ARG;
  return estimate_impl(p, d_offsets, d_t, d_logp, N, t0, t1, d_coeffs, d_sigma_or_null, d_R, N_used,
                       (cudaStream_t)stream);
}

// Device address of a host buffer of `bytes` bytes that kernels on device
// `dev` may read directly: pinned and mapped from its first to its last byte
// (page-locked memory from cudaHostAlloc or cudaMallocHost, or registered
// with cudaHostRegister); nullptr for pageable memory or anything else.
static const void* mapped_alias(const void* h, size_t bytes, int dev) {
  if (bytes == 0) return nullptr;
  cudaPointerAttributes a0{}, a1{};
  if (cudaPointerGetAttributes(&a0, h) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a0.type != cudaMemoryTypeHost || !a0.devicePointer || a0.device != dev) return nullptr;
  const char* last = static_cast<const char*>(h) + (bytes - 1);
  if (cudaPointerGetAttributes(&a1, last) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a1.type != cudaMemoryTypeHost || !a1.devicePointer ||
      static_cast<const char*>(a1.devicePointer) - static_cast<const char*>(a0.devicePointer) !=
          static_cast<ptrdiff_t>(bytes - 1))
    return nullptr;
  return a0.devicePointer;
}

mm_status mm_estimate_host(mm_plan p, const int64_t* h_offsets, const double* h_t, const double* h_logp, int32_t N,
                           double t0, double t1, void* h_coeffs_or_null, void* h_sigma_or_null, void* h_R,
                           int32_t* N_used, void* stream) {
  mm_status r = check_plan(p);
  if (r != MM_OK) return r;
  if (!h_offsets || !h_t || !h_logp || !h_R || !p->s_off) return MM_ERR_INVALID_ARG;
  const int D = p->D;
  const int64_t ne = h_offsets[D];
  if (h_offsets[0] != 0 || ne < 0 || ne > p->desc.max_events) return MM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  MM_CUDA(cudaMemcpyAsync(p->s_off, h_offsets, (size_t)(D + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  // Pinned, mapped event buffers are read by the kernels in place: on GB300
  // the host link is coherent and the kernels that read the events (bounds,
  // prep, Nyquist gaps) stream them from host memory at a higher rate than a
  // staging copy, and without a copy ahead of them. Pageable buffers are
  // copied to the plan's staging buffers first.
  const double* dt_ = p->s_t;
  const double* dp_ = p->s_p;
  if (ne > 0) {
    const size_t eb = (size_t)ne * sizeof(double);
    const void* at = mapped_alias(h_t, eb, p->dev);
    const void* ap = at ? mapped_alias(h_logp, eb, p->dev) : nullptr;
    if (at && ap) {
      dt_ = static_cast<const double*>(at);
      dp_ = static_cast<const double*>(ap);
    } else {
      MM_CUDA(cudaMemcpyAsync(p->s_t, h_t, eb, cudaMemcpyHostToDevice, st));
      MM_CUDA(cudaMemcpyAsync(p->s_p, h_logp, eb, cudaMemcpyHostToDevice, st));
    }
  }
  // pinned, mapped Sigma and R buffers are written by the correlation
  // epilogue in place; the coefficients stay in device memory (the
  // contraction reads them back) and are copied out when asked for
  const size_t dd = (size_t)D * D * p->rs;
  void* oR = const_cast<void*>(mapped_alias(h_R, dd, p->dev));
  void* oS = h_sigma_or_null ? const_cast<void*>(mapped_alias(h_sigma_or_null, dd, p->dev)) : nullptr;
  int32_t Nu = 0;
  r = mm_estimate(p, p->s_off, dt_, dp_, N, t0, t1, p->s_coef, oS ? oS : p->s_sigma, oR ? oR : p->s_R, &Nu,
                  stream);
  if (r != MM_OK) {
    cudaStreamSynchronize(st);
    return r;
  }
  if (!oR) MM_CUDA(cudaMemcpyAsync(h_R, p->s_R, dd, cudaMemcpyDeviceToHost, st));
  if (h_sigma_or_null && !oS)
    MM_CUDA(cudaMemcpyAsync(h_sigma_or_null, p->s_sigma, dd, cudaMemcpyDeviceToHost, st));
  if (h_coeffs_or_null)
    MM_CUDA(cudaMemcpyAsync(h_coeffs_or_null, p->s_coef, (size_t)D * (Nu + 1) * p->cs, cudaMemcpyDeviceToHost, st));
  if (N_used) *N_used = Nu;
  // the status word comes back with the results: one synchronisation
  MM_CUDA(cudaMemcpyAsync(p->h_status, p->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  MM_CUDA(cudaStreamSynchronize(st));
  const int f = *p->h_status;
  if (f) {
    // as mm_plan_sync: clear the status
    MM_CUDA(cudaMemsetAsync(p->status, 0, sizeof(int), st));
    MM_CUDA(cudaStreamSynchronize(st));
  }
  return flags_to_status(f);
}

mm_status mm_autotune(mm_plan p, const int64_t* d_offsets, const double* d_t, const double* d_logp, int32_t N,
                      double t0, double t1, void* d_coeffs, int32_t reps, void* stream) {
  mm_status r = check_plan(p);
  if (r != MM_OK) return r;
  if (!d_offsets || !d_t || !d_logp || !d_coeffs || N < 1 || N > p->desc.N_max) return MM_ERR_INVALID_ARG;
  if (reps < 1) reps = 1;
  cudaStream_t st = (cudaStream_t)stream;
  const bool prof = p->prof;
  p->prof = false;
  struct Cand { int algo, tile, lgc, rb, fft, split, maxr, poly = 1, perm = -1; };
  std::vector<Cand> cands;
  const int tmax = spread_max_tile(p->fp64);
  if (!p->fp64) {
    for (int split : {1, 3})  // 3: two CTAs per asset as a cluster
      for (int maxr : {16, 32}) {
        for (int tile : {tmax / 4, tmax / 2, tmax}) cands.push_back({0, tile, -1, -1, 0, split, maxr, 1});
        if (split == 1) cands.push_back({0, tmax / 2, -1, -1, 0, split, maxr, 1, 1});
        for (int tile : {tmax / 4, tmax / 2}) cands.push_back({0, tile, -1, -1, 0, split, maxr, 0});
        for (int tile : {tmax / 2, tmax}) cands.push_back({1, tile, -1, -1, 0, split, maxr, 1});
        cands.push_back({2, tmax, -1, -1, 0, split, maxr, 1});  // the resident row
      }
  }
  for (int tile : {tmax / 4, tmax / 2, tmax})
    for (int lgc : {3, 4, 5})
      for (int rb : {4, 8, 16}) cands.push_back({0, tile, lgc, rb, 1, -1, -1});
  for (int tile : {tmax / 2, tmax}) cands.push_back({1, tile, 4, 8, 1, -1, -1});
  for (int lgc : {3, 4})
    for (int rb : {4, 8}) cands.push_back({2, tmax, lgc, rb, 1, -1, -1});
  cudaEvent_t e0, e1;
  MM_CUDA(cudaEventCreate(&e0));
  MM_CUDA(cudaEventCreate(&e1));
  float best = 3.0e38f;
  Cand bestc{-1, -1, -1, -1, -1, -1, -1, -1, -1};
  const Cand saved{p->tune_algo, p->tune_tile, p->tune_lgcols, p->tune_rowblk, p->tune_fft, p->tune_split,
                   p->tune_maxr, p->tune_poly, p->tune_perm};
  for (const Cand& c : cands) {
    p->tune_algo = c.algo;
    p->tune_tile = c.tile;
    p->tune_lgcols = c.lgc;
    p->tune_rowblk = c.rb;
    p->tune_fft = c.fft;
    p->tune_split = c.split;
    p->tune_maxr = c.maxr;
    p->tune_poly = c.poly;
    p->tune_perm = c.perm;
    p->cfg_N = -1;  // force reconfiguration
    if (configure(p, N) != MM_OK) continue;
    if (c.algo == 2 && !p->sp.fused && !p->res_sub) continue;  // no fused variant fits
    if (c.fft == 0 && (!p->use_afft || p->afft.split != (c.split == 3 ? 2 : c.split) ||
                       p->afft.pair != (c.split == 3 ? 1 : 0)))
      continue;  // not available
    // warm-up (also builds the tables for N)
    if (coeffs_impl(p, d_offsets, d_t, d_logp, N, t0, t1, d_coeffs, nullptr, st) != MM_OK) continue;
    cudaEventRecord(e0, st);
    bool ok = true;
    for (int i = 0; i < reps && ok; ++i)
      ok = coeffs_impl(p, d_offsets, d_t, d_logp, N, t0, t1, d_coeffs, nullptr, st) == MM_OK;
    cudaEventRecord(e1, st);
    if (!ok || cudaEventSynchronize(e1) != cudaSuccess) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    if (ms < best) {
      best = ms;
      bestc = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p->prof = prof;
  if (bestc.algo < 0) {
    p->tune_algo = saved.algo;
    p->tune_tile = saved.tile;
    p->tune_lgcols = saved.lgc;
    p->tune_rowblk = saved.rb;
    p->tune_fft = saved.fft;
    p->tune_split = saved.split;
    p->tune_maxr = saved.maxr;
    p->tune_poly = saved.poly;
    p->tune_perm = saved.perm;
    p->cfg_N = -1;
    cudaGetLastError();
    return MM_ERR_CUDA;
  }
  p->tune_algo = bestc.algo;
  p->tune_tile = bestc.tile;
  p->tune_lgcols = bestc.lgc;
  p->tune_rowblk = bestc.rb;
  p->tune_fft = bestc.fft;
  p->tune_split = bestc.split;
  p->tune_maxr = bestc.maxr;
  p->tune_poly = bestc.poly;
  p->tune_perm = bestc.perm;
  p->tune_ms = best;
  p->cfg_N = -1;
  return configure(p, N);
}

mm_status mm_nyquist(mm_plan p, const int64_t* d_offsets, const double* d_t, double t0, double t1, int32_t* N_out,
                     void* stream) {
  mm_status r = check_plan(p);
  if (r != MM_OK) return r;
  if (!d_offsets || !d_t || !N_out) return MM_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  p->last = st;
  {
    StageScope sc(p, MM_STAGE_PREP, st);
    MM_CUDA(launch_bounds(d_offsets, d_t, p->D, p->gsize, p->desc.max_events, t0, t1, 0, p->bounds, p->status,
                          nullptr, st));
  }
  {
    StageScope sc(p, MM_STAGE_PREP, st, 2);
    MM_CUDA(launch_min_gap(d_offsets, d_t, p->D, p->bounds, p->gapbits, p->status + 2, p->status, st));
  }
  int hv[3];
  MM_CUDA(cudaMemcpyAsync(hv, p->status, sizeof(hv), cudaMemcpyDeviceToHost, st));
  MM_CUDA(cudaStreamSynchronize(st));
  if (hv[0] & (ST_DUPLICATE | ST_UNSORTED)) {
    int z = 0;
    cudaMemcpy(p->status, &z, sizeof(int), cudaMemcpyHostToDevice);
    return flags_to_status(hv[0]);
  }
  if (hv[1]) return hv[0] ? flags_to_status(hv[0]) : MM_ERR_INVALID_ARG;
  if (hv[2] < 0) return MM_ERR_CUTOFF;
  *N_out = hv[2];
  return MM_OK;
}

mm_status mm_plan_sync(mm_plan p) {
  mm_status r = check_plan(p);
  if (r != MM_OK) return r;
  if (p->last) MM_CUDA(cudaStreamSynchronize(p->last));
  else MM_CUDA(cudaDeviceSynchronize());
  int f = 0;
  MM_CUDA(cudaMemcpy(&f, p->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (f) MM_CUDA(cudaMemset(p->status, 0, sizeof(int)));
  // a timed-out wait may leave a split FFT's pair words set: clear them
  return flags_to_status(f);
}

mm_status mm_plan_set_wait_limit(mm_plan p, int64_t ns) {
  mm_status r = check_plan(p);
  if (r != MM_OK) return r;
  p->wait_ns = ns >= 0 ? (uint64_t)ns : kDefaultWaitNs;
  p->cfg_gen += 1;  // captured graphs hold the old limit
  return MM_OK;
}

mm_status mm_plan_set_graphs(mm_plan p, int32_t on) {
  mm_status r = check_plan(p);
  if (r != MM_OK) return r;
  if (on != 0 && on != 1) return MM_ERR_INVALID_ARG;
  p->graphs = on == 1;
  return MM_OK;
}

mm_status mm_plan_get_info(mm_plan p, mm_plan_info* info) {
  if (!p || !info) return MM_ERR_INVALID_ARG;
  memset(info, 0, sizeof(*info));
  info->msp = p->msp;
  info->N = p->cfg_N;
  info->Mr = p->Mr;
  info->fft_P = p->fft.P;
  info->fft_Q = p->fft.Q;
  info->workspace_bytes = p->workspace;
  info->launches = p->launches;
  info->gram_splits = p->gram.splits;
  info->spread_algo = (p->sp.fused || p->res_sub > 0) ? 3 : (p->sp.algo == 1 ? 2 : 1);
  info->res_sub = p->res_sub;
  info->spread_poly = p->poly_ok ? 1 : 0;
  info->spread_tile = p->sp.tile;
  info->fft_lg_cols = p->fft.lg_cols;
  info->fft_rowblk = p->fft.rowblk;
  info->tuned_ms = p->tune_ms;
  info->fft_algo = p->use_afft ? 0 : 1;
  info->fft_passes = p->use_afft ? p->afft.npass : 0;
  info->fft_split = p->use_afft ? (p->afft.pair ? 3 : 1) : 0;
  info->graphs = p->graphs ? 1 : 0;
  info->graph_launches = p->graph_launches;
  info->gram_algo = p->gram_used;
  for (int q = 0; q < 4; ++q) info->fft_radix[q] = p->use_afft && q < p->afft.npass ? p->afft.rad[q] : 0;
  return MM_OK;
}

mm_status mm_profile_enable(mm_plan p, int32_t on) {
  if (!p) return MM_ERR_INVALID_ARG;
  p->prof = on != 0;
  return MM_OK;
}

mm_status mm_profile_read(mm_plan p, double* ms, int64_t* launches, int32_t reset) {
  if (!p) return MM_ERR_INVALID_ARG;
  for (auto& e : p->pending) {
    float v = 0.f;
    if (cudaEventSynchronize(e.b) == cudaSuccess && cudaEventElapsedTime(&v, e.a, e.b) == cudaSuccess)
      p->ms[e.stage] += v;
    p->pool.push_back(e.a);
    p->pool.push_back(e.b);
  }
  p->pending.clear();
  for (int i = 0; i < MM_NUM_STAGES; ++i) {
    if (ms) ms[i] = p->ms[i];
    if (launches) launches[i] = p->nl[i];
  }
  if (reset) {
    for (int i = 0; i < MM_NUM_STAGES; ++i) {
      p->ms[i] = 0;
      p->nl[i] = 0;
    }
  }
  cudaGetLastError();
  return MM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ internal
namespace mmgpu {

mm_status plan_create_no_staging(const mm_plan_desc* desc, mm_plan* out) {
  if (!desc) return MM_ERR_INVALID_ARG;
  return plan_create_impl(desc, desc->D > 0 ? desc->D : 1, false, out, false);
}

mm_status plan_set_active_assets(mm_plan p, int D) {
  if (!p || D < 1 || D > p->desc.D || p->G != 1) return MM_ERR_INVALID_ARG;
  p->D = D;
  p->gsize = D;
  return MM_OK;
}

int* plan_status_word(mm_plan p) { return p ? p->status : nullptr; }

mm_status plan_flags_to_status(int flags) { return flags_to_status(flags); }

}  // namespace mmgpu

// ------------------------------------------------------------------ batch
struct mm_batch_s {
  mm_batch_desc desc{};
  mm_plan p = nullptr;
  void* coef = nullptr;           // [reps * D][N + 1] complex64 of the last call
  int ld = 0;
  int* d_cut = nullptr;           // cutoffs of the captured sweep (device)
  std::vector<int> cut;
  cudaStream_t cap = nullptr;     // capture stream
  cudaStream_t last = nullptr;    // caller's stream of the last call
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  const void* key[5] = {};        // inputs and outputs the graph was captured with
  int key_cfg = -1;               // plan configuration generation of the graph
  int cfg_gen = 0;
  int64_t graph_launches = 0;
  int captures = 0;
  int kernels = 0;
};

namespace {

void batch_drop_graph(mm_batch b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// Coefficients of every problem at the sweep's largest cutoff, then the
// prefix-weighted sweep contraction, enqueued on st.
mm_status batch_enqueue(mm_batch b, const int64_t* off, const double* t, const double* logp, int N, void* sigma,
                        void* R, cudaStream_t st) {
  mm_plan p = b->p;
  mm_status r = coeffs_impl(p, off, t, logp, N, 0.0, 0.0, b->coef, nullptr, st);
  if (r != MM_OK) return r;
  StageScope sc(p, MM_STAGE_GRAM, st);
  const int grid = std::max(1, std::min(p->G, 2 * kSMs));
  MM_CUDA(launch_epps(b->desc.D, b->desc.basis == MM_BASIS_FEJER, p->fp64, b->coef, N + 1, b->d_cut,
                      (int)b->cut.size(), p->G, sigma, R, p->status, grid, st));
  return MM_OK;
}

}  // namespace

extern "C" {

mm_status mm_batch_create(const mm_batch_desc* desc, mm_batch* out) {
  if (!out) return MM_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc) return MM_ERR_INVALID_ARG;
  const mm_batch_desc& d = *desc;
  if (d.reps < 1 || d.D < 1 || d.N_max < 1 || d.max_events < 0 || d.reserved0 != 0) return MM_ERR_INVALID_ARG;
  for (int i = 0; i < 4; ++i)
    if (d.reserved[i] != 0) return MM_ERR_INVALID_ARG;
  if (d.spread_algo < 0 || d.spread_algo > 3) return MM_ERR_INVALID_ARG;
  if (d.prec < MM_PREC_FP64 || d.prec > MM_PREC_MIXED_3XTF32) return MM_ERR_INVALID_ARG;
  if (d.D > epps_max_assets()) return MM_ERR_UNSUPPORTED;
  if ((int64_t)d.reps * d.D > (int64_t)1 << 30) return MM_ERR_UNSUPPORTED;
  mm_plan_desc pd{};
  pd.D = d.reps * d.D;
  pd.N_max = d.N_max;
  pd.max_events = d.max_events;
  pd.tol = d.tol;
  pd.kernel = d.kernel;
  pd.basis = d.basis;
  pd.prec = d.prec;
  pd.spread_algo = d.spread_algo;
  mm_batch b = new mm_batch_s();
  b->desc = d;
  mm_status r = plan_create_impl(&pd, d.D, true, &b->p);
  if (r != MM_OK) {
    delete b;
    return r;
  }
  const size_t coef_bytes = (size_t)pd.D * ((size_t)d.N_max + 1) * (d.prec == MM_PREC_FP64 ? 16 : 8);
  if (dalloc(b->p, &b->coef, coef_bytes) != MM_OK || dalloc(b->p, (void**)&b->d_cut, kMaxCutoffs * sizeof(int)) != MM_OK ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    if (b->coef) cudaFree(b->coef);
    if (b->d_cut) cudaFree(b->d_cut);
    mm_destroy(b->p);
    delete b;
    cudaGetLastError();
    return MM_ERR_OOM;
  }
  *out = b;
  return MM_OK;
}

mm_status mm_batch_destroy(mm_batch b) {
  if (!b) return MM_ERR_INVALID_ARG;
  if (check_plan(b->p) == MM_OK) cudaDeviceSynchronize();
  batch_drop_graph(b);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->coef) cudaFree(b->coef);
  if (b->d_cut) cudaFree(b->d_cut);
  mm_destroy(b->p);
  delete b;
  return MM_OK;
}

mm_status mm_batch_epps(mm_batch b, const int64_t* d_offsets, const double* d_t, const double* d_logp,
                        const int32_t* h_cutoffs, int32_t n_cutoffs, void* d_sigma_or_null, void* d_R, void* stream) {
  if (!b) return MM_ERR_INVALID_ARG;
  mm_plan p = b->p;
  mm_status r = check_plan(p);
  if (r != MM_OK) return r;
  if (!d_offsets || !d_t || !d_logp || !h_cutoffs || !d_R) return MM_ERR_INVALID_ARG;
  if (n_cutoffs < 1 || n_cutoffs > kMaxCutoffs) return MM_ERR_INVALID_ARG;
  const int lo = b->desc.basis == MM_BASIS_FEJER ? 1 : 0;
  for (int j = 0; j < n_cutoffs; ++j) {
    if (h_cutoffs[j] < lo || h_cutoffs[j] > b->desc.N_max) return MM_ERR_CUTOFF;
    if (j > 0 && h_cutoffs[j] <= h_cutoffs[j - 1]) return MM_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int N = h_cutoffs[n_cutoffs - 1];
  std::vector<int> cut(h_cutoffs, h_cutoffs + n_cutoffs);
  const bool new_cut = cut != b->cut;
  if (new_cut) {
    MM_CUDA(cudaStreamSynchronize(st));  // the previous sweep may still read the old cutoffs
    MM_CUDA(cudaMemcpy(b->d_cut, cut.data(), cut.size() * sizeof(int), cudaMemcpyHostToDevice));
    b->cut = cut;
  }
  const void* key[5] = {d_offsets, d_t, d_logp, d_sigma_or_null, d_R};
  if (p->prof) {
    // per-stage timing needs the eager launch sequence (graph nodes carry no
    // stage events): run without a graph
    b->last = st;
    b->ld = N + 1;
    return batch_enqueue(b, d_offsets, d_t, d_logp, N, d_sigma_or_null, d_R, st);
  }
  bool same = b->exec && !new_cut && b->key_cfg == b->cfg_gen && b->ld == N + 1;
  for (int i = 0; i < 5 && same; ++i) same = key[i] == b->key[i];
  b->last = st;
  if (same) {
    MM_CUDA(cudaGraphLaunch(b->exec, st));
    b->graph_launches += 1;
    p->launches += b->kernels;
    return MM_OK;
  }
  // first call with these inputs: run eagerly (this call's result; it also
  // builds the per-cutoff tables), then capture the same launches into a
  // graph that later calls replay with one launch
  batch_drop_graph(b);
  b->ld = N + 1;
  r = batch_enqueue(b, d_offsets, d_t, d_logp, N, d_sigma_or_null, d_R, st);
  if (r != MM_OK) return r;
  const bool prof = p->prof;
  p->prof = false;
  const int64_t l0 = p->launches;
  MM_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
  r = batch_enqueue(b, d_offsets, d_t, d_logp, N, d_sigma_or_null, d_R, b->cap);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(b->cap, &g);
  p->prof = prof;
  p->last = st;
  b->kernels = (int)(p->launches - l0);
  p->launches = l0;
  if (r != MM_OK || ce != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return r != MM_OK ? r : MM_ERR_CUDA;
  }
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    cudaGraphDestroy(g);
    b->exec = nullptr;
    cudaGetLastError();
    return MM_ERR_CUDA;
  }
  b->graph = g;
  for (int i = 0; i < 5; ++i) b->key[i] = key[i];
  b->key_cfg = b->cfg_gen;
  b->captures += 1;
  return MM_OK;
}

mm_status mm_batch_autotune(mm_batch b, const int64_t* d_offsets, const double* d_t, const double* d_logp,
                            int32_t N, int32_t reps, void* stream) {
  if (!b) return MM_ERR_INVALID_ARG;
  if (N < 1 || N > b->desc.N_max) return MM_ERR_CUTOFF;
  mm_status r = mm_autotune(b->p, d_offsets, d_t, d_logp, N, 0.0, 0.0, b->coef, reps, stream);
  b->cfg_gen += 1;  // a captured graph holds the old configuration
  return r;
}

mm_status mm_batch_coeffs(mm_batch b, const void** d_coeffs, int32_t* ld) {
  if (!b || !d_coeffs || !ld) return MM_ERR_INVALID_ARG;
  *d_coeffs = b->coef;
  *ld = b->ld;
  return MM_OK;
}

mm_status mm_batch_copy_coeffs(mm_batch b, void* d_dst, void* stream) {
  if (!b || !d_dst) return MM_ERR_INVALID_ARG;
  mm_status r = check_plan(b->p);
  if (r != MM_OK) return r;
  MM_CUDA(cudaMemcpyAsync(d_dst, b->coef, (size_t)b->p->desc.D * b->ld * (b->p->fp64 ? 16 : 8), cudaMemcpyDeviceToDevice,
                          (cudaStream_t)stream));
  return MM_OK;
}

mm_status mm_batch_profile_enable(mm_batch b, int32_t on) {
  if (!b) return MM_ERR_INVALID_ARG;
  return mm_profile_enable(b->p, on);
}

mm_status mm_batch_profile_read(mm_batch b, double* ms, int64_t* launches, int32_t reset) {
  if (!b) return MM_ERR_INVALID_ARG;
  return mm_profile_read(b->p, ms, launches, reset);
}

mm_status mm_batch_sync(mm_batch b) {
  if (!b) return MM_ERR_INVALID_ARG;
  b->p->last = b->last;
  return mm_plan_sync(b->p);
}

mm_status mm_batch_get_info(mm_batch b, mm_batch_info* info) {
  if (!b || !info) return MM_ERR_INVALID_ARG;
  memset(info, 0, sizeof(*info));
  mm_plan_info pi;
  mm_plan_get_info(b->p, &pi);
  info->graph_launches = b->graph_launches;
  info->graph_captures = b->captures;
  info->graph_kernels = b->kernels;
  info->launches = pi.launches;
  info->Mr = pi.Mr;
  info->spread_tile = pi.spread_tile;
  info->fft_algo = pi.fft_algo;
  info->fft_split = pi.fft_split;
  info->fft_passes = pi.fft_passes;
  info->tuned_ms = pi.tuned_ms;
  return MM_OK;
}

}  // extern "C"

