// mm_spread.cu -- stage (a) of the hot path: time rescaling and phase
// reduction to grid cells (Algorithm 4), returns (Algorithm 3 step F.3), the
// Nyquist cutoff (Algorithm 2) and the spreading of returns onto the
// oversampled grid (Eq. (12); Algorithms 8-10 step C) with the Gaussian (fast
// Gaussian gridding split, Eq. (17)), Kaiser-Bessel (Eq. (7)) or exponential
// of semicircle (Eq. (9)) kernel.
//
// Phase reduction. GB300 executes float64 at 1/64 of the float32 rate, and a
// float32 cell coordinate loses the phase at large N. The cell coordinate
// u = (t - t0) M_r / span is therefore computed in exact 64-bit fixed point on
// the integer pipes: t_fix = trunc(t 2^F) is read off the float64 bit pattern,
// and u_fix = ((t_fix - t0_fix) S) >> sh = floor(u 2^40) comes from one
// 64 x 64 -> 128-bit product (S, sh fixed per call). b0 and the offset d in
// [0, 1) follow with 2^-40-cell resolution, finer than float64's own rounding
// of u. Returns delta = logp[h+1] - logp[h] use float64 on the FP64 path and
// an exact hi/lo float32 split of each log-price on the mixed path (about 47
// significant bits, so the cancellation in the difference costs nothing).
//
// Spreading design: one block owns a contiguous tile of grid cells of one
// asset and accumulates into shared memory. Because an asset's times are
// sorted, the events whose stencil reaches the tile form at most three index
// ranges (the tile plus its halo, and the halo's periodic images), found by a
// block-parallel search on the same integer u_fix the accumulation uses. No
// global atomics; every shared-memory write is checked against the tile, so
// malformed input cannot write out of bounds.
#include <math.h>

#include "mm_common.cuh"

namespace mmgpu {

// ------------------------------------------------------------ fixed point
// trunc(x * 2^F) as int64 from the bit pattern (integer instructions only).
// Saturates when |x| >= 2^(62-F), which only out-of-window data can reach.
__device__ __forceinline__ long long to_fix(double x, int F) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  const long long M = (b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
  const int s = e - 1075 + F;
  long long v;
  if (e == 0) v = 0;
  else if (s > 9) v = 0x3FFFFFFFFFFFFFFFLL;
  else if (s >= 0) v = M << s;
  else if (s > -64) v = M >> (-s);
  else v = 0;
  return b < 0 ? -v : v;
}

// Per-call fixed-point scale for the cell coordinate (computed by every
// spreading block from the bounds, in float64: a handful of operations).
struct UScale {
  unsigned long long S;
  int sh;
};

__device__ __forceinline__ UScale make_uscale(const Rescale& r, int64_t Mr) {
  // u 2^40 = (t_fix - t0_fix) 2^-F (M_r/span) 2^40 = dt_fix * x with
  // x = (M_r/span) 2^(40-F) = f 2^ex (f in [0.5, 1)): S = f 2^64, sh = 64 - ex
  const double x = ldexp((double)Mr / (r.t1 - r.t0), 40 - r.F);
  int ex;
  const double f = frexp(x, &ex);
  UScale u;
  u.S = (unsigned long long)ldexp(f, 64);
  u.sh = 64 - ex;
  return u;
}

// u_fix = floor(u * 2^40) of an in-window time; times before t0 map to 0.
__device__ __forceinline__ unsigned long long u_fix_of(double t, long long t0_fix, int F, UScale us) {
  const long long d = to_fix(t, F) - t0_fix;
  if (d <= 0) return 0ull;
  const unsigned long long ud = (unsigned long long)d;
  const unsigned long long hi = __umul64hi(ud, us.S);
  const unsigned long long lo = ud * us.S;
  if (us.sh >= 128) return 0ull;
  if (us.sh >= 64) return hi >> (us.sh - 64);
  if (us.sh <= 0) return lo;
  return (lo >> us.sh) | (hi << (64 - us.sh));
}

// Float32 with the value of the 24 leading bits of the non-negative integer
// x (x < 2^63) and its exponent, built from bits (no int-to-float
// conversion, which GB300 issues to its narrow float64 pipe); *rest receives
// the bits below those 24 as an integer of the same scale.
__device__ __forceinline__ float lead24(unsigned long long x, unsigned long long* rest) {
  if (x == 0ull) {
    *rest = 0ull;
    return 0.0f;
  }
  const int lz = __clzll((long long)x);
  const int top = 63 - lz;  // index of the leading bit
  const int sh = top - 23;
  unsigned long long m24;
  if (sh >= 0) {
    m24 = x >> sh;
    *rest = x & ((1ull << sh) - 1ull);
  } else {
    m24 = x << (-sh);
    *rest = 0ull;
  }
  // value = m24 * 2^sh with m24 in [2^23, 2^24)
  return __uint_as_float(((unsigned)(top + 127) << 23) | ((unsigned)m24 & 0x7FFFFFu));
}

// Cell coordinate of the FP32 path: dt = t_fix - t0_fix (exact int64) as a
// float pair (hi + lo, 48 bits) times the scale M_r/span * 2^-F as a float
// pair, with the leading product's rounding error recovered by an FMA. The
// result b0 + d carries about 44 significant bits (u to ~1e-9 cells).
struct UScaleF {
  float s_hi, s_lo;  // (M_r / span) 2^-F = s_hi + s_lo
};

__device__ __forceinline__ UScaleF make_uscale_f(const Rescale& r, int64_t Mr) {
  const double x = ldexp((double)Mr / (r.t1 - r.t0), -r.F);
  UScaleF u;
  u.s_hi = (float)x;
  u.s_lo = (float)(x - (double)u.s_hi);
  return u;
}

__device__ __forceinline__ void cell_f32(long long dt, const UScaleF& us, int& b0, float& d) {
  if (dt <= 0) {
    b0 = 0;
    d = 0.0f;
    return;
  }
  unsigned long long rest;
  const float a_hi = lead24((unsigned long long)dt, &rest);
  unsigned long long rest2;
  const float a_lo = lead24(rest, &rest2);
  const float p = a_hi * us.s_hi;
  const float e = fmaf(a_hi, us.s_hi, -p);  // exact rounding error of p
  const float lo = fmaf(a_hi, us.s_lo, fmaf(a_lo, us.s_hi, e));
  float fb = floorf(p);
  float r = (p - fb) + lo;  // p - fb is exact
  if (r < 0.0f) { r += 1.0f; fb -= 1.0f; }
  if (r >= 1.0f) { r -= 1.0f; fb += 1.0f; }
  b0 = (int)fb;
  d = r;
}

// Exact split of a float64 into float32 hi + lo (hi = x truncated to 24
// significant bits, lo = the remaining 29 bits rounded to 24), by bit
// operations; hi_a - hi_b is exact for nearby values (Sterbenz), so a return
// keeps about 47 significant bits of the log-prices.
__device__ __forceinline__ void split_f64(double x, float& hi, float& lo) {
  const long long b = __double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e < 1023 - 125) {  // |x| < 2^-125 (log-prices this close to 0 are 0)
    hi = 0.0f;
    lo = 0.0f;
    return;
  }
  if (e > 1023 + 127) {  // beyond float range: infinity of the same sign
    hi = __uint_as_float(((unsigned)((unsigned long long)b >> 63) << 31) | 0x7F800000u);
    lo = 0.0f;
    return;
  }
  const unsigned long long m = (unsigned long long)b & 0xFFFFFFFFFFFFFULL;
  const unsigned sign = (unsigned)((unsigned long long)b >> 63) << 31;
  hi = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | (unsigned)(m >> 29));
  // the low 29 bits: their top 23 as an exact float (2^23 + x - 2^23), scaled
  const float r = __uint_as_float(0x4B000000u | (unsigned)((m >> 6) & 0x7FFFFFull)) - 8388608.0f;
  const float l = r * 1.4210854715202004e-14f * __uint_as_float((unsigned)(e - 1023 + 127) << 23);  // 2^-46 2^(e-1023)
  lo = sign ? -l : l;
}

// ------------------------------------------------------------------ bounds
// Validates the CSR offsets, finds t_min / t_max over all assets (Algorithm
// 4) or takes the caller's window, fixes the time fixed-point format and
// writes the per-call gate word (0 = proceed). One block.
__global__ void k_bounds(const int64_t* __restrict__ off, const double* __restrict__ t, int D,
                         int64_t max_events, double w0, double w1, Rescale* rs, int* status) {
  __shared__ double s_lo[256], s_hi[256];
  __shared__ int s_bad;
  int* gate = status + 1;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  // 1) the offsets alone: non-decreasing from 0 up to at most max_events.
  //    Only when all of them hold is any event time read.
  int bad = 0;
  for (int i = threadIdx.x; i < D; i += blockDim.x)
    if (off[i + 1] < off[i]) bad = 1;
  if (threadIdx.x == 0 && (off[0] != 0 || off[D] > max_events)) bad = 1;
  if (bad) atomicOr(&s_bad, 1);
  __syncthreads();
  if (s_bad) {
    if (threadIdx.x == 0) {
      atomicOr(status, ST_BAD_OFFSETS);
      rs->t0 = rs->t1 = 0.0;
      *gate = 1;
    }
    return;
  }
  // 2) t_min / t_max from each asset's first and last event (Algorithm 4)
  const bool window = w1 > w0;
  double lo = INFINITY, hi = -INFINITY;
  int outwin = 0;
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    const int64_t a = off[i], b = off[i + 1];
    if (b > a) {
      const double f = t[a], l = t[b - 1];
      lo = fmin(lo, f);
      hi = fmax(hi, l);
      if (window && (f < w0 || l > w1)) outwin = 1;
    }
  }
  if (outwin) atomicOr(&s_bad, 2);
  s_lo[threadIdx.x] = lo;
  s_hi[threadIdx.x] = hi;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s_lo[threadIdx.x] = fmin(s_lo[threadIdx.x], s_lo[threadIdx.x + w]);
      s_hi[threadIdx.x] = fmax(s_hi[threadIdx.x], s_hi[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double t0 = window ? w0 : s_lo[0];
    const double t1 = window ? w1 : s_hi[0];
    int g = 0;
    if (s_bad & 2) { atomicOr(status, ST_OUT_OF_WINDOW); g = 1; }
    if (!g && !(t1 > t0 && isfinite(t0) && isfinite(t1))) {
      // all assets empty, a single instant, or non-finite times
      if (s_hi[0] >= s_lo[0] || window || isnan(s_lo[0]) || isnan(s_hi[0])) atomicOr(status, ST_SPAN);
      g = 1;
    }
    Rescale r{};
    r.t0 = t0;
    r.t1 = t1;
    if (!g) {
      int ex;
      frexp(fmax(fabs(t0), fabs(t1)), &ex);  // max |t| < 2^ex
      r.F = 62 - (ex + 1);                   // |t_fix| < 2^61
      r.t0_fix = to_fix(t0, r.F);
    }
    *rs = r;
    *gate = g;
  }
}

cudaError_t launch_bounds(const int64_t* off, const double* t, int D, int64_t max_events, double w0,
                          double w1, Rescale* rs, int* status, cudaStream_t s) {
  k_bounds<<<1, 256, 0, s>>>(off, t, D, max_events, w0, w1, rs, status);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ Nyquist
// Algorithm 2: per-asset smallest gap (one block per asset), then
// N = floor(span / (2 max_i gap_i)) = min_i floor(span / (2 gap_i)).
__global__ void k_min_gap(const int64_t* __restrict__ off, const double* __restrict__ t,
                          const int* gate, unsigned long long* gapbits, int* status) {
  __shared__ double s[256];
  if (*gate) return;
  int i = blockIdx.x;
  int64_t a = off[i], b = off[i + 1];
  double g = INFINITY;
  int dup = 0;
  for (int64_t h = a + threadIdx.x; h + 1 < b; h += blockDim.x) {
    double d = t[h + 1] - t[h];
    if (!(d > 0)) dup = (d == 0) ? 1 : 2;
    g = fmin(g, d);
  }
  if (dup == 1) atomicOr(status, ST_DUPLICATE);
  if (dup == 2) atomicOr(status, ST_UNSORTED);
  s[threadIdx.x] = g;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] = fmin(s[threadIdx.x], s[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0 && b - a >= 2 && s[0] > 0 && isfinite(s[0])) {
    // positive doubles order like their bit patterns
    atomicMax(gapbits, (unsigned long long)__double_as_longlong(s[0]));
  }
}

__global__ void k_nyquist_final(const Rescale* rs, const int* gate, const unsigned long long* gapbits, int* nyq,
                                int* status) {
  if (*gate) { *nyq = -1; return; }
  unsigned long long gb = *gapbits;
  if (gb == 0ull) { *nyq = -1; atomicOr(status, ST_CUTOFF); return; }
  double g = __longlong_as_double((long long)gb);
  double span = rs->t1 - rs->t0;
  double v = floor(span / (2.0 * g));
  *nyq = (v > 2147483647.0) ? 2147483647 : (int)v;
}

cudaError_t launch_min_gap(const int64_t* off, const double* t, int D, const Rescale* rs,
                           unsigned long long* gapbits, int* nyq, int* status, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(gapbits, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_min_gap<<<D, 256, 0, s>>>(off, t, status + 1, gapbits, status);
  k_nyquist_final<<<1, 1, 0, s>>>(rs, status + 1, gapbits, nyq, status);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ kernels
template <typename T> struct Fn;
template <> struct Fn<float> {
  static __device__ __forceinline__ float exp_(float x) { return __expf(x); }
  static __device__ __forceinline__ float sqrt_(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }
  static __device__ __forceinline__ float sinh_(float x) { return sinhf(x); }
  static __device__ __forceinline__ float sin_(float x) { return sinf(x); }
};
template <> struct Fn<double> {
  static __device__ __forceinline__ double exp_(double x) { return exp(x); }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double sinh_(double x) { return sinh(x); }
  static __device__ __forceinline__ double sin_(double x) { return sin(x); }
};

// Return of event h (the log-price difference to event h+1).
template <typename T> __device__ __forceinline__ T return_of(double p0, double p1);
template <> __device__ __forceinline__ double return_of<double>(double p0, double p1) { return p1 - p0; }
template <> __device__ __forceinline__ float return_of<float>(double p0, double p1) {
  float h0, l0, h1, l1;
  split_f64(p0, h0, l0);
  split_f64(p1, h1, l1);
  return (h1 - h0) + (l1 - l0);
}

// Integer key with the same order as the float64 values (non-NaN).
__device__ __forceinline__ long long order_key(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}

// Non-finite check from the exponent bits (no float64 instruction).
__device__ __forceinline__ bool finite_bits(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7FF) != 0x7FF;
}

// Kernel value for the signed distance x = k - d (cells) between a grid
// point and a source: Eq. (9) rescaled to half-width M_sp (ES), Eq. (5) as
// exp(-t1 x^2) with t1 of Algorithm 8 (Gaussian), Eq. (7) normalised to
// phi(0) = 1 (Kaiser-Bessel). Each (event, cell) pair costs one evaluation,
// so the Gaussian needs no three-factor split.
template <typename T, int KERNEL>
__device__ __forceinline__ T kernel_value(T x, const SpreadParams& p) {
  if (KERNEL == MM_KERNEL_GAUSS) {
    return Fn<T>::exp_(-(T)p.g_t1 * x * x);
  } else if (KERNEL == MM_KERNEL_ES) {
    const T y = x * (T)p.es_inv_w;
    const T v = (T)1 - y * y;
    return v >= (T)0 ? Fn<T>::exp_((T)p.es_beta * (Fn<T>::sqrt_(v) - (T)1)) : (T)0;
  } else {
    const T b = (T)p.kb_b, ck = (T)(p.kb_inv_phi0 / kPi);
    const T s2 = (T)p.msp * (T)p.msp - x * x;
    if (s2 > (T)0) {
      const T sq = Fn<T>::sqrt_(s2);
      return Fn<T>::sinh_(b * sq) / sq * ck;
    } else if (s2 < (T)0) {
      const T sq = Fn<T>::sqrt_(-s2);
      return Fn<T>::sin_(b * sq) / sq * ck;
    }
    return b * ck;
  }
}

template <typename T> __device__ __forceinline__ T frac_to(unsigned long long frac);
template <> __device__ __forceinline__ float frac_to<float>(unsigned long long frac) {
  return (float)(unsigned)(frac >> (kUFrac - 24)) * 5.9604644775390625e-8f;  // 24 bits * 2^-24
}
template <> __device__ __forceinline__ double frac_to<double>(unsigned long long frac) {
  return (double)frac * 9.094947017729282e-13;  // * 2^-40
}

constexpr int kSpreadThreads = 256;
constexpr int kNoCell = -0x40000000;  // cell of a skipped event (outside every window)

// ------------------------------------------------------------------ prep
// Steps a0 / a1 of the hot path, one thread per event h: the rescaled cell
// coordinate in exact fixed point (Algorithm 4), split into the cell b0 and
// the offset d in [0, 1), and the return delta = logp[h+1] - logp[h]
// (Algorithm 3 step F.3), written once as a compact record (b0, d, delta) in
// event order. Since each asset's times are sorted, its records are sorted
// by cell: that order is the bin sort the spreading kernels search. The
// last event of an asset carries no return and its record is not read.
template <typename T>
__global__ void __launch_bounds__(256) k_prep(const int64_t* __restrict__ off, const double* __restrict__ t,
                                              const double* __restrict__ logp, const Rescale* __restrict__ rsp,
                                              const int* __restrict__ gate, int D, int64_t Mr, int* __restrict__ rb0,
                                              T* __restrict__ rd, T* __restrict__ rv, int* status) {
  __shared__ UScale s_us;
  __shared__ UScaleF s_usf;
  __shared__ Rescale s_rs;
  __shared__ int s_flags;
  if (*gate) return;  // uniform
  if (threadIdx.x == 0) {
    s_rs = *rsp;
    if (sizeof(T) == 8) s_us = make_uscale(s_rs, Mr);
    else s_usf = make_uscale_f(s_rs, Mr);
    s_flags = 0;
  }
  __syncthreads();
  const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ntot = off[D];
  // asset of the block's first event (binary search once per block), then
  // each thread walks forward to its own asset
  __shared__ int s_a0;
  if (threadIdx.x == 0) {
    const int64_t hb = min((int64_t)blockIdx.x * blockDim.x, ntot > 0 ? ntot - 1 : 0);
    int lo = 0, hi = D;  // off[lo] <= hb < off[hi]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (off[mid] <= hb) lo = mid;
      else hi = mid;
    }
    s_a0 = lo;
  }
  __syncthreads();
  int flags = 0;
  if (h < ntot) {
    int lo = s_a0;
    while (lo + 1 < D && off[lo + 1] <= h) ++lo;
    if (h + 1 < off[lo + 1]) {
      const Rescale rs = s_rs;
      const double th = t[h], tn = t[h + 1];
      const double p0 = logp[h], p1 = logp[h + 1];
      const long long kh = order_key(th), kn = order_key(tn);
      if (!(kh < kn)) flags |= (kh == kn) ? ST_DUPLICATE : ST_UNSORTED;
      int b0 = kNoCell;
      T d = (T)0, v = (T)0;
      if (!(finite_bits(th) && finite_bits(p0) && finite_bits(p1))) {
        flags |= ST_NONFINITE;
      } else {
        const long long dt = to_fix(th, rs.F) - rs.t0_fix;
        int cb;
        T cd;
        if (sizeof(T) == 8) {
          const unsigned long long uf = u_fix_of(th, rs.t0_fix, rs.F, s_us);
          cb = (int)(uf >> kUFrac);
          cd = frac_to<T>(uf & ((1ull << kUFrac) - 1));
        } else {
          float fd;
          cell_f32(dt, s_usf, cb, fd);
          cd = (T)fd;
        }
        if (dt < 0 || cb > Mr || (cb == Mr && cd > (T)0)) {
          flags |= ST_OUT_OF_WINDOW;
        } else {
          b0 = cb;
          d = cd;
          v = return_of<T>(p0, p1);
        }
      }
      rb0[h] = b0;
      rd[h] = d;
      rv[h] = v;
    }
  }
  if (flags) atomicOr(&s_flags, flags);
  __syncthreads();
  if (threadIdx.x == 0 && s_flags) atomicOr(status, s_flags);
}

template <typename T>
static cudaError_t launch_prep_t(const int64_t* off, const double* t, const double* logp, const Rescale* rs,
                                 int D, int64_t Mr, int64_t max_events, int* rb0, T* rd, T* rv, int* status,
                                 cudaStream_t s) {
  if (max_events <= 0) return cudaSuccess;
  const int64_t blocks = (max_events + 255) / 256;
  k_prep<T><<<(unsigned)blocks, 256, 0, s>>>(off, t, logp, rs, status + 1, D, Mr, rb0, rd, rv, status);
  return cudaGetLastError();
}

cudaError_t launch_prep_f32(const int64_t* off, const double* t, const double* logp, const Rescale* rs, int D,
                            int64_t Mr, int64_t max_events, int* rb0, void* rd, void* rv, int* status,
                            cudaStream_t s) {
  return launch_prep_t<float>(off, t, logp, rs, D, Mr, max_events, rb0, (float*)rd, (float*)rv, status, s);
}
cudaError_t launch_prep_f64(const int64_t* off, const double* t, const double* logp, const Rescale* rs, int D,
                            int64_t Mr, int64_t max_events, int* rb0, void* rd, void* rv, int* status,
                            cudaStream_t s) {
  return launch_prep_t<double>(off, t, logp, rs, D, Mr, max_events, rb0, (double*)rd, (double*)rv, status, s);
}

// ------------------------------------------------------------------ spread
template <typename T> struct EvChunk { static constexpr int n = 2048; };

// Event ranges of a tile [L, L + Tlen): image m = r - 1 (r = 0, 1, 2) holds
// the returns with b0 in [L - khi + m M_r, L + Tlen - klo + m M_r); taken in
// the order r = 2, 1, 0 their tile-relative positions p = b0 - L - m M_r are
// sorted. An event may sit in two images (a small grid seen through both of
// its periodic copies); each image feeds different cells.
struct TileRanges {
  int64_t lo[3], hi[3];
  int64_t n2, n1, n0;
};

// First index h in [e0, e1) with key[h] >= x (e1 if none), by one warp: each
// step the 32 lanes sample the bracket at 32 evenly spaced points and a
// ballot keeps the segment where the predicate turns true (32-ary search).
__device__ __forceinline__ int64_t warp_first_ge(const int* __restrict__ key, int64_t e0, int64_t e1, long long x) {
  const int lane = threadIdx.x & 31;
  int64_t lo = e0, hi = e1;  // answer in [lo, hi]
  for (int it = 0; it < 16 && hi > lo; ++it) {
    const int64_t len = hi - lo;
    const int64_t stride = (len + 31) / 32;
    const int64_t o = (int64_t)lane * stride;
    const bool below = o < len && (long long)key[lo + o] < x;
    const unsigned bal = __ballot_sync(0xffffffffu, below);
    const int c = __popc(bal);  // samples below x (a prefix when key is sorted)
    if (c == 0) {
      hi = lo;
    } else {
      const int64_t nlo = lo + (int64_t)(c - 1) * stride + 1;
      const int64_t nhi = min(lo + (int64_t)c * stride, hi);
      lo = min(nlo, nhi);
      hi = nhi;
    }
  }
  return lo;
}

__device__ __forceinline__ void tile_ranges(const int64_t* __restrict__ off, const int* __restrict__ rb0,
                                            const SpreadParams& p, int a, int64_t L, int Tlen, TileRanges& tr) {
  __shared__ int64_t s_res[6];
  const int64_t e0 = off[a], eend = off[a + 1];
  const int64_t e1 = eend > e0 ? eend - 1 : e0;  // returns live at h in [e0, e1)
  const int w = threadIdx.x >> 5;
  if (w < 6) {
    // warp w: threshold w of image m = w/2 - 1 (lower bound for even w)
    const int m = w / 2 - 1;
    long long A = L - p.khi + (long long)m * p.Mr;
    long long B = L + Tlen - p.klo + (long long)m * p.Mr;
    if (A < 0) A = 0;
    if (B > p.Mr + 1) B = p.Mr + 1;
    int64_t r = 0;
    if (A < B) r = warp_first_ge(rb0, e0, e1, (w & 1) ? B : A);
    else r = -1;  // empty image
    if ((threadIdx.x & 31) == 0) s_res[w] = r;
  }
  __syncthreads();
  for (int r = 0; r < 3; ++r) {
    const bool empty = s_res[2 * r] < 0;
    tr.lo[r] = empty ? 0 : s_res[2 * r];
    tr.hi[r] = empty ? 0 : s_res[2 * r + 1];
  }
  tr.n2 = tr.hi[2] - tr.lo[2];
  tr.n1 = tr.hi[1] - tr.lo[1];
  tr.n0 = tr.hi[0] - tr.lo[0];
}

// Record qi of the concatenation (r = 2, 1, 0) with its tile-relative position.
template <typename T>
__device__ __forceinline__ void load_record(const int* __restrict__ rb0, const T* __restrict__ rd,
                                            const T* __restrict__ rv, const SpreadParams& p, const TileRanges& tr,
                                            int64_t L, int64_t qi, int& pos, T& d, T& v) {
  int64_t h;
  long long shift;  // p = b0 - L - m M_r
  if (qi < tr.n2) { h = tr.lo[2] + qi; shift = -(long long)p.Mr; }
  else if (qi < tr.n2 + tr.n1) { h = tr.lo[1] + (qi - tr.n2); shift = 0; }
  else { h = tr.lo[0] + (qi - tr.n2 - tr.n1); shift = p.Mr; }
  const int b0 = rb0[h];
  pos = b0 == kNoCell ? kNoCell : (int)(b0 - L + shift);
  d = rd[h];
  v = rv[h];
}

// Gather spreading (Eq. (12)): thread t owns cells c = t CPT .. t CPT + CPT-1
// of the tile and sums, in registers, delta_e phi(c - p_e - d_e) over the
// events with c - p_e in [klo, khi], a sliding window over the sorted
// positions of each event chunk (no atomics, deterministic).
template <typename T, int KERNEL, int CPT>
__global__ void __launch_bounds__(kSpreadThreads) k_spread_gather(const int64_t* __restrict__ off,
                                                                 const int* __restrict__ rb0,
                                                                 const T* __restrict__ rd, const T* __restrict__ rv,
                                                                 const int* __restrict__ gate, SpreadParams p,
                                                                 T* __restrict__ grid) {
  constexpr int EC = EvChunk<T>::n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* ev_p = reinterpret_cast<int*>(smem_raw);
  T* ev_d = reinterpret_cast<T*>(smem_raw + EC * sizeof(int));
  T* ev_v = ev_d + EC;
  if (*gate) return;  // uniform: the whole block leaves
  const int a = blockIdx.y;
  const int64_t L = (int64_t)blockIdx.x * p.tile;
  const int Tlen = (int)min((int64_t)p.tile, p.Mr - L);
  TileRanges tr;
  tile_ranges(off, rb0, p, a, L, Tlen, tr);
  const int64_t ntot = tr.n2 + tr.n1 + tr.n0;
  const int c0 = threadIdx.x * CPT;
  T acc[CPT];
#pragma unroll
  for (int q = 0; q < CPT; ++q) acc[q] = (T)0;
  for (int64_t cs = 0; cs < ntot; cs += EC) {
    const int n = (int)min((int64_t)EC, ntot - cs);
    for (int i = threadIdx.x; i < n; i += kSpreadThreads) load_record<T>(rb0, rd, rv, p, tr, L, cs + i, ev_p[i], ev_d[i], ev_v[i]);
    __syncthreads();
    if (c0 < Tlen) {
      int lo = 0, hi = n;
      const int want = c0 - p.khi;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ev_p[mid] < want) lo = mid + 1;
        else hi = mid;
      }
#pragma unroll
      for (int q = 0; q < CPT; ++q) {
        const int c = c0 + q;
        while (lo < n && ev_p[lo] < c - p.khi) ++lo;
        T sum = (T)0;
        for (int e = lo; e < n; ++e) {
          const int k = c - ev_p[e];
          if (k < p.klo) break;
          sum += ev_v[e] * kernel_value<T, KERNEL>((T)k - ev_d[e], p);
        }
        acc[q] += sum;
      }
    }
    __syncthreads();
  }
  T* g = grid + (int64_t)a * p.Mr + L;
#pragma unroll
  for (int q = 0; q < CPT; ++q)
    if (c0 + q < Tlen) g[c0 + q] = acc[q];
}

// Scatter spreading (Eq. (12)): event records are staged per chunk in shared
// memory, then each thread adds one event's whole stencil into the shared-
// memory tile (at most KW points, unrolled; 32-bit indices). Lanes of a warp
// take consecutive events, so their cells rarely coincide.
template <typename T, int KERNEL, int KW>
__global__ void __launch_bounds__(kSpreadThreads) k_spread_scatter(const int64_t* __restrict__ off,
                                                                  const int* __restrict__ rb0,
                                                                  const T* __restrict__ rd, const T* __restrict__ rv,
                                                                  const int* __restrict__ gate, SpreadParams p,
                                                                  T* __restrict__ grid) {
  constexpr int EC = EvChunk<T>::n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* ev_p = reinterpret_cast<int*>(smem_raw);
  T* ev_d = reinterpret_cast<T*>(smem_raw + EC * sizeof(int));
  T* ev_v = ev_d + EC;
  T* tile = ev_v + EC;
  if (*gate) return;  // uniform: the whole block leaves
  const int a = blockIdx.y;
  const int64_t L = (int64_t)blockIdx.x * p.tile;
  const int Tlen = (int)min((int64_t)p.tile, p.Mr - L);
  {
    float4* t4 = reinterpret_cast<float4*>(tile);
    const int n4 = (int)(((size_t)Tlen * sizeof(T) + 15) / 16);
    for (int c = threadIdx.x; c < n4; c += kSpreadThreads) t4[c] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  TileRanges tr;
  tile_ranges(off, rb0, p, a, L, Tlen, tr);
  const int64_t ntot = tr.n2 + tr.n1 + tr.n0;
  const int klo = p.klo, nk = p.khi - p.klo + 1;
  for (int64_t cs = 0; cs < ntot; cs += EC) {
    const int n = (int)min((int64_t)EC, ntot - cs);
    for (int i = threadIdx.x; i < n; i += kSpreadThreads) load_record<T>(rb0, rd, rv, p, tr, L, cs + i, ev_p[i], ev_d[i], ev_v[i]);
    __syncthreads();
    for (int e = threadIdx.x; e < n; e += kSpreadThreads) {
      const int pe = ev_p[e];
      const T de = ev_d[e], ve = ev_v[e];
      T x = (T)klo - de;
#pragma unroll
      for (int j = 0; j < KW; ++j) {
        if (j >= nk) break;
        const unsigned c = (unsigned)(pe + klo + j);
        if (c < (unsigned)Tlen) atomicAdd(tile + c, ve * kernel_value<T, KERNEL>(x, p));
        x += (T)1;
      }
    }
    __syncthreads();
  }
  T* g = grid + (int64_t)a * p.Mr + L;
  // rows of M_r (even) cells start 8-byte aligned; tiles are multiples of 4 cells
  if (((reinterpret_cast<uintptr_t>(g) & 15) == 0) && (Tlen * sizeof(T)) % 16 == 0) {
    const float4* t4 = reinterpret_cast<const float4*>(tile);
    float4* g4 = reinterpret_cast<float4*>(g);
    const int n4 = (int)((size_t)Tlen * sizeof(T) / 16);
    for (int c = threadIdx.x; c < n4; c += kSpreadThreads) g4[c] = t4[c];
  } else {
    for (int c = threadIdx.x; c < Tlen; c += kSpreadThreads) g[c] = tile[c];
  }
}

template <typename T, int K>
static cudaError_t launch_variant(bool gather, int nk, dim3 grd, const int64_t* off, const int* rb0, const T* rd,
                                  const T* rv, const int* gate, const SpreadParams& p, T* grid, cudaStream_t s) {
  constexpr int CPT = sizeof(T) == 4 ? 16 : 8;
  const size_t ev_bytes = (size_t)EvChunk<T>::n * (sizeof(int) + 2 * sizeof(T));
  auto go = [&](auto fn, size_t smem) -> cudaError_t {
    if (smem > 48 * 1024) {
      cudaError_t r = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (r != cudaSuccess) return r;
    }
    fn<<<grd, kSpreadThreads, smem, s>>>(off, rb0, rd, rv, gate, p, grid);
    return cudaGetLastError();
  };
  if (gather) return go(k_spread_gather<T, K, CPT>, ev_bytes);
  const size_t smem = ev_bytes + (size_t)p.tile * sizeof(T);
  if (nk <= 8) return go(k_spread_scatter<T, K, 8>, smem);
  if (nk <= 16) return go(k_spread_scatter<T, K, 16>, smem);
  if (nk <= 32) return go(k_spread_scatter<T, K, 32>, smem);
  return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t launch_spread_t(const int64_t* off, const int* rb0, const void* rd, const void* rv,
                                   const SpreadParams& p, T* grid, const int* status, cudaStream_t s) {
  constexpr int CPT = sizeof(T) == 4 ? 16 : 8;
  if (p.tile > kSpreadThreads * CPT) return cudaErrorInvalidValue;
  dim3 grd(p.ntiles, p.D);
  const int* gate = status + 1;
  const bool gather = p.algo == 1;
  const int nk = p.khi - p.klo + 1;
  const T* d = (const T*)rd;
  const T* v = (const T*)rv;
  switch (p.kernel) {
    case MM_KERNEL_GAUSS: return launch_variant<T, MM_KERNEL_GAUSS>(gather, nk, grd, off, rb0, d, v, gate, p, grid, s);
    case MM_KERNEL_KB: return launch_variant<T, MM_KERNEL_KB>(gather, nk, grd, off, rb0, d, v, gate, p, grid, s);
    case MM_KERNEL_ES: return launch_variant<T, MM_KERNEL_ES>(gather, nk, grd, off, rb0, d, v, gate, p, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

int spread_max_tile(bool fp64) { return kSpreadThreads * (fp64 ? 8 : 16); }

cudaError_t launch_spread_f32(const int64_t* off, const int* rb0, const void* rd, const void* rv,
                              const SpreadParams& p, float* grid, const int* status, cudaStream_t s) {
  return launch_spread_t<float>(off, rb0, rd, rv, p, grid, status, s);
}
cudaError_t launch_spread_f64(const int64_t* off, const int* rb0, const void* rd, const void* rv,
                              const SpreadParams& p, double* grid, const int* status, cudaStream_t s) {
  return launch_spread_t<double>(off, rb0, rd, rv, p, grid, status, s);
}

}  // namespace mmgpu
