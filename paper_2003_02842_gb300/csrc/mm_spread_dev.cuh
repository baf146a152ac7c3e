// mm_spread_dev.cuh -- device helpers of stage (a): fixed-point time
// rescaling (Algorithm 4), returns (Algorithm 3 step F.3) and the averaging
// kernels of Sec. 2.2.5, shared by the multi-kernel and the fused paths.
#pragma once

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

// Fixed-point time format and cell scales of one problem of a batch.
struct GroupScale {
  UScale us;
  UScaleF usf;
  long long t0_fix;
  int F;
};

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

}  // namespace mmgpu
