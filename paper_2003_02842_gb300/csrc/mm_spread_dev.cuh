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

// ------------------------------------------------ spreading tiles
constexpr int kNoCell = -0x40000000;  // cell of a skipped event (outside every window)

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

// Shared-memory integer reduction without a returned value.
__device__ __forceinline__ void red_shared_add(uint32_t addr, int v) {
  asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// round(y) for |y| < 2^22 as y + 1.5 2^23 (float spacing 1 there): the
// integer is the result's bits minus those of 1.5 2^23.
constexpr float kRoundMagic = 12582912.0f;  // 1.5 * 2^23
constexpr int kRoundMagicBits = 0x4B400000;

// The cells of a tile one CTA accumulates: all of them (one CTA per grid
// row or tile), or, for the CTA c of a cluster pair that holds the complex
// points z[2m + c] of a row (cells 4m + 2c and 4m + 2c + 1), its own half,
// packed two cells per point (the tile starts at a multiple of 4).
struct AllCells {
  static constexpr bool kAll = true;
  __device__ __forceinline__ bool own(int) const { return true; }
  __device__ __forceinline__ uint32_t slot(int q) const { return (uint32_t)q; }
};
struct PairCells {
  static constexpr bool kAll = false;
  unsigned c;
  __device__ __forceinline__ bool own(int q) const { return (unsigned)((q >> 1) & 1) == c; }
  __device__ __forceinline__ uint32_t slot(int q) const { return (uint32_t)((q >> 2) * 2 + (q & 1)); }
};

// Scales of the exact hi/lo integer accumulation of one tile, from the sum
// B and the maximum V of |v| over its n records: every tap's x = v phi 2^eh
// has |x| < 2^21 and a cell's hi sum stays below 2^31 with
// eh = min(29 - ex(B), 21 - ex(V)); the residue (x - round(x)) 2^k, with
// k = min(20, 30 - bitlen(n)), keeps a cell's lo sum below 2^30.
struct TileScales {
  float scale, kscale, inv_h, inv_l;
};
template <int NTH>
__device__ __forceinline__ TileScales tile_scales(float part, float pmax, int64_t n, float* s_sum, float* s_max) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    part += __shfl_xor_sync(0xffffffffu, part, o);
    pmax = fmaxf(pmax, __shfl_xor_sync(0xffffffffu, pmax, o));
  }
  if ((threadIdx.x & 31) == 0) {
    s_sum[threadIdx.x >> 5] = part;
    s_max[threadIdx.x >> 5] = pmax;
  }
  __syncthreads();
  float B = 0.f, V = 0.f;
#pragma unroll
  for (int w = 0; w < NTH / 32; ++w) {
    B += s_sum[w];
    V = fmaxf(V, s_max[w]);
  }
  int eh = 0, k = 0;
  if (B > 0.f && B < 3.0e38f) {
    int exB, exV;
    frexpf(B, &exB);  // B < 2^exB
    frexpf(V, &exV);  // V < 2^exV
    eh = min(29 - exB, 21 - exV);
    const int bitlen = 64 - __clzll((long long)n);
    k = max(0, min(20, 30 - bitlen));
  }
  return TileScales{ldexpf(1.0f, eh), ldexpf(1.0f, k), ldexpf(1.0f, -eh), ldexpf(1.0f, -(eh + k))};
}

// Adds n staged records (tile-relative cell, offset d, return v) to the hi
// and lo integer tiles of a tile of Tlen cells (Eq. (12) with the averaging
// kernel's per-tap polynomials). Sparse chunks (fewer than one record per
// two cells) take one record per lane, its taps added at once: neighbouring
// lanes' records rarely share a cell. Dense chunks: each thread takes a
// contiguous, odd-length stretch of the cell-sorted records and, for each run
// of records in one cell, sums their taps in registers (exact integer sums,
// within the same per-cell bounds) before adding them to the tiles; one record
// per lane would have the lanes of a warp reduce into the same few cells at
// once. A run is swept twice, for the first and the second half of the taps,
// so that only half the sums are live; the odd stretch keeps the lanes'
// staged reads on distinct banks.
template <int NT, int NTH, class Cells>
__device__ __forceinline__ void spread_chunk(const int* ev_p, const float* ev_d, const float* ev_v, int n, int Tlen,
                                             int klo, const KernelPoly& poly, const TileScales& ts, uint32_t hi_s,
                                             uint32_t lo_s, Cells cells) {
  if (2 * n < Tlen) {
    for (int ei = threadIdx.x; ei < n; ei += NTH) {
      const int pe = ev_p[ei];
      if (pe == kNoCell) continue;
      const float z = ev_d[ei] - 0.5f;
      const float vs = ev_v[ei] * ts.scale;
      const int c0 = pe + klo;
      const bool inside = c0 >= 0 && c0 + NT <= Tlen;  // else test each tap's cell
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const int q = c0 + j;
        const bool take = (inside || (unsigned)q < (unsigned)Tlen) && cells.own(q);
        if (Cells::kAll || take) {
          float w = poly.c[j][kPolyDeg];
#pragma unroll
          for (int i = kPolyDeg - 1; i >= 0; --i) w = fmaf(w, z, poly.c[j][i]);
          const float h = fmaf(vs, w, kRoundMagic);      // round(vs w) + 1.5 2^23
          const float r = fmaf(vs, w, kRoundMagic - h);  // vs w - round(vs w), |r| <= 1/2
          const float l = fmaf(r, ts.kscale, kRoundMagic);
          if (take) {
            const uint32_t sl = cells.slot(q);
            red_shared_add(hi_s + 4u * sl, __float_as_int(h) - kRoundMagicBits);
            red_shared_add(lo_s + 4u * sl, __float_as_int(l) - kRoundMagicBits);
          }
        }
      }
    }
    return;
  }
  constexpr int H = (NT + 1) / 2;
  int cnt = (n + NTH - 1) / NTH;
  cnt |= 1;
  const int e0 = min(n, (int)threadIdx.x * cnt), e1 = min(n, e0 + cnt);
  for (int ei = e0; ei < e1;) {
    const int pe = ev_p[ei];
    int ej = ei + 1;
    while (ej < e1 && ev_p[ej] == pe) ++ej;
    if (pe != kNoCell) {
      const int c0 = pe + klo;
      const bool inside = c0 >= 0 && c0 + NT <= Tlen;  // else test each tap's cell
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        int ah[H], al[H];
#pragma unroll
        for (int q = 0; q < H; ++q) ah[q] = al[q] = 0;
        for (int e = ei; e < ej; ++e) {
          const float z = ev_d[e] - 0.5f;
          const float vs = ev_v[e] * ts.scale;
#pragma unroll
          for (int q = 0; q < H; ++q) {
            const int j = half * H + q;
            if (j < NT && (Cells::kAll || cells.own(c0 + j))) {
              float w = poly.c[j][kPolyDeg];
#pragma unroll
              for (int i = kPolyDeg - 1; i >= 0; --i) w = fmaf(w, z, poly.c[j][i]);
              const float h = fmaf(vs, w, kRoundMagic);      // round(vs w) + 1.5 2^23
              const float r = fmaf(vs, w, kRoundMagic - h);  // vs w - round(vs w), |r| <= 1/2
              const float l = fmaf(r, ts.kscale, kRoundMagic);
              ah[q] += __float_as_int(h) - kRoundMagicBits;
              al[q] += __float_as_int(l) - kRoundMagicBits;
            }
          }
        }
#pragma unroll
        for (int q = 0; q < H; ++q) {
          const int j = half * H + q;
          const int cq = c0 + j;
          if (j < NT && (inside || (unsigned)cq < (unsigned)Tlen) && cells.own(cq)) {
            const uint32_t sl = cells.slot(cq);
            red_shared_add(hi_s + 4u * sl, ah[q]);
            red_shared_add(lo_s + 4u * sl, al[q]);
          }
        }
      }
    }
    ei = ej;
  }
}

}  // namespace mmgpu
