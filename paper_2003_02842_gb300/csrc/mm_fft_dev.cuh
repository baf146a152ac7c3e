// mm_fft_dev.cuh -- device helpers of stage (b): small DFTs and the
// shared-memory Stockham FFT, shared by the multi-kernel and fused paths.
#pragma once

#include "mm_common.cuh"

namespace mmgpu {

// ------------------------------------------------------------ small DFTs
// Forward DFTs (exponent -2 pi i j k / R) of R = 2, 3, 4, 5, 8 points.
template <typename T>
__device__ __forceinline__ void dft2(Cplx<T>& a, Cplx<T>& b) {
  Cplx<T> s = cadd(a, b), d = csub(a, b);
  a = s;
  b = d;
}

template <typename T, int R>
struct Dft;

template <typename T>
struct Dft<T, 2> {
  static __device__ __forceinline__ void run(Cplx<T>* v) { dft2(v[0], v[1]); }
};

template <typename T>
struct Dft<T, 3> {
  static __device__ __forceinline__ void run(Cplx<T>* v) {
    const T c = (T)-0.5, s = (T)0.866025403784438646763723170752936183;  // cos, sin of 2 pi / 3
    Cplx<T> p = cadd(v[1], v[2]), m = csub(v[1], v[2]);
    Cplx<T> y0 = cadd(v[0], p);
    Cplx<T> a = {v[0].x + c * p.x, v[0].y + c * p.y};
    Cplx<T> b = {s * m.x, s * m.y};
    Cplx<T> jb = cmul_mi(b);  // -i s (x1 - x2)
    v[0] = y0;
    v[1] = cadd(a, jb);
    v[2] = csub(a, jb);
  }
};

template <typename T>
struct Dft<T, 4> {
  static __device__ __forceinline__ void run(Cplx<T>* v) {
    Cplx<T> s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    Cplx<T> s13 = cadd(v[1], v[3]), d13 = cmul_mi(csub(v[1], v[3]));
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13);
    v[3] = csub(d02, d13);
  }
};

template <typename T>
struct Dft<T, 5> {
  static __device__ __forceinline__ void run(Cplx<T>* v) {
    const T c1 = (T)0.309016994374947424102293417182819059;   // cos(2 pi/5)
    const T c2 = (T)-0.809016994374947424102293417182819059;  // cos(4 pi/5)
    const T s1 = (T)0.951056516295153572116439333379382143;   // sin(2 pi/5)
    const T s2 = (T)0.587785252292473129168705954639072769;   // sin(4 pi/5)
    Cplx<T> p14 = cadd(v[1], v[4]), m14 = csub(v[1], v[4]);
    Cplx<T> p23 = cadd(v[2], v[3]), m23 = csub(v[2], v[3]);
    Cplx<T> y0 = cadd(v[0], cadd(p14, p23));
    Cplx<T> a1 = {v[0].x + c1 * p14.x + c2 * p23.x, v[0].y + c1 * p14.y + c2 * p23.y};
    Cplx<T> a2 = {v[0].x + c2 * p14.x + c1 * p23.x, v[0].y + c2 * p14.y + c1 * p23.y};
    Cplx<T> b1 = {s1 * m14.x + s2 * m23.x, s1 * m14.y + s2 * m23.y};
    Cplx<T> b2 = {s2 * m14.x - s1 * m23.x, s2 * m14.y - s1 * m23.y};
    Cplx<T> jb1 = cmul_mi(b1), jb2 = cmul_mi(b2);
    v[0] = y0;
    v[1] = cadd(a1, jb1);
    v[4] = csub(a1, jb1);
    v[2] = cadd(a2, jb2);
    v[3] = csub(a2, jb2);
  }
};

template <typename T>
struct Dft<T, 8> {
  static __device__ __forceinline__ void run(Cplx<T>* v) {
    const T r = (T)0.707106781186547524400844362104849039;  // sqrt(1/2)
    Cplx<T> e[4] = {v[0], v[2], v[4], v[6]};
    Cplx<T> o[4] = {v[1], v[3], v[5], v[7]};
    Dft<T, 4>::run(e);
    Dft<T, 4>::run(o);
    // o_k *= w8^k, w8 = e^{-i pi/4}
    Cplx<T> o1 = {r * (o[1].x + o[1].y), r * (o[1].y - o[1].x)};
    Cplx<T> o2 = cmul_mi(o[2]);
    Cplx<T> o3 = {r * (o[3].y - o[3].x), -r * (o[3].x + o[3].y)};
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
  }
};

// j / d for j, d < 2^16 with m = ceil(2^32 / d): floor(j m / 2^32) is exact,
// because the rounding of m adds less than 2^-16 < 1/d to j / d.
__device__ __forceinline__ unsigned magic_of(unsigned d) { return d <= 1u ? 0u : 0xFFFFFFFFu / d + 1u; }
__device__ __forceinline__ int fast_div(int j, int d, unsigned m) { return d == 1 ? j : (int)__umulhi((unsigned)j, m); }

// Shared-memory slot of element j of column c when B = 2^lgB columns are
// interleaved: row j holds the B columns, permuted by an XOR with the row
// index so that reading one column down many rows (the transposed loads of
// pass 2) touches distinct banks while a row stays one contiguous segment.
__device__ __forceinline__ int swz(int j, int c, int lgB) { return (j << lgB) | (c ^ (j & ((1 << lgB) - 1))); }

// One autosorting Stockham stage of radix R over L-point sequences stored as
// B = 2^lgB interleaved columns (element j of column c at swz(j, c)).
// Ns is the product of the radices already applied; tw[j] = e^{-2 pi i j / L}.
template <typename T, int R>
__device__ __forceinline__ void stockham_stage(const Cplx<T>* __restrict__ in, Cplx<T>* __restrict__ out,
                                               const Cplx<T>* __restrict__ tw, int L, int lgB, int Ns) {
  const int nb = L / R;
  const int twstep = L / (Ns * R);
  const unsigned mNs = magic_of((unsigned)Ns);
  const int B = 1 << lgB;
  for (int idx = threadIdx.x; idx < (nb << lgB); idx += blockDim.x) {
    const int j = idx >> lgB, c = idx & (B - 1);
    const int q = fast_div(j, Ns, mNs);
    const int k = j - q * Ns;
    Cplx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[swz(j + r * nb, c, lgB)];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[r * k * twstep]);
    }
    Dft<T, R>::run(v);
    const int base = q * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) out[swz(base + r * Ns, c, lgB)] = v[r];
  }
}

// Full L-point FFT of 2^lgB columns; returns the buffer holding the result.
template <typename T>
__device__ Cplx<T>* stockham_fft(Cplx<T>* a, Cplx<T>* b, const Cplx<T>* tw, int L, int lgB, const int* rad,
                                 int nrad) {
  int Ns = 1;
  Cplx<T>* in = a;
  Cplx<T>* out = b;
  for (int s = 0; s < nrad; ++s) {
    const int r = rad[s];
    switch (r) {
      case 2: stockham_stage<T, 2>(in, out, tw, L, lgB, Ns); break;
      case 3: stockham_stage<T, 3>(in, out, tw, L, lgB, Ns); break;
      case 4: stockham_stage<T, 4>(in, out, tw, L, lgB, Ns); break;
      case 5: stockham_stage<T, 5>(in, out, tw, L, lgB, Ns); break;
      default: stockham_stage<T, 8>(in, out, tw, L, lgB, Ns); break;
    }
    __syncthreads();
    Cplx<T>* x = in;
    in = out;
    out = x;
    Ns *= r;
  }
  return in;
}

}  // namespace mmgpu
