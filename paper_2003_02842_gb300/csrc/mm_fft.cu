// mm_fft.cu -- stages (b) and (c) of the hot path: the FFT of every asset's
// oversampled grid (Eq. (13)) and the deconvolution with truncation to
// 0 <= k <= N (Eq. (14); step D of Algorithms 8-10), plus the per-cutoff
// tables they use.
//
// The real grid f (length M_r) of asset a is read as n = M_r/2 complex points
// z_m = f_{2m} + i f_{2m+1}. Its length-n DFT Z is taken in two passes over
// L2-resident data (n = P Q, index m = Q j1 + j2, k = k1 + P k2):
//   pass 1 (columns): length-P Stockham FFTs over j1 for a block of adjacent
//     j2, times the twiddle w_n^{j2 k1}, written back in place;
//   pass 2 (rows): length-Q Stockham FFTs over j2 for a block of rows k1 and
//     their mirrors P - k1, then the real-input unpack
//       G(k) = (Z_k + conj Z_{n-k})/2 + w_{2n}^k (Z_k - conj Z_{n-k})/(2i)
//     and F(k) = G(k) * decon(k) for k <= N, written with coalesced stores.
// Both passes keep their rows in shared memory and ping-pong between two
// buffers (autosorting Stockham), so no bit reversal is needed.
#include <math.h>

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

// ------------------------------------------------------------ pass 1
template <typename T>
__global__ void __launch_bounds__(256) k_fft_cols(Cplx<T>* __restrict__ z, FftParams f,
                                                  const Cplx<T>* __restrict__ W, const int* __restrict__ gate) {
  if (*gate) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = f.P, Q = f.Q, lgB = f.lg_cols, B = 1 << lgB;
  Cplx<T>* buf0 = reinterpret_cast<Cplx<T>*>(smem_raw);
  Cplx<T>* buf1 = buf0 + P * B;
  Cplx<T>* tw = buf1 + P * B;
  const int j20 = blockIdx.x * B;
  Cplx<T>* za = z + (int64_t)blockIdx.y * f.n;
  for (int j = threadIdx.x; j < P; j += blockDim.x) tw[j] = W[j * Q];
  for (int idx = threadIdx.x; idx < (P << lgB); idx += blockDim.x) {
    const int j1 = idx >> lgB, c = idx & (B - 1), j2 = j20 + c;
    buf0[swz(j1, c, lgB)] = (j2 < Q) ? za[Q * j1 + j2] : Cplx<T>{(T)0, (T)0};
  }
  __syncthreads();
  const Cplx<T>* X = stockham_fft(buf0, buf1, tw, P, lgB, f.rad_p, f.nrad_p);
  for (int idx = threadIdx.x; idx < (P << lgB); idx += blockDim.x) {
    const int k1 = idx >> lgB, c = idx & (B - 1), j2 = j20 + c;
    // j2 k1 <= (Q-1)(P-1) < n: the twiddle index needs no reduction
    if (j2 < Q) za[Q * k1 + j2] = cmul(X[swz(k1, c, lgB)], W[j2 * k1]);
  }
}

// ------------------------------------------------------------ pass 2
template <typename T>
__global__ void __launch_bounds__(256) k_fft_rows(const Cplx<T>* __restrict__ z, FftParams f,
                                                  const Cplx<T>* __restrict__ W, const Cplx<T>* __restrict__ U,
                                                  const T* __restrict__ decon, Cplx<T>* __restrict__ out,
                                                  const int* __restrict__ gate) {
  if (*gate) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_row[64], s_partner[64];
  __shared__ int s_nrows;
  const int P = f.P, Q = f.Q;
  const int lgB = f.lg_rowcols, B = 1 << lgB;  // padded number of rows held
  const int r0 = blockIdx.x * f.rowblk;
  const int r1 = min(r0 + f.rowblk, f.H);
  if (threadIdx.x == 0) {
    // lower rows first (ascending k1), then the mirrors P - k1 that are not
    // lower rows themselves (descending), so output segments stay contiguous
    int nr = 0;
    for (int k1 = r0; k1 < r1; ++k1) s_row[nr++] = k1;
    const int nlow = nr;
    for (int i = 0; i < nlow; ++i) {
      const int k1 = s_row[i];
      const int m = (P - k1) % P;
      if (m >= f.H) s_row[nr++] = m;
    }
    for (int i = 0; i < nr; ++i) {
      const int m = (P - s_row[i]) % P;
      int pi = i;
      for (int q = 0; q < nr; ++q)
        if (s_row[q] == m) pi = q;
      s_partner[i] = pi;
    }
    for (int i = nr; i < B; ++i) s_row[i] = -1;
    s_nrows = nr;
  }
  __syncthreads();
  const int nr = s_nrows;
  Cplx<T>* buf0 = reinterpret_cast<Cplx<T>*>(smem_raw);
  Cplx<T>* buf1 = buf0 + B * Q;
  Cplx<T>* tw = buf1 + B * Q;
  const Cplx<T>* za = z + (int64_t)blockIdx.y * f.n;
  for (int j = threadIdx.x; j < Q; j += blockDim.x) tw[j] = W[j * P];
  const unsigned mQ = magic_of((unsigned)Q);
  for (int idx = threadIdx.x; idx < B * Q; idx += blockDim.x) {
    const int ri = fast_div(idx, Q, mQ), j2 = idx - ri * Q;
    const int row = s_row[ri];
    buf0[swz(j2, ri, lgB)] = row >= 0 ? za[Q * row + j2] : Cplx<T>{(T)0, (T)0};
  }
  __syncthreads();
  const Cplx<T>* X = stockham_fft(buf0, buf1, tw, Q, lgB, f.rad_q, f.nrad_q);
  Cplx<T>* oa = out + (int64_t)blockIdx.y * (f.N + 1);
  for (int idx = threadIdx.x; idx < (Q << lgB); idx += blockDim.x) {
    const int k2 = idx >> lgB, ri = idx & (B - 1);
    if (ri >= nr) continue;
    const int k1 = s_row[ri];
    const int k = k1 + P * k2;
    if (k > f.N) continue;
    const int pri = s_partner[ri];
    const int pk2 = (k1 == 0) ? ((k2 == 0) ? 0 : Q - k2) : Q - 1 - k2;
    const Cplx<T> Zk = X[swz(k2, ri, lgB)];
    const Cplx<T> Zc = cconj(X[swz(pk2, pri, lgB)]);
    const Cplx<T> E = {(T)0.5 * (Zk.x + Zc.x), (T)0.5 * (Zk.y + Zc.y)};
    const Cplx<T> dlt = csub(Zk, Zc);
    const Cplx<T> O = {(T)0.5 * dlt.y, (T)-0.5 * dlt.x};  // (Zk - Zc) / (2i)
    const Cplx<T> G = cadd(E, cmul(U[k], O));
    const T sc = decon[k];
    oa[k] = Cplx<T>{G.x * sc, G.y * sc};
  }
}

// ------------------------------------------------------------ tables
// Gauss-Legendre nodes on [-1, 1] by Newton's method on P_nq (one thread per node).
__global__ void k_gl_nodes(int nq, double* x, double* w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  double zz = cos(kPi * (i + 0.75) / (nq + 0.5));
  double dp = 1.0;
  for (int it = 0; it < 100; ++it) {
    double p0 = 1.0, p1 = zz;
    for (int k = 2; k <= nq; ++k) {
      const double p2 = ((2.0 * k - 1.0) * zz * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = nq * (zz * p1 - p0) / (zz * zz - 1.0);
    const double dz = p1 / dp;
    zz -= dz;
    if (fabs(dz) < 1e-16) break;
  }
  double p0 = 1.0, p1 = zz;
  for (int k = 2; k <= nq; ++k) {
    const double p2 = ((2.0 * k - 1.0) * zz * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  dp = nq * (zz * p1 - p0) / (zz * zz - 1.0);
  x[i] = zz;
  w[i] = 2.0 / ((1.0 - zz * zz) * dp * dp);
}

cudaError_t launch_gl_nodes(int nq, double* x, double* w, cudaStream_t s) {
  k_gl_nodes<<<(nq + 127) / 128, 128, 0, s>>>(nq, x, w);
  return cudaGetLastError();
}

// W[j] = e^{-2 pi i j / n} (j < n); U[k] = e^{-i pi k / n} (k <= N);
// decon[k]: the F-convention deconvolution factor of Eq. (14) for the kernel
// as spread by mm_spread.cu (so F(k) = G(k) decon(k)).
template <typename T>
__global__ void k_setup_tables(int kernel, int msp, int64_t Mr, int N, int64_t n, double es_beta, double kb_b,
                               double kb_inv_phi0, double tau, const double* __restrict__ glx,
                               const double* __restrict__ glw, int nq, Cplx<T>* W, Cplx<T>* U, T* decon) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    double s, c;
    sincospi(-2.0 * (double)i / (double)n, &s, &c);
    W[i] = Cplx<T>{(T)c, (T)s};
  }
  if (i <= N) {
    const double k = (double)i;
    double s, c;
    sincospi(-k / (double)n, &s, &c);
    U[i] = Cplx<T>{(T)c, (T)s};
    double v;
    if (kernel == MM_KERNEL_GAUSS) {
      // step D.1 of Algorithm 8: c_k = sqrt(pi/tau) e^{k^2 tau} G(k) / M_r
      v = sqrt(kPi / tau) * exp(k * k * tau) / ((double)Mr * 2.0 * kPi);
    } else if (kernel == MM_KERNEL_KB) {
      // step D.1 of Algorithm 9 with Eq. (8): c_k = G(k) / I0(m sqrt(b^2 - (2 pi k/M_r)^2))
      const double a = 2.0 * kPi * k / (double)Mr;
      const double arg = (double)msp * sqrt(fmax(kb_b * kb_b - a * a, 0.0));
      v = 1.0 / (2.0 * kPi * kb_inv_phi0 * cyl_bessel_i0(arg));
    } else {
      // steps D.1-D.2 of Algorithm 10: phihat(k) = 2 alpha int_0^1
      // exp(beta (sqrt(1-y^2) - 1)) cos(alpha k y) dy, Gauss-Legendre in y
      const double alpha = kPi * 2.0 * msp / (double)Mr;
      double acc = 0.0;
      for (int q = 0; q < nq; ++q) {
        const double y = 0.5 * (glx[q] + 1.0);
        acc += 0.5 * glw[q] * exp(es_beta * (sqrt(fmax(1.0 - y * y, 0.0)) - 1.0)) * cos(alpha * k * y);
      }
      const double ph = 2.0 * alpha * acc;
      v = 1.0 / ((double)Mr * ph);
    }
    decon[i] = (T)v;
  }
}

cudaError_t launch_setup_tables(int kernel, int msp, int64_t Mr, int N, int64_t n, const SpreadParams& sp,
                                double tau, const double* glx, const double* glw, int nq, void* W, void* U,
                                void* decon, bool fp64, cudaStream_t s) {
  const int64_t m = n > (int64_t)N + 1 ? n : (int64_t)N + 1;
  const int blocks = (int)((m + 255) / 256);
  if (fp64)
    k_setup_tables<double><<<blocks, 256, 0, s>>>(kernel, msp, Mr, N, n, sp.es_beta, sp.kb_b, sp.kb_inv_phi0, tau,
                                                  glx, glw, nq, (Cplx<double>*)W, (Cplx<double>*)U, (double*)decon);
  else
    k_setup_tables<float><<<blocks, 256, 0, s>>>(kernel, msp, Mr, N, n, sp.es_beta, sp.kb_b, sp.kb_inv_phi0, tau,
                                                 glx, glw, nq, (Cplx<float>*)W, (Cplx<float>*)U, (float*)decon);
  return cudaGetLastError();
}

// ------------------------------------------------------------ launchers
size_t fft_cols_smem(const FftParams& f, bool fp64) {
  const size_t cs = fp64 ? 16 : 8;
  return cs * ((size_t)2 * f.P * ((size_t)1 << f.lg_cols) + f.P);
}
size_t fft_rows_smem(const FftParams& f, bool fp64) {
  const size_t cs = fp64 ? 16 : 8;
  return cs * ((size_t)2 * ((size_t)1 << f.lg_rowcols) * f.Q + f.Q);
}

template <typename T>
static cudaError_t launch_cols_t(T* grid, const FftParams& f, int D, const void* W, const int* status,
                                 cudaStream_t s) {
  const size_t smem = fft_cols_smem(f, sizeof(T) == 8);
  auto fn = k_fft_cols<T>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int B = 1 << f.lg_cols;
  dim3 grd((f.Q + B - 1) / B, D);
  fn<<<grd, 256, smem, s>>>(reinterpret_cast<Cplx<T>*>(grid), f, (const Cplx<T>*)W, status + 1);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_rows_t(const T* grid, const FftParams& f, int D, const void* W, const void* U,
                                 const void* decon, void* coeffs, const int* status, cudaStream_t s) {
  const size_t smem = fft_rows_smem(f, sizeof(T) == 8);
  auto fn = k_fft_rows<T>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grd((f.H + f.rowblk - 1) / f.rowblk, D);
  fn<<<grd, 256, smem, s>>>(reinterpret_cast<const Cplx<T>*>(grid), f, (const Cplx<T>*)W, (const Cplx<T>*)U,
                            (const T*)decon, (Cplx<T>*)coeffs, status + 1);
  return cudaGetLastError();
}

cudaError_t launch_fft_cols_f32(float* grid, const FftParams& f, int D, const void* W, const int* status,
                                cudaStream_t s) {
  return launch_cols_t<float>(grid, f, D, W, status, s);
}
cudaError_t launch_fft_cols_f64(double* grid, const FftParams& f, int D, const void* W, const int* status,
                                cudaStream_t s) {
  return launch_cols_t<double>(grid, f, D, W, status, s);
}
cudaError_t launch_fft_rows_f32(const float* grid, const FftParams& f, int D, const void* W, const void* U,
                                const void* decon, void* coeffs, const int* status, cudaStream_t s) {
  return launch_rows_t<float>(grid, f, D, W, U, decon, coeffs, status, s);
}
cudaError_t launch_fft_rows_f64(const double* grid, const FftParams& f, int D, const void* W, const void* U,
                                const void* decon, void* coeffs, const int* status, cudaStream_t s) {
  return launch_rows_t<double>(grid, f, D, W, U, decon, coeffs, status, s);
}

}  // namespace mmgpu
