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
#include "mm_fft_dev.cuh"

namespace mmgpu {

// Elements per thread held in registers between the batched global loads
// and the shared-memory stages (the host keeps P 2^lg_cols and 2^lg_rowcols Q
// at most kFftThreads * kFftPer).
constexpr int kFftThreads = 256;
constexpr int kFftPer = 16;

// ------------------------------------------------------------ pass 1
// Every global load of a block (its column values and the write-back
// twiddles) is issued in one batch into registers before the first barrier,
// so the block waits for memory once.
template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_fft_cols(Cplx<T>* __restrict__ z, FftParams f,
                                                          const Cplx<T>* __restrict__ W, const int* __restrict__ gate) {
  if (*gate) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = f.P, Q = f.Q, lgB = f.lg_cols, B = 1 << lgB;
  Cplx<T>* buf0 = reinterpret_cast<Cplx<T>*>(smem_raw);
  Cplx<T>* buf1 = buf0 + P * B;
  Cplx<T>* tw = buf1 + P * B;
  const int j20 = blockIdx.x * B;
  Cplx<T>* za = z + (int64_t)blockIdx.y * f.n;
  const int total = P << lgB;
  Cplx<T> v[kFftPer], wt[kFftPer];
#pragma unroll
  for (int i = 0; i < kFftPer; ++i) {
    const int idx = threadIdx.x + i * kFftThreads;
    v[i] = Cplx<T>{(T)0, (T)0};
    wt[i] = Cplx<T>{(T)1, (T)0};
    if (idx < total) {
      const int j1 = idx >> lgB, j2 = j20 + (idx & (B - 1));
      if (j2 < Q) {
        v[i] = za[Q * j1 + j2];
        wt[i] = W[j2 * j1];  // j2 k1 <= (Q-1)(P-1) < n: no reduction
      }
    }
  }
  for (int j = threadIdx.x; j < P; j += kFftThreads) tw[j] = W[j * Q];
#pragma unroll
  for (int i = 0; i < kFftPer; ++i) {
    const int idx = threadIdx.x + i * kFftThreads;
    if (idx < total) buf0[swz(idx >> lgB, idx & (B - 1), lgB)] = v[i];
  }
  __syncthreads();
  const Cplx<T>* X = stockham_fft(buf0, buf1, tw, P, lgB, f.rad_p, f.nrad_p);
#pragma unroll
  for (int i = 0; i < kFftPer; ++i) {
    const int idx = threadIdx.x + i * kFftThreads;
    if (idx < total) {
      const int k1 = idx >> lgB, c = idx & (B - 1), j2 = j20 + c;
      if (j2 < Q) za[Q * k1 + j2] = cmul(X[swz(k1, c, lgB)], wt[i]);
    }
  }
}

// Rows held by a pass-2 block: lower rows k1 = r0 .. r1-1, then the mirrors
// P - k1 that are not lower rows (k1 in [max(r0,1), min(r1, P-H+1))), so the
// block's output segments are contiguous. Closed forms, no search.
struct RowSet {
  int r0, nlow, mlo, nr;
};
__device__ __forceinline__ RowSet row_set(int r0, int rowblk, int P, int H) {
  RowSet r;
  const int r1 = min(r0 + rowblk, H);
  r.r0 = r0;
  r.nlow = r1 - r0;
  r.mlo = max(r0, 1);
  const int mhi = min(r1, P - H + 1);
  r.nr = r.nlow + max(0, mhi - r.mlo);
  return r;
}
__device__ __forceinline__ int row_of(const RowSet& r, int ri, int P) {
  if (ri < r.nlow) return r.r0 + ri;
  if (ri < r.nr) return P - (r.mlo + (ri - r.nlow));
  return -1;
}
// index of the row holding Z_{n-k} for the rows of the block
__device__ __forceinline__ int partner_of(const RowSet& r, int ri, int P, int H) {
  if (ri < r.nlow) {
    const int k1 = r.r0 + ri;
    if (k1 >= 1 && P - k1 >= H) return r.nlow + (k1 - r.mlo);
    return ri;  // row 0 and the self-mirrored row P/2
  }
  return (r.mlo + (ri - r.nlow)) - r.r0;
}

// ------------------------------------------------------------ pass 2
template <typename T>
__global__ void __launch_bounds__(kFftThreads) k_fft_rows(const Cplx<T>* __restrict__ z, FftParams f,
                                                          const Cplx<T>* __restrict__ W, const Cplx<T>* __restrict__ U,
                                                          const T* __restrict__ decon, Cplx<T>* __restrict__ out,
                                                          const int* __restrict__ gate) {
  if (*gate) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int P = f.P, Q = f.Q;
  const int lgB = f.lg_rowcols, B = 1 << lgB;  // padded number of rows held
  const RowSet rs = row_set(blockIdx.x * f.rowblk, f.rowblk, P, f.H);
  Cplx<T>* buf0 = reinterpret_cast<Cplx<T>*>(smem_raw);
  Cplx<T>* buf1 = buf0 + B * Q;
  Cplx<T>* tw = buf1 + B * Q;
  const Cplx<T>* za = z + (int64_t)blockIdx.y * f.n;
  const int total = B * Q;
  const unsigned mQ = magic_of((unsigned)Q);
  // batched loads: row values (load order: row-major, coalesced), and for
  // the unpack (order: k2-major) the U and deconvolution factors
  Cplx<T> v[kFftPer], uk[kFftPer];
  T dk[kFftPer];
#pragma unroll
  for (int i = 0; i < kFftPer; ++i) {
    const int idx = threadIdx.x + i * kFftThreads;
    v[i] = Cplx<T>{(T)0, (T)0};
    uk[i] = Cplx<T>{(T)0, (T)0};
    dk[i] = (T)0;
    if (idx < total) {
      const int ri = fast_div(idx, Q, mQ), j2 = idx - ri * Q;
      const int row = row_of(rs, ri, P);
      if (row >= 0) v[i] = za[Q * row + j2];
      const int k2 = idx >> lgB, ro = idx & (B - 1);
      const int k1 = row_of(rs, ro, P);
      const int k = k1 + P * k2;
      if (k1 >= 0 && k <= f.N) {
        uk[i] = U[k];
        dk[i] = decon[k];
      }
    }
  }
  for (int j = threadIdx.x; j < Q; j += kFftThreads) tw[j] = W[j * P];
#pragma unroll
  for (int i = 0; i < kFftPer; ++i) {
    const int idx = threadIdx.x + i * kFftThreads;
    if (idx < total) {
      const int ri = fast_div(idx, Q, mQ), j2 = idx - ri * Q;
      buf0[swz(j2, ri, lgB)] = v[i];
    }
  }
  __syncthreads();
  const Cplx<T>* X = stockham_fft(buf0, buf1, tw, Q, lgB, f.rad_q, f.nrad_q);
  Cplx<T>* oa = out + (int64_t)blockIdx.y * (f.N + 1);
#pragma unroll
  for (int i = 0; i < kFftPer; ++i) {
    const int idx = threadIdx.x + i * kFftThreads;
    if (idx >= total) continue;
    const int k2 = idx >> lgB, ri = idx & (B - 1);
    const int k1 = row_of(rs, ri, P);
    const int k = k1 + P * k2;
    if (k1 < 0 || k > f.N) continue;
    const int pri = partner_of(rs, ri, P, f.H);
    const int pk2 = (k1 == 0) ? ((k2 == 0) ? 0 : Q - k2) : Q - 1 - k2;
    const Cplx<T> Zk = X[swz(k2, ri, lgB)];
    const Cplx<T> Zc = cconj(X[swz(pk2, pri, lgB)]);
    const Cplx<T> E = {(T)0.5 * (Zk.x + Zc.x), (T)0.5 * (Zk.y + Zc.y)};
    const Cplx<T> dlt = csub(Zk, Zc);
    const Cplx<T> O = {(T)0.5 * dlt.y, (T)-0.5 * dlt.x};  // (Zk - Zc) / (2i)
    const Cplx<T> G = cadd(E, cmul(uk[i], O));
    oa[k] = Cplx<T>{G.x * dk[i], G.y * dk[i]};
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
  if ((f.P << f.lg_cols) > kFftThreads * kFftPer) return cudaErrorInvalidValue;
  fn<<<grd, kFftThreads, smem, s>>>(reinterpret_cast<Cplx<T>*>(grid), f, (const Cplx<T>*)W, status + 1);
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
  if (((1 << f.lg_rowcols) * f.Q) > kFftThreads * kFftPer) return cudaErrorInvalidValue;
  fn<<<grd, kFftThreads, smem, s>>>(reinterpret_cast<const Cplx<T>*>(grid), f, (const Cplx<T>*)W, (const Cplx<T>*)U,
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
