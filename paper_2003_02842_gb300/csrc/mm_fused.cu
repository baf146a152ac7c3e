// mm_fused.cu -- stages (a)-(c) of the hot path in one kernel for grids that
// fit in shared memory: one CTA per asset rescales its events and forms the
// returns (Algorithm 4, Algorithm 3 step F.3), spreads them onto the
// oversampled grid held in shared memory (Eq. (12)), takes the two-pass FFT
// of the grid in place (Eq. (13)) and writes the deconvolved, truncated
// coefficients (Eq. (14)). The grid never leaves the SM: global traffic is
// the events in and the coefficients out.
//
// Shared memory: the real grid (M_r cells, read as n = M_r/2 complex points),
// one work area for a block of FFT columns or rows (ping-pong), and the two
// stage-twiddle tables. The FFT passes are the ones of mm_fft.cu with the
// grid's home in shared instead of global memory.
#include <algorithm>

#include "mm_common.cuh"
#include "mm_fft_dev.cuh"
#include "mm_spread_dev.cuh"

namespace mmgpu {

constexpr int kFusedThreads = 1024;

template <typename T, int KERNEL, int KW>
__global__ void __launch_bounds__(kFusedThreads, 1)
    k_coeff_fused(const int64_t* __restrict__ off, const double* __restrict__ t, const double* __restrict__ logp,
                  const Rescale* __restrict__ rsp, const int* __restrict__ gate, SpreadParams sp, FftParams f,
                  const Cplx<T>* __restrict__ W, const Cplx<T>* __restrict__ U, const T* __restrict__ decon,
                  Cplx<T>* __restrict__ out, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_row[64], s_partner[64];
  __shared__ int s_nrows, s_flags;
  __shared__ UScale s_us;
  __shared__ UScaleF s_usf;
  if (*gate) return;  // uniform: the whole block leaves
  const int P = f.P, Q = f.Q;
  const int Mr = (int)sp.Mr;
  T* grid = reinterpret_cast<T*>(smem_raw);
  Cplx<T>* z = reinterpret_cast<Cplx<T>*>(smem_raw);
  const int lgC = f.lg_cols, Bc = 1 << lgC;
  const int lgR = f.lg_rowcols, Br = 1 << lgR;
  const int work_elems = max(2 * P * Bc, 2 * Br * Q);
  Cplx<T>* work = z + f.n;
  Cplx<T>* twP = work + work_elems;
  Cplx<T>* twQ = twP + P;
  const int a = blockIdx.x;
  const Rescale rs = *rsp;

  // zero the grid; stage twiddle tables
  {
    float4* g4 = reinterpret_cast<float4*>(grid);
    const int n4 = (int)(((size_t)Mr * sizeof(T) + 15) / 16);
    for (int c = threadIdx.x; c < n4; c += kFusedThreads) g4[c] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (int j = threadIdx.x; j < P; j += kFusedThreads) twP[j] = W[j * Q];
  for (int j = threadIdx.x; j < Q; j += kFusedThreads) twQ[j] = W[j * P];
  if (threadIdx.x == 0) {
    s_flags = 0;
    if (sizeof(T) == 8) s_us = make_uscale(rs, sp.Mr);
    else s_usf = make_uscale_f(rs, sp.Mr);
  }
  __syncthreads();

  // ---- spreading: one event per thread per pass, its whole stencil into the
  // shared grid (periodic wrap of Eq. (11) by one conditional add)
  const int64_t e0 = off[a], eend = off[a + 1];
  const int64_t e1 = eend > e0 ? eend - 1 : e0;
  const int klo = sp.klo, nk = sp.khi - sp.klo + 1;
  int flags = 0;
  for (int64_t h = e0 + threadIdx.x; h < e1; h += kFusedThreads) {
    const double th = t[h], tn = t[h + 1];
    const double p0 = logp[h], p1 = logp[h + 1];
    const long long kh = order_key(th), kn = order_key(tn);
    if (!(kh < kn)) flags |= (kh == kn) ? ST_DUPLICATE : ST_UNSORTED;
    if (!(finite_bits(th) && finite_bits(p0) && finite_bits(p1))) {
      flags |= ST_NONFINITE;
      continue;
    }
    const long long dt = to_fix(th, rs.F) - rs.t0_fix;
    int b0;
    T d;
    if (sizeof(T) == 8) {
      const unsigned long long uf = u_fix_of(th, rs.t0_fix, rs.F, s_us);
      b0 = (int)(uf >> kUFrac);
      d = frac_to<T>(uf & ((1ull << kUFrac) - 1));
    } else {
      float fd;
      cell_f32(dt, s_usf, b0, fd);
      d = (T)fd;
    }
    if (dt < 0 || b0 > Mr || (b0 == Mr && d > (T)0)) {
      flags |= ST_OUT_OF_WINDOW;
      continue;
    }
    const T v = return_of<T>(p0, p1);
    T x = (T)klo - d;
#pragma unroll
    for (int j = 0; j < KW; ++j) {
      if (j >= nk) break;
      int c = b0 + klo + j;
      if (c < 0) c += Mr;
      else if (c >= Mr) c -= Mr;
      atomicAdd(grid + c, v * kernel_value<T, KERNEL>(x, sp));
      x += (T)1;
    }
  }
  if (flags) atomicOr(&s_flags, flags);
  __syncthreads();
  if (threadIdx.x == 0 && s_flags) atomicOr(status, s_flags);

  // ---- FFT pass 1: columns j2 in blocks of Bc, length-P FFTs over j1, then
  // the twiddle w_n^{j2 k1}, written back in place
  for (int j20 = 0; j20 < Q; j20 += Bc) {
    for (int idx = threadIdx.x; idx < (P << lgC); idx += kFusedThreads) {
      const int j1 = idx >> lgC, c = idx & (Bc - 1), j2 = j20 + c;
      work[swz(j1, c, lgC)] = (j2 < Q) ? z[Q * j1 + j2] : Cplx<T>{(T)0, (T)0};
    }
    __syncthreads();
    const Cplx<T>* X = stockham_fft(work, work + P * Bc, twP, P, lgC, f.rad_p, f.nrad_p);
    for (int idx = threadIdx.x; idx < (P << lgC); idx += kFusedThreads) {
      const int k1 = idx >> lgC, c = idx & (Bc - 1), j2 = j20 + c;
      if (j2 < Q) z[Q * k1 + j2] = cmul(X[swz(k1, c, lgC)], W[j2 * k1]);
    }
    __syncthreads();
  }

  // ---- FFT pass 2: blocks of rows k1 and their mirrors P - k1, length-Q
  // FFTs over j2, real-input unpack and deconvolution into the coefficients
  Cplx<T>* oa = out + (int64_t)a * (f.N + 1);
  for (int r0 = 0; r0 < f.H; r0 += f.rowblk) {
    if (threadIdx.x == 0) {
      const int r1 = min(r0 + f.rowblk, f.H);
      int nr = 0;
      for (int k1 = r0; k1 < r1; ++k1) s_row[nr++] = k1;
      const int nlow = nr;
      for (int i = 0; i < nlow; ++i) {
        const int m = (P - s_row[i]) % P;
        if (m >= f.H) s_row[nr++] = m;
      }
      for (int i = 0; i < nr; ++i) {
        const int m = (P - s_row[i]) % P;
        int pi = i;
        for (int q = 0; q < nr; ++q)
          if (s_row[q] == m) pi = q;
        s_partner[i] = pi;
      }
      for (int i = nr; i < Br; ++i) s_row[i] = -1;
      s_nrows = nr;
    }
    __syncthreads();
    const int nr = s_nrows;
    const unsigned mQ = magic_of((unsigned)Q);
    for (int idx = threadIdx.x; idx < Br * Q; idx += kFusedThreads) {
      const int ri = fast_div(idx, Q, mQ), j2 = idx - ri * Q;
      const int row = s_row[ri];
      work[swz(j2, ri, lgR)] = row >= 0 ? z[Q * row + j2] : Cplx<T>{(T)0, (T)0};
    }
    __syncthreads();
    const Cplx<T>* X = stockham_fft(work, work + Br * Q, twQ, Q, lgR, f.rad_q, f.nrad_q);
    for (int idx = threadIdx.x; idx < (Q << lgR); idx += kFusedThreads) {
      const int k2 = idx >> lgR, ri = idx & (Br - 1);
      if (ri >= nr) continue;
      const int k1 = s_row[ri];
      const int k = k1 + P * k2;
      if (k > f.N) continue;
      const int pri = s_partner[ri];
      const int pk2 = (k1 == 0) ? ((k2 == 0) ? 0 : Q - k2) : Q - 1 - k2;
      const Cplx<T> Zk = X[swz(k2, ri, lgR)];
      const Cplx<T> Zc = cconj(X[swz(pk2, pri, lgR)]);
      const Cplx<T> E = {(T)0.5 * (Zk.x + Zc.x), (T)0.5 * (Zk.y + Zc.y)};
      const Cplx<T> dlt = csub(Zk, Zc);
      const Cplx<T> O = {(T)0.5 * dlt.y, (T)-0.5 * dlt.x};  // (Zk - Zc) / (2i)
      const Cplx<T> G = cadd(E, cmul(U[k], O));
      const T s = decon[k];
      oa[k] = Cplx<T>{G.x * s, G.y * s};
    }
    __syncthreads();
  }
}

size_t fused_smem(const FftParams& f, int64_t Mr, bool fp64) {
  const size_t cs = fp64 ? 16 : 8, rs = fp64 ? 8 : 4;
  const size_t work = std::max((size_t)2 * f.P * ((size_t)1 << f.lg_cols), (size_t)2 * ((size_t)1 << f.lg_rowcols) * f.Q);
  const size_t grid = ((size_t)Mr * rs + 15) / 16 * 16;
  return grid + cs * (work + f.P + f.Q);
}

template <typename T, int K>
static cudaError_t launch_fused_k(int nk, const int64_t* off, const double* t, const double* logp, const Rescale* rs,
                                  const SpreadParams& sp, const FftParams& f, const void* W, const void* U,
                                  const void* decon, void* coeffs, int* status, cudaStream_t s) {
  const size_t smem = fused_smem(f, sp.Mr, sizeof(T) == 8);
  auto go = [&](auto fn) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<sp.D, kFusedThreads, smem, s>>>(off, t, logp, rs, status + 1, sp, f, (const Cplx<T>*)W, (const Cplx<T>*)U,
                                        (const T*)decon, (Cplx<T>*)coeffs, status);
    return cudaGetLastError();
  };
  if (nk <= 8) return go(k_coeff_fused<T, K, 8>);
  if (nk <= 16) return go(k_coeff_fused<T, K, 16>);
  if (nk <= 32) return go(k_coeff_fused<T, K, 32>);
  return cudaErrorInvalidValue;
}

template <typename T>
static cudaError_t launch_fused_t(const int64_t* off, const double* t, const double* logp, const Rescale* rs,
                                  const SpreadParams& sp, const FftParams& f, const void* W, const void* U,
                                  const void* decon, void* coeffs, int* status, cudaStream_t s) {
  const int nk = sp.khi - sp.klo + 1;
  switch (sp.kernel) {
    case MM_KERNEL_GAUSS: return launch_fused_k<T, MM_KERNEL_GAUSS>(nk, off, t, logp, rs, sp, f, W, U, decon, coeffs, status, s);
    case MM_KERNEL_KB: return launch_fused_k<T, MM_KERNEL_KB>(nk, off, t, logp, rs, sp, f, W, U, decon, coeffs, status, s);
    case MM_KERNEL_ES: return launch_fused_k<T, MM_KERNEL_ES>(nk, off, t, logp, rs, sp, f, W, U, decon, coeffs, status, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_coeff_fused(bool fp64, const int64_t* off, const double* t, const double* logp, const Rescale* rs,
                               const SpreadParams& sp, const FftParams& f, const void* W, const void* U,
                               const void* decon, void* coeffs, int* status, cudaStream_t s) {
  if (fp64) return launch_fused_t<double>(off, t, logp, rs, sp, f, W, U, decon, coeffs, status, s);
  return launch_fused_t<float>(off, t, logp, rs, sp, f, W, U, decon, coeffs, status, s);
}

}  // namespace mmgpu
