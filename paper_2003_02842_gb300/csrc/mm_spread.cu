// mm_spread.cu -- stage (a) of the hot path: FP64 time rescaling and phase
// reduction (Algorithm 4), returns (Algorithm 3 step F.3), the Nyquist cutoff
// (Algorithm 2) and the spreading of returns onto the oversampled grid
// (Eq. (12); Algorithms 8-10 step C) with the Gaussian (fast Gaussian
// gridding split, Eq. (17)), Kaiser-Bessel (Eq. (7)) or exponential of
// semicircle (Eq. (9)) kernel.
//
// Spreading design: one block owns a contiguous tile of grid cells of one
// asset and accumulates into shared memory. Because an asset's times are
// sorted, the events whose stencil reaches the tile form at most three index
// ranges (the tile plus its halo, and the halo's periodic images), found by
// binary search on the same FP64 cell coordinate u = (t - t0) M_r / span that
// the accumulation uses. No global atomics; every shared-memory write is
// checked against the tile, so malformed input cannot write out of bounds.
#include <math.h>

#include "mm_common.cuh"

namespace mmgpu {

// ------------------------------------------------------------------ bounds
// Validates the CSR offsets, finds t_min / t_max over all assets (Algorithm
// 4) or takes the caller's window, and writes the per-call gate word
// (0 = proceed). One block.
__global__ void k_bounds(const int64_t* __restrict__ off, const double* __restrict__ t, int D,
                         int64_t max_events, double w0, double w1, double* bounds, int* status) {
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
      bounds[0] = bounds[1] = 0.0;
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
    bounds[0] = t0;
    bounds[1] = t1;
    *gate = g;
  }
}

cudaError_t launch_bounds(const int64_t* off, const double* t, int D, int64_t max_events, double w0,
                          double w1, double* bounds, int* status, cudaStream_t s) {
  k_bounds<<<1, 256, 0, s>>>(off, t, D, max_events, w0, w1, bounds, status);
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

__global__ void k_nyquist_final(const double* bounds, const int* gate, const unsigned long long* gapbits,
                                int* nyq, int* status) {
  if (*gate) { *nyq = -1; return; }
  unsigned long long gb = *gapbits;
  if (gb == 0ull) { *nyq = -1; atomicOr(status, ST_CUTOFF); return; }
  double g = __longlong_as_double((long long)gb);
  double span = bounds[1] - bounds[0];
  double v = floor(span / (2.0 * g));
  *nyq = (v > 2147483647.0) ? 2147483647 : (int)v;
}

cudaError_t launch_min_gap(const int64_t* off, const double* t, int D, const double* bounds,
                           unsigned long long* gapbits, int* nyq, int* status, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(gapbits, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_min_gap<<<D, 256, 0, s>>>(off, t, status + 1, gapbits, status);
  k_nyquist_final<<<1, 1, 0, s>>>(bounds, status + 1, gapbits, nyq, status);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ kernels
template <typename T> struct Fn;
template <> struct Fn<float> {
  static __device__ __forceinline__ float exp_(float x) { return __expf(x); }
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float sinh_(float x) { return sinhf(x); }
  static __device__ __forceinline__ float sin_(float x) { return sinf(x); }
};
template <> struct Fn<double> {
  static __device__ __forceinline__ double exp_(double x) { return exp(x); }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double sinh_(double x) { return sinh(x); }
  static __device__ __forceinline__ double sin_(double x) { return sin(x); }
};

// First index h in [e0, e1) with u(h) = (t[h] - t0) * scale >= xs[m] (e1 if
// none), for NX thresholds at once. Each level samples the current bracket at
// blockDim.x evenly spaced points and keeps the segment where the predicate
// turns true, so a bracket of n events closes after ceil(log_256 n) levels of
// parallel loads. On unsorted input the result is still inside [e0, e1].
template <int NX>
__device__ void block_first_ge(const double* __restrict__ t, int64_t e0, int64_t e1, double t0,
                               double scale, const double* xs, int64_t* res) {
  __shared__ int64_t s_lo[NX], s_hi[NX];
  __shared__ int s_cnt[NX];
  __shared__ int s_open;
  if (threadIdx.x < NX) {
    s_lo[threadIdx.x] = e0;
    s_hi[threadIdx.x] = e1;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  for (int level = 0; level < 8; ++level) {
    if (threadIdx.x < NX) s_cnt[threadIdx.x] = 0;
    if (threadIdx.x == 0) s_open = 0;
    __syncthreads();
    for (int m = 0; m < NX; ++m) {
      const int64_t lo = s_lo[m], len = s_hi[m] - s_lo[m];
      if (len <= 0) continue;  // uniform across the block
      const int64_t stride = (len + blockDim.x - 1) / blockDim.x;
      const int64_t off = (int64_t)threadIdx.x * stride;
      bool below = false;
      if (off < len) below = (t[lo + off] - t0) * scale < xs[m];
      unsigned bal = __ballot_sync(0xffffffffu, below);
      if (lane == 0 && bal) atomicAdd(&s_cnt[m], __popc(bal));
    }
    __syncthreads();
    if (threadIdx.x < NX) {
      const int m = threadIdx.x;
      const int64_t lo = s_lo[m], len = s_hi[m] - s_lo[m];
      if (len > 0) {
        const int64_t stride = (len + blockDim.x - 1) / blockDim.x;
        const int64_t c = s_cnt[m];
        if (c == 0) {
          s_hi[m] = lo;
        } else {
          int64_t nlo = lo + (c - 1) * stride + 1;
          int64_t nhi = min(lo + c * stride, s_hi[m]);
          if (nlo > nhi) nlo = nhi;
          s_lo[m] = nlo;
          s_hi[m] = nhi;
          if (nhi > nlo) atomicAdd(&s_open, 1);
        }
      }
    }
    __syncthreads();
    if (s_open == 0) break;
    __syncthreads();
  }
  if (threadIdx.x < NX) res[threadIdx.x] = s_lo[threadIdx.x];
  __syncthreads();
}

// Spread one return (cell coordinate u, value delta) into the tile.
template <typename T, int KERNEL>
__device__ __forceinline__ void spread_one(T* tile, const T* E3, const SpreadParams& p, int64_t L,
                                           int Tlen, double u, double delta) {
  const double fb = floor(u);
  int64_t b0 = (int64_t)fb;
  const T d = (T)(u - fb);   // offset of the source from cell b0, in [0, 1)
  const T dl = (T)delta;
  auto put = [&](int k, T v) {
    int64_t c = b0 + k;
    if (c < 0) c += p.Mr;
    else if (c >= p.Mr) c -= p.Mr;
    int64_t lc = c - L;
    if (lc >= 0 && lc < Tlen) atomicAdd(tile + lc, dl * v);
  };
  if (KERNEL == MM_KERNEL_GAUSS) {
    // Eq. (17) / Algorithm 8: exp(-t1 (k - d)^2) = E3_k * E1 * E2^k
    const T t1 = (T)p.g_t1;
    const T E1 = Fn<T>::exp_(-t1 * d * d);
    const T E2 = Fn<T>::exp_((T)2 * t1 * d);
    const T E2i = Fn<T>::exp_((T)-2 * t1 * d);
    put(0, E1);
    T pw = (T)1;
    for (int k = 1; k <= p.khi; ++k) { pw *= E2; put(k, E3[k] * E1 * pw); }
    pw = (T)1;
    for (int k = 1; k <= -p.klo; ++k) { pw *= E2i; put(-k, E3[k] * E1 * pw); }
  } else if (KERNEL == MM_KERNEL_ES) {
    // Eq. (9) rescaled to half-width M_sp cells: exp(beta (sqrt(1 - x^2) - 1))
    const T beta = (T)p.es_beta, iw = (T)p.es_inv_w;
    for (int k = p.klo; k <= p.khi; ++k) {
      T x = ((T)k - d) * iw;
      T v = (T)1 - x * x;
      if (v >= (T)0) put(k, Fn<T>::exp_(beta * (Fn<T>::sqrt_(v) - (T)1)));
    }
  } else {
    // Eq. (7) with the distance in cells, normalised to phi(0) = 1
    const T b = (T)p.kb_b, m2 = (T)p.msp * (T)p.msp, ck = (T)(p.kb_inv_phi0 / kPi);
    for (int k = p.klo; k <= p.khi; ++k) {
      T x = (T)k - d;
      T s2 = m2 - x * x;
      T v;
      if (s2 > (T)0) {
        T s = Fn<T>::sqrt_(s2);
        v = Fn<T>::sinh_(b * s) / s * ck;
      } else if (s2 < (T)0) {
        T s = Fn<T>::sqrt_(-s2);
        v = Fn<T>::sin_(b * s) / s * ck;
      } else {
        v = b * ck;
      }
      put(k, v);
    }
  }
}

template <typename T, int KERNEL>
__global__ void __launch_bounds__(256) k_spread(const int64_t* __restrict__ off, const double* __restrict__ t,
                                                const double* __restrict__ logp, const double* __restrict__ bounds,
                                                const int* __restrict__ gate, SpreadParams p, T* __restrict__ grid,
                                                int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tile = reinterpret_cast<T*>(smem_raw);
  __shared__ T E3[32];
  __shared__ int64_t r_lo[3], r_hi[3];
  __shared__ int s_flags;
  if (*gate) return;  // uniform: the whole block leaves
  const int a = blockIdx.y;
  const int64_t L = (int64_t)blockIdx.x * p.tile;
  const int Tlen = (int)min((int64_t)p.tile, p.Mr - L);
  for (int c = threadIdx.x; c < Tlen; c += blockDim.x) tile[c] = (T)0;
  if (KERNEL == MM_KERNEL_GAUSS && threadIdx.x <= p.msp && threadIdx.x < 32)
    E3[threadIdx.x] = (T)exp(-p.g_t1 * (double)threadIdx.x * (double)threadIdx.x);

  const double t0 = bounds[0];
  const double scale = (double)p.Mr / (bounds[1] - t0);
  const int64_t e0 = off[a], eend = off[a + 1];
  const int64_t e1 = eend > e0 ? eend - 1 : e0;  // returns live at h in [e0, e1)
  // Event ranges whose stencils reach this tile: b0 in [L - khi, L + Tlen - klo)
  // and its two periodic images, clipped to b0 in [0, M_r].
  __shared__ double s_x[6];
  if (threadIdx.x == 0) {
    s_flags = 0;
    const double top = (double)p.Mr + 1.0;
    for (int m = -1; m <= 1; ++m) {
      double A = fmax((double)(L - p.khi + m * p.Mr), 0.0);
      double B = fmin((double)(L + Tlen - p.klo + m * p.Mr), top);
      if (!(A < B)) { A = 0.0; B = 0.0; }
      s_x[2 * (m + 1)] = A;
      s_x[2 * (m + 1) + 1] = B;
    }
  }
  __syncthreads();
  if (p.single_tile) {
    if (threadIdx.x == 0) {
      r_lo[0] = e0; r_hi[0] = e1;
      r_lo[1] = r_hi[1] = r_lo[2] = r_hi[2] = 0;
    }
  } else {
    __shared__ int64_t s_res[6];
    block_first_ge<6>(t, e0, e1, t0, scale, s_x, s_res);
    if (threadIdx.x == 0) {
      for (int r = 0; r < 3; ++r) {
        bool empty = !(s_x[2 * r] < s_x[2 * r + 1]);
        r_lo[r] = empty ? 0 : s_res[2 * r];
        r_hi[r] = empty ? 0 : s_res[2 * r + 1];
      }
    }
  }
  __syncthreads();
  int flags = 0;
  for (int r = 0; r < 3; ++r) {
    for (int64_t h = r_lo[r] + threadIdx.x; h < r_hi[r]; h += blockDim.x) {
      const double th = t[h];
      const double tn = t[h + 1];
      if (!(th < tn)) flags |= (th == tn) ? ST_DUPLICATE : ST_UNSORTED;
      const double u = (th - t0) * scale;
      const double delta = logp[h + 1] - logp[h];
      if (!(isfinite(u) && isfinite(delta)) || u < 0.0 || u > (double)p.Mr) {
        flags |= ST_NONFINITE;
        continue;
      }
      spread_one<T, KERNEL>(tile, E3, p, L, Tlen, u, delta);
    }
  }
  if (flags) atomicOr(&s_flags, flags);
  __syncthreads();
  if (threadIdx.x == 0 && s_flags) atomicOr(status, s_flags);
  T* g = grid + (int64_t)a * p.Mr + L;
  for (int c = threadIdx.x; c < Tlen; c += blockDim.x) g[c] = tile[c];
}

template <typename T>
static cudaError_t launch_spread_t(const int64_t* off, const double* t, const double* logp,
                                   const double* bounds, const SpreadParams& p, T* grid, int* status,
                                   cudaStream_t s) {
  dim3 grd(p.ntiles, p.D);
  size_t smem = (size_t)p.tile * sizeof(T);
  const int* gate = status + 1;
  cudaError_t e = cudaSuccess;
#define MM_SPREAD_CASE(K)                                                                        \
  case K: {                                                                                      \
    auto fn = k_spread<T, K>;                                                                    \
    if (smem > 48 * 1024) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (e != cudaSuccess) return e;                                                              \
    fn<<<grd, 256, smem, s>>>(off, t, logp, bounds, gate, p, grid, status);                       \
    break;                                                                                       \
  }
  switch (p.kernel) {
    MM_SPREAD_CASE(MM_KERNEL_GAUSS)
    MM_SPREAD_CASE(MM_KERNEL_KB)
    MM_SPREAD_CASE(MM_KERNEL_ES)
    default: return cudaErrorInvalidValue;
  }
#undef MM_SPREAD_CASE
  return cudaGetLastError();
}

cudaError_t launch_spread_f32(const int64_t* off, const double* t, const double* logp, const double* bounds,
                              const SpreadParams& p, float* grid, int* status, cudaStream_t s) {
  return launch_spread_t<float>(off, t, logp, bounds, p, grid, status, s);
}
cudaError_t launch_spread_f64(const int64_t* off, const double* t, const double* logp, const double* bounds,
                              const SpreadParams& p, double* grid, int* status, cudaStream_t s) {
  return launch_spread_t<double>(off, t, logp, bounds, p, grid, status, s);
}

}  // namespace mmgpu
