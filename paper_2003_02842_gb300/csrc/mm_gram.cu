// mm_gram.cu -- stage (d) of the hot path: the covariance of Algorithm 3
// step C (Eqs. (2)/(3)) as a Hermitian rank-(2N+1) update of the
// coefficients, and the correlation of its last step.
//
// With F-convention coefficients F_i(k) (k = 0..N) and basis weights w_k,
//   Sigma_ij = (2 pi)^2 sum_{|k|<=N} w_k conj(F_i(k)) F_j(k)
//            = sum_{k=0..N} W_k (Re F_i Re F_j + Im F_i Im F_j) (2 pi)^2,
// W_0 = w_0, W_k = 2 w_k (k >= 1), because the terms of k and -k are complex
// conjugates. So Sigma = A A^T for the real D x 2(N+1) matrix A whose row i
// is (F_i(k) interleaved re, im) scaled by s_k = 2 pi sqrt(W_k): a real SYRK
// whose K-major operand is exactly the complex64 coefficient array.
//
// Mixed precision: one CTA per (output tile pair, K-split) stages 128-row
// tiles of A in shared memory (converted to split bf16 or split tf32 in the
// canonical 128-byte-swizzled K-major layout), and one thread issues
// tcgen05.mma (hi*hi + hi*lo + lo*hi) into a TMEM accumulator; commits are
// tracked by mbarriers so the next tile is staged while the tensor core runs.
// Every wait is bounded: after the plan's wait limit (1 s unless
// mm_plan_set_wait_limit changed it) it records MM_ERR_TIMEOUT, and the CTA
// lets the MMAs it issued finish before it frees its TMEM.
// The split-K partial products meet in an FP32 accumulator through vector
// reductions in L2 (red.global.add.v4.f32); k_corr_acc then normalises in
// FP64. FP64 path: a CUDA-core tiled kernel writing per-split partial tiles
// that k_reduce_corr sums in FP64 before the same normalisation.
#include <cuda_bf16.h>
#include <math.h>

#include "mm_async.cuh"
#include "mm_common.cuh"
#include "mm_tc.cuh"

namespace mmgpu {

// ------------------------------------------------------------ weights
template <typename T>
__global__ void k_gram_weights(int basis, int N, T* wsq) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > N) return;
  const double w = (basis == MM_BASIS_DIRICHLET) ? 1.0 / (2.0 * N + 1.0)
                                                 : (1.0 - (double)k / (double)N) / (N + 1.0);
  const double W = (k == 0) ? w : 2.0 * w;
  wsq[k] = (T)(2.0 * kPi * sqrt(fmax(W, 0.0)));
}

cudaError_t launch_gram_weights(int basis, int N, bool fp64, void* wsq, cudaStream_t s) {
  const int blocks = (N + 1 + 255) / 256;
  if (fp64) k_gram_weights<double><<<blocks, 256, 0, s>>>(basis, N, (double*)wsq);
  else k_gram_weights<float><<<blocks, 256, 0, s>>>(basis, N, (float*)wsq);
  return cudaGetLastError();
}

// ------------------------------------------------------------ FP64 path
// 64 x 64 output tile per block, 256 threads with a 4 x 4 micro-tile each,
// K in chunks of 16 complex modes.
__global__ void __launch_bounds__(256) k_gram_f64(const double2* __restrict__ F, GramParams g,
                                                  const double* __restrict__ wsq, double* __restrict__ partial) {
  __shared__ double As[32][65];
  __shared__ double Bs[32][65];
  int I, J;
  pair_of(blockIdx.y, g.ntiles, I, J);
  const int s = blockIdx.x;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  const int c0 = s * g.chunks_per_split;
  const int c1 = min(c0 + g.chunks_per_split, g.nchunks);
  for (int c = c0; c < c1; ++c) {
    const int kb = c * 16;
    for (int idx = threadIdx.x; idx < 2 * 64 * 16; idx += 256) {
      const int which = idx >> 10;  // 0: A rows, 1: B rows
      const int r = (idx >> 4) & 63, kk = idx & 15;
      const int row = (which ? J : I) * 64 + r;
      const int k = kb + kk;
      double2 v = {0.0, 0.0};
      if (row < g.D && k <= g.N) {
        v = F[(int64_t)row * g.ld + k];
        const double sc = wsq[k];
        v.x *= sc;
        v.y *= sc;
      }
      if (which) { Bs[2 * kk][r] = v.x; Bs[2 * kk + 1][r] = v.y; }
      else { As[2 * kk][r] = v.x; As[2 * kk + 1][r] = v.y; }
    }
    __syncthreads();
#pragma unroll 4
    for (int kr = 0; kr < 32; ++kr) {
      double a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) { a[q] = As[kr][ty * 4 + q]; b[q] = Bs[kr][tx * 4 + q]; }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
  }
  double* out = partial + ((int64_t)blockIdx.y * g.splits + s) * 64 * 64;
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) out[(ty * 4 + x) * 64 + tx * 4 + y] = acc[x][y];
}

cudaError_t launch_gram_f64(const void* coeffs, const GramParams& g, const double* wsq, double* partial,
                            cudaStream_t s) {
  dim3 grd(g.splits, g.npairs);
  k_gram_f64<<<grd, 256, 0, s>>>((const double2*)coeffs, g, wsq, partial);
  return cudaGetLastError();
}

// ------------------------------------------------------------ tcgen05 path
constexpr int kTcThreads = 512;
constexpr int kTcWarps = kTcThreads / 32;
constexpr int kRowsPerWarp = 128 / kTcWarps;  // operand rows a warp converts

size_t gram_tc_smem(int, bool two_tiles) {
  return (size_t)2 /*stages*/ * (two_tiles ? 4 : 2) * kTileBytes + 1024 /*alignment slack*/;
}

// Byte offset of the 4-byte (bf16 pair) or 8-byte (tf32 pair) element at
// row r, byte column cb of a 128B-swizzled K-major tile.
__device__ __forceinline__ uint32_t sw128_off(int r, int cb) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((cb >> 4) ^ (r & 7)) << 4) | (cb & 15)));
}

// One K-chunk of the operand rows a thread owns, held in registers between
// the global load and the conversion into shared memory, so that the loads
// of chunk c+1 are in flight while chunk c is converted and multiplied.
// MODE 0: 32 complex modes per chunk, one per lane, kRowsPerWarp rows per warp.
// MODE 1: 16 complex modes per chunk, two rows per warp step, kRowsPerWarp rows per warp.
template <int MODE>
struct Chunk {
  static constexpr int R = MODE == 0 ? kRowsPerWarp : kRowsPerWarp / 2;
  float2 v[R];
  float sc;
};

template <int MODE>
__device__ __forceinline__ void load_chunk(const float2* __restrict__ F, const GramParams& g,
                                           const float* __restrict__ wsq, int row0, int kbase, Chunk<MODE>& c) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = MODE == 0 ? lane : (lane & 15);
  const int half = MODE == 0 ? 0 : (lane >> 4);
  const int k = kbase + l;
  const bool kin = k <= g.N;
  c.sc = kin ? __ldg(wsq + k) : 0.0f;
#pragma unroll
  for (int rr = 0; rr < Chunk<MODE>::R; ++rr) {
    const int r = warp * kRowsPerWarp + (MODE == 0 ? rr : rr * 2 + half);
    const int row = row0 + r;
    c.v[rr] = (kin && row < g.D) ? __ldg(F + (int64_t)row * g.ld + k) : make_float2(0.f, 0.f);
  }
}

// Scale by s_k = 2 pi sqrt(W_k), split into hi + lo (bf16 or tf32) and write
// both into the 128B-swizzled K-major tiles.
template <int MODE>
__device__ __forceinline__ void store_chunk(const Chunk<MODE>& c, uint8_t* hi, uint8_t* lo) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (MODE == 0) {
#pragma unroll
    for (int rr = 0; rr < kRowsPerWarp; ++rr) {
      const int r = warp * kRowsPerWarp + rr;
      const float xr = c.v[rr].x * c.sc, xi = c.v[rr].y * c.sc;
      // (re, im) rounded as one packed pair, then the pair of residuals
      const __nv_bfloat162 H = __floats2bfloat162_rn(xr, xi);
      const __nv_bfloat162 L = __floats2bfloat162_rn(xr - __low2float(H), xi - __high2float(H));
      const uint32_t off = sw128_off(r, lane * 4);
      *reinterpret_cast<__nv_bfloat162*>(hi + off) = H;
      *reinterpret_cast<__nv_bfloat162*>(lo + off) = L;
    }
  } else {
    const int half = lane >> 4, l = lane & 15;
#pragma unroll
    for (int rr = 0; rr < kRowsPerWarp / 2; ++rr) {
      const int r = warp * kRowsPerWarp + rr * 2 + half;
      const float xr = c.v[rr].x * c.sc, xi = c.v[rr].y * c.sc;
      const uint32_t hr = f32_to_tf32(xr), hi_ = f32_to_tf32(xi);
      const uint32_t lr = f32_to_tf32(xr - __uint_as_float(hr));
      const uint32_t li = f32_to_tf32(xi - __uint_as_float(hi_));
      const uint32_t off = sw128_off(r, l * 8);
      *reinterpret_cast<uint2*>(hi + off) = make_uint2(hr, hi_);
      *reinterpret_cast<uint2*>(lo + off) = make_uint2(lr, li);
    }
  }
}

// One CTA per (output tile pair I <= J, K-split): the split's partial
// 128 x 128 product accumulates in TMEM and is then added into the FP32
// accumulator acc (row stride Dp) with vector reductions in L2.
// 1 / sqrt(v) in float64 for a float32 v > 0: the single-precision
// reciprocal square root as a seed (relative error below 2^-21), then two
// Newton-Raphson steps y <- y (3 - v y^2) / 2, each of which squares the
// relative error (to below 2^-40, then to float64 rounding). GB300 runs
// float64 at a small fraction of the float32 rate, and its float64 square
// root and division are long instruction sequences.
__device__ __forceinline__ double inv_sqrt_f64(float v) {
  const double x = (double)v;
  double y = (double)rsqrtf(v);
  y = y * fma(-0.5 * x, y * y, 1.5);
  y = y * fma(-0.5 * x, y * y, 1.5);
  return y;
}

// Sigma and R from the accumulator by one CTA (the last split to finish):
// the same arithmetic as k_corr_acc, block-strided over the D x Dp entries.
__device__ void corr_epilogue_block(const float* __restrict__ acc, const GramParams& g, float* __restrict__ sigma,
                                    float* __restrict__ R, float* __restrict__ zero_next, double* s_inv, int* status) {
  for (int d = threadIdx.x; d < g.D; d += blockDim.x) {
    const float v = __ldcg(acc + (int64_t)d * g.Dp + d);
    s_inv[d] = v > 0.0f ? inv_sqrt_f64(v) : 0.0;
  }
  __syncthreads();
  bool zero = false;
  for (int e = threadIdx.x; e < g.D * g.Dp; e += blockDim.x) {
    const int i = e / g.Dp, j = e - i * g.Dp;
    if (zero_next) zero_next[e] = 0.0f;
    if (j >= g.D) continue;
    // (min, max) is in an accumulated tile pair; reading it for both (i, j)
    // and (j, i), with the commuting product a * b, makes Sigma and R exactly
    // symmetric (the split-K sums of acc[i][j] and acc[j][i] within a
    // diagonal tile round in different orders)
    const double v = (double)__ldcg(acc + (int64_t)min(i, j) * g.Dp + max(i, j));
    const double a = s_inv[i], b = s_inv[j];
    double r;
    if (a > 0.0 && b > 0.0) r = (i == j) ? 1.0 : v * (a * b);
    else {
      r = __longlong_as_double(0x7ff8000000000000ll);
      if (i == j) zero = true;
    }
    if (sigma) sigma[(int64_t)i * g.D + j] = (float)v;
    if (R) R[(int64_t)i * g.D + j] = (float)r;
  }
  if (zero) atomicOr(status, ST_ZERO_VAR);
}

template <int MODE>
__global__ void __launch_bounds__(kTcThreads, 2) k_gram_tc(const float2* __restrict__ F, GramParams g,
                                                           const float* __restrict__ wsq, float* __restrict__ acc,
                                                           int* status, int* done, float* sigma, float* Rout,
                                                           float* zero_next) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;

  int I, J;
  pair_of(blockIdx.y, g.ntiles, I, J);
  const bool two = I != J;
  // the K-chunks spread evenly over the splits (at most chunks_per_split each)
  const int s = blockIdx.x;
  const int c0 = (int)((int64_t)s * g.nchunks / g.splits);
  const int c1 = (int)((int64_t)(s + 1) * g.nchunks / g.splits);
  const int nit = c1 - c0;

  // 1024-byte aligned staging area: per stage [A_hi][A_lo]([B_hi][B_lo])
  const uint32_t base_s = smem_u32(smem_raw);
  uint8_t* base = smem_raw + (((base_s + 1023u) & ~1023u) - base_s);
  const int tiles_per_stage = two ? 4 : 2;

  const int rowsI = min(kTile, g.D - I * kTile);
  const int rowsJ = min(kTile, g.D - J * kTile);
  const int Nmma = ((rowsJ + 15) / 16) * 16;
  const uint32_t fmt = (MODE == 0) ? 1u : 2u;  // bf16 / tf32 operands
  const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(Nmma >> 3) << 17) |
                         ((uint32_t)(kTile >> 4) << 24);

  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  pdl_wait();     // the coefficients come from the FFT kernel
  pdl_trigger();  // the correlation epilogue may be scheduled

  const int chunk = g.chunk;
  Chunk<MODE> ca, cb;
  if (nit > 0) {
    load_chunk<MODE>(F, g, wsq, I * kTile, c0 * chunk, ca);
    if (two) load_chunk<MODE>(F, g, wsq, J * kTile, c0 * chunk, cb);
  }
  bool ok = true;
  int committed = -1;  // last K-chunk whose MMAs were issued and committed
  for (int it = 0; it < nit; ++it) {
    const int st = it & 1;
    if (it >= 2) {
      if (!mbar_wait(&bars[st], (uint32_t)(((it >> 1) - 1) & 1), g.wait_ns)) ok = false;
    }
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
    uint8_t* stg = base + (size_t)st * tiles_per_stage * kTileBytes;
    store_chunk<MODE>(ca, stg, stg + kTileBytes);
    if (two) store_chunk<MODE>(cb, stg + 2 * kTileBytes, stg + 3 * kTileBytes);
    if (it + 1 < nit) {
      const int kb = (c0 + it + 1) * chunk;
      load_chunk<MODE>(F, g, wsq, I * kTile, kb, ca);
      if (two) load_chunk<MODE>(F, g, wsq, J * kTile, kb, cb);
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint32_t a_hi = smem_u32(stg), a_lo = a_hi + kTileBytes;
      const uint32_t b_hi = two ? a_hi + 2 * kTileBytes : a_hi;
      const uint32_t b_lo = two ? a_hi + 3 * kTileBytes : a_lo;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {  // four 32-byte K steps per 128-byte row
        const uint32_t o = ks * 32;
        tc_mma<MODE>(tmem, sw128_desc(a_hi + o), sw128_desc(b_hi + o), idesc, (it > 0 || ks > 0) ? 1u : 0u);
        tc_mma<MODE>(tmem, sw128_desc(a_hi + o), sw128_desc(b_lo + o), idesc, 1u);
        tc_mma<MODE>(tmem, sw128_desc(a_lo + o), sw128_desc(b_hi + o), idesc, 1u);
      }
      tc_commit(&bars[st]);
    }
    committed = it;
  }
  // drain: the last commit covers every MMA issued before it. A wait that
  // gives up still lets those MMAs finish (at the fixed limit) before the
  // CTA frees its TMEM and shared memory.
  if (committed >= 0) {
    uint64_t* bar = &bars[committed & 1];
    const uint32_t par = (uint32_t)((committed >> 1) & 1);
    if (!mbar_wait(bar, par, g.wait_ns)) {
      ok = false;
      mbar_wait(bar, par, kWaitLimitNs);
    }
  }
  if (!ok) atomicOr(&s_fail, 1);
  tc_fence_after();
  __syncthreads();

  // warp w reads TMEM lanes 32 (w mod 4) .. + 31 (its lane quadrant); the
  // warps sharing a quadrant take alternate 16-column groups
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quad = warp & 3;
  const int r = quad * 32 + lane;
  if (!s_fail && nit > 0) {
    float* out = acc + (int64_t)(I * kTile + r) * g.Dp + J * kTile;
    for (int c = 16 * (warp >> 2); c < Nmma; c += 16 * (kTcWarps / 4)) {
      uint32_t v[16];
      tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c, v);
      if (r < rowsI) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (c + 4 * q < rowsJ)
            red_add_v4(out + c + 4 * q, __uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                       __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
      }
    }
  } else if (threadIdx.x == 0 && nit > 0) {
    atomicOr(status, ST_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
  if (done) {
    // the last CTA to finish turns the accumulator into Sigma and R (the
    // correlation epilogue without a separate launch) and re-arms the counter
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(done, 1) == (int)(gridDim.x * gridDim.y) - 1;
    __syncthreads();
    if (s_last) {
      __threadfence();
      corr_epilogue_block(acc, g, sigma, Rout, zero_next, reinterpret_cast<double*>(base), status);
      if (threadIdx.x == 0) *done = 0;
    }
  }
}

cudaError_t launch_gram_tc(int mode, const void* coeffs, const GramParams& g, const float* wsq, float* acc,
                           int* status, int* done, float* sigma, float* R, float* zero_next, cudaStream_t s) {
  const bool two = g.ntiles > 1;
  const size_t smem = gram_tc_smem(mode, two);
  dim3 grd(g.splits, g.npairs);
  cudaError_t e;
  if (mode == 0) {
    e = cudaFuncSetAttribute(k_gram_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_gram_tc<0>, grd, dim3(kTcThreads), smem, s, (const float2*)coeffs, g, wsq, acc, status, done,
                      sigma, R, zero_next);
  }
  e = cudaFuncSetAttribute(k_gram_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_gram_tc<1>, grd, dim3(kTcThreads), smem, s, (const float2*)coeffs, g, wsq, acc, status, done,
                    sigma, R, zero_next);
}

// Sigma and R from the FP32 accumulator of k_gram_tc (upper tile pairs only:
// entry (i, j) lives at acc[i][j] when tile(i) <= tile(j), else acc[j][i];
// both triangles read acc[min(i, j)][max(i, j)]).
// The normalisation R_ij = Sigma_ij / (sqrt(Sigma_ii) sqrt(Sigma_jj)) is in
// FP64; R_ii = 1 exactly; zero variance gives NaN and a status. The block
// also clears the matching entries of zero_next, the accumulator the next
// call will use.
__global__ void __launch_bounds__(256) k_corr_acc(const float* __restrict__ acc, GramParams g, float* __restrict__ sigma,
                                                  float* __restrict__ R, float* __restrict__ zero_next, int* status) {
  __shared__ double s_inv_i[16], s_inv_j[16];
  pdl_wait();  // the accumulator comes from the contraction kernel
  pdl_trigger();
  const int li = threadIdx.x >> 4, lj = threadIdx.x & 15;
  const int j = blockIdx.x * 16 + lj;
  const int i = blockIdx.y * 16 + li;
  // 1 / sqrt(Sigma_dd) in FP64 once per row and column of the block
  if (threadIdx.x < 32) {
    const int q = threadIdx.x & 15;
    const int d = (threadIdx.x < 16 ? blockIdx.y : blockIdx.x) * 16 + q;
    double inv = 0.0;
    if (d < g.D) {
      const float v = acc[(int64_t)d * g.Dp + d];
      inv = v > 0.0f ? inv_sqrt_f64(v) : 0.0;
    }
    if (threadIdx.x < 16) s_inv_i[q] = inv;
    else s_inv_j[q] = inv;
  }
  __syncthreads();
  if (i >= g.D || j >= g.Dp) return;
  if (zero_next) zero_next[(int64_t)i * g.Dp + j] = 0.0f;
  if (j >= g.D) return;
  // read (min, max) for both triangles: exactly symmetric Sigma and R
  const double v = (double)acc[(int64_t)min(i, j) * g.Dp + max(i, j)];
  const double a = s_inv_i[li], b = s_inv_j[lj];
  double r;
  if (a > 0.0 && b > 0.0) r = (i == j) ? 1.0 : v * (a * b);
  else {
    r = __longlong_as_double(0x7ff8000000000000ll);
    if (i == j) atomicOr(status, ST_ZERO_VAR);
  }
  if (sigma) sigma[(int64_t)i * g.D + j] = (float)v;
  if (R) R[(int64_t)i * g.D + j] = (float)r;
}

cudaError_t launch_corr_acc(const float* acc, const GramParams& g, float* sigma, float* R, float* zero_next,
                            int* status, cudaStream_t s) {
  dim3 grd((g.Dp + 15) / 16, (g.D + 15) / 16);
  return launch_pdl(k_corr_acc, grd, dim3(256), 0, s, acc, g, sigma, R, zero_next, status);
}

// ------------------------------------------------------------ reduce + R
// Sums the split partials in FP64 for a 16 x 16 block of (i, j), i-block <=
// j-block, and writes Sigma and R = Sigma_ij / (sqrt(Sigma_ii) sqrt(Sigma_jj))
// to both triangles. R_ii is exactly 1; zero variance gives NaN and a status.
template <typename TP>
__device__ __forceinline__ double sum_splits(const TP* __restrict__ partial, const GramParams& g, int i, int j) {
  const int I = i / g.tile, J = j / g.tile;
  const int p = I * g.ntiles - I * (I - 1) / 2 + (J - I);
  const int64_t base = (int64_t)p * g.splits * g.tile * g.tile + (int64_t)(i % g.tile) * g.tile + (j % g.tile);
  const int64_t step = (int64_t)g.tile * g.tile;
  double acc = 0.0;
  for (int s = 0; s < g.splits; ++s) acc += (double)partial[base + s * step];
  return acc;
}

template <typename TP, typename TO>
__global__ void __launch_bounds__(256) k_reduce_corr(const TP* __restrict__ partial, GramParams g,
                                                     TO* __restrict__ sigma, TO* __restrict__ R, int* status) {
  __shared__ double s_di[16], s_dj[16];
  const int nb = (g.D + 15) / 16;
  int bi, bj;
  pair_of(blockIdx.x, nb, bi, bj);
  const int li = threadIdx.x >> 4, lj = threadIdx.x & 15;
  if (threadIdx.x < 32) {
    const int q = threadIdx.x & 15;
    const int d = (threadIdx.x < 16 ? bi : bj) * 16 + q;
    const double v = (d < g.D) ? sum_splits(partial, g, d, d) : 1.0;
    if (threadIdx.x < 16) s_di[q] = v;
    else s_dj[q] = v;
  }
  __syncthreads();
  const int i = bi * 16 + li, j = bj * 16 + lj;
  if (i >= g.D || j >= g.D || (bi == bj && j < i)) return;
  const double v = (i == j) ? s_di[li] : sum_splits(partial, g, i, j);
  const double a = s_di[li], b = s_dj[lj];
  double r;
  if (a > 0.0 && b > 0.0) r = (i == j) ? 1.0 : v / (sqrt(a) * sqrt(b));
  else {
    r = __longlong_as_double(0x7ff8000000000000ll);
    atomicOr(status, ST_ZERO_VAR);
  }
  if (sigma) {
    sigma[(int64_t)i * g.D + j] = (TO)v;
    sigma[(int64_t)j * g.D + i] = (TO)v;
  }
  if (R) {
    R[(int64_t)i * g.D + j] = (TO)r;
    R[(int64_t)j * g.D + i] = (TO)r;
  }
}

cudaError_t launch_reduce_corr(bool fp64, const void* partial, const GramParams& g, void* sigma, void* R,
                               int* status, cudaStream_t s) {
  const int nb = (g.D + 15) / 16;
  const int blocks = nb * (nb + 1) / 2;
  if (fp64)
    k_reduce_corr<double, double><<<blocks, 256, 0, s>>>((const double*)partial, g, (double*)sigma, (double*)R,
                                                          status);
  else
    k_reduce_corr<float, float><<<blocks, 256, 0, s>>>((const float*)partial, g, (float*)sigma, (float*)R, status);
  return cudaGetLastError();
}

}  // namespace mmgpu
