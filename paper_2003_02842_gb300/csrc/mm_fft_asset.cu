// mm_fft_asset.cu -- stages (b) and (c) of the hot path for grids that fit in
// shared memory: each asset's spread grid (Eq. (12)) is read once from global
// memory (L2) into shared memory, transformed there by the length-M_r real FFT
// of Eq. (13) taken as an n = M_r/2-point complex FFT, and its deconvolved,
// truncated coefficients of Eq. (14) are written for k = 0..N.
//
// An asset is handled by one CTA when its row fits one CTA's shared memory,
// else by a cluster of two CTAs (decimation in time by 2, the halves joined
// through distributed shared memory; k_fft_asset_pair below). Two or three
// CTAs per asset with the first radix-2 or radix-3 step done while loading
// were measured slower on every workload and are not built: each CTA's time
// is set by latency, so splitting an asset only added load work.

// The local transform of L = R_1 R_2 ... R_s points (every R_p <= 32) runs in
// place in shared memory, pass p working on blocks of length L_p = R_p m_p
// with stride m_p = L / (R_1 ... R_p): each butterfly's R_p points are
// transformed in registers by a fully unrolled R_p-point DFT (a compile-time
// Cooley-Tukey split into 2-, 3-, 4-, 5- and 8-point DFTs with its twiddles
// folded into immediates) and stored back. With k = q_1 + R_1 (q_2 + R_2 (q_3
// + ...)) and rev(k) = sum_p q_p m_p, two orders are used:
//  - decimation in frequency (the default): natural-order input, so the grid
//    row lands in shared memory by bulk asynchronous copies; passes p = 1..s multiply output q of butterfly j by
//    w_{L_p}^{j q} after the DFT; output k ends up at position rev(k), which
//    the unpacking step reads;
//  - decimation in time: input k stored at position rev(k) (as the polynomial
//    scatter can write it, or by per-point asynchronous copies), passes p =
//    s..1 multiplying input r by w_{L_p}^{j r} before the DFT, output in
//    natural order.
#include <algorithm>
#include <utility>

#include "mm_async.cuh"
#include "mm_common.cuh"
#include "mm_fft_dev.cuh"
#include "mm_spread_dev.cuh"

namespace mmgpu {

namespace {

// ------------------------------------------------------------------------
// cos and sin of 2 pi p / q for integers, evaluated at compile time in double
// precision: the angle is reduced exactly to an eighth of a turn plus
// x = pi s / (4 q) in [0, pi/4], then Taylor series (error < 1e-17).
__host__ __device__ constexpr double ct_sin_series(double x) {
  double x2 = x * x, term = x, sum = x;
  for (int k = 1; k < 14; ++k) {
    term *= -x2 / (double)((2 * k) * (2 * k + 1));
    sum += term;
  }
  return sum;
}
__host__ __device__ constexpr double ct_cos_series(double x) {
  double x2 = x * x, term = 1.0, sum = 1.0;
  for (int k = 1; k < 14; ++k) {
    term *= -x2 / (double)((2 * k - 1) * (2 * k));
    sum += term;
  }
  return sum;
}
// which = 0: cos, 1: sin
__host__ __device__ constexpr double ct_trig(long p, long q, int which) {
  long r = p % q;
  if (r < 0) r += q;
  const long o = (8 * r) / q;       // octant
  const long s = 8 * r - o * q;     // remainder, angle = o pi/4 + pi s/(4q)
  const double x = kPi * (double)s / (4.0 * (double)q);
  const double y = kPi * (double)(q - s) / (4.0 * (double)q);  // pi/4 - x
  double c = 0, sn = 0;
  switch (o) {
    case 0: c = ct_cos_series(x); sn = ct_sin_series(x); break;
    case 1: c = ct_sin_series(y); sn = ct_cos_series(y); break;
    case 2: c = -ct_sin_series(x); sn = ct_cos_series(x); break;
    case 3: c = -ct_cos_series(y); sn = ct_sin_series(y); break;
    case 4: c = -ct_cos_series(x); sn = -ct_sin_series(x); break;
    case 5: c = -ct_sin_series(y); sn = -ct_cos_series(y); break;
    case 6: c = ct_sin_series(x); sn = -ct_cos_series(x); break;
    default: c = ct_cos_series(y); sn = -ct_sin_series(y); break;
  }
  return which == 0 ? c : sn;
}
constexpr double ct_abs(double x) { return x < 0 ? -x : x; }
static_assert(ct_abs(ct_trig(1, 6, 0) - 0.5) < 1e-15, "cos(pi/3)");
static_assert(ct_abs(ct_trig(1, 4, 1) - 1.0) < 1e-15, "sin(pi/2)");
static_assert(ct_abs(ct_trig(3, 8, 0) + 0.70710678118654752) < 1e-15, "cos(3pi/4)");
static_assert(ct_abs(ct_trig(2, 5, 1) - 0.58778525229247313) < 1e-15, "sin(4pi/5)");

template <int... I, typename F>
__device__ __forceinline__ void static_for_impl(std::integer_sequence<int, I...>, F&& f) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(std::make_integer_sequence<int, N>{}, f);
}

// u * w_R^E with w_R = e^{-2 pi i / R}; trivial angles cost no multiply.
template <int E, int R>
__device__ __forceinline__ Cplx<float> twmul(Cplx<float> u) {
  constexpr int e = ((E % R) + R) % R;
  if constexpr (e == 0) {
    return u;
  } else if constexpr (4 * e == R) {
    return Cplx<float>{u.y, -u.x};  // -i
  } else if constexpr (2 * e == R) {
    return Cplx<float>{-u.x, -u.y};
  } else if constexpr (4 * e == 3 * R) {
    return Cplx<float>{-u.y, u.x};  // +i
  } else {
    constexpr float c = (float)ct_trig(e, R, 0);
    constexpr float s = (float)ct_trig(e, R, 1);
    // (u.x + i u.y)(c - i s)
    return Cplx<float>{fmaf(u.x, c, u.y * s), fmaf(u.y, c, -u.x * s)};
  }
}

// Outer radix of the compile-time split R = A * (R / A).
__host__ __device__ constexpr int outer_radix(int R) {
  return (R % 8 == 0 && R > 8) ? 8 : (R % 5 == 0 && R > 5) ? 5 : (R % 4 == 0 && R > 4) ? 4 : (R % 3 == 0 && R > 3) ? 3 : 2;
}

// Forward R-point DFT in registers, natural order in and out.
template <int R>
struct Codelet {
  static __device__ __forceinline__ void run(Cplx<float>* v) {
    constexpr int A = outer_radix(R);
    constexpr int B = R / A;
    Cplx<float> t[R];
    static_for<A>([&](auto ia) {
      constexpr int a = decltype(ia)::value;
      Cplx<float> u[B];
#pragma unroll
      for (int m = 0; m < B; ++m) u[m] = v[A * m + a];
      Codelet<B>::run(u);
      static_for<B>([&](auto ib) {
        constexpr int b = decltype(ib)::value;
        t[a * B + b] = twmul<a * b, R>(u[b]);
      });
    });
#pragma unroll
    for (int b = 0; b < B; ++b) {
      Cplx<float> w[A];
#pragma unroll
      for (int a = 0; a < A; ++a) w[a] = t[a * B + b];
      Dft<float, A>::run(w);
#pragma unroll
      for (int c = 0; c < A; ++c) v[b + B * c] = w[c];
    }
  }
};
template <> struct Codelet<2> { static __device__ __forceinline__ void run(Cplx<float>* v) { Dft<float, 2>::run(v); } };
template <> struct Codelet<3> { static __device__ __forceinline__ void run(Cplx<float>* v) { Dft<float, 3>::run(v); } };
template <> struct Codelet<4> { static __device__ __forceinline__ void run(Cplx<float>* v) { Dft<float, 4>::run(v); } };
template <> struct Codelet<5> { static __device__ __forceinline__ void run(Cplx<float>* v) { Dft<float, 5>::run(v); } };
template <> struct Codelet<8> { static __device__ __forceinline__ void run(Cplx<float>* v) { Dft<float, 8>::run(v); } };

// The twiddles w^r (w = w_{L_p}^j, row j of the pass's anchors), r = 1..R-1,
// applied to v[r]: built from the four anchors w, w^2, w^3, w^4 of row j
// (shared memory) as (w^4)^(r/4) w^(r mod 4), at most R/4 + 1 rounded
// complex products per twiddle.
template <int R>
__device__ __forceinline__ void apply_twiddles(Cplx<float>* v, const float4* __restrict__ anc, int j) {
  const float4 a01 = anc[2 * j], a23 = anc[2 * j + 1];
  const Cplx<float> w1{a01.x, a01.y}, w2{a01.z, a01.w}, w3{a23.x, a23.y}, w4{a23.z, a23.w};
  Cplx<float> pw = w4;  // (w^4)^(q4) for q4 >= 1
#pragma unroll
  for (int q4 = 0; 4 * q4 < R; ++q4) {
#pragma unroll
    for (int rr = 0; rr < 4; ++rr) {
      const int r = 4 * q4 + rr;
      if (r == 0 || r >= R) continue;
      Cplx<float> t;
      if (q4 == 0) t = rr == 1 ? w1 : (rr == 2 ? w2 : w3);
      else if (rr == 0) t = pw;
      else t = cmul(pw, rr == 1 ? w1 : (rr == 2 ? w2 : w3));
      v[r] = cmul(v[r], t);
    }
    if (q4 >= 1) pw = cmul(pw, w4);
  }
}

// One pass of radix R and stride m over L points in place: decimation in
// time twiddles the inputs, decimation in frequency the outputs.
template <int R, bool DIF>
__device__ __forceinline__ void fft_pass(Cplx<float>* __restrict__ s, int L, int m, const float4* __restrict__ anc,
                                         int nth) {
  const int nbf = L / R;
  const unsigned mm = magic_of((unsigned)m);
  for (int i = threadIdx.x; i < nbf; i += nth) {
    const int b = fast_div(i, m, mm);
    const int j = i - b * m;
    const int base = b * (R * m) + j;
    Cplx<float> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s[base + r * m];
    if (!DIF && m > 1) apply_twiddles<R>(v, anc, j);
    Codelet<R>::run(v);
    if (DIF && m > 1) apply_twiddles<R>(v, anc, j);
#pragma unroll
    for (int q = 0; q < R; ++q) s[base + q * m] = v[q];
  }
}

template <bool DIF, bool BIG>
__device__ __forceinline__ void run_pass_t(int R, Cplx<float>* s, int L, int m, const float4* anc, int nth) {
  if constexpr (BIG) {
    switch (R) {
      case 18: fft_pass<18, DIF>(s, L, m, anc, nth); return;
      case 20: fft_pass<20, DIF>(s, L, m, anc, nth); return;
      case 24: fft_pass<24, DIF>(s, L, m, anc, nth); return;
      case 25: fft_pass<25, DIF>(s, L, m, anc, nth); return;
      case 27: fft_pass<27, DIF>(s, L, m, anc, nth); return;
      case 30: fft_pass<30, DIF>(s, L, m, anc, nth); return;
      case 32: fft_pass<32, DIF>(s, L, m, anc, nth); return;
      default: break;
    }
  }
  switch (R) {
    case 2: fft_pass<2, DIF>(s, L, m, anc, nth); break;
    case 3: fft_pass<3, DIF>(s, L, m, anc, nth); break;
    case 4: fft_pass<4, DIF>(s, L, m, anc, nth); break;
    case 5: fft_pass<5, DIF>(s, L, m, anc, nth); break;
    case 6: fft_pass<6, DIF>(s, L, m, anc, nth); break;
    case 8: fft_pass<8, DIF>(s, L, m, anc, nth); break;
    case 9: fft_pass<9, DIF>(s, L, m, anc, nth); break;
    case 10: fft_pass<10, DIF>(s, L, m, anc, nth); break;
    case 12: fft_pass<12, DIF>(s, L, m, anc, nth); break;
    case 15: fft_pass<15, DIF>(s, L, m, anc, nth); break;
    case 16: fft_pass<16, DIF>(s, L, m, anc, nth); break;
    default: break;  // the host plans only the radices above
  }
}

// Entry p of a per-pass array, selected without indexing it at run time (a
// run-time index would move the kernel parameter into local memory).
__device__ __forceinline__ int pick(const int (&a)[kMaxAssetPasses], int p) {
  static_assert(kMaxAssetPasses == 4, "pick() selects among four entries");
  return p == 0 ? a[0] : p == 1 ? a[1] : p == 2 ? a[2] : a[3];
}

// All passes of the local transform in the plan's order for its direction.
template <bool BIG>
__device__ __forceinline__ void run_passes(const AssetFft& f, Cplx<float>* s, const float4* anc, int nth) {
  for (int i = 0; i < f.npass; ++i) {
    const int p = f.dif ? i : f.npass - 1 - i;
    const int R = pick(f.rad, p), m = pick(f.stride, p);
    const float4* a = anc + 2 * pick(f.tw_off, p);
    if (f.dif) run_pass_t<true, BIG>(R, s, f.nl, m, a, nth);
    else run_pass_t<false, BIG>(R, s, f.nl, m, a, nth);
    __syncthreads();
  }
}

// Position of local input j in digit-reversed order.
__device__ __forceinline__ int digit_rev(int j, const AssetFft& f, const unsigned* mr) {
  int pos = 0;
#pragma unroll
  for (int p = 0; p < kMaxAssetPasses; ++p) {
    if (p < f.npass) {
      const int R = f.rad[p];
      const int q = fast_div(j, R, mr[p]);
      pos += (j - q * R) * f.stride[p];
      j = q;
    }
  }
  return pos;
}

// Shared-memory position of local output k: rev(k) after decimation in
// frequency (from the two digit-reversal tables: k = x + rev_lo y has
// rev(k) = T_lo[x] + T_hi[y], T_lo holding the first two digits' terms and
// T_hi the rest), k after decimation in time.
struct RevTab {
  const int* lo;
  const int* hi;
  int B;
  unsigned mB;
};
__device__ __forceinline__ int out_pos(int k, const AssetFft& f, const RevTab& t) {
  if (!f.dif) return k;
  const int y = fast_div(k, t.B, t.mB);
  return t.lo[k - y * t.B] + t.hi[y];
}

// Byte offset of the anchor rows in shared memory: after the nl complex
// points, rounded up to 16 bytes (nl may be odd) for the float4 accesses.
__host__ __device__ __forceinline__ size_t anchor_offset(int nl) { return ((size_t)nl * 8 + 15) & ~(size_t)15; }

// The two digit-reversal tables of a decimation-in-frequency plan, built in
// shared memory after the anchor rows (from the plan alone: no global reads).
template <int NTH>
__device__ __forceinline__ RevTab build_rev_tables(const AssetFft& f, unsigned char* smem_raw, const unsigned* mr) {
  RevTab rt{};
  if (!f.dif) return rt;
  int* tlo = reinterpret_cast<int*>(smem_raw + anchor_offset(f.nl) + (size_t)f.tw_rows * 32);
  int* thi = tlo + f.rev_lo;
  const int R0 = f.rad[0], R1 = f.npass >= 2 ? f.rad[1] : 1;
  for (int x = threadIdx.x; x < f.rev_lo; x += NTH) {
    const int q1 = fast_div(x, R0, mr[0]);
    tlo[x] = (x - q1 * R0) * f.stride[0] + (R1 > 1 ? q1 * f.stride[1] : 0);
  }
  for (int y = threadIdx.x; y < f.rev_hi; y += NTH) {
    int pos = 0, r = y;
#pragma unroll
    for (int p = 2; p < kMaxAssetPasses; ++p) {
      if (p < f.npass) {
        const int R = f.rad[p];
        const int q = fast_div(r, R, mr[p]);
        pos += (r - q * R) * f.stride[p];
        r = q;
      }
    }
    thi[y] = pos;
  }
  rt.lo = tlo;
  rt.hi = thi;
  rt.B = f.rev_lo;
  rt.mB = magic_of((unsigned)f.rev_lo);
  return rt;
}

// Distributed shared memory of a thread-block cluster.
__device__ __forceinline__ uint32_t peer_addr(const void* p, unsigned rank) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(p), r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ Cplx<float> ld_cluster(uint32_t addr) {
  float x, y;
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(x), "=f"(y) : "r"(addr) : "memory");
  return Cplx<float>{x, y};
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

constexpr uint32_t kBulkChunk = 32768;  // bytes per bulk copy instruction
// table reads in flight per thread in the unpacking step (fewer with more threads)
template <int NTH> constexpr int kUnpackBatch = NTH >= 1024 ? 4 : 8;
template <int NTH> constexpr int kPairBatch = NTH >= 1024 ? 2 : 4;  // the cluster variant (more values per mode)
constexpr int kPairThreads = 512; // one CTA of a pair per SM (each holds half an asset's grid)

// The local transform of a row held whole by one CTA, then the unpacking
// of the real-input transform and the deconvolution of the modes k <= N.
template <int NTH, bool BIG>
__device__ __forceinline__ void single_finish(const AssetFft& f, Cplx<float>* s, const float4* anc, int a,
                                              const RevTab& rt, const Cplx<float>* __restrict__ U,
                                              const float* __restrict__ decon, Cplx<float>* __restrict__ out) {
  constexpr int kUB = kUnpackBatch<NTH>;
  const int L = f.nl;
  run_passes<BIG>(f, s, anc, NTH);

  // unpack the real-input transform and deconvolve (Eq. (14)):
  // G(k) = (Z_k + conj Z_{n-k}) / 2 + w_{2n}^k (Z_k - conj Z_{n-k}) / (2i)
  //      = alpha_k Z_k + beta_k conj Z_{n-k},
  // alpha_k = (1 - i w_{2n}^k) / 2, beta_k = (1 + i w_{2n}^k) / 2, for the
  // modes k <= N (Z_0 pairs with itself). U[k] = w_{2n}^k and the
  // deconvolution factors are read kUB at a time per thread.
  Cplx<float>* oa = out + (size_t)a * (f.N + 1);
  for (int k0 = threadIdx.x; k0 <= f.N; k0 += NTH * kUB) {
    float dk[kUB];
    Cplx<float> Uk[kUB];
#pragma unroll
    for (int u = 0; u < kUB; ++u) {
      const int k = k0 + u * NTH;
      if (k <= f.N) {
        dk[u] = __ldg(decon + k);
        Uk[u] = U[k];
      }
    }
#pragma unroll
    for (int u = 0; u < kUB; ++u) {
      const int k = k0 + u * NTH;
      if (k <= f.N) {
        const int kn = k == 0 ? 0 : L - k;
        const Cplx<float> Zk = s[out_pos(k, f, rt)];
        const Cplx<float> Zc = cconj(s[out_pos(kn, f, rt)]);
        const Cplx<float> E = {0.5f * (Zk.x + Zc.x), 0.5f * (Zk.y + Zc.y)};
        const Cplx<float> dlt = csub(Zk, Zc);
        const Cplx<float> O = {0.5f * dlt.y, -0.5f * dlt.x};  // (Z_k - conj Z_{n-k}) / (2i)
        const Cplx<float> G = cadd(E, cmul(Uk[u], O));
        oa[k] = Cplx<float>{G.x * dk[u], G.y * dk[u]};
      }
    }
  }
}

template <int NTH, bool BIG>
__global__ void __launch_bounds__(NTH, 1)
    k_fft_asset(const float* __restrict__ grid, AssetFft f, const Cplx<float>* __restrict__ W,
                const Cplx<float>* __restrict__ tw, const Cplx<float>* __restrict__ U,
                const float* __restrict__ decon, Cplx<float>* __restrict__ out, const int* __restrict__ gate,
                int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cplx<float>* s = reinterpret_cast<Cplx<float>*>(smem_raw);
  float4* anc = reinterpret_cast<float4*>(smem_raw + anchor_offset(f.nl));  // twiddle anchors, 32 B per row
  unsigned mr[kMaxAssetPasses];
#pragma unroll
  for (int p = 0; p < kMaxAssetPasses; ++p) mr[p] = magic_of((unsigned)f.rad[p]);
  const RevTab rt = build_rev_tables<NTH>(f, smem_raw, mr);
  pdl_wait();         // the grid comes from the spreading kernel
  if (*gate) return;  // uniform: the whole block leaves
  pdl_trigger();      // the contraction may take the SMs this launch leaves free
  {
    // anchor rows: 16-byte asynchronous copies, waited for with the grid
    const float4* src = reinterpret_cast<const float4*>(tw);
    for (int i = threadIdx.x; i < 2 * f.tw_rows; i += NTH) {
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(anc + i);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src + i) : "memory");
    }
  }
  const int a = blockIdx.y;
  const int L = f.nl;

  // load in the order of the transform's direction
  const Cplx<float>* z = reinterpret_cast<const Cplx<float>*>(grid) + (size_t)a * f.n;
  if (f.pre_perm || (f.dif && f.split == 1)) {
    // the row as stored (natural order, or digit-reversed by the polynomial
    // scatter): bulk asynchronous copies of the whole row, 16-byte aligned
    // since n is even (the anchors' cp.async copies are waited for below)
    __shared__ __align__(8) uint64_t bar;
    const uint32_t bytes = (uint32_t)f.n * 8u;
    if (threadIdx.x == 0) {
      mbar_init(&bar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      mbar_expect_tx(&bar, bytes);
      const unsigned char* src = reinterpret_cast<const unsigned char*>(z);
      for (uint32_t o = 0; o < bytes; o += kBulkChunk) {
        const uint32_t cb = bytes - o < kBulkChunk ? bytes - o : kBulkChunk;
        bulk_g2s(smem_raw + o, src + o, cb, &bar);
      }
    }
    const bool ok = mbar_wait(&bar, 0, kWaitLimitNs);
    if (!__syncthreads_and(ok)) {
      // the copy did not land in time: report it, give it a bounded second
      // wait so no write into shared memory stays in flight, and leave
      if (threadIdx.x == 0) {
        atomicOr(status, ST_TIMEOUT);
        mbar_wait(&bar, 0, kWaitLimitNs);
      }
      asm volatile("cp.async.wait_all;" ::: "memory");
      __syncthreads();
      return;
    }
  } else {
    // asynchronous 8-byte copies straight into their shared-memory slots:
    // the whole grid row is in flight at once, no registers held
    for (int j = threadIdx.x; j < L; j += NTH) {
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(s + digit_rev(j, f, mr));
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(z + j) : "memory");
    }
  }
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  single_finish<NTH, BIG>(f, s, anc, a, rt, U, decon, out);
}

// The pair's local transform, the join of the two halves through
// distributed shared memory and the unpacking and deconvolution of the
// modes k = c, c + 2, ... <= N (CTA c of the cluster).
template <int NTH, bool BIG>
__device__ __forceinline__ void pair_finish(const AssetFft& f, Cplx<float>* s, const float4* anc, unsigned c, int a,
                                            const RevTab& rt, const Cplx<float>* __restrict__ W,
                                            const Cplx<float>* __restrict__ U, const float* __restrict__ decon,
                                            Cplx<float>* __restrict__ out) {
  constexpr int kPB = kPairBatch<NTH>;
  const int L = f.nl;
  run_passes<BIG>(f, s, anc, NTH);
  cluster_sync_all();  // both halves transformed and visible to the partner
  const uint32_t peer = peer_addr(s, c ^ 1u);
  Cplx<float>* oa = out + (size_t)a * (f.N + 1);
  for (int k0 = (int)c + 2 * (int)threadIdx.x; k0 <= f.N; k0 += 2 * NTH * kPB) {
    float dk[kPB];
    Cplx<float> Uk[kPB], Wk[kPB], A0[kPB], A1[kPB], B0[kPB],
        B1[kPB];
#pragma unroll
    for (int u = 0; u < kPB; ++u) {
      const int k = k0 + u * 2 * NTH;
      if (k <= f.N) {
        const int j = k == 0 ? 0 : L - k;  // (n - k) mod L
        dk[u] = __ldg(decon + k);
        Uk[u] = U[k];
        Wk[u] = W[k];
        const int pk = out_pos(k, f, rt), pj = out_pos(j, f, rt);  // the same layout in both CTAs
        const Cplx<float> lk = s[pk], lj = s[pj];
        const Cplx<float> rk = ld_cluster(peer + 8u * (uint32_t)pk), rj = ld_cluster(peer + 8u * (uint32_t)pj);
        A0[u] = c == 0 ? lk : rk;  // X_0[k]
        A1[u] = c == 0 ? rk : lk;  // X_1[k]
        B0[u] = c == 0 ? lj : rj;  // X_0[(n-k) mod L]
        B1[u] = c == 0 ? rj : lj;  // X_1[(n-k) mod L]
      }
    }
#pragma unroll
    for (int u = 0; u < kPB; ++u) {
      const int k = k0 + u * 2 * NTH;
      if (k <= f.N) {
        const Cplx<float> Zk = cadd(A0[u], cmul(Wk[u], A1[u]));
        const Cplx<float> Znk = cadd(B0[u], cmul(cconj(Wk[u]), B1[u]));  // w_n^{n-k} = conj(w_n^k)
        const Cplx<float> Zc = cconj(Znk);
        const Cplx<float> E = {0.5f * (Zk.x + Zc.x), 0.5f * (Zk.y + Zc.y)};
        const Cplx<float> dlt = csub(Zk, Zc);
        const Cplx<float> O = {0.5f * dlt.y, -0.5f * dlt.x};  // (Z_k - conj Z_{n-k}) / (2i)
        const Cplx<float> G = cadd(E, cmul(Uk[u], O));
        oa[k] = Cplx<float>{G.x * dk[u], G.y * dk[u]};
      }
    }
  }
  cluster_sync_all();  // the partner has finished reading this CTA's shared memory
}

// Two CTAs per asset as a thread-block cluster (decimation in time by 2):
// CTA c transforms x_c[m] = z[2m + c], m < L = n/2, loaded straight into
// its shared memory by asynchronous copies; then
//   Z_k = X_0[k mod L] + w_n^k X_1[k mod L]
// joins the halves, each CTA reading its partner's X through distributed
// shared memory while it unpacks and deconvolves every other mode.
template <int NTH, bool BIG>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NTH, 1)
    k_fft_asset_pair(const float* __restrict__ grid, AssetFft f, const Cplx<float>* __restrict__ W,
                     const Cplx<float>* __restrict__ tw, const Cplx<float>* __restrict__ U,
                     const float* __restrict__ decon, Cplx<float>* __restrict__ out, const int* __restrict__ gate) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cplx<float>* s = reinterpret_cast<Cplx<float>*>(smem_raw);
  float4* anc = reinterpret_cast<float4*>(smem_raw + anchor_offset(f.nl));
  unsigned c;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(c));
  const int a = blockIdx.y;
  const int L = f.nl;
  unsigned mr[kMaxAssetPasses];
#pragma unroll
  for (int p = 0; p < kMaxAssetPasses; ++p) mr[p] = magic_of((unsigned)f.rad[p]);
  const RevTab rt = build_rev_tables<NTH>(f, smem_raw, mr);
  pdl_wait();  // the grid comes from the spreading kernel
  // every CTA of the cluster reads the same gate word: both leave or neither
  if (*gate) return;
  pdl_trigger();
  {
    const float4* src = reinterpret_cast<const float4*>(tw);
    for (int i = threadIdx.x; i < 2 * f.tw_rows; i += NTH) {
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(anc + i);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src + i) : "memory");
    }
  }
  const Cplx<float>* z = reinterpret_cast<const Cplx<float>*>(grid) + (size_t)a * f.n + c;
  for (int m = threadIdx.x; m < L; m += NTH) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(s + (f.dif ? m : digit_rev(m, f, mr)));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(z + 2 * (size_t)m) : "memory");
  }
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  pair_finish<NTH, BIG>(f, s, anc, c, a, rt, W, U, decon, out);
}

// Stages (a2)-(c) in one launch with the grid row resident in shared
// memory: each CTA spreads its asset's records (Eq. (12)) straight into the
// complex points of the row it transforms, so only the records come in and
// only the coefficients go out. One CTA per asset holds the whole row; for
// rows too large for one CTA, CTA c of a cluster pair holds the points
// z[2m + c] (cells 4m + 2c, 4m + 2c + 1) and adds only the taps that land in
// its own cells. The row's cells are taken in sub-ranges [A, A + sub): the
// records whose stencils reach a sub-range (found for all sub-ranges at once
// before the first) are scaled and accumulated exactly as for a spreading
// tile (the same per-tap polynomials, the same hi/lo int32 accumulation),
// then the sub-range's points become float32 in the row at their positions
// for the transform. The staging area and integer tiles live where the
// twiddle anchors (and digit-reversal tables) go afterwards.
constexpr int kResChunk = 1024;   // records staged per pass
constexpr int kResMaxSub = 64;    // sub-ranges per row

template <int NT, int NTH, class Cells>
__device__ __forceinline__ void spread_resident(const int64_t* __restrict__ off, const int* __restrict__ rb0,
                                                const float* __restrict__ rd, const float* __restrict__ rv,
                                                const SpreadParams& sp, const KernelPoly& poly, int sub,
                                                const AssetFft& f, const unsigned* mr, int a, Cells cells,
                                                Cplx<float>* s, unsigned char* work) {
  constexpr int EC = kResChunk;
  constexpr int kPer = Cells::kAll ? 2 : 4;  // cells per complex point of this CTA
  int* ev_p = reinterpret_cast<int*>(work);
  float* ev_d = reinterpret_cast<float*>(ev_p + EC);
  float* ev_v = ev_d + EC;
  const int nslot = sub / (kPer / 2);  // integer cells per tile held by this CTA
  int* tile_hi = reinterpret_cast<int*>(ev_v + EC);
  int* tile_lo = tile_hi + nslot;
  const uint32_t hi_s = (uint32_t)__cvta_generic_to_shared(tile_hi);
  const uint32_t lo_s = (uint32_t)__cvta_generic_to_shared(tile_lo);
  __shared__ float s_sum[NTH / 32], s_max[NTH / 32];
  __shared__ int64_t s_rng[kResMaxSub][6];
  const int nsub = (int)((sp.Mr + sub - 1) / sub);
  // record ranges of every sub-range: for image m = w/2 - 1 the returns with
  // b0 in [A - khi + m M_r, A + Tlen - klo + m M_r), clipped to [0, M_r + 1)
  // (a search per bound and one warp per search; empty images skipped)
  {
    const int64_t e0 = off[a], eend = off[a + 1];
    const int64_t e1 = eend > e0 ? eend - 1 : e0;  // returns live at h in [e0, e1)
    for (int job = threadIdx.x >> 5; job < 6 * nsub; job += NTH / 32) {
      const int r = job / 6, w = job - 6 * (job / 6);
      const int64_t A = (int64_t)r * sub;
      const int Tlen = (int)min((int64_t)sub, sp.Mr - A);
      const int m = w / 2 - 1;
      long long lo = A - sp.khi + (long long)m * sp.Mr;
      long long hi = A + Tlen - sp.klo + (long long)m * sp.Mr;
      if (lo < 0) lo = 0;
      if (hi > sp.Mr + 1) hi = sp.Mr + 1;
      const int64_t res = lo < hi ? warp_first_ge(rb0, e0, e1, (w & 1) ? hi : lo) : -1;
      if ((threadIdx.x & 31) == 0) s_rng[r][w] = res;
    }
  }
  __syncthreads();
  for (int r = 0; r < nsub; ++r) {
    const int64_t A = (int64_t)r * sub;
    const int Tlen = (int)min((int64_t)sub, sp.Mr - A);  // even (a multiple of 4 for the pair)
    {
      int4* t4 = reinterpret_cast<int4*>(tile_hi);
      for (int i = threadIdx.x; i < nslot / 2; i += NTH) t4[i] = make_int4(0, 0, 0, 0);  // both tiles
    }
    TileRanges tr;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const bool empty = s_rng[r][2 * q] < 0;
      tr.lo[q] = empty ? 0 : s_rng[r][2 * q];
      tr.hi[q] = empty ? 0 : s_rng[r][2 * q + 1];
    }
    tr.n2 = tr.hi[2] - tr.lo[2];
    tr.n1 = tr.hi[1] - tr.lo[1];
    tr.n0 = tr.hi[0] - tr.lo[0];
    const int64_t ntot = tr.n2 + tr.n1 + tr.n0;
    float part = 0.f, pmax = 0.f;
    const int n_first = (int)min((int64_t)EC, ntot);
    for (int i = threadIdx.x; i < n_first; i += NTH) {
      load_record<float>(rb0, rd, rv, sp, tr, A, i, ev_p[i], ev_d[i], ev_v[i]);
      part += fabsf(ev_v[i]);
      pmax = fmaxf(pmax, fabsf(ev_v[i]));
    }
    for (int64_t i = EC + threadIdx.x; i < ntot; i += NTH) {
      int pp;
      float dd, vv;
      load_record<float>(rb0, rd, rv, sp, tr, A, i, pp, dd, vv);
      part += fabsf(vv);
      pmax = fmaxf(pmax, fabsf(vv));
    }
    const TileScales ts = tile_scales<NTH>(part, pmax, ntot, s_sum, s_max);
    for (int64_t cs = 0; cs < ntot; cs += EC) {
      const int n = (int)min((int64_t)EC, ntot - cs);
      if (cs > 0) {
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += NTH)
          load_record<float>(rb0, rd, rv, sp, tr, A, cs + i, ev_p[i], ev_d[i], ev_v[i]);
      }
      __syncthreads();
      spread_chunk<NT, NTH>(ev_p, ev_d, ev_v, n, Tlen, sp.klo, poly, ts, hi_s, lo_s, cells);
    }
    __syncthreads();
    // this CTA's points of the sub-range, m = A / kPer + i (two integer cells each)
    const int m0 = (int)(A / kPer);
    const int2* h2 = reinterpret_cast<const int2*>(tile_hi);
    const int2* l2 = reinterpret_cast<const int2*>(tile_lo);
    for (int i = threadIdx.x; i < Tlen / kPer; i += NTH) {
      const int2 hv = h2[i], lv = l2[i];
      const int m = m0 + i;
      s[f.dif ? m : digit_rev(m, f, mr)] = Cplx<float>{fmaf((float)lv.x, ts.inv_l, (float)hv.x * ts.inv_h),
                                                       fmaf((float)lv.y, ts.inv_l, (float)hv.y * ts.inv_h)};
    }
    __syncthreads();  // the tiles are cleared for the next sub-range
  }
}

// Anchor rows (16-byte asynchronous copies) into their place after the row.
template <int NTH>
__device__ __forceinline__ void load_anchors(const AssetFft& f, const Cplx<float>* __restrict__ tw, float4* anc) {
  const float4* src = reinterpret_cast<const float4*>(tw);
  for (int i = threadIdx.x; i < 2 * f.tw_rows; i += NTH) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(anc + i);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src + i) : "memory");
  }
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

template <int NT>
__global__ void __launch_bounds__(512, 1)
    k_spread_fft(const int64_t* __restrict__ off, const int* __restrict__ rb0, const float* __restrict__ rd,
                 const float* __restrict__ rv, SpreadParams sp, KernelPoly poly, int sub, AssetFft f,
                 const Cplx<float>* __restrict__ tw, const Cplx<float>* __restrict__ U,
                 const float* __restrict__ decon, Cplx<float>* __restrict__ out, const int* __restrict__ gate) {
  constexpr int NTH = 512;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cplx<float>* s = reinterpret_cast<Cplx<float>*>(smem_raw);
  float4* anc = reinterpret_cast<float4*>(smem_raw + anchor_offset(f.nl));
  const int a = blockIdx.y;
  unsigned mr[kMaxAssetPasses];
#pragma unroll
  for (int p = 0; p < kMaxAssetPasses; ++p) mr[p] = magic_of((unsigned)f.rad[p]);
  pdl_wait();         // the records come from the prep kernel
  if (*gate) return;  // uniform: the whole block leaves
  pdl_trigger();
  spread_resident<NT, NTH>(off, rb0, rd, rv, sp, poly, sub, f, mr, a, AllCells{}, s,
                           smem_raw + anchor_offset(f.nl));
  load_anchors<NTH>(f, tw, anc);
  const RevTab rt = build_rev_tables<NTH>(f, smem_raw, mr);
  __syncthreads();
  single_finish<NTH, true>(f, s, anc, a, rt, U, decon, out);
}

template <int NT>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kPairThreads, 1)
    k_spread_fft_pair(const int64_t* __restrict__ off, const int* __restrict__ rb0, const float* __restrict__ rd,
                      const float* __restrict__ rv, SpreadParams sp, KernelPoly poly, int sub, AssetFft f,
                      const Cplx<float>* __restrict__ W, const Cplx<float>* __restrict__ tw,
                      const Cplx<float>* __restrict__ U, const float* __restrict__ decon,
                      Cplx<float>* __restrict__ out, const int* __restrict__ gate) {
  constexpr int NTH = kPairThreads;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cplx<float>* s = reinterpret_cast<Cplx<float>*>(smem_raw);
  float4* anc = reinterpret_cast<float4*>(smem_raw + anchor_offset(f.nl));
  unsigned c;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(c));
  const int a = blockIdx.y;
  unsigned mr[kMaxAssetPasses];
#pragma unroll
  for (int p = 0; p < kMaxAssetPasses; ++p) mr[p] = magic_of((unsigned)f.rad[p]);
  pdl_wait();  // the records come from the prep kernel
  // every CTA of the cluster reads the same gate word: both leave or neither
  if (*gate) return;
  pdl_trigger();
  spread_resident<NT, NTH>(off, rb0, rd, rv, sp, poly, sub, f, mr, a, PairCells{c}, s,
                           smem_raw + anchor_offset(f.nl));
  load_anchors<NTH>(f, tw, anc);
  const RevTab rt = build_rev_tables<NTH>(f, smem_raw, mr);  // none: decimation in time
  __syncthreads();
  pair_finish<NTH, true>(f, s, anc, c, a, rt, W, U, decon, out);
}

// Twiddle anchors of each pass: row j < m_p holds w^1..w^4 of w = w_{L_p}^j,
// from float64 angles.
__global__ void k_asset_twiddles(AssetFft f, Cplx<float>* tw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  for (int p = 0; p < f.npass; ++p) {
    const int R = f.rad[p], m = f.stride[p];
    if (m <= 1) continue;
    if (i < 4 * m) {
      const int j = i >> 2, e = (i & 3) + 1;
      const long Lp = (long)R * m;
      const long x = ((long)j * e) % Lp;
      double sn, cs;
      sincospi(-2.0 * (double)x / (double)Lp, &sn, &cs);
      tw[4 * f.tw_off[p] + i] = Cplx<float>{(float)cs, (float)sn};
    }
  }
}

}  // namespace

bool asset_fft_radix_ok(int R) {
  switch (R) {
    case 2: case 3: case 4: case 5: case 6: case 8: case 9: case 10: case 12: case 15:
    case 16: case 18: case 20: case 24: case 25: case 27: case 30: case 32:
      return true;
    default:
      return false;
  }
}

size_t asset_fft_smem(const AssetFft& f) {
  return anchor_offset(f.nl) + (size_t)f.tw_rows * 32 + (f.dif ? (size_t)(f.rev_lo + f.rev_hi) * 4 : 0);
}

cudaError_t launch_asset_twiddles(const AssetFft& f, void* tw, cudaStream_t s) {
  int cnt = 1;
  for (int p = 0; p < f.npass; ++p) cnt = std::max(cnt, 4 * f.stride[p]);
  k_asset_twiddles<<<(cnt + 255) / 256, 256, 0, s>>>(f, (Cplx<float>*)tw);
  return cudaGetLastError();
}

// Cells per sub-range of the resident spread + FFT kernels (a multiple of
// 8) for a shared-memory limit on the dynamic allocation; 0 when the row
// leaves no room for the staging area and a useful sub-range, or when the row
// would take more than kResMaxSub sub-ranges.
int spread_fft_sub(const AssetFft& f, int64_t Mr, size_t smem_limit) {
  const size_t row = anchor_offset(f.nl) + (size_t)kResChunk * 12;
  const size_t per_cell = f.pair ? 4 : 8;  // hi + lo of this CTA's cells
  if (row + 1024 * per_cell > smem_limit) return 0;
  int64_t sub = (int64_t)((smem_limit - row) / per_cell) / 8 * 8;
  sub = std::min<int64_t>(sub, (Mr + 7) / 8 * 8);
  if ((Mr + sub - 1) / sub > kResMaxSub) return 0;
  if (asset_fft_smem(f) > smem_limit) return 0;
  return (int)sub;
}

size_t spread_fft_smem(const AssetFft& f, int sub) {
  const size_t work = anchor_offset(f.nl) + (size_t)kResChunk * 12 + (size_t)sub * (f.pair ? 4 : 8);
  return std::max(work, asset_fft_smem(f));
}

cudaError_t launch_spread_fft(const int64_t* off, const int* rb0, const void* rd, const void* rv,
                              const SpreadParams& sp, const KernelPoly& poly, int sub, const AssetFft& f, int D,
                              const void* W, const void* tw, const void* U, const void* decon, void* coeffs,
                              const int* status, cudaStream_t s) {
  if (sub < 8 || sub % 8 || (f.pair && f.dif) || f.split != (f.pair ? 2 : 1)) return cudaErrorInvalidValue;
  const size_t smem = spread_fft_smem(f, sub);
  const int nt = sp.khi - sp.klo + 1;
  auto go = [&](auto single, auto pair) -> cudaError_t {
    cudaError_t e;
    if (f.pair) {
      if ((e = cudaFuncSetAttribute(pair, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
      return launch_pdl(pair, dim3(2, D), dim3(kPairThreads), smem, s, off, rb0, (const float*)rd, (const float*)rv,
                        sp, poly, sub, f, (const Cplx<float>*)W, (const Cplx<float>*)tw, (const Cplx<float>*)U,
                        (const float*)decon, (Cplx<float>*)coeffs, status + 1);
    }
    if ((e = cudaFuncSetAttribute(single, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
      return e;
    return launch_pdl(single, dim3(1, D), dim3(512), smem, s, off, rb0, (const float*)rd, (const float*)rv, sp, poly,
                      sub, f, (const Cplx<float>*)tw, (const Cplx<float>*)U, (const float*)decon,
                      (Cplx<float>*)coeffs, status + 1);
  };
  switch (nt) {
    case 9: return go(k_spread_fft<9>, k_spread_fft_pair<9>);
    case 13: return go(k_spread_fft<13>, k_spread_fft_pair<13>);
    case 14: return go(k_spread_fft<14>, k_spread_fft_pair<14>);
    default: break;
  }
  if (nt <= 8) return go(k_spread_fft<8>, k_spread_fft_pair<8>);
  if (nt <= 16) return go(k_spread_fft<16>, k_spread_fft_pair<16>);
  if (nt <= 24) return go(k_spread_fft<24>, k_spread_fft_pair<24>);
  if (nt <= 32) return go(k_spread_fft<32>, k_spread_fft_pair<32>);
  return cudaErrorInvalidValue;
}

int asset_fft_max_radix(const AssetFft& f) {
  int r = 1;
  for (int p = 0; p < f.npass; ++p) r = std::max(r, f.rad[p]);
  return r;
}

cudaError_t launch_fft_asset(const float* grid, const AssetFft& f, int D, const void* W, const void* tw,
                             const void* U, const void* decon, void* coeffs, int* status, cudaStream_t s) {
  const size_t smem = asset_fft_smem(f);
  auto go = [&](auto fn, dim3 grd, int nth, auto... extra) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(fn, grd, dim3(nth), smem, s, grid, f, (const Cplx<float>*)W, (const Cplx<float>*)tw,
                      (const Cplx<float>*)U, (const float*)decon, (Cplx<float>*)coeffs, (const int*)(status + 1),
                      extra...);
  };
  // plans of radices up to 16 run a kernel without the larger codelets
  // (fewer registers); the one-CTA kernel then runs 1024 threads, twice the
  // warps to hide its shared-memory and barrier latency (measured on the
  // block workload: 28.5 us with 512 threads and every codelet, 26.7 us
  // without the large ones, 25.3 us with 1024 threads). The cluster pair
  // measured fastest with 512 threads and radices up to 32.
  const bool big = asset_fft_max_radix(f) > 16;
  if (f.pair) {
    if (big) return go(k_fft_asset_pair<kPairThreads, true>, dim3(2, D), kPairThreads);
    return go(k_fft_asset_pair<kPairThreads, false>, dim3(2, D), kPairThreads);
  }
  if (big) return go(k_fft_asset<512, true>, dim3(1, D), 512, status);
  return go(k_fft_asset<1024, false>, dim3(1, D), 1024, status);
}

}  // namespace mmgpu
