// mm_spread.cu -- stage (a) of the hot path: time rescaling and phase
// reduction to grid cells (Algorithm 4), returns (Algorithm 3 step F.3), the
// Nyquist cutoff (Algorithm 2) and the spreading of returns onto the
// oversampled grid (Eq. (12); Algorithms 8-10 step C) with the Gaussian (fast
// Gaussian gridding split, Eq. (17)), Kaiser-Bessel (Eq. (7)) or exponential
// of semicircle (Eq. (9)) kernel.
//
// Phase reduction. GB300 executes float64 at about 1/47 of the float32 rate
// (measured: 4.8e11 float64 FMAs per second over the chip), and a
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
#include "mm_spread_dev.cuh"

namespace mmgpu {

// ------------------------------------------------------------------ bounds
// Validates the CSR offsets, finds t_min / t_max (Algorithm 4) or takes the
// caller's window, fixes the time fixed-point format and writes the gate word
// (0 = proceed). Block g handles problem g of a batch (assets g*gsize ..
// (g+1)*gsize - 1; a single problem has one block with gsize = D). A block
// reads event times only after checking that its own offsets are
// non-decreasing and lie in [0, max_events], so a malformed offsets array
// anywhere leaves every read in bounds.
__global__ void k_bounds(const int64_t* __restrict__ off, const double* __restrict__ t, int D, int gsize,
                         int64_t max_events, double w0, double w1, int64_t Mr, Rescale* rs, int* status,
                         int* __restrict__ order) {
  __shared__ double s_lo[8], s_hi[8];
  __shared__ int s_bad;
  pdl_wait();     // the previous call's kernels may still read the gate
  pdl_trigger();  // prep may be scheduled (it waits for this kernel)
  int* gate = status + 1;
  const int g = blockIdx.x;
  const int i0 = g * gsize, i1 = min(i0 + gsize, D);
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  // 1) the offsets alone: non-decreasing from 0 up to at most max_events.
  //    Only when all of them hold is any event time read.
  int bad = 0;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x)
    if (off[i + 1] < off[i]) bad = 1;
  if (threadIdx.x == 0 && (off[i0] < 0 || off[i1] > max_events || (g == 0 && off[0] != 0))) bad = 1;
  if (bad) atomicOr(&s_bad, 1);
  __syncthreads();
  if (s_bad) {
    if (threadIdx.x == 0) {
      atomicOr(status, ST_BAD_OFFSETS);
      rs[g].t0 = rs[g].t1 = 0.0;
      if (gridDim.x == 1) *gate = 1;
      else atomicOr(gate, 1);
    }
    return;
  }
  // 2) t_min / t_max from each asset's first and last event (Algorithm 4);
  //    the first asset's two times are loaded before the ranking below and
  //    used after it, so that the load latency overlaps the ranking
  const bool window = w1 > w0;
  double lo = INFINITY, hi = -INFINITY;
  int outwin = 0;
  double f0 = INFINITY, l0 = -INFINITY;
  bool has0 = false;
  {
    const int i = i0 + (int)threadIdx.x;
    if (i < i1) {
      const int64_t a = off[i], b = off[i + 1];
      if (b > a) {
        f0 = t[a];
        l0 = t[b - 1];
        has0 = true;
      }
    }
  }
  // the spreading tiles' dispatch order: assets ranked by event count,
  // heaviest first (ties by index), so that the longest tiles start first
  if (order) {  // uniform: a single problem, D <= kOrderMaxAssets
    __shared__ int s_cnt[kOrderMaxAssets];
    for (int i = threadIdx.x; i < D; i += blockDim.x) {
      const int64_t c = off[i + 1] - off[i];
      s_cnt[i] = (int)min(c, (int64_t)0x7fffffff);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < D; i += blockDim.x) {
      const int ci = s_cnt[i];
      int r = 0;
      for (int j = 0; j < D; ++j) {
        const int cj = s_cnt[j];
        r += (cj > ci || (cj == ci && j < i)) ? 1 : 0;
      }
      order[r] = i;
    }
  }
  if (has0) {
    lo = fmin(lo, f0);
    hi = fmax(hi, l0);
    if (window && (f0 < w0 || l0 > w1)) outwin = 1;
  }
  for (int i = i0 + (int)threadIdx.x + (int)blockDim.x; i < i1; i += blockDim.x) {
    const int64_t a = off[i], b = off[i + 1];
    if (b > a) {
      const double f = t[a], l = t[b - 1];
      lo = fmin(lo, f);
      hi = fmax(hi, l);
      if (window && (f < w0 || l > w1)) outwin = 1;
    }
  }
  if (outwin) atomicOr(&s_bad, 2);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    s_lo[threadIdx.x >> 5] = lo;
    s_hi[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      lo = fmin(lo, s_lo[w]);
      hi = fmax(hi, s_hi[w]);
    }
    s_lo[0] = lo;
    s_hi[0] = hi;
    const double t0 = window ? w0 : s_lo[0];
    const double t1 = window ? w1 : s_hi[0];
    int gt = 0;
    if (s_bad & 2) { atomicOr(status, ST_OUT_OF_WINDOW); gt = 1; }
    if (!gt && !(t1 > t0 && isfinite(t0) && isfinite(t1))) {
      // all assets empty, a single instant, or non-finite times
      if (s_hi[0] >= s_lo[0] || window || isnan(s_lo[0]) || isnan(s_hi[0])) atomicOr(status, ST_SPAN);
      gt = 1;
    }
    Rescale r{};
    r.t0 = t0;
    r.t1 = t1;
    if (!gt) {
      int ex;
      frexp(fmax(fabs(t0), fabs(t1)), &ex);  // max |t| < 2^ex
      r.F = 62 - (ex + 1);                   // |t_fix| < 2^61
      r.t0_fix = to_fix(t0, r.F);
      if (Mr > 0) {
        // the cell scales of this call's grid, once (float64 is slow here)
        const UScale us = make_uscale(r, Mr);
        const UScaleF usf = make_uscale_f(r, Mr);
        r.S = us.S;
        r.sh = us.sh;
        r.s_hi = usf.s_hi;
        r.s_lo = usf.s_lo;
        r.scale_Mr = Mr;
      }
    }
    rs[g] = r;
    if (gridDim.x == 1) *gate = gt;  // one problem: this call's gate
    else if (gt) atomicOr(gate, 1);  // batched: cleared before the launch
  }
}

cudaError_t launch_bounds(const int64_t* off, const double* t, int D, int gsize, int64_t max_events, double w0,
                          double w1, int64_t Mr, Rescale* rs, int* status, int* order, cudaStream_t s) {
  const int G = (D + gsize - 1) / gsize;
  if (order && (G != 1 || D > kOrderMaxAssets)) return cudaErrorInvalidValue;
  if (G > 1) {
    cudaError_t e = cudaMemsetAsync(status + 1, 0, sizeof(int), s);  // the gate of this call
    if (e != cudaSuccess) return e;
  }
  return launch_pdl(k_bounds, dim3(G), dim3(256), 0, s, off, t, D, gsize, max_events, w0, w1, Mr, rs, status,
                    order);
}

// Per-problem fixed-point cell scales for the grid size of this call.
__global__ void k_group_scales(const Rescale* __restrict__ rs, int G, int64_t Mr, const int* __restrict__ gate,
                               GroupScale* out) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G || *gate) return;
  const Rescale r = rs[g];
  GroupScale q;
  q.us = make_uscale(r, Mr);
  q.usf = make_uscale_f(r, Mr);
  q.t0_fix = r.t0_fix;
  q.F = r.F;
  out[g] = q;
}

size_t group_scale_bytes() { return sizeof(GroupScale); }

cudaError_t launch_group_scales(const Rescale* rs, int G, int64_t Mr, GroupScale* out, const int* status,
                                cudaStream_t s) {
  k_group_scales<<<(G + 127) / 128, 128, 0, s>>>(rs, G, Mr, status + 1, out);
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

constexpr int kSpreadThreads = 256;

// ------------------------------------------------------------------ prep
// Steps a0 / a1 of the hot path: for each event h, the rescaled cell
// coordinate in exact fixed point (Algorithm 4), split into the cell b0 and
// the offset d in [0, 1), and the return delta = logp[h+1] - logp[h]
// (Algorithm 3 step F.3), written once as a compact record (b0, d, delta) in
// event order. Since each asset's times are sorted, its records are sorted
// by cell: that order is the bin sort the spreading kernels search. The
// last event of an asset carries no return and its record is never read
// (it holds kNoCell or is left as it was).
//
// Each thread takes kPrepE consecutive events: it loads kPrepE + 1 times and
// log-prices, orders, checks and splits each value once (every value but the
// last serves two returns), and writes its records with vector stores.
constexpr int kPrepE = 4;
constexpr int kPrepThreads = 256;

template <typename T> struct Rec4;
template <> struct Rec4<float> {
  static __device__ __forceinline__ void store(float* p, const float* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <> struct Rec4<double> {
  static __device__ __forceinline__ void store(double* p, const double* v) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
};

template <typename T>
__global__ void __launch_bounds__(kPrepThreads, 5) k_prep(const int64_t* __restrict__ off, const double* __restrict__ t,
                                                       const double* __restrict__ logp,
                                                       const Rescale* __restrict__ rsp,
                                                       const GroupScale* __restrict__ gsc, int gsize,
                                                       const int* __restrict__ gate, int D, int64_t Mr,
                                                       int* __restrict__ rb0, T* __restrict__ rd,
                                                       T* __restrict__ rv, int* status) {
  static_assert(kPrepE == 4, "records are stored as 4-vectors");
  __shared__ UScale s_us;
  __shared__ UScaleF s_usf;
  __shared__ int s_flags;
  __shared__ int s_a0;
  // one round of loads: the gate, the event count and the call's rescaling
  // (with its cell scales when k_bounds knew the grid); then each thread's
  // event loads are in flight while warp 0 finds the block's asset. No event
  // is read before the gate (k_bounds' validation of the offsets) is known.
  pdl_wait();
  const int gated = *gate;
  const int64_t ntot = off[D];
  Rescale rs0{};
  if (!gsc) rs0 = *rsp;
  if (gated) return;  // uniform
  const bool scales = gsc || rs0.scale_Mr == Mr;  // uniform
  const int64_t hb = (int64_t)blockIdx.x * (kPrepThreads * kPrepE);
  const int64_t h0 = hb + (int64_t)threadIdx.x * kPrepE;
  double tv[kPrepE + 1], pv[kPrepE + 1];
#pragma unroll
  for (int j = 0; j <= kPrepE; ++j) {
    tv[j] = 0.0;
    pv[j] = 0.0;
    if (h0 + j < ntot) {
      tv[j] = t[h0 + j];
      pv[j] = logp[h0 + j];
    }
  }
  if (threadIdx.x == 0) {
    if (!scales) {
      if (sizeof(T) == 8) s_us = make_uscale(rs0, Mr);
      else s_usf = make_uscale_f(rs0, Mr);
    }
    s_flags = 0;
  }
  // asset of the block's first event (a 32-ary search by warp 0, a couple of
  // dependent loads), then each thread walks forward to its own events' assets
  if (threadIdx.x < 32) {
    const int64_t hs = min(hb, ntot > 0 ? ntot - 1 : 0);
    // first index in [1, D] with off[idx] > hs (D when none): the asset is idx - 1
    const int lane = threadIdx.x;
    int64_t lo = 1, hi = D;
    for (int it = 0; it < 16 && hi > lo; ++it) {
      const int64_t len = hi - lo;
      const int64_t stride = (len + 31) / 32;
      const int64_t o = (int64_t)lane * stride;
      const bool below = o < len && off[lo + o] <= hs;
      const int cnt = __popc(__ballot_sync(0xffffffffu, below));
      if (cnt == 0) {
        hi = lo;
      } else {
        const int64_t nlo = lo + (int64_t)(cnt - 1) * stride + 1;
        const int64_t nhi = min(lo + (int64_t)cnt * stride, hi);
        lo = min(nlo, nhi);
        hi = nhi;
      }
    }
    if (lane == 0) s_a0 = (int)lo - 1;
  }
  // per value, once: order key, finiteness and (float32 path) the exact
  // hi + lo split of the log-price
  long long key[kPrepE + 1];
  bool fin_t[kPrepE + 1], fin_p[kPrepE + 1];
  float ph[kPrepE + 1], pl[kPrepE + 1];
#pragma unroll
  for (int j = 0; j <= kPrepE; ++j) {
    key[j] = order_key(tv[j]);
    fin_t[j] = finite_bits(tv[j]);
    fin_p[j] = finite_bits(pv[j]);
    if (sizeof(T) == 4) split_f64(pv[j], ph[j], pl[j]);
  }
  __syncthreads();
  int flags = 0;
  int b0v[kPrepE];
  T dv[kPrepE], vv[kPrepE];
  int lo = s_a0;
#pragma unroll
  for (int j = 0; j < kPrepE; ++j) {
    const int64_t h = h0 + j;
    b0v[j] = kNoCell;
    dv[j] = (T)0;
    vv[j] = (T)0;
    if (h >= ntot) continue;
    while (lo + 1 < D && off[lo + 1] <= h) ++lo;
    if (!(h + 1 < off[lo + 1])) continue;  // the asset's last event: no return
    // this event's problem: its fixed-point scale (batched form) or the
    // call's single one
    Rescale rs = rs0;
    UScale us;
    UScaleF usf;
    if (gsc) {
      const GroupScale q = gsc[lo / gsize];
      rs.t0_fix = q.t0_fix;
      rs.F = q.F;
      us = q.us;
      usf = q.usf;
    } else if (scales) {
      us.S = rs0.S;
      us.sh = rs0.sh;
      usf.s_hi = rs0.s_hi;
      usf.s_lo = rs0.s_lo;
    } else {
      us = s_us;
      usf = s_usf;
    }
    if (!(key[j] < key[j + 1])) flags |= (key[j] == key[j + 1]) ? ST_DUPLICATE : ST_UNSORTED;
    if (!(fin_t[j] && fin_p[j] && fin_p[j + 1])) {
      flags |= ST_NONFINITE;
      continue;
    }
    const long long dt = to_fix(tv[j], rs.F) - rs.t0_fix;
    int cb;
    T cd;
    if (sizeof(T) == 8) {
      const unsigned long long uf = u_fix_of(tv[j], rs.t0_fix, rs.F, us);
      cb = (int)(uf >> kUFrac);
      cd = frac_to<T>(uf & ((1ull << kUFrac) - 1));
    } else {
      float fd;
      cell_f32(dt, usf, cb, fd);
      cd = (T)fd;
    }
    if (dt < 0 || cb > Mr || (cb == Mr && cd > (T)0)) {
      flags |= ST_OUT_OF_WINDOW;
      continue;
    }
    b0v[j] = cb;
    dv[j] = cd;
    if (sizeof(T) == 8) vv[j] = (T)(pv[j + 1] - pv[j]);
    else vv[j] = (T)((ph[j + 1] - ph[j]) + (pl[j + 1] - pl[j]));
  }
  if (h0 + kPrepE <= ntot) {
    // h0 is a multiple of 4 and the record arrays are the plan's own
    // (256-byte aligned) allocations: 16-byte vector stores
    *reinterpret_cast<int4*>(rb0 + h0) = make_int4(b0v[0], b0v[1], b0v[2], b0v[3]);
    Rec4<T>::store(rd + h0, dv);
    Rec4<T>::store(rv + h0, vv);
  } else {
#pragma unroll
    for (int j = 0; j < kPrepE; ++j) {
      if (h0 + j < ntot) {
        rb0[h0 + j] = b0v[j];
        rd[h0 + j] = dv[j];
        rv[h0 + j] = vv[j];
      }
    }
  }
  if (flags) atomicOr(&s_flags, flags);
  __syncthreads();
  if (threadIdx.x == 0 && s_flags) atomicOr(status, s_flags);
  pdl_trigger();
}

template <typename T>
static cudaError_t launch_prep_t(const int64_t* off, const double* t, const double* logp, const Rescale* rs,
                                 const GroupScale* gsc, int gsize, int D, int64_t Mr, int64_t max_events, int* rb0,
                                 T* rd, T* rv, int* status, cudaStream_t s) {
  if (max_events <= 0) return cudaSuccess;
  if ((((uintptr_t)rb0) | ((uintptr_t)rd) | ((uintptr_t)rv)) & 15) return cudaErrorMisalignedAddress;
  const int64_t per_block = (int64_t)kPrepThreads * kPrepE;
  const int64_t blocks = (max_events + per_block - 1) / per_block;
  return launch_pdl(k_prep<T>, dim3((unsigned)blocks), dim3(kPrepThreads), 0, s, off, t, logp, rs, gsc, gsize,
                    status + 1, D, Mr, rb0, rd, rv, status);
}

cudaError_t launch_prep_f32(const int64_t* off, const double* t, const double* logp, const Rescale* rs,
                            const GroupScale* gsc, int gsize, int D,
                            int64_t Mr, int64_t max_events, int* rb0, void* rd, void* rv, int* status,
                            cudaStream_t s) {
  return launch_prep_t<float>(off, t, logp, rs, gsc, gsize, D, Mr, max_events, rb0, (float*)rd, (float*)rv, status, s);
}
cudaError_t launch_prep_f64(const int64_t* off, const double* t, const double* logp, const Rescale* rs,
                            const GroupScale* gsc, int gsize, int D,
                            int64_t Mr, int64_t max_events, int* rb0, void* rd, void* rv, int* status,
                            cudaStream_t s) {
  return launch_prep_t<double>(off, t, logp, rs, gsc, gsize, D, Mr, max_events, rb0, (double*)rd, (double*)rv, status,
                               s);
}

// ------------------------------------------------------------------ spread
template <typename T> struct EvChunk { static constexpr int n = 1536; };  // 6 spreading blocks per SM

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

// Float32 scatter with polynomial taps and exact integer accumulation.
// Shared-memory float atomics run as compare-and-swap loops and 64-bit
// integer reductions are slower still (3.4x and 5.6x the time of an int32
// reduction on GB300), so each tap's product x = v phi 2^eh goes to two int32
// tiles by native int32 reductions: hi = round(x) and lo = round((x - hi) 2^k).
// Both sums are exact and independent of the order of the atomics; a cell
// holds (hi + lo 2^-k) 2^-eh with one quantum 2^-(eh + k) per tap.
//
// Scales (B = sum |v|, V = max |v| over the tile's n events, |phi| <= 1 + 1e-6):
//  * eh = min(29 - ex(B), 21 - ex(V)) with B < 2^ex(B), V < 2^ex(V): every
//    |x| < 2^21 (the rounding below needs |x| < 2^22) and a cell's hi sum is
//    below 2^29 (1 + 1e-6) + n/2 < 2^31;
//  * k = min(20, 30 - bitlen(n)): |lo| <= 2^(k-1) + 1 per tap, so a cell's lo
//    sum is below n (2^(k-1) + 1) < 2^30.
// The quantum per tap, 2^-(eh + k), is therefore at most
// max(B 2^-(28 + k), V 2^-(20 + k)): max(B 2^-48, V 2^-40) for tiles of up to
// 1023 events, and for larger tiles at most max(B n 2^-58, V n 2^-50)
// (2^-k < 2n 2^-30). Against float32 rounding of a tap's product (2^-24 of
// it) this is negligible up to about 2^20 events per tile.
//
// round(y) for |y| < 2^22 is taken as y + 1.5 2^23, whose float spacing is 1
// (one FMA, no conversion instruction; kRoundMagic).

// Records staged per pass of the polynomial scatter: with two 4096-cell
// tiles, 44 KB of shared memory per block and five blocks per SM. On the
// block workload 512 to 1536 records and 2048- or 4096-cell tiles all ran
// the stage within 2 us of one another: its time is the reductions.
constexpr int kPolyChunk = 1024;

template <int NT>
__global__ void __launch_bounds__(kSpreadThreads, 5) k_spread_poly(const int64_t* __restrict__ off,
                                                               const int* __restrict__ rb0,
                                                               const float* __restrict__ rd,
                                                               const float* __restrict__ rv,
                                                               const int* __restrict__ gate, SpreadParams p,
                                                               KernelPoly poly, float* __restrict__ grid) {
  constexpr int EC = kPolyChunk;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* ev_p = reinterpret_cast<int*>(smem_raw);
  float* ev_d = reinterpret_cast<float*>(smem_raw + EC * sizeof(int));
  float* ev_v = ev_d + EC;
  const int tpad = (p.tile + 3) & ~3;  // tile cells rounded up to whole int4
  int* tile_hi = reinterpret_cast<int*>(ev_v + EC);
  int* tile_lo = tile_hi + tpad;
  const uint32_t hi_s = (uint32_t)__cvta_generic_to_shared(tile_hi);
  const uint32_t lo_s = (uint32_t)__cvta_generic_to_shared(tile_lo);
  __shared__ float s_sum[kSpreadThreads / 32], s_max[kSpreadThreads / 32];
  const int64_t L = (int64_t)blockIdx.x * p.tile;
  const int Tlen = (int)min((int64_t)p.tile, p.Mr - L);
  {
    int4* t4 = reinterpret_cast<int4*>(tile_hi);
    const int n4 = tpad / 2;  // both tiles
    for (int c = threadIdx.x; c < n4; c += kSpreadThreads) t4[c] = make_int4(0, 0, 0, 0);
  }
  pdl_wait();         // the records come from the prep kernel
  if (*gate) return;  // uniform: the whole block leaves
  const int a = p.order ? p.order[blockIdx.y] : (int)blockIdx.y;
  TileRanges tr;
  tile_ranges(off, rb0, p, a, L, Tlen, tr);
  const int64_t ntot = tr.n2 + tr.n1 + tr.n0;
  // the tile's scales: sum and maximum of |v| over its records (staged with
  // the first chunk when one chunk holds them all, else a pass over the returns)
  float part = 0.f, pmax = 0.f;
  const int n_first = (int)min((int64_t)EC, ntot);
  for (int i = threadIdx.x; i < n_first; i += kSpreadThreads) {
    load_record<float>(rb0, rd, rv, p, tr, L, i, ev_p[i], ev_d[i], ev_v[i]);
    part += fabsf(ev_v[i]);
    pmax = fmaxf(pmax, fabsf(ev_v[i]));
  }
  for (int64_t i = EC + threadIdx.x; i < ntot; i += kSpreadThreads) {
    int pp;
    float dd, vv;
    load_record<float>(rb0, rd, rv, p, tr, L, i, pp, dd, vv);
    part += fabsf(vv);
    pmax = fmaxf(pmax, fabsf(vv));
  }
  const TileScales ts = tile_scales<kSpreadThreads>(part, pmax, ntot, s_sum, s_max);
  const float inv_h = ts.inv_h, inv_l = ts.inv_l;
  for (int64_t cs = 0; cs < ntot; cs += EC) {
    const int n = (int)min((int64_t)EC, ntot - cs);
    if (cs > 0) {
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += kSpreadThreads)
        load_record<float>(rb0, rd, rv, p, tr, L, cs + i, ev_p[i], ev_d[i], ev_v[i]);
    }
    __syncthreads();
    spread_chunk<NT, kSpreadThreads>(ev_p, ev_d, ev_v, n, Tlen, p.klo, poly, ts, hi_s, lo_s, AllCells{});
  }
  __syncthreads();
  if (p.perm_np > 0) {
    // the per-asset FFT's input order: complex point m = (L + c) / 2 goes to
    // its digit reversal (tiles and M_r are even, so cells pair up)
    float2* gz = reinterpret_cast<float2*>(grid + (int64_t)a * p.Mr);
    const int2* h2 = reinterpret_cast<const int2*>(tile_hi);
    const int2* l2 = reinterpret_cast<const int2*>(tile_lo);
    const int m0 = (int)(L >> 1);
    for (int c2 = threadIdx.x; c2 < (Tlen >> 1); c2 += kSpreadThreads) {
      int m = m0 + c2, pos = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (q < p.perm_np) {
          const int R = p.perm_rad[q];
          const int h = (int)__umulhi((unsigned)m, p.perm_magic[q]);
          pos += (m - h * R) * p.perm_stride[q];
          m = h;
        }
      }
      const int2 hv = h2[c2], lv = l2[c2];
      gz[pos] = make_float2(fmaf((float)lv.x, inv_l, (float)hv.x * inv_h),
                            fmaf((float)lv.y, inv_l, (float)hv.y * inv_h));
    }
    pdl_trigger();
    return;
  }
  float* g = grid + (int64_t)a * p.Mr + L;
  if (((reinterpret_cast<uintptr_t>(g) & 15) == 0) && (Tlen & 3) == 0) {
    const int4* h4 = reinterpret_cast<const int4*>(tile_hi);
    const int4* l4 = reinterpret_cast<const int4*>(tile_lo);
    float4* g4 = reinterpret_cast<float4*>(g);
    for (int c = threadIdx.x; c < Tlen / 4; c += kSpreadThreads) {
      const int4 hq = h4[c], lq = l4[c];
      g4[c] = make_float4(fmaf((float)lq.x, inv_l, (float)hq.x * inv_h), fmaf((float)lq.y, inv_l, (float)hq.y * inv_h),
                          fmaf((float)lq.z, inv_l, (float)hq.z * inv_h), fmaf((float)lq.w, inv_l, (float)hq.w * inv_h));
    }
  } else {
    for (int c = threadIdx.x; c < Tlen; c += kSpreadThreads)
      g[c] = fmaf((float)tile_lo[c], inv_l, (float)tile_hi[c] * inv_h);
  }
  pdl_trigger();
}

bool spread_poly_supported(int ntaps) {
  return ntaps == 9 || ntaps == 13 || ntaps == 14 || (ntaps >= 1 && ntaps <= kPolyMaxTaps);
}

cudaError_t launch_spread_poly(const int64_t* off, const int* rb0, const void* rd, const void* rv,
                               const SpreadParams& p, const KernelPoly& poly, float* grid, const int* status,
                               cudaStream_t s) {
  if (p.tile > spread_max_tile(false)) return cudaErrorInvalidValue;
  const int nt = p.khi - p.klo + 1;
  // staged records, then the hi and lo tiles (each rounded up to whole int4)
  const size_t smem = (size_t)kPolyChunk * (sizeof(int) + 2 * sizeof(float)) + 2 * (((size_t)p.tile + 3) / 4 * 16);
  dim3 grd(p.ntiles, p.D);
  auto go = [&](auto fn) -> cudaError_t {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(fn, grd, dim3(kSpreadThreads), smem, s, off, rb0, (const float*)rd, (const float*)rv,
                      (const int*)(status + 1), p, poly, grid);
  };
  switch (nt) {
    case 9: return go(k_spread_poly<9>);
    case 13: return go(k_spread_poly<13>);
    case 14: return go(k_spread_poly<14>);
    default: break;
  }
  // other tap counts: the next instantiation up, padded with zero taps
  if (nt <= 8) return go(k_spread_poly<8>);
  if (nt <= 16) return go(k_spread_poly<16>);
  if (nt <= 24) return go(k_spread_poly<24>);
  if (nt <= 32) return go(k_spread_poly<32>);
  return cudaErrorInvalidValue;
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
