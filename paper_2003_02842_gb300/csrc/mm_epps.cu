// mm_epps.cu -- the cutoff sweep of the batched form: for every problem of a
// batch (G problems of Dg assets each) and every cutoff N_j of an ascending
// list, the covariance and correlation of Algorithm 3 step C (Eqs. (2), (3))
// from ONE set of coefficients computed at N_max = max_j N_j.
//
// Prefix-weighted contraction. With the Hermitian half (the -k term of each
// pair k, -k folded into a factor 2 for k >= 1, no factor for k = 0) and
// Q_k = Re(F(k) F(k)^H) (a Dg x Dg matrix),
//   Dirichlet  Sigma(N) = (2 pi)^2 / (2N + 1) * P(N),
//   Fejer      Sigma(N) = (2 pi)^2 / (N + 1) * (P(N) - P1(N) / N),
//   P(N) = sum_{k<=N} d_k Q_k,  P1(N) = sum_{k<=N} d_k k Q_k,  d_0 = 1, d_k = 2,
// so one pass over k accumulating the segments (N_{j-1}, N_j] followed by a
// prefix sum over segments gives every cutoff: the work is that of a single
// contraction at N_max plus O(#cutoffs Dg^2) additions, not one contraction
// per cutoff.
//
// One CTA per problem (grid-stride over problems). Thread t of a 256-mode
// tile takes mode k = tile + t, loads the Dg coefficients F_i(k) (coalesced
// across threads) and adds the Dg (Dg+1)/2 products into registers; a warp
// whose 32 modes lie in one segment keeps accumulating, and a warp-wide
// shuffle reduction flushes its registers into the segment's shared-memory
// slots when its segment changes. Accumulation is float32 (the products are
// well within range; the sums run over at most N_max + 1 modes); the
// correlation normalisation is float64.
#include "mm_common.cuh"

namespace mmgpu {

namespace {

constexpr int kEppsThreads = 256;

template <int DG>
struct Pairs {
  static constexpr int n = DG * (DG + 1) / 2;
};

// First segment j with cut[j] >= k (k <= cut[ncut - 1]).
__device__ __forceinline__ int segment_of(const int* cut, int ncut, int k) {
  int lo = 0, hi = ncut - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cut[mid] >= k) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

template <int DG, bool FEJER>
__global__ void __launch_bounds__(kEppsThreads) k_epps(const float2* __restrict__ coef, int ld, const int* __restrict__ cut_g,
                                                       int ncut, int G, float* __restrict__ sigma,
                                                       float* __restrict__ Rout, const int* __restrict__ gate,
                                                       int* status) {
  constexpr int NP = Pairs<DG>::n;
  constexpr int NS = FEJER ? 2 : 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sacc = reinterpret_cast<float*>(smem_raw);                     // [NS][ncut][NP]
  double* ssig = reinterpret_cast<double*>(smem_raw + (((size_t)NS * ncut * NP * 4 + 15) & ~(size_t)15));  // [ncut][NP]
  __shared__ int scut[kMaxCutoffs];
  if (*gate) return;  // uniform
  const int lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < ncut; i += kEppsThreads) scut[i] = cut_g[i];
  int zero_var = 0;
  for (int g = blockIdx.x; g < G; g += gridDim.x) {
    for (int i = threadIdx.x; i < NS * ncut * NP; i += kEppsThreads) sacc[i] = 0.f;
    __syncthreads();
    const int Kuse = scut[ncut - 1] + 1;
    const float2* cg = coef + (size_t)g * DG * ld;
    float acc[NP], acc1[FEJER ? NP : 1];
#pragma unroll
    for (int p = 0; p < NP; ++p) acc[p] = 0.f;
#pragma unroll
    for (int p = 0; p < (FEJER ? NP : 1); ++p) acc1[p] = 0.f;
    int cs = -1;  // segment held in the registers (uniform across the warp)
    auto flush = [&]() {
      if (cs >= 0) {
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          float v = acc[p];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) atomicAdd(&sacc[cs * NP + p], v);
          acc[p] = 0.f;
          if (FEJER) {
            float w = acc1[p];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
            if (lane == 0) atomicAdd(&sacc[(ncut + cs) * NP + p], w);
            acc1[p] = 0.f;
          }
        }
      }
      cs = -1;
    };
    for (int t0 = 0; t0 < Kuse; t0 += kEppsThreads) {
      const int k = t0 + threadIdx.x;
      const bool valid = k < Kuse;
      float2 c[DG];
      const float sc = k == 0 ? 1.0f : 1.41421356237309515f;  // sqrt(d_k)
#pragma unroll
      for (int i = 0; i < DG; ++i) {
        const float2 v = valid ? __ldg(cg + (size_t)i * ld + k) : make_float2(0.f, 0.f);
        c[i] = make_float2(v.x * sc, v.y * sc);
      }
      const int seg = valid ? segment_of(scut, ncut, k) : -1;
      const int s0 = __shfl_sync(0xffffffffu, seg, 0), s31 = __shfl_sync(0xffffffffu, seg, 31);
      const float kf = (float)k;
      if (s0 == s31 && s0 >= 0) {
        if (s0 != cs) {
          flush();
          cs = s0;
        }
        int p = 0;
#pragma unroll
        for (int i = 0; i < DG; ++i)
#pragma unroll
          for (int j = i; j < DG; ++j, ++p) {
            const float q = fmaf(c[i].x, c[j].x, c[i].y * c[j].y);
            acc[p] += q;
            if (FEJER) acc1[p] = fmaf(kf, q, acc1[p]);
          }
      } else {
        // the warp straddles a cutoff (or the end): per-lane shared atomics
        flush();
        if (seg >= 0) {
          int p = 0;
#pragma unroll
          for (int i = 0; i < DG; ++i)
#pragma unroll
            for (int j = i; j < DG; ++j, ++p) {
              const float q = fmaf(c[i].x, c[j].x, c[i].y * c[j].y);
              atomicAdd(&sacc[seg * NP + p], q);
              if (FEJER) atomicAdd(&sacc[(ncut + seg) * NP + p], kf * q);
            }
        }
      }
    }
    flush();
    __syncthreads();
    // prefix over segments and the basis weights (float64 from here on)
    const double four_pi2 = 4.0 * kPi * kPi;
    for (int p = threadIdx.x; p < NP; p += kEppsThreads) {
      double P = 0.0, P1 = 0.0;
      for (int j = 0; j < ncut; ++j) {
        P += (double)sacc[j * NP + p];
        if (FEJER) P1 += (double)sacc[(ncut + j) * NP + p];
        const double Nj = (double)scut[j];
        ssig[j * NP + p] = FEJER ? four_pi2 / (Nj + 1.0) * (P - P1 / Nj) : four_pi2 / (2.0 * Nj + 1.0) * P;
      }
    }
    __syncthreads();
    // Sigma and R for every cutoff, both triangles
    for (int e = threadIdx.x; e < ncut * DG * DG; e += kEppsThreads) {
      const int j = e / (DG * DG), r = e - j * DG * DG;
      const int a = r / DG, b = r - a * DG;
      const int lo = a < b ? a : b, hi = a < b ? b : a;
      const int p = lo * DG - lo * (lo - 1) / 2 + (hi - lo);  // index of pair (lo, hi)
      const int pa = a * DG - a * (a - 1) / 2, pb = b * DG - b * (b - 1) / 2;  // (a, a), (b, b)
      const double s = ssig[j * NP + p];
      const double da = ssig[j * NP + pa], db = ssig[j * NP + pb];
      const size_t o = ((size_t)g * ncut + j) * DG * DG + r;
      if (sigma) sigma[o] = (float)s;
      double rv;
      if (a == b) rv = da > 0.0 ? 1.0 : __longlong_as_double(0x7ff8000000000000LL);
      else rv = (da > 0.0 && db > 0.0) ? s / (sqrt(da) * sqrt(db)) : __longlong_as_double(0x7ff8000000000000LL);
      if (!(da > 0.0)) zero_var = 1;
      Rout[o] = (float)rv;
    }
    __syncthreads();
  }
  if (zero_var) atomicOr(status, ST_ZERO_VAR);
}

template <int DG>
cudaError_t launch_dg(bool fejer, const void* coef, int ld, const int* cut, int ncut, int G, float* sigma, float* R,
                      const int* status_gate, int* status, int grid, cudaStream_t s) {
  constexpr int NP = Pairs<DG>::n;
  const int NS = fejer ? 2 : 1;
  const size_t smem = (((size_t)NS * ncut * NP * 4 + 15) & ~(size_t)15) + (size_t)ncut * NP * 8;
  auto go = [&](auto fn) -> cudaError_t {
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    fn<<<grid, kEppsThreads, smem, s>>>((const float2*)coef, ld, cut, ncut, G, sigma, R, status_gate, status);
    return cudaGetLastError();
  };
  return fejer ? go(k_epps<DG, true>) : go(k_epps<DG, false>);
}

}  // namespace

int epps_max_assets() { return kMaxEppsAssets; }

cudaError_t launch_epps(int Dg, bool fejer, const void* coef, int ld, const int* cut, int ncut, int G, float* sigma,
                        float* R, int* status, int grid, cudaStream_t s) {
  if (ncut < 1 || ncut > kMaxCutoffs || G < 1) return cudaErrorInvalidValue;
  const int* gate = status + 1;
  switch (Dg) {
    case 1: return launch_dg<1>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 2: return launch_dg<2>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 3: return launch_dg<3>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 4: return launch_dg<4>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 5: return launch_dg<5>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 6: return launch_dg<6>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 7: return launch_dg<7>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 8: return launch_dg<8>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 9: return launch_dg<9>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 10: return launch_dg<10>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 11: return launch_dg<11>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 12: return launch_dg<12>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mmgpu
