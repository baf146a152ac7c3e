// mm_epps.cu -- the cutoff sweep of the batched form: for every problem of a
// batch (G problems of Dg assets each) and every cutoff N_j of an ascending
// list, the covariance and correlation of Algorithm 3 step C (Eqs. (2), (3))
// from ONE set of coefficients computed at N_max = max_j N_j.
//
// Prefix-weighted contraction. With the Hermitian half (the -k term of each
// pair k, -k folded into a factor 2 for k >= 1, no factor for k = 0) and
// Q_k = Re(F(k) F(k)^H) (a Dg x Dg matrix),
//   Dirichlet  Sigma(N) = (2 pi)^2 / (2N + 1) * P(N),
//   Fejer      Sigma(N) = (2 pi)^2 / ((N + 1) N) * sum_{k<=N} d_k (N - k) Q_k,
//   P(N) = sum_{k<=N} d_k Q_k,  d_0 = 1, d_k = 2.
// One pass over k accumulates, for each segment s = (e_{s-1}, e_s] of the
// cutoff list, S_s = sum d_k Q_k and T_s = sum d_k (e_s - k) Q_k; then
//   sum_{k<=N_j} d_k (N_j - k) Q_k = sum_{s<=j} ((N_j - e_s) S_s + T_s)
//                                  = A_j + sum_{s<=j} T_s,
//   A_j = A_{j-1} + (e_j - e_{j-1}) P_{j-1},  P_j = P_{j-1} + S_j,
// every cutoff from one contraction at N_max plus O(#cutoffs Dg^2) additions.
// All weights here are non-negative, so a diagonal entry is a sum of
// non-negative terms: the form P(N) - sum d_k k Q_k / N, which cancels when
// Q_0 dominates (a small total return at N = 1), is not used.
//
// One CTA per problem (grid-stride over problems). The modes are cut into
// chunks of at most 512 that never cross a cutoff; each warp takes whole
// chunks, its lanes step through the chunk's modes (coalesced loads of the
// Dg coefficients F_i(k)) adding the Dg (Dg+1)/2 products into registers,
// and one warp-shuffle reduction per chunk adds them into the chunk's segment
// in shared memory. Accumulation is float32 (the sums run over at most
// N_max + 1 modes); the diagonal normalisation is float64. The FP64 form
// (the comparator of the mixed one) runs the same sweep on complex128
// coefficients with float64 accumulation and float64 Sigma and R.
#include "mm_common.cuh"

namespace mmgpu {

namespace {

constexpr int kEppsThreads = 256;
constexpr int kChunkModes = 512;  // modes per warp work item (16 per lane)

template <int DG>
struct Pairs {
  static constexpr int n = DG * (DG + 1) / 2;
};

template <typename T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };

template <typename T, int DG, bool FEJER>
__global__ void __launch_bounds__(kEppsThreads) k_epps(const typename Cx<T>::type* __restrict__ coef, int ld,
                                                       const int* __restrict__ cut_g, int ncut, int G,
                                                       T* __restrict__ sigma, T* __restrict__ Rout,
                                                       const int* __restrict__ gate, int* status) {
  using C2 = typename Cx<T>::type;
  constexpr int NP = Pairs<DG>::n;
  constexpr int NS = FEJER ? 2 : 1;
  constexpr int NW = kEppsThreads / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sacc = reinterpret_cast<T*>(smem_raw);  // [NS][ncut][NP]
  double* ssig =
      reinterpret_cast<double*>(smem_raw + (((size_t)NS * ncut * NP * sizeof(T) + 15) & ~(size_t)15));  // [ncut][NP]
  __shared__ int scut[kMaxCutoffs];
  __shared__ int cstart[kMaxCutoffs + 1];                  // first chunk of each segment
  __shared__ double swt[kMaxCutoffs];                      // basis weight per cutoff
  __shared__ T sinv[kMaxCutoffs * DG];                     // 1 / sqrt(Sigma_aa(N_j))
  if (*gate) return;  // uniform
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < ncut; i += kEppsThreads) {
    const int c = cut_g[i];
    scut[i] = c;
    const double four_pi2 = 4.0 * kPi * kPi;
    swt[i] = FEJER ? four_pi2 / (((double)c + 1.0) * (double)c) : four_pi2 / (2.0 * (double)c + 1.0);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // segment j holds the modes (N_{j-1}, N_j] (j = 0: [0, N_0]), in chunks
    // of at most kChunkModes
    int c = 0;
    for (int j = 0; j < ncut; ++j) {
      cstart[j] = c;
      const int len = scut[j] - (j ? scut[j - 1] : -1);
      c += (len + kChunkModes - 1) / kChunkModes;
    }
    cstart[ncut] = c;
  }
  __syncthreads();
  const int nchunks = cstart[ncut];
  int zero_var = 0;
  for (int g = blockIdx.x; g < G; g += gridDim.x) {
    for (int i = threadIdx.x; i < NS * ncut * NP; i += kEppsThreads) sacc[i] = (T)0;
    __syncthreads();
    const C2* cg = coef + (size_t)g * DG * ld;
    // each warp takes whole chunks: all 32 lanes in one segment, registers
    // accumulate over the chunk, one warp reduction per chunk
    for (int ch = warp; ch < nchunks; ch += NW) {
      int sj = 0;
      {
        int lo = 0, hi = ncut - 1;  // last segment with cstart <= ch
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (cstart[mid] <= ch) lo = mid;
          else hi = mid - 1;
        }
        sj = lo;
      }
      const int kb = (sj ? scut[sj - 1] + 1 : 0) + (ch - cstart[sj]) * kChunkModes;
      const int ke = min(kb + kChunkModes, scut[sj] + 1);
      const int es = scut[sj];  // the segment's end cutoff: weights e_s - k >= 0
      T acc[NP], acc1[FEJER ? NP : 1];
#pragma unroll
      for (int p = 0; p < NP; ++p) acc[p] = (T)0;
#pragma unroll
      for (int p = 0; p < (FEJER ? NP : 1); ++p) acc1[p] = (T)0;
      for (int k = kb + lane; k < ke; k += 32) {
        C2 c[DG];
        const T sc = k == 0 ? (T)1 : (T)1.41421356237309515;  // sqrt(d_k)
#pragma unroll
        for (int i = 0; i < DG; ++i) {
          const C2 v = __ldg(cg + (size_t)i * ld + k);
          c[i].x = v.x * sc;
          c[i].y = v.y * sc;
        }
        const T kf = (T)(es - k);
        int p = 0;
#pragma unroll
        for (int i = 0; i < DG; ++i)
#pragma unroll
          for (int j = i; j < DG; ++j, ++p) {
            const T q = fma(c[i].x, c[j].x, c[i].y * c[j].y);
            acc[p] += q;
            if (FEJER) acc1[p] = fma(kf, q, acc1[p]);
          }
      }
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        T v = acc[p];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) atomicAdd(&sacc[sj * NP + p], v);
        if (FEJER) {
          T w = acc1[p];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
          if (lane == 0) atomicAdd(&sacc[(ncut + sj) * NP + p], w);
        }
      }
    }
    __syncthreads();
    // prefix over segments with the basis weights (float64), then the
    // diagonal normalisation: 1/sqrt(Sigma_aa) in float64 once per asset and
    // cutoff, the off-diagonal products in float32
    for (int p = threadIdx.x; p < NP; p += kEppsThreads) {
      double P = 0.0, A = 0.0, Ts = 0.0;
      for (int j = 0; j < ncut; ++j) {
        if (FEJER && j > 0) A += (double)(scut[j] - scut[j - 1]) * P;
        P += (double)sacc[j * NP + p];
        if (FEJER) Ts += (double)sacc[(ncut + j) * NP + p];
        ssig[j * NP + p] = FEJER ? swt[j] * (A + Ts) : swt[j] * P;
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ncut * DG; e += kEppsThreads) {
      const int j = e / DG, a = e - j * DG;
      const double d = ssig[j * NP + a * DG - a * (a - 1) / 2];
      sinv[e] = d > 0.0 ? (T)rsqrt(d) : (T)__longlong_as_double(0x7ff8000000000000ll);
      if (!(d > 0.0)) zero_var = 1;
    }
    __syncthreads();
    // Sigma and R for every cutoff, both triangles
    for (int e = threadIdx.x; e < ncut * DG * DG; e += kEppsThreads) {
      const int j = e / (DG * DG), r = e - j * DG * DG;
      const int a = r / DG, b = r - a * DG;
      const int lo = a < b ? a : b, hi = a < b ? b : a;
      const int p = lo * DG - lo * (lo - 1) / 2 + (hi - lo);  // index of pair (lo, hi)
      const T sv = (T)ssig[j * NP + p];
      const size_t o = ((size_t)g * ncut + j) * DG * DG + r;
      if (sigma) sigma[o] = sv;
      Rout[o] = a == b ? (sinv[j * DG + a] == sinv[j * DG + a] ? (T)1 : sinv[j * DG + a])
                       : sv * sinv[j * DG + a] * sinv[j * DG + b];
    }
    __syncthreads();
  }
  if (zero_var) atomicOr(status, ST_ZERO_VAR);
}

template <typename T, int DG>
cudaError_t launch_dg(bool fejer, const void* coef, int ld, const int* cut, int ncut, int G, void* sigma, void* R,
                      const int* status_gate, int* status, int grid, cudaStream_t s) {
  constexpr int NP = Pairs<DG>::n;
  const int NS = fejer ? 2 : 1;
  const size_t smem = (((size_t)NS * ncut * NP * sizeof(T) + 15) & ~(size_t)15) + (size_t)ncut * NP * 8;
  auto go = [&](auto fn) -> cudaError_t {
    // static + dynamic shared memory may pass 48 KB: always opt in
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, kEppsThreads, smem, s>>>((const typename Cx<T>::type*)coef, ld, cut, ncut, G, (T*)sigma, (T*)R,
                                        status_gate, status);
    return cudaGetLastError();
  };
  return fejer ? go(k_epps<T, DG, true>) : go(k_epps<T, DG, false>);
}

template <typename T>
cudaError_t launch_t(int Dg, bool fejer, const void* coef, int ld, const int* cut, int ncut, int G, void* sigma,
                     void* R, int* status, int grid, cudaStream_t s) {
  const int* gate = status + 1;
  switch (Dg) {
    case 1: return launch_dg<T, 1>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 2: return launch_dg<T, 2>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 3: return launch_dg<T, 3>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 4: return launch_dg<T, 4>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 5: return launch_dg<T, 5>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 6: return launch_dg<T, 6>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 7: return launch_dg<T, 7>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 8: return launch_dg<T, 8>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 9: return launch_dg<T, 9>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 10: return launch_dg<T, 10>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 11: return launch_dg<T, 11>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    case 12: return launch_dg<T, 12>(fejer, coef, ld, cut, ncut, G, sigma, R, gate, status, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

int epps_max_assets() { return kMaxEppsAssets; }

cudaError_t launch_epps(int Dg, bool fejer, bool fp64, const void* coef, int ld, const int* cut, int ncut, int G,
                        void* sigma, void* R, int* status, int grid, cudaStream_t s) {
  if (ncut < 1 || ncut > kMaxCutoffs || G < 1) return cudaErrorInvalidValue;
  return fp64 ? launch_t<double>(Dg, fejer, coef, ld, cut, ncut, G, sigma, R, status, grid, s)
              : launch_t<float>(Dg, fejer, coef, ld, cut, ncut, G, sigma, R, status, grid, s);
}

}  // namespace mmgpu
