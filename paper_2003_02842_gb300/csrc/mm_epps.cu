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
// N_max + 1 modes); the diagonal normalisation is float64.
#include "mm_common.cuh"

namespace mmgpu {

namespace {

constexpr int kEppsThreads = 256;
constexpr int kChunkModes = 512;  // modes per warp work item (16 per lane)

template <int DG>
struct Pairs {
  static constexpr int n = DG * (DG + 1) / 2;
};

template <int DG, bool FEJER>
__global__ void __launch_bounds__(kEppsThreads) k_epps(const float2* __restrict__ coef, int ld, const int* __restrict__ cut_g,
                                                       int ncut, int G, float* __restrict__ sigma,
                                                       float* __restrict__ Rout, const int* __restrict__ gate,
                                                       int* status) {
  constexpr int NP = Pairs<DG>::n;
  constexpr int NS = FEJER ? 2 : 1;
  constexpr int NW = kEppsThreads / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sacc = reinterpret_cast<float*>(smem_raw);                     // [NS][ncut][NP]
  double* ssig = reinterpret_cast<double*>(smem_raw + (((size_t)NS * ncut * NP * 4 + 15) & ~(size_t)15));  // [ncut][NP]
  __shared__ int scut[kMaxCutoffs];
  __shared__ int cstart[kMaxCutoffs + 1];                  // first chunk of each segment
  __shared__ double swt[kMaxCutoffs];                      // basis weight per cutoff
  __shared__ float sinv[kMaxCutoffs * DG];                 // 1 / sqrt(Sigma_aa(N_j))
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
    for (int i = threadIdx.x; i < NS * ncut * NP; i += kEppsThreads) sacc[i] = 0.f;
    __syncthreads();
    const float2* cg = coef + (size_t)g * DG * ld;
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
      float acc[NP], acc1[FEJER ? NP : 1];
#pragma unroll
      for (int p = 0; p < NP; ++p) acc[p] = 0.f;
#pragma unroll
      for (int p = 0; p < (FEJER ? NP : 1); ++p) acc1[p] = 0.f;
      for (int k = kb + lane; k < ke; k += 32) {
        float2 c[DG];
        const float sc = k == 0 ? 1.0f : 1.41421356237309515f;  // sqrt(d_k)
#pragma unroll
        for (int i = 0; i < DG; ++i) {
          const float2 v = __ldg(cg + (size_t)i * ld + k);
          c[i] = make_float2(v.x * sc, v.y * sc);
        }
        const float kf = (float)(es - k);
        int p = 0;
#pragma unroll
        for (int i = 0; i < DG; ++i)
#pragma unroll
          for (int j = i; j < DG; ++j, ++p) {
            const float q = fmaf(c[i].x, c[j].x, c[i].y * c[j].y);
            acc[p] += q;
            if (FEJER) acc1[p] = fmaf(kf, q, acc1[p]);
          }
      }
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        float v = acc[p];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) atomicAdd(&sacc[sj * NP + p], v);
        if (FEJER) {
          float w = acc1[p];
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
      sinv[e] = d > 0.0 ? (float)rsqrt(d) : __int_as_float(0x7fc00000);
      if (!(d > 0.0)) zero_var = 1;
    }
    __syncthreads();
    // Sigma and R for every cutoff, both triangles
    for (int e = threadIdx.x; e < ncut * DG * DG; e += kEppsThreads) {
      const int j = e / (DG * DG), r = e - j * DG * DG;
      const int a = r / DG, b = r - a * DG;
      const int lo = a < b ? a : b, hi = a < b ? b : a;
      const int p = lo * DG - lo * (lo - 1) / 2 + (hi - lo);  // index of pair (lo, hi)
      const float sv = (float)ssig[j * NP + p];
      const size_t o = ((size_t)g * ncut + j) * DG * DG + r;
      if (sigma) sigma[o] = sv;
      Rout[o] = a == b ? (sinv[j * DG + a] == sinv[j * DG + a] ? 1.0f : sinv[j * DG + a])
                       : sv * sinv[j * DG + a] * sinv[j * DG + b];
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
    // static + dynamic shared memory may pass 48 KB: always opt in
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
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
