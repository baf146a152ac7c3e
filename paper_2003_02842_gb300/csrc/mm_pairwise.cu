// mm_pairwise.cu -- covariance with a cutoff per pair of assets and the
// repair to the nearest positive semi-definite matrix (Sec. 3.1: when each
// asset has its own cutoff, e.g. its own Nyquist cutoff in the arrival-time
// representation, each entry is a pairwise estimate, and neither basis then
// guarantees a positive semi-definite matrix).
//
// Sigma_ij is Eq. (2) (Dirichlet) or Eq. (3) (Fejer) at N_ij = min(N_i, N_j)
// from coefficients computed once at max_i N_i:
//   Dirichlet  (2 pi)^2 / (2N + 1)      * sum_{k<=N} d_k Re(F_i(k) conj F_j(k)),
//   Fejer      (2 pi)^2 / ((N + 1) N)   * sum_{k<=N} d_k (N - k) Re(F_i(k) conj F_j(k)),
// d_0 = 1, d_k = 2 (the -k half folded in); every weight is non-negative.
// One CTA per 16 x 16 tile of pairs (upper tiles), the two tiles' coefficient
// rows staged in shared memory 128 modes at a time; a thread owns one pair,
// sums a chunk in the coefficients' precision and adds it to a float64 sum.
//
// Repair: the matrix closest to Sigma in the Frobenius norm among the positive
// semi-definite ones is V max(Lambda, 0) V^T (Sigma = V Lambda V^T), the
// eigenvalue method the paper points to. The eigendecomposition is a cyclic
// Jacobi iteration in one CTA: each step applies D/2 disjoint
// rotations in parallel (round-robin pairing), a sweep is D - 1 steps, and
// the sweeps stop when the off-diagonal norm is below 2 D eps of the matrix
// norm (eps of the working type: float64 for FP64 plans, float32 for the
// mixed precisions' float32 Sigma) or after kJacobiSweeps. GB300 issues
// float64 at a small fraction of the float32 rate, so the mixed path works
// in float32.
#include <math.h>

#include "mm_common.cuh"

namespace mmgpu {

namespace {

constexpr int kPT = 16;        // tile edge (pairs per tile: 16 x 16)
constexpr int kPChunk = 128;   // modes staged per chunk
constexpr int kJacobiThreads = 1024;
constexpr int kJacobiSweeps = 40;
constexpr int kPsdMaxD = 256;  // rotation arrays of the one-CTA repair (it takes what fits 200 KB)
constexpr size_t kPsdSmemBytes = 200 * 1024;  // the working matrix and eigenvectors in shared memory up to this

__device__ __forceinline__ void tile_of(int p, int nt, int& I, int& J) {
  int i = 0;
  while (p >= nt - i) {
    p -= nt - i;
    ++i;
  }
  I = i;
  J = i + p;
}

template <typename T2>
__device__ __forceinline__ T2 zero2() {
  T2 z;
  z.x = 0;
  z.y = 0;
  return z;
}

template <typename T2, typename T, bool FEJER>
__global__ void __launch_bounds__(256) k_pairwise(const T2* __restrict__ F, int ld, const int* __restrict__ Nv,
                                                  int D, int nt, double* __restrict__ sig) {
  __shared__ T2 a[kPT][kPChunk + 1], b[kPT][kPChunk + 1];
  __shared__ int s_nmax;
  int I, J;
  tile_of(blockIdx.x, nt, I, J);
  const int ti = threadIdx.x / kPT, tj = threadIdx.x % kPT;
  const int i = I * kPT + ti, j = J * kPT + tj;
  const bool valid = i < D && j < D && (I < J || ti <= tj);
  const int Nij = valid ? min(Nv[i], Nv[j]) : -1;
  if (threadIdx.x == 0) s_nmax = -1;
  __syncthreads();
  if (valid) atomicMax(&s_nmax, Nij);
  __syncthreads();
  const int nmax = s_nmax;  // the tile's largest pairwise cutoff
  double acc = 0.0;
  for (int k0 = 0; k0 <= nmax; k0 += kPChunk) {
    for (int e = threadIdx.x; e < kPT * kPChunk; e += blockDim.x) {
      const int r = e / kPChunk, c = e - r * kPChunk;
      const int k = k0 + c;
      const int ra = I * kPT + r, rb = J * kPT + r;
      a[r][c] = (k <= nmax && ra < D) ? F[(size_t)ra * ld + k] : zero2<T2>();
      b[r][c] = (k <= nmax && rb < D) ? F[(size_t)rb * ld + k] : zero2<T2>();
    }
    __syncthreads();
    T part = 0;
    const int cend = min(kPChunk - 1, Nij - k0);  // last mode of this pair in the chunk
    for (int c = 0; c <= cend; ++c) {
      const int k = k0 + c;
      T w = k == 0 ? (T)1 : (T)2;
      if (FEJER) w *= (T)(Nij - k);
      part += w * (a[ti][c].x * b[tj][c].x + a[ti][c].y * b[tj][c].y);
    }
    acc += (double)part;
    __syncthreads();
  }
  if (valid) {
    const double fp2 = 4.0 * kPi * kPi;
    const double v = acc * (FEJER ? fp2 / (((double)Nij + 1.0) * (double)Nij) : fp2 / (2.0 * Nij + 1.0));
    sig[(size_t)i * D + j] = v;
    sig[(size_t)j * D + i] = v;
  }
}

// The Jacobi iteration (Golub and Van Loan, the cyclic Jacobi algorithm with
// a parallel ordering): rotation (p, q) with tau = (a_qq - a_pp) / (2 a_pq),
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c
// zeroes a_pq in J^T A J, J = [[c, s], [-s, c]] on rows and columns p, q;
// V accumulates V J. A is a float64 copy of Sigma, V the eigenvectors (both
// in shared memory up to D = 112, else in global scratch); sig is replaced by
// V max(Lambda, 0) V^T only when an eigenvalue is negative.
template <typename W>
__global__ void __launch_bounds__(kJacobiThreads) k_psd_repair(double* __restrict__ sig, W* Ag, W* Vg, int D,
                                                               int* clipped) {
  // the working matrix and the eigenvectors in shared memory when both fit,
  // else in the global scratch
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const bool in_smem = (size_t)2 * D * D * sizeof(W) <= kPsdSmemBytes;
  W* A = in_smem ? reinterpret_cast<W*>(smem_raw) : Ag;
  W* V = in_smem ? reinterpret_cast<W*>(smem_raw) + (size_t)D * D : Vg;
  __shared__ int sp[kPsdMaxD / 2], sq[kPsdMaxD / 2];
  __shared__ W sc[kPsdMaxD / 2], ss[kPsdMaxD / 2];
  __shared__ double s_lam[kPsdMaxD];
  __shared__ double s_red[kJacobiThreads / 32];
  __shared__ int s_neg;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int m = (D + 1) & ~1;  // players of the round-robin (one idle when D is odd)
  const int nh = m / 2;
  for (int e = tid; e < D * D; e += nth) {
    A[e] = (W)sig[e];
    const int r = e / D;
    V[e] = (r == e - r * D) ? (W)1 : (W)0;
  }
  __syncthreads();
  auto block_sum = [&](double v) -> double {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) s_red[tid >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (nth >> 5); ++w) t += s_red[w];
    __syncthreads();
    return t;
  };
  double nrm = 0.0;
  for (int e = tid; e < D * D; e += nth) nrm += (double)A[e] * (double)A[e];
  const double norm2 = block_sum(nrm);
  // converged when the off-diagonal norm reaches the level rounding leaves in
  // a D x D rotation sequence, 2 D eps of the norm (eps of the working type)
  const double eps = sizeof(W) == 8 ? 1.1102230246251565e-16 : 5.9604644775390625e-8;
  const double rel2 = (2.0 * D * eps) * (2.0 * D * eps);
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    double off = 0.0;
    for (int e = tid; e < D * D; e += nth) {
      const int r = e / D;
      if (r != e - r * D) off += (double)A[e] * (double)A[e];
    }
    if (!(block_sum(off) > rel2 * norm2)) break;  // uniform
    for (int step = 0; step < m - 1; ++step) {
      // round-robin: player m-1 meets player `step`; the others pair up
      // symmetrically around it
      if (tid < nh) {
        int p, q;
        if (tid == 0) {
          p = step;
          q = m - 1;
        } else {
          p = (step + tid) % (m - 1);
          q = (step - tid + (m - 1)) % (m - 1);
        }
        if (p > q) {
          const int x = p;
          p = q;
          q = x;
        }
        W c = 1, sn = 0;
        if (q < D) {
          const W apq = A[(size_t)p * D + q];
          if (apq != (W)0) {
            const W tau = (A[(size_t)q * D + q] - A[(size_t)p * D + p]) / ((W)2 * apq);
            const W t = (tau >= (W)0 ? (W)1 : (W)-1) / (fabs(tau) + sqrt((W)1 + tau * tau));
            c = (W)1 / sqrt((W)1 + t * t);
            sn = t * c;
          }
        }
        sp[tid] = p;
        sq[tid] = q;
        sc[tid] = c;
        ss[tid] = sn;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int e = tid; e < nh * D; e += nth) {
        const int r = e / D, x = e - r * D;
        const int p = sp[r], q = sq[r];
        if (q >= D) continue;
        const W c = sc[r], sn = ss[r];
        const W ap = A[(size_t)p * D + x], aq = A[(size_t)q * D + x];
        A[(size_t)p * D + x] = c * ap - sn * aq;
        A[(size_t)q * D + x] = sn * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int e = tid; e < nh * D; e += nth) {
        const int r = e / D, x = e - r * D;
        const int p = sp[r], q = sq[r];
        if (q >= D) continue;
        const W c = sc[r], sn = ss[r];
        const W ap = A[(size_t)x * D + p], aq = A[(size_t)x * D + q];
        A[(size_t)x * D + p] = c * ap - sn * aq;
        A[(size_t)x * D + q] = sn * ap + c * aq;
        const W vp = V[(size_t)x * D + p], vq = V[(size_t)x * D + q];
        V[(size_t)x * D + p] = c * vp - sn * vq;
        V[(size_t)x * D + q] = sn * vp + c * vq;
      }
      __syncthreads();
    }
  }
  if (tid == 0) s_neg = 0;
  __syncthreads();
  for (int i = tid; i < D; i += nth) {
    const double l = (double)A[(size_t)i * D + i];
    s_lam[i] = l > 0.0 ? l : 0.0;
    if (l < 0.0) atomicAdd(&s_neg, 1);
  }
  __syncthreads();
  if (tid == 0 && clipped) *clipped = s_neg;
  if (s_neg == 0) return;  // already positive semi-definite: Sigma unchanged
  for (int e = tid; e < D * D; e += nth) {
    const int i = e / D, j = e - i * D;
    if (j < i) continue;
    W v = 0;
    for (int k = 0; k < D; ++k) v += V[(size_t)i * D + k] * (W)s_lam[k] * V[(size_t)j * D + k];
    sig[(size_t)i * D + j] = v;
    sig[(size_t)j * D + i] = v;
  }
}

// The same cyclic Jacobi iteration over the whole GPU, for matrices larger
// than one CTA's shared memory holds: one CTA per SM under a cooperative
// launch (every CTA resident), A and V in global memory (read through L2).
// A round-robin step's rotations act on disjoint index pairs, so J^T A J
// splits into independent 2 x 2 blocks (rows p_i, q_i; columns p_j, q_j):
// after a grid barrier every CTA recomputes the step's D/2 rotations from
// A's current diagonal and pivot entries, and the threads of the grid update
// the blocks of A and the column pairs of V (each element written by one
// thread). One barrier per step, one reduction per sweep; every barrier wait
// is bounded (ST_TIMEOUT, and the CTA leaves).
struct GridSync {
  unsigned count;  // arrivals at the current barrier
  unsigned gen;    // barriers completed
  int neg;         // negative eigenvalues
  int pad;
  double red[3];   // [0] squared norm, [1], [2] off-diagonal sums of alternate sweeps
};

__device__ __forceinline__ uint64_t grid_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier for a cooperative launch; false when the wait timed out.
__device__ bool grid_barrier(GridSync* gs, unsigned nblocks, int* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &gs->gen;
    const unsigned g = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&gs->count, 1u) == nblocks - 1) {
      atomicExch(&gs->count, 0u);
      __threadfence();
      atomicAdd(&gs->gen, 1u);
    } else {
      const uint64_t t0 = grid_timer_ns();
      while (*vgen == g) {
        if (grid_timer_ns() - t0 > kDefaultWaitNs) {
          ok = 0;
          atomicOr(status, ST_TIMEOUT);
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

constexpr int kGridJacobiThreads = 512;
constexpr int kGridMaxD = 4000;  // rotations of one step fit 48 KB of shared memory

template <typename W>
__global__ void __launch_bounds__(kGridJacobiThreads) k_psd_repair_grid(double* __restrict__ sig, W* __restrict__ A,
                                                                        W* __restrict__ V, int D, int* clipped,
                                                                        GridSync* gs, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = (D + 1) & ~1, nh = m / 2;
  W* rc = reinterpret_cast<W*>(smem_raw);
  W* rs = rc + nh;
  int* rp = reinterpret_cast<int*>(rs + nh);
  int* rq = rp + nh;
  __shared__ double s_red[kGridJacobiThreads / 32];
  const unsigned nb = gridDim.x;
  const int tid = threadIdx.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + tid, gnth = (int64_t)gridDim.x * blockDim.x;
  const int64_t DD = (int64_t)D * D;
  auto block_sum_to = [&](double v, double* dst) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) s_red[tid >> 5] = v;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < kGridJacobiThreads / 32; ++w) t += s_red[w];
      atomicAdd(dst, t);
    }
    __syncthreads();
  };
  double nrm = 0.0;
  for (int64_t e = gtid; e < DD; e += gnth) {
    const W a = (W)sig[e];
    A[e] = a;
    const int64_t r = e / D;
    V[e] = (r == e - r * D) ? (W)1 : (W)0;
    nrm += (double)a * (double)a;
  }
  block_sum_to(nrm, &gs->red[0]);
  if (!grid_barrier(gs, nb, status)) return;
  const double norm2 = __ldcg(&gs->red[0]);
  const double eps = sizeof(W) == 8 ? 1.1102230246251565e-16 : 5.9604644775390625e-8;
  const double rel2 = (2.0 * D * eps) * (2.0 * D * eps);
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    double* slot = &gs->red[1 + (sweep & 1)];
    double off = 0.0;
    for (int64_t e = gtid; e < DD; e += gnth) {
      const int64_t r = e / D;
      if (r != e - r * D) {
        const double a = (double)__ldcg(A + e);
        off += a * a;
      }
    }
    block_sum_to(off, slot);
    if (!grid_barrier(gs, nb, status)) return;
    const double off_all = __ldcg(slot);
    // the other slot was last read before this barrier: clear it for the next sweep
    if (blockIdx.x == 0 && tid == 0) gs->red[1 + ((sweep + 1) & 1)] = 0.0;
    if (!(off_all > rel2 * norm2)) break;  // uniform: every CTA read the same sum
    for (int step = 0; step < m - 1; ++step) {
      for (int i = tid; i < nh; i += blockDim.x) {
        int p, q;
        if (i == 0) {
          p = step;
          q = m - 1;
        } else {
          p = (step + i) % (m - 1);
          q = (step - i + (m - 1)) % (m - 1);
        }
        if (p > q) {
          const int x = p;
          p = q;
          q = x;
        }
        W c = 1, sn = 0;
        if (q < D) {
          const W apq = __ldcg(A + (int64_t)p * D + q);
          if (apq != (W)0) {
            const W tau = (__ldcg(A + (int64_t)q * D + q) - __ldcg(A + (int64_t)p * D + p)) / ((W)2 * apq);
            const W t = (tau >= (W)0 ? (W)1 : (W)-1) / (fabs(tau) + sqrt((W)1 + tau * tau));
            c = (W)1 / sqrt((W)1 + t * t);
            sn = t * c;
          }
        }
        rp[i] = p;
        rq[i] = q;
        rc[i] = c;
        rs[i] = sn;
      }
      __syncthreads();
      // A <- J^T A J by 2 x 2 blocks (rows of pair i, columns of pair j)
      const int64_t nblk = (int64_t)nh * nh;
      for (int64_t e = gtid; e < nblk; e += gnth) {
        const int i = (int)(e / nh), j = (int)(e - (int64_t)i * nh);
        const int pi = rp[i], qi = rq[i], pj = rp[j], qj = rq[j];
        const bool vi = qi < D, vj = qj < D;
        const W ci = rc[i], si = rs[i], cj = rc[j], sj = rs[j];
        const W app = __ldcg(A + (int64_t)pi * D + pj);
        const W apq = vj ? __ldcg(A + (int64_t)pi * D + qj) : (W)0;
        const W aqp = vi ? __ldcg(A + (int64_t)qi * D + pj) : (W)0;
        const W aqq = (vi && vj) ? __ldcg(A + (int64_t)qi * D + qj) : (W)0;
        // rows: J_i^T, then columns: J_j
        const W bpp = ci * app - si * aqp, bpq = ci * apq - si * aqq;
        const W bqp = si * app + ci * aqp, bqq = si * apq + ci * aqq;
        A[(int64_t)pi * D + pj] = cj * bpp - sj * bpq;
        if (vj) A[(int64_t)pi * D + qj] = sj * bpp + cj * bpq;
        if (vi) A[(int64_t)qi * D + pj] = cj * bqp - sj * bqq;
        if (vi && vj) A[(int64_t)qi * D + qj] = sj * bqp + cj * bqq;
      }
      // V <- V J by column pairs
      const int64_t nv = (int64_t)D * nh;
      for (int64_t e = gtid; e < nv; e += gnth) {
        const int x = (int)(e / nh), j = (int)(e - (int64_t)x * nh);
        const int pj = rp[j], qj = rq[j];
        if (qj >= D) continue;
        const W cj = rc[j], sj = rs[j];
        const W vp = __ldcg(V + (int64_t)x * D + pj), vq = __ldcg(V + (int64_t)x * D + qj);
        V[(int64_t)x * D + pj] = cj * vp - sj * vq;
        V[(int64_t)x * D + qj] = sj * vp + cj * vq;
      }
      if (!grid_barrier(gs, nb, status)) return;
    }
  }
  // eigenvalues: the diagonal, negatives clipped
  int neg = 0;
  for (int i = (int)gtid; i < D; i += (int)gnth)
    if (__ldcg(A + (int64_t)i * D + i) < (W)0) ++neg;
  if (neg) atomicAdd(&gs->neg, neg);
  if (!grid_barrier(gs, nb, status)) return;
  const int negs = *(volatile int*)&gs->neg;
  if (blockIdx.x == 0 && tid == 0 && clipped) *clipped = negs;
  if (negs == 0) return;  // already positive semi-definite: Sigma unchanged
  // the clipped eigenvalues in this CTA's shared memory (the rotation arrays
  // hold at least 8 D bytes)
  double* lam = reinterpret_cast<double*>(smem_raw);
  for (int k = tid; k < D; k += blockDim.x) {
    const double l = (double)__ldcg(A + (int64_t)k * D + k);
    lam[k] = l > 0.0 ? l : 0.0;
  }
  __syncthreads();
  const int64_t npairs = (int64_t)D * (D + 1) / 2;
  for (int64_t e = gtid; e < npairs; e += gnth) {
    // pair (i, j), i <= j, in row-major order of the upper triangle
    int i = (int)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
    while ((int64_t)(i + 1) * (i + 2) / 2 <= e) ++i;
    while ((int64_t)i * (i + 1) / 2 > e) --i;
    const int jj = (int)(e - (int64_t)i * (i + 1) / 2);  // 0..i
    const int r = jj, c = i;                             // r <= c
    double v = 0.0;
    for (int k = 0; k < D; ++k)
      if (lam[k] > 0.0) v += (double)__ldcg(V + (int64_t)r * D + k) * lam[k] * (double)__ldcg(V + (int64_t)c * D + k);
    sig[(int64_t)r * D + c] = v;
    sig[(int64_t)c * D + r] = v;
  }
}

// Sigma and R in the output precision: R_ij = Sigma_ij / sqrt(Sigma_ii Sigma_jj)
// (float64), R_ii = 1; a non-positive variance gives NaN and ST_ZERO_VAR.
template <typename T>
__global__ void k_pairwise_out(const double* __restrict__ sig, int D, T* __restrict__ sigma, T* __restrict__ R,
                               int* status) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= D * D) return;
  const int i = e / D, j = e - i * D;
  const double v = sig[e], a = sig[(size_t)i * D + i], b = sig[(size_t)j * D + j];
  if (sigma) sigma[e] = (T)v;
  double r;
  if (a > 0.0 && b > 0.0) {
    r = (i == j) ? 1.0 : v / (sqrt(a) * sqrt(b));
  } else {
    r = __longlong_as_double(0x7ff8000000000000ll);
    if (i == j) atomicOr(status, ST_ZERO_VAR);
  }
  R[e] = (T)r;
}

}  // namespace

}  // namespace mmgpu

namespace mmgpu {

int pairwise_psd_max_assets() { return kGridMaxD; }

cudaError_t launch_pairwise(bool fp64, bool fejer, const void* coeffs, int ld, const int* Nv, int D,
                            double* sig, cudaStream_t s) {
  const int nt = (D + kPT - 1) / kPT;
  const int grid = nt * (nt + 1) / 2;
  if (fp64) {
    if (fejer) k_pairwise<double2, double, true><<<grid, 256, 0, s>>>((const double2*)coeffs, ld, Nv, D, nt, sig);
    else k_pairwise<double2, double, false><<<grid, 256, 0, s>>>((const double2*)coeffs, ld, Nv, D, nt, sig);
  } else {
    if (fejer) k_pairwise<float2, float, true><<<grid, 256, 0, s>>>((const float2*)coeffs, ld, Nv, D, nt, sig);
    else k_pairwise<float2, float, false><<<grid, 256, 0, s>>>((const float2*)coeffs, ld, Nv, D, nt, sig);
  }
  return cudaGetLastError();
}

cudaError_t launch_psd_repair(bool fp64, double* sig, double* A, double* V, int D, int* clipped, void* sync,
                              int* status, cudaStream_t s) {
  if (D > kGridMaxD) return cudaErrorInvalidValue;
  const size_t wb = fp64 ? 8 : 4;
  const size_t need = 2 * (size_t)D * D * wb;
  if (need <= kPsdSmemBytes) {
    // the working matrix and eigenvectors in one CTA's shared memory
    auto one = [&](auto kern) -> cudaError_t {
      const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
      if (e != cudaSuccess) return e;
      return cudaSuccess;
    };
    cudaError_t e;
    if (fp64) {
      if ((e = one(k_psd_repair<double>)) != cudaSuccess) return e;
      k_psd_repair<double><<<1, kJacobiThreads, need, s>>>(sig, A, V, D, clipped);
    } else {
      if ((e = one(k_psd_repair<float>)) != cudaSuccess) return e;
      k_psd_repair<float><<<1, kJacobiThreads, need, s>>>(sig, (float*)A, (float*)V, D, clipped);
    }
    return cudaGetLastError();
  }
  // the whole GPU: one CTA per SM, every CTA resident (cooperative launch)
  cudaError_t e = cudaMemsetAsync(sync, 0, sizeof(GridSync), s);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int nh = ((D + 1) & ~1) / 2;
  const size_t smem = (size_t)nh * (2 * wb + 2 * sizeof(int));
  GridSync* gs = reinterpret_cast<GridSync*>(sync);
  auto launch = [&](auto kern, void* Aw, void* Vw) -> cudaError_t {
    int per_sm = 0;
    cudaError_t r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGridJacobiThreads, smem);
    if (r != cudaSuccess) return r;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    void* args[] = {(void*)&sig, &Aw, &Vw, (void*)&D, (void*)&clipped, (void*)&gs, (void*)&status};
    return cudaLaunchCooperativeKernel((const void*)kern, dim3(sms), dim3(kGridJacobiThreads), args, smem, s);
  };
  if (fp64) return launch(k_psd_repair_grid<double>, (void*)A, (void*)V);
  return launch(k_psd_repair_grid<float>, (void*)A, (void*)V);
}

size_t psd_sync_bytes() { return sizeof(GridSync); }

cudaError_t launch_pairwise_out(bool fp64, const double* sig, int D, void* sigma, void* R, int* status,
                                cudaStream_t s) {
  const int n = D * D, grid = (n + 255) / 256;
  if (fp64) k_pairwise_out<double><<<grid, 256, 0, s>>>(sig, D, (double*)sigma, (double*)R, status);
  else k_pairwise_out<float><<<grid, 256, 0, s>>>(sig, D, (float*)sigma, (float*)R, status);
  return cudaGetLastError();
}

}  // namespace mmgpu
