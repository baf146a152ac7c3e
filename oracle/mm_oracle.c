/*
 * mm_oracle.c -- plain, slow, FP64 CPU oracle for the Malliavin-Mancino
 * Fourier covariance estimator computed with type-1 NUFFTs
 * (Chang, Pienaar & Gebbie, "Malliavin-Mancino estimators implemented with
 * non-uniform fast Fourier transforms", arXiv:2003.02842).
 *
 * TEST INFRASTRUCTURE. This file states what the GPU library must compute,
 * written from the paper's definitions. It shares no code, header, table or
 * constant generator with the CUDA path. Only tests/, __graft_entry__.smoke()
 * and bench.py's CPU-baseline / reference legs may load it; the product never
 * calls it.
 *
 * Every function cites the passage it follows. Equation numbers follow the
 * paper's display order: (2) Dirichlet estimator, (3) Fejer estimator,
 * (4) Fourier coefficients, (5)-(10) averaging kernels, (12) spreading,
 * (13) FFT on the grid, (14) deconvolution, (15) relative l2 error,
 * (19) Delta-t -> N. Algorithms follow the appendix order: 2 Nyquist,
 * 3 MM estimators, 4 time rescaling, 8 FGG NUFFT, 9 Kaiser-Bessel NUFFT,
 * 10 exponential-of-semicircle NUFFT.
 *
 * Parity status: every exported function is pinned by tests/test_oracle_*.py
 * against closed forms, brute force, printed constants or library routines;
 * none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846264338327950288

enum { ORC_KERNEL_GAUSS = 0, ORC_KERNEL_KB = 1, ORC_KERNEL_ES = 2 };
enum { ORC_BASIS_DIRICHLET = 0, ORC_BASIS_FEJER = 1 };

/* ------------------------------------------------------------------------- */
/* Compensated (Neumaier) summation: keeps the oracle's own rounding far below */
/* the 1e-10 tolerance of the FP64 GPU path.                                   */
/* ------------------------------------------------------------------------- */
typedef struct { double s, c; } orc_sum;
static void sum_add(orc_sum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}
static double sum_get(const orc_sum* a) { return a->s + a->c; }

/* Fraction of k * (t - t0) / span in cycles, reduced to [-1/2, 1/2], computed
 * in double-double so that e^{-i k t~} is evaluated at the exact rescaled time
 * t~ = 2 pi (t - t0) / span of Algorithm 4, with an absolute phase error near
 * 1e-16 cycles even for k * t~ of order 1e6. */
static double cycles_frac(double k, double t, double t0, double span) {
  /* a = t - t0 exactly (TwoSum) */
  double a_hi = t - t0;
  double bb = a_hi - t;
  double a_lo = (t - (a_hi - bb)) + (-t0 - bb);
  /* q = a / span as a double-double */
  double q_hi = a_hi / span;
  double r = fma(-q_hi, span, a_hi);
  double q_lo = (r + a_lo) / span;
  /* x = k * q */
  double p_hi = k * q_hi;
  double p_lo = fma(k, q_hi, -p_hi) + k * q_lo;
  double f = p_hi - nearbyint(p_hi); /* exact */
  f += p_lo;
  f -= nearbyint(f);
  return f;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 4 (time rescaling): t_min, t_max over all assets' times.          */
/* ------------------------------------------------------------------------- */
void orc_bounds(int D, const int64_t* off, const double* t, double* tmin, double* tmax) {
  double lo = INFINITY, hi = -INFINITY;
  for (int i = 0; i < D; ++i)
    for (int64_t h = off[i]; h < off[i + 1]; ++h) {
      if (t[h] < lo) lo = t[h];
      if (t[h] > hi) hi = t[h];
    }
  *tmin = lo;
  *tmax = hi;
}

/* Algorithm 4: t~ = 2 pi (t - t_min) / (t_max - t_min). */
void orc_rescale(int64_t n, const double* t, double t0, double t1, double* tt) {
  double span = t1 - t0;
  for (int64_t h = 0; h < n; ++h) tt[h] = 2.0 * ORC_PI * (t[h] - t0) / span;
}

/* Returns (Sec. 2.1 below Eq. (2); Algorithm 3 step F.3): delta_i(I_h) =
 * p_i(t_{h+1}) - p_i(t_h), attached to the left end point t_h (previous-tick
 * interpolation). Writes, per asset, its n_i - 1 returns and their times into
 * CSR arrays (roff has D+1 entries). */
void orc_returns(int D, const int64_t* off, const double* t, const double* logp,
                 int64_t* roff, double* rt, double* rd) {
  int64_t o = 0;
  roff[0] = 0;
  for (int i = 0; i < D; ++i) {
    for (int64_t h = off[i]; h + 1 < off[i + 1]; ++h) {
      rt[o] = t[h];
      rd[o] = logp[h + 1] - logp[h];
      ++o;
    }
    roff[i + 1] = o;
  }
}

/* Algorithm 2 (Nyquist cutoff): Delta t0_i = smallest gap of asset i,
 * N_i = floor((2 pi / Delta t~0_i) / 2), N = min_i N_i. In raw time units this
 * is floor(span / (2 Delta t0_i)) (the footnote of Sec. 3.1), which avoids a
 * spurious floor() flip when span / Delta t0 is an even integer. Assets with
 * fewer than two events impose no limit. Returns -1 when no asset has a gap. */
int64_t orc_nyquist(int D, const int64_t* off, const double* t, double t0, double t1) {
  double span = t1 - t0;
  int64_t best = -1;
  for (int i = 0; i < D; ++i) {
    double g = INFINITY;
    for (int64_t h = off[i]; h + 1 < off[i + 1]; ++h) {
      double d = t[h + 1] - t[h];
      if (d < g) g = d;
    }
    if (!(g < INFINITY) || !(g > 0.0)) continue;
    int64_t Ni = (int64_t)floor(span / (2.0 * g));
    if (best < 0 || Ni < best) best = Ni;
  }
  return best;
}

/* Eq. (4) without the 1/(2 pi) (Algorithm 3 step F.4, c^-_k):
 *   c_k = sum_h delta_h e^{-i k t~_h},  t~_h = 2 pi (t_h - t0) / span,
 * for k = kmin..kmax. Output interleaved (re, im). Direct O(n (kmax-kmin+1))
 * sum with exact phase reduction and compensated accumulation. */
void orc_coeffs(int64_t n, const double* t, const double* delta, double t0, double span,
                int64_t kmin, int64_t kmax, double* out) {
  int64_t K = kmax - kmin + 1;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t kk = 0; kk < K; ++kk) {
    double k = (double)(kmin + kk);
    orc_sum re = {0, 0}, im = {0, 0};
    for (int64_t h = 0; h < n; ++h) {
      double f = cycles_frac(k, t[h], t0, span);
      double th = 2.0 * ORC_PI * f;
      sum_add(&re, delta[h] * cos(th));
      sum_add(&im, -delta[h] * sin(th));
    }
    out[2 * kk] = sum_get(&re);
    out[2 * kk + 1] = sum_get(&im);
  }
}

/* Same sum at an arbitrary list of (asset-local) modes k_list[0..nk). */
void orc_coeffs_at(int64_t n, const double* t, const double* delta, double t0, double span,
                   int64_t nk, const int64_t* k_list, double* out) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t q = 0; q < nk; ++q) {
    double k = (double)k_list[q];
    orc_sum re = {0, 0}, im = {0, 0};
    for (int64_t h = 0; h < n; ++h) {
      double f = cycles_frac(k, t[h], t0, span);
      double th = 2.0 * ORC_PI * f;
      sum_add(&re, delta[h] * cos(th));
      sum_add(&im, -delta[h] * sin(th));
    }
    out[2 * q] = sum_get(&re);
    out[2 * q + 1] = sum_get(&im);
  }
}

/* Basis weights of Algorithm 3 step C: Dirichlet 1/(2N+1) (C.1, Eq. (2));
 * Fejer (1 - |k|/N) / (N+1) (C.2, Eq. (3)), taken literally. */
double orc_weight(int basis, int64_t N, int64_t k) {
  if (basis == ORC_BASIS_DIRICHLET) return 1.0 / (double)(2 * N + 1);
  double ak = (double)(k < 0 ? -k : k);
  return (1.0 - ak / (double)N) / (double)(N + 1);
}

/* Algorithm 3 step C: Sigma_ij = sum_{k=-N..N} w_k c^+_k(i) c^-_k(j), with
 * c^-_k = c_k of Eq. (4) (times 2 pi) and c^+_k = c_{-k}. c holds, per asset,
 * the 2N+1 complex values for k = -N..N. Sigma is real; the largest |Im|
 * relative to sqrt(Sigma_ii Sigma_jj) is returned as a self-check. */
double orc_cov_from_coeffs(int D, int64_t N, int basis, const double* c, double* S) {
  int64_t M = 2 * N + 1;
  double worst = 0.0;
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      orc_sum re = {0, 0}, im = {0, 0};
      for (int64_t k = -N; k <= N; ++k) {
        const double* cp = c + 2 * ((int64_t)i * M + (-k + N)); /* c^+_k(i) = c_{-k}(i) */
        const double* cm = c + 2 * ((int64_t)j * M + (k + N));  /* c^-_k(j) = c_k(j)  */
        double w = orc_weight(basis, N, k);
        sum_add(&re, w * (cp[0] * cm[0] - cp[1] * cm[1]));
        sum_add(&im, w * (cp[0] * cm[1] + cp[1] * cm[0]));
      }
      S[(int64_t)i * D + j] = sum_get(&re);
      S[(int64_t)D * D + (int64_t)i * D + j] = sum_get(&im); /* scratch: imaginary parts */
    }
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      double sc = sqrt(fabs(S[(int64_t)i * D + i] * S[(int64_t)j * D + j]));
      double v = fabs(S[(int64_t)D * D + (int64_t)i * D + j]);
      if (sc > 0 && v / sc > worst) worst = v / sc;
    }
  return worst;
}

/* sin(pi * x) for any x, by exact reduction of x modulo 2. */
static double sinpi_red(double x) {
  double r = x - 2.0 * nearbyint(0.5 * x); /* exact, r in [-1, 1] */
  return sin(ORC_PI * r);
}

/* Eq. (2) and Eq. (3) with the sum over s done in closed form (an independent
 * second route to Sigma):
 *   Dirichlet  K(x) = (1/(2N+1)) sum_{|s|<=N} e^{isx} = sin((N+1/2)x) / ((2N+1) sin(x/2)),
 *   Fejer      K(x) = (1/(N+1)) sum_{|s|<=N} (1-|s|/N) e^{isx} = sin^2(Nx/2) / (N(N+1) sin^2(x/2)),
 * Sigma_ij = sum_{h,l} delta^i_h delta^j_l K(t~^j_l - t~^i_h). Returns (rt, rd)
 * are CSR arrays of return times (raw units) and returns. O(n_i n_j). */
void orc_cov_pairwise(int D, const int64_t* roff, const double* rt, const double* rd,
                      double t0, double span, int64_t N, int basis, double* S) {
  (void)t0;
  double Nd = (double)N;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t ij = 0; ij < (int64_t)D * D; ++ij) {
    int i = (int)(ij / D), j = (int)(ij % D);
    orc_sum acc = {0, 0};
    for (int64_t h = roff[i]; h < roff[i + 1]; ++h)
      for (int64_t l = roff[j]; l < roff[j + 1]; ++l) {
        double y = (rt[l] - rt[h]) / span; /* x = 2 pi y */
        double K;
        if (y == 0.0) {
          K = (basis == ORC_BASIS_DIRICHLET) ? 1.0 : Nd / (Nd + 1.0);
        } else {
          double den = sinpi_red(y); /* sin(x/2) */
          if (basis == ORC_BASIS_DIRICHLET) {
            K = sinpi_red((2.0 * Nd + 1.0) * y) / ((2.0 * Nd + 1.0) * den);
          } else {
            double num = sinpi_red(Nd * y);
            K = (num * num) / (Nd * (Nd + 1.0) * den * den);
          }
        }
        sum_add(&acc, rd[h] * rd[l] * K);
      }
    S[ij] = sum_get(&acc);
  }
}

/* Algorithm 3, last step: R_ij = Sigma_ij / (sqrt(Sigma_ii) sqrt(Sigma_jj)).
 * A zero-variance asset gives NaN entries in its row and column. */
void orc_corr(int D, const double* S, double* R) {
  for (int i = 0; i < D; ++i)
    for (int j = 0; j < D; ++j) {
      double a = S[(int64_t)i * D + i], b = S[(int64_t)j * D + j];
      R[(int64_t)i * D + j] = (a > 0 && b > 0) ? S[(int64_t)i * D + j] / (sqrt(a) * sqrt(b)) : NAN;
    }
}

/* ------------------------------------------------------------------------- */
/* NUFFT parameters, Sec. 2.2.5                                               */
/* ------------------------------------------------------------------------- */

/* Spreading half-width M_sp(eps) (Sec. 2.2.5, the paragraph after Eq. (15)),
 * with sigma = 2 as in step I.1 of Algorithms 8-10. */
int orc_msp(int kernel, double eps) {
  const double sigma = 2.0;
  if (kernel == ORC_KERNEL_GAUSS)
    return (int)floor(-log(eps) * (sigma - 0.5) / (ORC_PI * (sigma - 1.0)) + 0.5);
  int digits = (int)ceil(log10(1.0 / eps) - 1e-9);
  int m = (int)floor(0.5 * (double)(digits + 2));
  return kernel == ORC_KERNEL_ES ? m + 2 : m;
}

/* Modified Bessel function I_0 by its power series sum_j ((x/2)^{2j}) / (j!)^2
 * (all terms positive, so the series is accurate for the arguments used). */
double orc_bessel_i0(double x) {
  double q = 0.25 * x * x, term = 1.0, s = 1.0;
  for (int j = 1; j < 500; ++j) {
    term *= q / ((double)j * (double)j);
    s += term;
    if (term < 1e-18 * s) break;
  }
  return s;
}

/* Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on P_n. */
void orc_gauss_legendre(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(ORC_PI * ((double)i + 0.75) / ((double)n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / (double)k;
        p0 = p1;
        p1 = p2;
      }
      dp = (double)n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / (double)k;
        p0 = p1;
        p1 = p2;
      }
      dp = (double)n * (z * p1 - p0) / (z * z - 1.0);
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* ES kernel parameters (Eqs. (9)-(10)), reading omega = 2 M_sp:
 * beta = 2.3 omega, alpha = pi omega / M_r (support half-width in radians). */
static void es_params(int msp, int64_t Mr, double* beta, double* alpha) {
  double omega = 2.0 * (double)msp;
  *beta = 2.3 * omega;
  *alpha = ORC_PI * omega / (double)Mr;
}

/* Eq. (10) scaled as in Sec. 2.2.5: phihat_ES(k) = alpha * int_{-1}^{1}
 * exp(beta (sqrt(1-y^2) - 1)) e^{i alpha k y} dy, by Gauss-Legendre quadrature
 * in theta with y = cos(theta) (smooth integrand exp(beta(sin th - 1))
 * cos(alpha k cos th) sin th on [0, pi]). nq nodes. */
double orc_es_phihat(int msp, int64_t Mr, double k, int nq) {
  double beta, alpha;
  es_params(msp, Mr, &beta, &alpha);
  double* x = (double*)malloc(sizeof(double) * nq);
  double* w = (double*)malloc(sizeof(double) * nq);
  orc_gauss_legendre(nq, x, w);
  orc_sum s = {0, 0};
  for (int q = 0; q < nq; ++q) {
    double th = 0.5 * ORC_PI * (x[q] + 1.0);
    double f = exp(beta * (sin(th) - 1.0)) * cos(alpha * k * cos(th)) * sin(th);
    sum_add(&s, 0.5 * ORC_PI * w[q] * f);
  }
  free(x);
  free(w);
  return alpha * sum_get(&s);
}

/* Kernel value phi(x) with x the signed distance (grid point - source) in
 * grid cells, for the three averaging kernels on the 2 pi or 1 periodic
 * domain as each algorithm states them. */
static double kb_phi(double xg, int m, double b) {
  /* Eq. (7) with M_r x = xg (distance in cells), m = M_sp */
  double s2 = (double)m * m - xg * xg;
  if (s2 > 0) {
    double s = sqrt(s2);
    return sinh(b * s) / (ORC_PI * s);
  } else if (s2 < 0) {
    double s = sqrt(-s2);
    return sin(b * s) / (ORC_PI * s);
  }
  return b / ORC_PI;
}

/* Plain DFT of the real grid f (Eq. (13)) at modes k = -N..N; exact integer
 * reduction of k*l modulo M_r before the trigonometric call. */
static void grid_dft(int64_t Mr, const double* f, int64_t N, double* G) {
#pragma omp parallel for schedule(static)
  for (int64_t kk = 0; kk <= 2 * N; ++kk) {
    int64_t k = kk - N;
    int64_t km = ((k % Mr) + Mr) % Mr;
    orc_sum re = {0, 0}, im = {0, 0};
    for (int64_t l = 0; l < Mr; ++l) {
      int64_t r = (km * l) % Mr;
      double th = 2.0 * ORC_PI * (double)r / (double)Mr;
      sum_add(&re, f[l] * cos(th));
      sum_add(&im, -f[l] * sin(th));
    }
    G[2 * kk] = sum_get(&re);
    G[2 * kk + 1] = sum_get(&im);
  }
}

/* Paper-faithful CPU type-1 NUFFT for one asset (Algorithms 8, 9, 10), with
 * the readings: the spread index wraps modulo M_r for every stencil offset
 * (Sec. 2.2.5, paragraph after Eq. (15)); the ES algorithm works on the 2 pi
 * domain (b0 = floor(t/h), argument d - k h); sigma = M_r / M when an
 * explicit grid size Mr > 0 is given (else M_r = 2M), with M_sp always from
 * the sigma = 2 rule.
 * tt: rescaled return times in [0, 2 pi]; d: returns. Output: c_k (no 1/2pi)
 * for k = -N..N interleaved. Returns the grid size used. */
int64_t orc_nufft(int kernel, double eps, int64_t n, const double* tt, const double* d,
                  int64_t N, int64_t Mr_in, double* out) {
  int64_t M = 2 * N + 1;
  int64_t Mr = Mr_in > 0 ? Mr_in : 2 * M; /* step I.2 */
  double sigma = (double)Mr / (double)M;
  int msp = orc_msp(kernel, eps);
  double hx = 2.0 * ORC_PI / (double)Mr;
  double* f = (double*)calloc((size_t)Mr, sizeof(double));
  double* G = (double*)malloc(sizeof(double) * 2 * (size_t)M);

  if (kernel == ORC_KERNEL_GAUSS) {
    /* Algorithm 8, steps I.3-I.4 and C */
    double lam = sigma * sigma * (double)msp / (sigma * (sigma - 0.5));
    double t1 = ORC_PI / lam;
    double tau = ORC_PI * lam / ((double)Mr * (double)Mr);
    double* E3 = (double*)malloc(sizeof(double) * (msp + 1));
    double* E0 = (double*)malloc(sizeof(double) * (2 * msp + 1));
    for (int k = 1; k <= msp; ++k) E3[k] = exp(-t1 * (double)k * k);
    for (int64_t h = 0; h < n; ++h) {
      double u = tt[h] / hx;
      double b0 = floor(u);
      double dd = u - b0;
      double E1 = exp(-t1 * dd * dd), E2 = exp(2.0 * t1 * dd);
      E0[msp] = E1;
      double pw = 1.0;
      for (int k = 1; k <= msp; ++k) { pw *= E2; E0[msp + k] = E3[k] * E1 * pw; }
      pw = 1.0;
      for (int k = 1; k <= msp - 1; ++k) { pw /= E2; E0[msp - k] = E3[k] * E1 * pw; }
      int64_t ib = (int64_t)b0;
      for (int k = -msp + 1; k <= msp; ++k) {
        int64_t l = ((ib + k) % Mr + Mr) % Mr;
        f[l] += d[h] * E0[msp + k];
      }
    }
    grid_dft(Mr, f, N, G);
    /* step D.1 */
    for (int64_t kk = 0; kk < M; ++kk) {
      double k = (double)(kk - N);
      double s = sqrt(ORC_PI / tau) * exp(k * k * tau) / (double)Mr;
      out[2 * kk] = s * G[2 * kk];
      out[2 * kk + 1] = s * G[2 * kk + 1];
    }
    free(E3);
    free(E0);
  } else if (kernel == ORC_KERNEL_KB) {
    /* Algorithm 9 on the 1-periodic domain, b = pi (2 - 1/sigma), m = M_sp */
    double b = ORC_PI * (2.0 - 1.0 / sigma);
    for (int64_t h = 0; h < n; ++h) {
      double uu = tt[h] / (2.0 * ORC_PI); /* [0,1] domain */
      double b0 = floor(uu * (double)Mr);
      double dd = uu - b0 / (double)Mr;
      int64_t ib = (int64_t)b0;
      for (int k = -msp; k <= msp; ++k) {
        double x = dd - (double)k / (double)Mr; /* argument of Algorithm 9 */
        int64_t l = ((ib + k) % Mr + Mr) % Mr;
        f[l] += d[h] * kb_phi(x * (double)Mr, msp, b);
      }
    }
    grid_dft(Mr, f, N, G);
    /* step D.1 with Eq. (8) */
    for (int64_t kk = 0; kk < M; ++kk) {
      double k = (double)(kk - N);
      double a = 2.0 * ORC_PI * k / (double)Mr;
      double phihat = orc_bessel_i0((double)msp * sqrt(b * b - a * a)) / (double)Mr;
      double s = 1.0 / ((double)Mr * phihat);
      out[2 * kk] = s * G[2 * kk];
      out[2 * kk + 1] = s * G[2 * kk + 1];
    }
  } else {
    /* Algorithm 10 on the 2 pi domain */
    double beta, alpha;
    es_params(msp, Mr, &beta, &alpha);
    for (int64_t h = 0; h < n; ++h) {
      double b0 = floor(tt[h] / hx);
      double dd = tt[h] - b0 * hx;
      int64_t ib = (int64_t)b0;
      for (int k = -msp; k <= msp; ++k) {
        double x = (dd - (double)k * hx) / alpha;
        double phi = (fabs(x) <= 1.0) ? exp(beta * (sqrt(1.0 - x * x) - 1.0)) : 0.0;
        int64_t l = ((ib + k) % Mr + Mr) % Mr;
        f[l] += d[h] * phi;
      }
    }
    grid_dft(Mr, f, N, G);
    /* steps D.1-D.2 */
    for (int64_t kk = 0; kk < M; ++kk) {
      double k = (double)(kk - N);
      double ph = orc_es_phihat(msp, Mr, k, 200);
      double s = (2.0 * ORC_PI / (double)Mr) / ph;
      out[2 * kk] = s * G[2 * kk];
      out[2 * kk + 1] = s * G[2 * kk + 1];
    }
  }
  free(f);
  free(G);
  return Mr;
}

/* Eq. (15): relative l2 error ||F - F_ref||_2 / ||F_ref||_2 over interleaved
 * complex vectors of length m. */
double orc_rel_l2(int64_t m, const double* F, const double* Fref) {
  orc_sum num = {0, 0}, den = {0, 0};
  for (int64_t q = 0; q < 2 * m; ++q) {
    double e = F[q] - Fref[q];
    sum_add(&num, e * e);
    sum_add(&den, Fref[q] * Fref[q]);
  }
  return sqrt(sum_get(&num)) / sqrt(sum_get(&den));
}

/* Eq. (19): N = floor((T / Delta t - 1) / 2). */
int64_t orc_n_from_dt(double T, double dt) { return (int64_t)floor(0.5 * (T / dt - 1.0)); }

/* Number of threads the parallel loops above use (1 without OpenMP). */
int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
