/*
 * stokes_oracle.c -- plain, slow, FP64 CPU oracle for the regularized Stokes
 * single- and double-layer sums of arXiv 2310.13908.
 *
 * TEST INFRASTRUCTURE ONLY. The test-suite, the smoke check and the CPU
 * baseline leg of the benchmark use this file; the CUDA library never links,
 * loads or calls it, and shares no code, header or constant with it.
 *
 * What is computed:
 *
 *  Single layer (Sec. 3.4, Eq. regstokes, discretized with the smooth POU
 *  trapezoid rule of Sec. 3.3, Eq. smoothint, whose weights w_y = psi W h^2
 *  are inputs):
 *
 *    u(x) = 1/(8 pi mu) sum_y w_y [ f_y s1(r/delta)/r + (f_y . d) d s2(r/delta)/r^3 ],
 *    d = x - y, r = |d|, delta = delta of the TARGET x (Sec. 3.4, Eq. regparam),
 *
 *    s1(p) = erf p - (2/3) p (2p^2 - 5) e^{-p^2} / sqrt(pi),
 *    s2(p) = erf p - (2/3) p (4p^4 - 14p^2 + 3) e^{-p^2} / sqrt(pi)   (Sec. 3.4).
 *
 *  Double layer (the paper names the regularized double layer of its
 *  reference [beale2019] in Sec. 1, Limitations (ii), but prints no formula):
 *
 *    D(x) = 1/(8 pi) sum_y w_y (-6) (d . q_y)(d . n_y) d s3(r/delta)/r^5,
 *    s3(p) = erf p - (2/9) p (8p^6 - 36p^4 + 6p^2 + 9) e^{-p^2} / sqrt(pi).
 *
 *  Small r: s1(p)/p, s2(p)/p^3 and s3(p)/p^5 are even power series in p.
 *  Their coefficients are built below from the erf and exp series, term by
 *  term; for p < 1 the series is summed instead of the closed form, which
 *  loses digits to cancellation there. At p = 0 the series gives the limits
 *  printed in Sec. 3.4: s1/r -> 16/(3 delta sqrt(pi)), s2/r^3 -> 32/(3 delta^3 sqrt(pi)).
 *
 *  Each target's three components are summed over the sources in input
 *  order with Neumaier's compensated summation. Sources with w_y == 0 add
 *  exactly zero and are skipped. Targets are spread over OpenMP threads;
 *  that does not change any target's arithmetic.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846
#define N_SERIES 30
#define SERIES_SWITCH 1.0

/* c1[n]: s1(p)/p = (2/sqrt(pi)) sum_{n>=0} c1[n] p^{2n}
 * c2[n]: s2(p)/p^3 = (2/sqrt(pi)) sum_{n>=0} c2[n] p^{2n}
 * c3[n]: s3(p)/p^5 = (2/sqrt(pi)) sum_{n>=0} c3[n] p^{2n}            */
static double c1[N_SERIES], c2[N_SERIES], c3[N_SERIES];
static int series_ready = 0;

/* e_k = (-1)^k / k!, the coefficient of p^{2k} in exp(-p^2); zero for k < 0. */
static double exp_coef(int k) {
  if (k < 0) return 0.0;
  double v = 1.0;
  for (int i = 1; i <= k; ++i) v /= (double)i;
  return (k % 2) ? -v : v;
}

/* E_n = (-1)^n / (n! (2n+1)): erf p = (2/sqrt(pi)) sum_n E_n p^{2n+1}. */
static double erf_coef(int n) { return exp_coef(n) / (double)(2 * n + 1); }

static void build_series(void) {
  if (series_ready) return;
  /* Coefficient of p^{2n+1} in s_i / (2/sqrt(pi)): erf part minus the
   * polynomial-times-exp part, whose p^{2n+1} coefficient is a short sum of
   * shifted exp coefficients. */
  double a1[N_SERIES + 3], a2[N_SERIES + 3], a3[N_SERIES + 3];
  for (int n = 0; n < N_SERIES + 3; ++n) {
    /* s1: (1/3) p (2p^2 - 5) e^{-p^2} */
    a1[n] = erf_coef(n) - (2.0 * exp_coef(n - 1) - 5.0 * exp_coef(n)) / 3.0;
    /* s2: (1/3) p (4p^4 - 14p^2 + 3) e^{-p^2} */
    a2[n] = erf_coef(n) - (4.0 * exp_coef(n - 2) - 14.0 * exp_coef(n - 1) + 3.0 * exp_coef(n)) / 3.0;
    /* s3: (1/9) p (8p^6 - 36p^4 + 6p^2 + 9) e^{-p^2} */
    a3[n] = erf_coef(n) - (8.0 * exp_coef(n - 3) - 36.0 * exp_coef(n - 2) + 6.0 * exp_coef(n - 1)
                           + 9.0 * exp_coef(n)) / 9.0;
  }
  /* s1 = sum a1[n] p^{2n+1}            -> s1/p   = sum a1[n]   p^{2n}
   * s2 = sum a2[n] p^{2n+1}, a2[0]=0   -> s2/p^3 = sum a2[n+1] p^{2n}
   * s3 = sum a3[n] p^{2n+1}, a3[0..1]=0-> s3/p^5 = sum a3[n+2] p^{2n} */
  for (int n = 0; n < N_SERIES; ++n) {
    c1[n] = a1[n];
    c2[n] = a2[n + 1];
    c3[n] = a3[n + 2];
  }
  series_ready = 1;
}

static double horner(const double* c, double x) {
  double s = 0.0;
  for (int n = N_SERIES - 1; n >= 0; --n) s = s * x + c[n];
  return s;
}

/* Closed forms of s1, s2, s3 (Sec. 3.4 and the double-layer reading above). */
double oracle_s1(double p) {
  return erf(p) - (2.0 / 3.0) * p * (2.0 * p * p - 5.0) * exp(-p * p) / sqrt(ORACLE_PI);
}
double oracle_s2(double p) {
  double p2 = p * p;
  return erf(p) - (2.0 / 3.0) * p * (4.0 * p2 * p2 - 14.0 * p2 + 3.0) * exp(-p2) / sqrt(ORACLE_PI);
}
double oracle_s3(double p) {
  double p2 = p * p;
  return erf(p) - (2.0 / 9.0) * p * (8.0 * p2 * p2 * p2 - 36.0 * p2 * p2 + 6.0 * p2 + 9.0) * exp(-p2)
                      / sqrt(ORACLE_PI);
}

/* k_i(p): which = 1 -> s1(p)/p, 2 -> s2(p)/p^3, 3 -> s3(p)/p^5.
 * branch: 0 = automatic (series below SERIES_SWITCH), 1 = series, 2 = closed form. */
double oracle_k(int which, int branch, double p) {
  build_series();
  int use_series = (branch == 1) || (branch == 0 && p < SERIES_SWITCH);
  if (use_series) {
    const double* c = (which == 1) ? c1 : (which == 2) ? c2 : c3;
    return 2.0 / sqrt(ORACLE_PI) * horner(c, p * p);
  }
  if (which == 1) return oracle_s1(p) / p;
  if (which == 2) return oracle_s2(p) / (p * p * p);
  return oracle_s3(p) / (p * p * p * p * p);
}

void oracle_k_batch(int which, int branch, int64_t n, const double* p, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = oracle_k(which, branch, p[i]);
}

/* Neumaier compensated summation step. */
static void nsum_add(double* s, double* c, double x) {
  double t = *s + x;
  if (fabs(*s) >= fabs(x)) *c += (*s - t) + x;
  else *c += (x - t) + *s;
  *s = t;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static int check_common(int64_t n_src, int64_t n_tgt, const double* delta, int64_t n_delta) {
  if (n_src < 0 || n_tgt < 0) return -1;
  if (n_tgt > 0 && !(n_delta == 1 || n_delta == n_tgt)) return -1;
  for (int64_t i = 0; i < n_delta; ++i)
    if (!(delta[i] > 0.0)) return -1;
  return 0;
}

/* Regularized single layer at n_tgt targets (row-major xyz triples).
 * Returns 0, or -1 on invalid arguments. */
int oracle_sl(int64_t n_src, const double* src_xyz, const double* w, const double* f,
              int64_t n_tgt, const double* tgt_xyz, const double* delta, int64_t n_delta,
              double mu, double* u_out, int n_threads) {
  if (check_common(n_src, n_tgt, delta, n_delta) != 0 || !(mu > 0.0)) return -1;
  build_series();
  const double pref = 1.0 / (8.0 * ORACLE_PI * mu);
#ifdef _OPENMP
  int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
#endif
  for (int64_t t = 0; t < n_tgt; ++t) {
    const double dl = delta[n_delta == 1 ? 0 : t];
    const double x0 = tgt_xyz[3 * t], x1 = tgt_xyz[3 * t + 1], x2 = tgt_xyz[3 * t + 2];
    double s[3] = {0.0, 0.0, 0.0}, c[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < n_src; ++j) {
      if (w[j] == 0.0) continue;
      const double d0 = x0 - src_xyz[3 * j], d1 = x1 - src_xyz[3 * j + 1], d2 = x2 - src_xyz[3 * j + 2];
      const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      const double p = r / dl;
      const double a = oracle_k(1, 0, p) / dl;              /* s1(r/delta) / r   */
      const double b = oracle_k(2, 0, p) / (dl * dl * dl);  /* s2(r/delta) / r^3 */
      const double f0 = f[3 * j], f1 = f[3 * j + 1], f2 = f[3 * j + 2];
      const double fd = f0 * d0 + f1 * d1 + f2 * d2;
      const double wp = w[j] * pref;
      nsum_add(&s[0], &c[0], wp * (f0 * a + fd * d0 * b));
      nsum_add(&s[1], &c[1], wp * (f1 * a + fd * d1 * b));
      nsum_add(&s[2], &c[2], wp * (f2 * a + fd * d2 * b));
    }
    u_out[3 * t] = s[0] + c[0];
    u_out[3 * t + 1] = s[1] + c[1];
    u_out[3 * t + 2] = s[2] + c[2];
  }
  return 0;
}

/* Regularized double layer at n_tgt targets. Returns 0, or -1 on invalid arguments. */
int oracle_dl(int64_t n_src, const double* src_xyz, const double* w, const double* nrm,
              const double* q, int64_t n_tgt, const double* tgt_xyz, const double* delta,
              int64_t n_delta, double* u_out, int n_threads) {
  if (check_common(n_src, n_tgt, delta, n_delta) != 0) return -1;
  build_series();
  const double pref = 1.0 / (8.0 * ORACLE_PI);
#ifdef _OPENMP
  int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
#endif
  for (int64_t t = 0; t < n_tgt; ++t) {
    const double dl = delta[n_delta == 1 ? 0 : t];
    const double dl5 = dl * dl * dl * dl * dl;
    const double x0 = tgt_xyz[3 * t], x1 = tgt_xyz[3 * t + 1], x2 = tgt_xyz[3 * t + 2];
    double s[3] = {0.0, 0.0, 0.0}, c[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < n_src; ++j) {
      if (w[j] == 0.0) continue;
      const double d0 = x0 - src_xyz[3 * j], d1 = x1 - src_xyz[3 * j + 1], d2 = x2 - src_xyz[3 * j + 2];
      const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      const double p = r / dl;
      const double a = oracle_k(3, 0, p) / dl5;  /* s3(r/delta) / r^5 */
      const double dq = d0 * q[3 * j] + d1 * q[3 * j + 1] + d2 * q[3 * j + 2];
      const double dn = d0 * nrm[3 * j] + d1 * nrm[3 * j + 1] + d2 * nrm[3 * j + 2];
      const double coef = w[j] * pref * (-6.0) * dq * dn * a;
      nsum_add(&s[0], &c[0], coef * d0);
      nsum_add(&s[1], &c[1], coef * d1);
      nsum_add(&s[2], &c[2], coef * d2);
    }
    u_out[3 * t] = s[0] + c[0];
    u_out[3 * t + 1] = s[1] + c[1];
    u_out[3 * t + 2] = s[2] + c[2];
  }
  return 0;
}

/* Plain (unregularized) Stokeslet sum of Sec. 2.2 without the 1/(8 pi mu)
 * factor: v(x) = sum_y [ g_y / r + (g_y . d) d / r^3 ], d = x - y, for
 * targets away from every source (r > 0). The single-level FMM's equivalent
 * sources (Sec. 5) act through this kernel. Neumaier sums in input order.
 * Returns 0, or -1 on invalid arguments. */
int oracle_plain_stokeslet(int64_t n_src, const double* src_xyz, const double* g,
                           int64_t n_tgt, const double* tgt_xyz, double* v_out, int n_threads) {
  if (n_src < 0 || n_tgt < 0) return -1;
#ifdef _OPENMP
  int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
#endif
  for (int64_t t = 0; t < n_tgt; ++t) {
    const double x0 = tgt_xyz[3 * t], x1 = tgt_xyz[3 * t + 1], x2 = tgt_xyz[3 * t + 2];
    double s[3] = {0.0, 0.0, 0.0}, c[3] = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < n_src; ++j) {
      const double d0 = x0 - src_xyz[3 * j], d1 = x1 - src_xyz[3 * j + 1], d2 = x2 - src_xyz[3 * j + 2];
      const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
      const double r = sqrt(r2);
      const double g0 = g[3 * j], g1 = g[3 * j + 1], g2 = g[3 * j + 2];
      const double gd = (g0 * d0 + g1 * d1 + g2 * d2) / (r2 * r);
      nsum_add(&s[0], &c[0], g0 / r + gd * d0);
      nsum_add(&s[1], &c[1], g1 / r + gd * d1);
      nsum_add(&s[2], &c[2], g2 / r + gd * d2);
    }
    v_out[3 * t] = s[0] + c[0];
    v_out[3 * t + 1] = s[1] + c[1];
    v_out[3 * t + 2] = s[2] + c[2];
  }
  return 0;
}
