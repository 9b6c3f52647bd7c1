// sk_series.cuh -- FP64 kernel factors of the regularized Stokes kernels.
//
// The smoothing factors of Sec. 3.4 (s1, s2) and of the regularized
// stresslet (s3) have derivatives of the form  poly(p) e^{-p^2}:
//
//   s1'(p) = (8 /(3 sqrt pi))       (p^4 - 4 p^2 + 2)  e^{-p^2}
//   s2'(p) = (16/(3 sqrt pi)) p^2   (p^4 - 6 p^2 + 6)  e^{-p^2}
//   s3'(p) = (32/(9 sqrt pi)) p^4   (p^4 - 8 p^2 + 12) e^{-p^2}
//
// (differentiate s_i = erf p - p P_i(p) e^{-p^2}/sqrt(pi) and collect terms).
// Expanding e^{-p^2} = sum_k (-1)^k p^{2k}/k! and integrating from 0 term by
// term gives even power series for s1/p, s2/p^3 and s3/p^5:
//
//   s1/p   = (8 /(3 sqrt pi)) sum_n (2 e_n - 4 e_{n-1} +    e_{n-2}) p^{2n} / (2n+1)
//   s2/p^3 = (16/(3 sqrt pi)) sum_n (6 e_n - 6 e_{n-1} +    e_{n-2}) p^{2n} / (2n+3)
//   s3/p^5 = (32/(9 sqrt pi)) sum_n (12 e_n - 8 e_{n-1} +   e_{n-2}) p^{2n} / (2n+5)
//
// with e_k = (-1)^k / k! (zero for k < 0). At p = 0 the first two give the
// limits printed in Sec. 3.4: s1/r -> 16/(3 delta sqrt pi) and
// s2/r^3 -> 32/(3 delta^3 sqrt pi). The coefficients are evaluated at compile
// time; kernels use them in Horner form in x = p^2 (no square root needed).
#pragma once

namespace sk {

constexpr double INV_SQRT_PI = 0.56418958354775628695;  // 1/sqrt(pi)
constexpr double PI_D = 3.14159265358979323846;

__host__ __device__ constexpr double ecoef(int k) {
  if (k < 0) return 0.0;
  double v = 1.0;
  for (int i = 1; i <= k; ++i) v /= (double)i;
  return (k & 1) ? -v : v;
}

template <int N>
struct Poly {
  double c[N];
};

// which = 1: s1/p, 2: s2/p^3, 3: s3/p^5 (prefactor included)
template <int WHICH, int N>
__host__ __device__ constexpr Poly<N> series_coefs() {
  Poly<N> P{};
  for (int n = 0; n < N; ++n) {
    double v = 0.0;
    if (WHICH == 1)
      v = (8.0 / 3.0) * INV_SQRT_PI * (2.0 * ecoef(n) - 4.0 * ecoef(n - 1) + ecoef(n - 2)) /
          (2.0 * n + 1.0);
    else if (WHICH == 2)
      v = (16.0 / 3.0) * INV_SQRT_PI * (6.0 * ecoef(n) - 6.0 * ecoef(n - 1) + ecoef(n - 2)) /
          (2.0 * n + 3.0);
    else
      v = (32.0 / 9.0) * INV_SQRT_PI * (12.0 * ecoef(n) - 8.0 * ecoef(n - 1) + ecoef(n - 2)) /
          (2.0 * n + 5.0);
    P.c[n] = v;
  }
  return P;
}

template <int WHICH, int N>
__device__ __forceinline__ double horner(double x) {
  constexpr Poly<N> P = series_coefs<WHICH, N>();
  double s = P.c[N - 1];
#pragma unroll
  for (int n = N - 2; n >= 0; --n) s = fma(s, x, P.c[n]);
  return s;
}

// Series switch points in x = p^2. Relative truncation error of the three
// series (exact rational arithmetic): 13 terms 1.3e-17 at x = 0.25 (p = 0.5,
// the default rho_T of SK_FP32C); 16 terms 2.8e-20 at x = 0.36; 40 terms for
// x < 4.84 (p < 2.2); beyond that the closed forms are used.
constexpr double SERIES_X_TINY = 0.25;
constexpr double SERIES_X_SHORT = 0.36;
constexpr double SERIES_X_MAX = 4.84;

template <int WHICH>
__device__ __forceinline__ double series_factor(double x) {
  if (x < SERIES_X_TINY) return horner<WHICH, 13>(x);
  return x < SERIES_X_SHORT ? horner<WHICH, 16>(x) : horner<WHICH, 40>(x);
}

// Closed forms, FP64 (Sec. 3.4 for s1, s2; s3 as in the header).
__device__ __forceinline__ void closed_s12(double p, double& s1, double& s2) {
  const double p2 = p * p;
  const double e = exp(-p2) * INV_SQRT_PI;
  const double er = erf(p);
  s1 = er - (2.0 / 3.0) * p * (2.0 * p2 - 5.0) * e;
  s2 = er - (2.0 / 3.0) * p * ((4.0 * p2 - 14.0) * p2 + 3.0) * e;
}

__device__ __forceinline__ double closed_s3(double p) {
  const double p2 = p * p;
  return erf(p) - (2.0 / 9.0) * p * (((8.0 * p2 - 36.0) * p2 + 6.0) * p2 + 9.0) * exp(-p2) *
                      INV_SQRT_PI;
}

// One single-layer pair in FP64: u += ws * [ f s1/r + (f.d) d s2/r^3 ],
// d = x - y, ws = w / (8 pi mu). invd = 1/delta.
__device__ __forceinline__ void sl_pair64(double dx, double dy, double dz, double fx, double fy,
                                          double fz, double ws, double invd, double& u0,
                                          double& u1, double& u2) {
  const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
  const double x = r2 * invd * invd;
  double k1, k2;  // s1/r, s2/r^3
  if (x < SERIES_X_MAX) {
    k1 = series_factor<1>(x) * invd;
    k2 = series_factor<2>(x) * invd * invd * invd;
  } else {
    const double r = sqrt(r2);
    double s1, s2;
    closed_s12(r * invd, s1, s2);
    k1 = s1 / r;
    k2 = s2 / (r2 * r);
  }
  const double fd = fma(fz, dz, fma(fy, dy, fx * dx));
  u0 = fma(ws, fma(fx, k1, fd * dx * k2), u0);
  u1 = fma(ws, fma(fy, k1, fd * dy * k2), u1);
  u2 = fma(ws, fma(fz, k1, fd * dz * k2), u2);
}

// One double-layer pair in FP64: u += ws (d.q)(d.n) d s3/r^5, ws = -6 w / (8 pi).
__device__ __forceinline__ void dl_pair64(double dx, double dy, double dz, double qx, double qy,
                                          double qz, double nx, double ny, double nz, double ws,
                                          double invd, double& u0, double& u1, double& u2) {
  const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
  const double x = r2 * invd * invd;
  double k3;  // s3/r^5
  if (x < SERIES_X_MAX) {
    const double i2 = invd * invd;
    k3 = series_factor<3>(x) * i2 * i2 * invd;
  } else {
    const double r = sqrt(r2);
    k3 = closed_s3(r * invd) / (r2 * r2 * r);
  }
  const double dq = fma(qz, dz, fma(qy, dy, qx * dx));
  const double dn = fma(nz, dz, fma(ny, dy, nx * dx));
  const double c = ws * dq * dn * k3;
  u0 = fma(c, dx, u0);
  u1 = fma(c, dy, u1);
  u2 = fma(c, dz, u2);
}

}  // namespace sk
