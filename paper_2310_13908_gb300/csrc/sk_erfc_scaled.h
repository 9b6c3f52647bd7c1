// Generated by fit_erfc_scaled.py (least-squares fit; do not edit by hand).
// E(rho) = exp(rho^2) erfc(rho) for 0.2 <= rho <= 8.5, as t * P(t) with
// t = 1 / (1 + 0.4 rho), P of degree 8; largest absolute error of the fit
// in double precision: 1.2e-08. The pair kernels' smoothing factors use it.
#pragma once

__device__ __forceinline__ float erfc_scaled(float rho) {
  float t;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(fmaf(0.4f, rho, 1.f)));
  return t * fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(fmaf(4.784089457e-02f, t, -1.683306099e-01f),
             t, 1.341372371e-01f), t, 3.880643045e-02f), t, 1.084623046e-01f), t, 1.832297197e-01f),
             t, 2.040023261e-01f), t, 2.262090106e-01f), t, 2.256446329e-01f);
}
