// sk_fmm.cu -- single-level kernel-independent FMM for the regularized single
// layer (Sec. 5), FP64.
//
//   1. k-means (Lloyd) clustering of the sources with nonzero weight, from
//      caller-given initial centres;
//   2. per cluster a cube (centre = midpoint of the points' bounding box,
//      half width a = half the largest extent), equivalent sources on a
//      p-per-edge grid of the surface of the 1.05 a cube and check points on
//      the 2.95 a cube; equivalent densities phi solve, in the Tikhonov
//      sense, K phi = u_check (plain Stokeslet), u_check being the cluster's
//      potential at the check points;
//   3. box against box: each target joins the box of its nearest final
//      centre (a target box is the bounding box of its targets, with their
//      largest delta); the box takes a cluster's equivalent sources when it
//      lies wholly outside the cluster's check cube and at least 7 delta
//      from the cluster cube (the regularized kernel then equals the plain
//      one to double precision), else the direct regularized sum over the
//      cluster's points (neighbouring boxes).
// The Tikhonov operator P1 = (K1^T K1 + alpha^2 I)^{-1} K1^T of the unit cube
// (alpha = 1e-8 |K1|_F) is built once per p on the host by Householder QR of
// [K1; alpha I]; K scales like 1/a, so phi = a P1 u_check for a cube of half
// width a. Every reduction runs in a fixed order, so results are
// deterministic.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "sk_internal.h"
#include "sk_series.cuh"

namespace sk {

struct FmmOp {
  int p = 0, Np = 0;         // points per edge, surface points
  double* unit = nullptr;    // [Np][3] surface grid of [-1, 1]^3
  double* P1 = nullptr;      // [3 Np][3 Np]
};

namespace {

constexpr double R_EQUIV = 1.05, R_CHECK = 2.95, RHO_FAR = 7.0, TIKHONOV = 1e-8;
constexpr int FMM_TPB = 256;

inline unsigned nblk(int64_t n, int t = FMM_TPB) { return (unsigned)((n + t - 1) / t); }

// ---- host: surface grid and the Tikhonov operator ---------------------------
std::vector<double> h_cube_surface(int p) {
  std::vector<double> pts;
  for (int i = 0; i < p; ++i)
    for (int j = 0; j < p; ++j)
      for (int l = 0; l < p; ++l) {
        if (!(i == 0 || i == p - 1 || j == 0 || j == p - 1 || l == 0 || l == p - 1)) continue;
        const double s = 2.0 / (p - 1);
        pts.insert(pts.end(), {-1.0 + s * i, -1.0 + s * j, -1.0 + s * l});
      }
  return pts;
}

// plain Stokeslet block (I/r + d d^T / r^3) for d = x - y
inline void h_stokeslet(const double* x, const double* y, double G[9]) {
  const double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
  const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const double ir = 1.0 / std::sqrt(r2), ir3 = ir / r2;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) G[3 * a + b] = (a == b ? ir : 0.0) + d[a] * d[b] * ir3;
}

// P1 = argmin_phi |K phi - u|^2 + alpha^2 |phi|^2 as an n x n matrix, by
// Householder QR of the 2n x n matrix A = [K; alpha I]: A = Q R, and
// P1 = R^{-1} (Q^T [I; 0])_{first n rows}.
std::vector<double> h_tikhonov_operator(const std::vector<double>& K, int n, double alpha) {
  const int m = 2 * n;
  std::vector<double> A((size_t)m * n, 0.0), B((size_t)m * n, 0.0);  // row-major
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = K[(size_t)i * n + j];
  for (int i = 0; i < n; ++i) {
    A[(size_t)(n + i) * n + i] = alpha;
    B[(size_t)i * n + i] = 1.0;  // [I; 0]
  }
  std::vector<double> v(m);
  for (int c = 0; c < n; ++c) {
    double nrm = 0.0;
    for (int i = c; i < m; ++i) nrm += A[(size_t)i * n + c] * A[(size_t)i * n + c];
    nrm = std::sqrt(nrm);
    const double a0 = A[(size_t)c * n + c];
    const double beta = a0 >= 0.0 ? -nrm : nrm;
    for (int i = c; i < m; ++i) v[i] = A[(size_t)i * n + c];
    v[c] -= beta;
    double vv = 0.0;
    for (int i = c; i < m; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    // apply H = I - 2 v v^T / (v^T v) to A (columns c..n-1) and to B
    for (int j = c; j < n; ++j) {
      double s = 0.0;
      for (int i = c; i < m; ++i) s += v[i] * A[(size_t)i * n + j];
      s *= 2.0 / vv;
      for (int i = c; i < m; ++i) A[(size_t)i * n + j] -= s * v[i];
    }
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int i = c; i < m; ++i) s += v[i] * B[(size_t)i * n + j];
      s *= 2.0 / vv;
      for (int i = c; i < m; ++i) B[(size_t)i * n + j] -= s * v[i];
    }
  }
  // back substitution R P1 = B[0:n, :]
  std::vector<double> P((size_t)n * n);
  for (int j = 0; j < n; ++j)
    for (int i = n - 1; i >= 0; --i) {
      double s = B[(size_t)i * n + j];
      for (int l = i + 1; l < n; ++l) s -= A[(size_t)i * n + l] * P[(size_t)l * n + j];
      P[(size_t)i * n + j] = s / A[(size_t)i * n + i];
    }
  return P;
}

int build_fmm_op(int p, FmmOp** out, std::string& err) {
  FmmOp* op = new (std::nothrow) FmmOp();
  if (!op) return SK_ENOMEM;
  const std::vector<double> unit = h_cube_surface(p);
  const int Np = (int)(unit.size() / 3), n = 3 * Np;
  std::vector<double> K((size_t)n * n);
  double fro = 0.0;
  for (int i = 0; i < Np; ++i)
    for (int j = 0; j < Np; ++j) {
      const double c[3] = {R_CHECK * unit[3 * i], R_CHECK * unit[3 * i + 1], R_CHECK * unit[3 * i + 2]};
      const double e[3] = {R_EQUIV * unit[3 * j], R_EQUIV * unit[3 * j + 1], R_EQUIV * unit[3 * j + 2]};
      double G[9];
      h_stokeslet(c, e, G);
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          K[(size_t)(3 * i + a) * n + 3 * j + b] = G[3 * a + b];
          fro += G[3 * a + b] * G[3 * a + b];
        }
    }
  const std::vector<double> P = h_tikhonov_operator(K, n, TIKHONOV * std::sqrt(fro));
  op->p = p;
  op->Np = Np;
  cudaError_t e = cudaMalloc(&op->unit, unit.size() * sizeof(double));
  if (e == cudaSuccess)
    e = cudaMemcpy(op->unit, unit.data(), unit.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&op->P1, P.size() * sizeof(double));
  if (e == cudaSuccess)
    e = cudaMemcpy(op->P1, P.data(), P.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    err = std::string("fmm operator: ") + cudaGetErrorString(e);
    if (op->unit) cudaFree(op->unit);
    if (op->P1) cudaFree(op->P1);
    delete op;
    return e == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA;
  }
  *out = op;
  return SK_OK;
}

// ---- device ------------------------------------------------------------------
// nearest centre (lowest index on ties); -1 for zero weight
__global__ void k_km_assign(const double* __restrict__ X, const double* __restrict__ w, int64_t N,
                            const double* __restrict__ C, int k, int* __restrict__ lab) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (w && w[i] == 0.0) {
    lab[i] = -1;
    return;
  }
  const double x = X[3 * i], y = X[3 * i + 1], z = X[3 * i + 2];
  double best = INFINITY;
  int bj = 0;
  for (int j = 0; j < k; ++j) {
    // (dx^2 + dy^2) + dz^2, each step rounded (no contraction): the same
    // decisions as any plain evaluation of the definition
    const double dx = x - C[3 * j], dy = y - C[3 * j + 1], dz = z - C[3 * j + 2];
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    if (d2 < best) {
      best = d2;
      bj = j;
    }
  }
  lab[i] = bj;
}

// block per cluster: sums over its points in a fixed order; move = update centre
__global__ void k_km_update(const double* __restrict__ X, const int* __restrict__ lab, int64_t N,
                            double* __restrict__ C, int* __restrict__ count, int move) {
  __shared__ double s[4][FMM_TPB];
  const int c = blockIdx.x, t = threadIdx.x;
  double sx = 0.0, sy = 0.0, sz = 0.0, sn = 0.0;
  for (int64_t i = t; i < N; i += FMM_TPB)
    if (lab[i] == c) {
      sx += X[3 * i];
      sy += X[3 * i + 1];
      sz += X[3 * i + 2];
      sn += 1.0;
    }
  s[0][t] = sx;
  s[1][t] = sy;
  s[2][t] = sz;
  s[3][t] = sn;
  __syncthreads();
  for (int o = FMM_TPB / 2; o > 0; o >>= 1) {
    if (t < o)
      for (int q = 0; q < 4; ++q) s[q][t] += s[q][t + o];
    __syncthreads();
  }
  if (t == 0) {
    const double n = s[3][0];
    if (move && n > 0.0) {
      C[3 * c] = s[0][0] / n;
      C[3 * c + 1] = s[1][0] / n;
      C[3 * c + 2] = s[2][0] / n;
    }
    count[c] = (int)n;
  }
}

__global__ void k_km_offsets(const int* __restrict__ count, int k, int* __restrict__ off) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int s = 0;
  for (int j = 0; j < k; ++j) {
    off[j] = s;
    s += count[j];
  }
  off[k] = s;
}

// block per cluster: indices of its points in ascending order
__global__ void k_km_list(const int* __restrict__ lab, int64_t N, const int* __restrict__ off,
                          int* __restrict__ list) {
  __shared__ int sc[FMM_TPB];
  const int c = blockIdx.x, t = threadIdx.x;
  int base = off[c];
  for (int64_t i0 = 0; i0 < N; i0 += FMM_TPB) {
    const int64_t i = i0 + t;
    const int flag = (i < N && lab[i] == c) ? 1 : 0;
    sc[t] = flag;
    __syncthreads();
    for (int o = 1; o < FMM_TPB; o <<= 1) {  // inclusive scan
      const int v = t >= o ? sc[t - o] : 0;
      __syncthreads();
      sc[t] += v;
      __syncthreads();
    }
    if (flag) list[base + sc[t] - 1] = (int)i;
    const int tot = sc[FMM_TPB - 1];
    __syncthreads();
    base += tot;
  }
}

// block per cluster: cube centre and half width
__global__ void k_km_box(const double* __restrict__ X, const int* __restrict__ off,
                         const int* __restrict__ list, double* __restrict__ box) {
  __shared__ double s[6][FMM_TPB];
  const int c = blockIdx.x, t = threadIdx.x;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int q = off[c] + t; q < off[c + 1]; q += FMM_TPB) {
    const int i = list[q];
    for (int a = 0; a < 3; ++a) {
      lo[a] = fmin(lo[a], X[3 * i + a]);
      hi[a] = fmax(hi[a], X[3 * i + a]);
    }
  }
  for (int a = 0; a < 3; ++a) {
    s[a][t] = lo[a];
    s[3 + a][t] = hi[a];
  }
  __syncthreads();
  for (int o = FMM_TPB / 2; o > 0; o >>= 1) {
    if (t < o)
      for (int a = 0; a < 3; ++a) {
        s[a][t] = fmin(s[a][t], s[a][t + o]);
        s[3 + a][t] = fmax(s[3 + a][t], s[3 + a][t + o]);
      }
    __syncthreads();
  }
  if (t == 0) {
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) {
      box[4 * c + a] = 0.5 * (s[a][0] + s[3 + a][0]);
      ext = fmax(ext, s[3 + a][0] - s[a][0]);
    }
    box[4 * c + 3] = fmax(0.5 * ext, 1e-12);
  }
}

// block per target box: bounding box of its targets and their largest delta
__global__ void k_tgt_box(const double* __restrict__ Y, const double* __restrict__ delta,
                          int64_t n_delta, const int* __restrict__ off,
                          const int* __restrict__ list, double* __restrict__ tbox) {
  __shared__ double s[7][FMM_TPB];
  const int c = blockIdx.x, t = threadIdx.x;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  double dmax = 0.0;
  for (int q = off[c] + t; q < off[c + 1]; q += FMM_TPB) {
    const int i = list[q];
    for (int a = 0; a < 3; ++a) {
      lo[a] = fmin(lo[a], Y[3 * i + a]);
      hi[a] = fmax(hi[a], Y[3 * i + a]);
    }
    dmax = fmax(dmax, delta[n_delta == 1 ? 0 : i]);
  }
  for (int a = 0; a < 3; ++a) {
    s[a][t] = lo[a];
    s[3 + a][t] = hi[a];
  }
  s[6][t] = dmax;
  __syncthreads();
  for (int o = FMM_TPB / 2; o > 0; o >>= 1) {
    if (t < o) {
      for (int a = 0; a < 3; ++a) {
        s[a][t] = fmin(s[a][t], s[a][t + o]);
        s[3 + a][t] = fmax(s[3 + a][t], s[3 + a][t + o]);
      }
      s[6][t] = fmax(s[6][t], s[6][t + o]);
    }
    __syncthreads();
  }
  if (t < 7) tbox[8 * c + t] = s[t][0];
}

// One thread per (target box i, source cluster j): near[i k + j] = 1 when
// the cluster is a neighbour of the box (direct sum), 0 when the box lies
// wholly outside the cluster's check cube and at least RHO_FAR delta_i from
// its cube. Plain IEEE operations (no contraction), as the definition reads.
__global__ void k_fmm_neighbours(const double* __restrict__ tbox, const int* __restrict__ toff,
                                 const double* __restrict__ box, const int* __restrict__ off,
                                 int k, unsigned char* __restrict__ near) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= (int64_t)k * k) return;
  const int i = (int)(q / k), j = (int)(q % k);
  if (toff[i + 1] == toff[i] || off[j + 1] == off[j]) {
    near[q] = 0;  // an empty box or cluster contributes nothing either way
    return;
  }
  const double* tb = tbox + 8 * i;
  const double a = box[4 * j + 3], ca = __dmul_rn(R_CHECK, a);
  bool outside = false;
  double g2 = 0.0;
  for (int ax = 0; ax < 3; ++ax) {
    const double c = box[4 * j + ax], lo = tb[ax], hi = tb[3 + ax];
    outside |= (lo > __dadd_rn(c, ca)) || (hi < __dsub_rn(c, ca));
    const double g = fmax(fmax(__dsub_rn(lo, __dadd_rn(c, a)), __dsub_rn(__dsub_rn(c, a), hi)), 0.0);
    g2 = ax == 0 ? __dmul_rn(g, g) : __dadd_rn(g2, __dmul_rn(g, g));
  }
  const double rf = __dmul_rn(RHO_FAR, tb[6]);
  near[q] = (outside && g2 >= __dmul_rn(rf, rf)) ? 0 : 1;
}

// block per cluster: potential of its points (plain Stokeslet, w f) at the
// check points, then phi = a P1 u_check
__global__ void k_fmm_upward(const double* __restrict__ X, const double* __restrict__ w,
                             const double* __restrict__ f, const int* __restrict__ off,
                             const int* __restrict__ list, const double* __restrict__ box,
                             const double* __restrict__ unit, int Np,
                             const double* __restrict__ P1, double* __restrict__ ucheck,
                             double* __restrict__ phi) {
  const int c = blockIdx.x, t = threadIdx.x;
  const int n = 3 * Np;
  const double cx = box[4 * c], cy = box[4 * c + 1], cz = box[4 * c + 2], a = box[4 * c + 3];
  double* uc = ucheck + (int64_t)c * n;
  for (int j = t; j < Np; j += blockDim.x) {
    const double px = cx + R_CHECK * a * unit[3 * j], py = cy + R_CHECK * a * unit[3 * j + 1],
                 pz = cz + R_CHECK * a * unit[3 * j + 2];
    double u0 = 0.0, u1 = 0.0, u2 = 0.0;
    for (int q = off[c]; q < off[c + 1]; ++q) {
      const int i = list[q];
      const double dx = px - X[3 * i], dy = py - X[3 * i + 1], dz = pz - X[3 * i + 2];
      const double r2 = dx * dx + dy * dy + dz * dz;
      const double ir = rsqrt(r2), ir3 = ir * ir * ir;
      const double gx = w[i] * f[3 * i], gy = w[i] * f[3 * i + 1], gz = w[i] * f[3 * i + 2];
      const double gd = (gx * dx + gy * dy + gz * dz) * ir3;
      u0 += gx * ir + gd * dx;
      u1 += gy * ir + gd * dy;
      u2 += gz * ir + gd * dz;
    }
    uc[3 * j] = u0;
    uc[3 * j + 1] = u1;
    uc[3 * j + 2] = u2;
  }
  __syncthreads();
  for (int r = t; r < n; r += blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += P1[(int64_t)r * n + j] * uc[j];
    phi[(int64_t)c * n + r] = a * s;
  }
}

// One thread per target, targets in box order (tlist), so a warp's targets
// share their box's decisions: a far cluster through its equivalent
// sources, a neighbouring one by the direct regularized sum over its points
// (beyond 7 delta the regularized pair is the plain Stokeslet).
__global__ void k_fmm_eval(const double* __restrict__ Y, const double* __restrict__ delta,
                           int64_t n_delta, int64_t M, int k, const double* __restrict__ box,
                           const int* __restrict__ off, const int* __restrict__ list,
                           const int* __restrict__ tlab, const int* __restrict__ tlist,
                           const unsigned char* __restrict__ near,
                           const double* __restrict__ unit, int Np, const double* __restrict__ phi,
                           const double* __restrict__ X, const double* __restrict__ w,
                           const double* __restrict__ f, double scale, double* __restrict__ u) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= M) return;
  const int t = tlist[q];
  const int bi = tlab[t];
  const double x = Y[3 * t], y = Y[3 * t + 1], z = Y[3 * t + 2];
  const double d = delta[n_delta == 1 ? 0 : t], invd = 1.0 / d;
  const double rf = RHO_FAR * d, rf2 = rf * rf;
  double fx0 = 0.0, fx1 = 0.0, fx2 = 0.0;  // far, without 1/(8 pi mu)
  double n0 = 0.0, n1 = 0.0, n2 = 0.0;     // near
  for (int c = 0; c < k; ++c) {
    if (off[c + 1] == off[c]) continue;
    const double cx = box[4 * c], cy = box[4 * c + 1], cz = box[4 * c + 2], a = box[4 * c + 3];
    if (!near[(int64_t)bi * k + c]) {
      const double* ph = phi + (int64_t)c * 3 * Np;
      for (int j = 0; j < Np; ++j) {
        const double dx = x - (cx + R_EQUIV * a * unit[3 * j]);
        const double dy = y - (cy + R_EQUIV * a * unit[3 * j + 1]);
        const double dz = z - (cz + R_EQUIV * a * unit[3 * j + 2]);
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double ir = rsqrt(r2), ir3 = ir * ir * ir;
        const double px = ph[3 * j], py = ph[3 * j + 1], pz = ph[3 * j + 2];
        const double pd = (px * dx + py * dy + pz * dz) * ir3;
        fx0 += px * ir + pd * dx;
        fx1 += py * ir + pd * dy;
        fx2 += pz * ir + pd * dz;
      }
    } else {
      for (int qq = off[c]; qq < off[c + 1]; ++qq) {
        const int i = list[qq];
        const double dx = x - X[3 * i], dy = y - X[3 * i + 1], dz = z - X[3 * i + 2];
        const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
        if (r2 >= rf2) {  // s1 = s2 = 1 to double precision
          const double ir = rsqrt(r2), ir3 = ir * ir * ir;
          const double ws = w[i] * scale;
          const double fx = f[3 * i], fy = f[3 * i + 1], fz = f[3 * i + 2];
          const double fd = (fx * dx + fy * dy + fz * dz) * ir3;
          n0 = fma(ws, fx * ir + fd * dx, n0);
          n1 = fma(ws, fy * ir + fd * dy, n1);
          n2 = fma(ws, fz * ir + fd * dz, n2);
        } else {
          sl_pair64(dx, dy, dz, f[3 * i], f[3 * i + 1], f[3 * i + 2], w[i] * scale, invd, n0, n1,
                    n2);
        }
      }
    }
  }
  u[3 * t] = scale * fx0 + n0;
  u[3 * t + 1] = scale * fx1 + n1;
  u[3 * t + 2] = scale * fx2 + n2;
}

}  // namespace

int fmm_op(sk_ctx* ctx, int p, FmmOp** out) {
  for (auto& kv : ctx->fmm_ops)
    if (kv.first == p) {
      *out = kv.second;
      return SK_OK;
    }
  FmmOp* op = nullptr;
  const int rc = build_fmm_op(p, &op, ctx->err);
  if (rc != SK_OK) return rc;
  ctx->fmm_ops.push_back({p, op});
  *out = op;
  return SK_OK;
}

void free_fmm_ops(sk_ctx* ctx) {
  for (auto& kv : ctx->fmm_ops) {
    cudaFree(kv.second->unit);
    cudaFree(kv.second->P1);
    delete kv.second;
  }
  ctx->fmm_ops.clear();
}

}  // namespace sk

using namespace sk;

extern "C" {

int stokes_sl_eval_fmm(sk_ctx* ctx, int mem, int64_t n_src, const double* src_xyz,
                       const double* src_w, const double* f, int64_t n_tgt, const double* tgt_xyz,
                       const double* delta, int64_t n_delta, double mu, int k,
                       const double* centers0, int lloyd_iters, int p, double* u_out,
                       void* stream) {
  if (!ctx) return SK_EINVAL;
  if (n_src < 1 || n_tgt < 1 || n_src > (1LL << 30) || n_tgt > (1LL << 30) || !src_xyz ||
      !src_w || !f || !tgt_xyz || !delta || !u_out || !centers0 || k < 1 || k > 65536 ||
      lloyd_iters < 0 || p < 3 || p > 10 || !(n_delta == 1 || n_delta == n_tgt) ||
      !(mu > 0.0 && mu < INFINITY) || (mem != SK_HOST && mem != SK_DEVICE)) {
    ctx->err = "stokes_sl_eval_fmm: invalid argument (sizes, pointers, 1 <= k <= 65536, "
               "3 <= p <= 10, n_delta in {1, n_tgt}, mu > 0, mem)";
    return SK_EINVAL;
  }
  if (mem == SK_HOST)
    for (int64_t i = 0; i < n_delta; ++i)
      if (!(delta[i] > 0.0 && delta[i] < INFINITY)) {
        ctx->err = "stokes_sl_eval_fmm: delta must be positive and finite";
        return SK_EINVAL;
      }
  FmmOp* op = nullptr;
  int rc = fmm_op(ctx, p, &op);
  if (rc != SK_OK) return rc;
  cudaSetDevice(ctx->device);
  cudaStream_t st = (mem == SK_DEVICE && stream) ? (cudaStream_t)stream : ctx->stream;
  const int n3 = 3 * op->Np;
  // workspace: inputs and output (host calls), labels, counts, offsets,
  // point lists, centres, boxes, check potentials, densities
  struct Carve {
    double *tX = nullptr, *tW = nullptr, *tF = nullptr, *tY = nullptr, *tD = nullptr, *U = nullptr;
    int *lab = nullptr, *count = nullptr, *offs = nullptr, *list = nullptr;
    int *tlab = nullptr, *tcount = nullptr, *toffs = nullptr, *tlist = nullptr;
    double *C = nullptr, *box = nullptr, *tbox = nullptr, *ucheck = nullptr, *phi = nullptr;
    unsigned char* near = nullptr;
  };
  auto carve = [&](Bump& b, Carve& c) {
    if (mem == SK_HOST) {
      c.tX = b.take<double>(3 * n_src);
      c.tW = b.take<double>(n_src);
      c.tF = b.take<double>(3 * n_src);
      c.tY = b.take<double>(3 * n_tgt);
      c.tD = b.take<double>(n_delta);
      c.U = b.take<double>(3 * n_tgt);
    }
    c.lab = b.take<int>(n_src);
    c.count = b.take<int>(k);
    c.offs = b.take<int>(k + 1);
    c.list = b.take<int>(n_src);
    c.tlab = b.take<int>(n_tgt);
    c.tcount = b.take<int>(k);
    c.toffs = b.take<int>(k + 1);
    c.tlist = b.take<int>(n_tgt);
    c.C = b.take<double>(3 * (size_t)k);
    c.box = b.take<double>(4 * (size_t)k);
    c.tbox = b.take<double>(8 * (size_t)k);
    c.near = b.take<unsigned char>((size_t)k * k);
    c.ucheck = b.take<double>((size_t)k * n3);
    c.phi = b.take<double>((size_t)k * n3);
  };
  Carve cv;
  Bump measure;
  carve(measure, cv);
  rc = ensure_workspace(ctx, measure.off + 256);
  if (rc != SK_OK) return rc;
  Bump b;
  b.base = ctx->ws;
  carve(b, cv);
  const double *X = src_xyz, *W = src_w, *F = f, *Y = tgt_xyz, *D = delta;
  double* U = u_out;
  if (mem == SK_HOST) {
    cudaMemcpyAsync(cv.tX, src_xyz, 3 * n_src * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(cv.tW, src_w, n_src * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(cv.tF, f, 3 * n_src * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(cv.tY, tgt_xyz, 3 * n_tgt * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(cv.tD, delta, n_delta * sizeof(double), cudaMemcpyHostToDevice, st);
    X = cv.tX;
    W = cv.tW;
    F = cv.tF;
    Y = cv.tY;
    D = cv.tD;
    U = cv.U;
  }
  int* lab = cv.lab;
  int* count = cv.count;
  int* offs = cv.offs;
  int* list = cv.list;
  double* C = cv.C;
  double* box = cv.box;
  double* ucheck = cv.ucheck;
  double* phi = cv.phi;
  cudaMemcpyAsync(C, centers0, 3 * (size_t)k * sizeof(double),
                  mem == SK_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st);
  for (int it = 0; it < lloyd_iters; ++it) {
    k_km_assign<<<nblk(n_src), FMM_TPB, 0, st>>>(X, W, n_src, C, k, lab);
    k_km_update<<<k, FMM_TPB, 0, st>>>(X, lab, n_src, C, count, 1);
  }
  k_km_assign<<<nblk(n_src), FMM_TPB, 0, st>>>(X, W, n_src, C, k, lab);
  k_km_update<<<k, FMM_TPB, 0, st>>>(X, lab, n_src, C, count, 0);
  k_km_offsets<<<1, 32, 0, st>>>(count, k, offs);
  k_km_list<<<k, FMM_TPB, 0, st>>>(lab, n_src, offs, list);
  k_km_box<<<k, FMM_TPB, 0, st>>>(X, offs, list, box);
  k_fmm_upward<<<k, FMM_TPB, 0, st>>>(X, W, F, offs, list, box, op->unit, op->Np, op->P1, ucheck,
                                      phi);
  // target boxes: nearest final centre, ordered lists, boxes, neighbour matrix
  k_km_assign<<<nblk(n_tgt), FMM_TPB, 0, st>>>(Y, nullptr, n_tgt, C, k, cv.tlab);
  k_km_update<<<k, FMM_TPB, 0, st>>>(Y, cv.tlab, n_tgt, C, cv.tcount, 0);
  k_km_offsets<<<1, 32, 0, st>>>(cv.tcount, k, cv.toffs);
  k_km_list<<<k, FMM_TPB, 0, st>>>(cv.tlab, n_tgt, cv.toffs, cv.tlist);
  k_tgt_box<<<k, FMM_TPB, 0, st>>>(Y, D, n_delta, cv.toffs, cv.tlist, cv.tbox);
  k_fmm_neighbours<<<nblk((int64_t)k * k), FMM_TPB, 0, st>>>(cv.tbox, cv.toffs, box, offs, k,
                                                              cv.near);
  const double scale = 1.0 / (8.0 * PI_CONST * mu);
  k_fmm_eval<<<nblk(n_tgt, 128), 128, 0, st>>>(Y, D, n_delta, n_tgt, k, box, offs, list, cv.tlab,
                                               cv.tlist, cv.near, op->unit, op->Np, phi, X, W, F,
                                               scale, U);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && mem == SK_HOST)
    e = cudaMemcpyAsync(u_out, U, 3 * n_tgt * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && (mem == SK_HOST || !stream)) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    ctx->err = std::string("stokes_sl_eval_fmm: ") + cudaGetErrorString(e);
    return SK_ECUDA;
  }
  return SK_OK;
}

}  // extern "C"
