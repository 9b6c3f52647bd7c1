// sk_fmm.cu -- single-level kernel-independent FMM for the regularized single
// layer (Sec. 5), in FP64 or FP32C.
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
// k-means: the nearest centre is decided in FP64 (FP32 distances only select
// the candidates); a centre moves to the mean of its points, summed exactly
// in fixed point so that the order of the additions does not matter. A
// stable radix sort by label lists each cluster's points.
// The Tikhonov operator P1 = (K1^T K1 + alpha^2 I)^{-1} K1^T of the unit cube
// (alpha = 1e-8 |K1|_F) is built once per p on the host by Householder QR of
// [K1; alpha I]; K scales like 1/a, so phi = a P1 u_check for a cube of half
// width a. Every reduction runs in a fixed order, so results are
// deterministic.
//
// FP64: one thread per target sums its box's neighbouring clusters directly
// and the far clusters' equivalent sources. FP32C: the pair kernel of the
// direct sum processes, per target block, one list of source tiles: the
// neighbouring clusters' points (same regimes and FP64 near lists as
// stokes_sl_eval) and the far clusters' equivalent sources (far loop).
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "sk_decomp.h"
#include "sk_internal.h"
#include "sk_pair32.cuh"
#include "sk_series.cuh"

namespace sk {

struct FmmOp {
  int p = 0, Np = 0;         // points per edge, surface points
  double* unit = nullptr;    // [Np][3] surface grid of [-1, 1]^3
  double* P1 = nullptr;      // [3 Np][3 Np]
  double* P1T = nullptr;     // its transpose (coalesced rows for the FP32C path's product)
};

namespace {

constexpr double R_EQUIV = 1.05, R_CHECK = 2.95, RHO_FAR = 7.0, TIKHONOV = 1e-8;
constexpr int FMM_TPB = 256;
constexpr int FMM_MAX_N3 = 3 * (6 * 10 * 10 - 12 * 10 + 8);  // p <= 10

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
  std::vector<double> PT(P.size());
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) PT[(size_t)c * n + r] = P[(size_t)r * n + c];
  if (e == cudaSuccess) e = cudaMalloc(&op->P1T, PT.size() * sizeof(double));
  if (e == cudaSuccess)
    e = cudaMemcpy(op->P1T, PT.data(), PT.size() * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    err = std::string("fmm operator: ") + cudaGetErrorString(e);
    if (op->unit) cudaFree(op->unit);
    if (op->P1) cudaFree(op->P1);
    if (op->P1T) cudaFree(op->P1T);
    delete op;
    return e == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA;
  }
  *out = op;
  return SK_OK;
}

// ---- device ------------------------------------------------------------------
// ---- clustering (both precisions) ------------------------------------------
constexpr int KM_SMEM_CENTRES = 1024;  // centres staged per pass of the assignment
constexpr int KM_SMEM_SUMS = 512;      // clusters whose sums a block gathers in shared memory

// Nearest centre of point i (lowest index on ties), decided in FP64 by the
// plain squared distance (dx^2 + dy^2) + dz^2. FP32 distances to every
// centre select the candidates: their error is below 1e-6 (d^2 + S^2), S the
// largest coordinate magnitude of point and centres, so every centre within
// 2^-16 (m + S^2) of the FP32 minimum m is a candidate and the FP64 minimum is
// always among them. A point with a single candidate takes it (the FP64
// minimum then is that centre); the FP64 distances decide between several,
// in a pass that only blocks holding such points run. -1 for a zero-weight
// point. C32: FP32 centres (x, y, z, largest |coordinate|).
__global__ void __launch_bounds__(FMM_TPB) k_km_assign32(const double* __restrict__ X,
                                                         const double* __restrict__ w, int64_t N,
                                                         const double* __restrict__ C,
                                                         const float4* __restrict__ C32, int k,
                                                         int* __restrict__ lab) {
  __shared__ float4 sc[KM_SMEM_CENTRES];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool live = i < N && !(w && w[i] == 0.0);
  const int64_t ii = i < N ? i : N - 1;
  const double x = X[3 * ii], y = X[3 * ii + 1], z = X[3 * ii + 2];
  const float xf = (float)x, yf = (float)y, zf = (float)z;
  float m1 = INFINITY, m2 = INFINITY, cmax = 0.f;  // smallest, second smallest
  int j1 = 0;
  for (int j0 = 0; j0 < k; j0 += KM_SMEM_CENTRES) {
    const int nj = min(KM_SMEM_CENTRES, k - j0);
    __syncthreads();
    for (int j = threadIdx.x; j < nj; j += blockDim.x) sc[j] = C32[j0 + j];
    __syncthreads();
    for (int j = 0; j < nj; ++j) {
      const float4 c = sc[j];
      const float dx = xf - c.x, dy = yf - c.y, dz = zf - c.z;
      const float d = dx * dx + dy * dy + dz * dz;
      if (d < m1) {
        m2 = m1;
        m1 = d;
        j1 = j0 + j;
      } else {
        m2 = fminf(m2, d);
      }
      cmax = fmaxf(cmax, c.w);
    }
  }
  const float S = fmaxf(fabsf(xf), fmaxf(fabsf(yf), fabsf(zf))) + cmax;
  const float lim = m1 + 1.52587890625e-05f * (m1 + S * S);  // 2^-16
  const bool several = m2 <= lim;
  int bj = j1;
  if (__syncthreads_or(several)) {
    double best = INFINITY;
    for (int j0 = 0; j0 < k; j0 += KM_SMEM_CENTRES) {
      const int nj = min(KM_SMEM_CENTRES, k - j0);
      if (k > KM_SMEM_CENTRES) {  // restage (the staged centres are the last chunk otherwise)
        __syncthreads();
        for (int j = threadIdx.x; j < nj; j += blockDim.x) sc[j] = C32[j0 + j];
        __syncthreads();
      }
      if (!several) continue;
      for (int j = 0; j < nj; ++j) {
        const float4 c = sc[j];
        const float fx = xf - c.x, fy = yf - c.y, fz = zf - c.z;
        if (fx * fx + fy * fy + fz * fz > lim) continue;
        const int jj = j0 + j;
        const double dx = x - C[3 * jj], dy = y - C[3 * jj + 1], dz = z - C[3 * jj + 2];
        const double d2 =
            __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        if (d2 < best) {
          best = d2;
          bj = jj;
        }
      }
    }
  }
  if (i < N) lab[i] = live ? bj : -1;
}

// FP32 copies of the centres, with their largest |coordinate| in .w.
__global__ void k_km_centres32(const double* __restrict__ C, int k, float4* __restrict__ C32) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  const float x = (float)C[3 * j], y = (float)C[3 * j + 1], z = (float)C[3 * j + 2];
  C32[j] = make_float4(x, y, z, fmaxf(fabsf(x), fmaxf(fabsf(y), fabsf(z))));
}

// FP64 bounding box of the active points: per-block partial boxes, then one
// block combines them into frame = (lo[3], quantum q), q = (largest extent) *
// 2^-34, the unit of the fixed-point sums below.
__global__ void k_km_frame_part(const double* __restrict__ X, const double* __restrict__ w,
                                int64_t N, double* __restrict__ part) {
  __shared__ double s[6][FMM_TPB];
  const int t = threadIdx.x;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = blockIdx.x * (int64_t)FMM_TPB + t; i < N; i += (int64_t)gridDim.x * FMM_TPB) {
    if (w && w[i] == 0.0) continue;
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
  if (t < 6) part[6 * blockIdx.x + t] = s[t][0];
}

__global__ void k_km_frame(const double* __restrict__ part, int nblk, double* __restrict__ frame) {
  // one warp: lane-strided minima and maxima, then a butterfly (exact in any order)
  const int lane = threadIdx.x & 31;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int b = lane; b < nblk; b += 32)
    for (int a = 0; a < 3; ++a) {
      lo[a] = fmin(lo[a], part[6 * b + a]);
      hi[a] = fmax(hi[a], part[6 * b + 3 + a]);
    }
  for (int o = 16; o > 0; o >>= 1)
    for (int a = 0; a < 3; ++a) {
      lo[a] = fmin(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
      hi[a] = fmax(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
    }
  if (threadIdx.x != 0) return;
  double ext = 0.0;
  for (int a = 0; a < 3; ++a) {
    frame[a] = lo[a] <= hi[a] ? lo[a] : 0.0;
    ext = fmax(ext, hi[a] - lo[a]);
  }
  frame[3] = (ext > 0.0 ? ext : 1.0) * 5.820766091346741e-11;  // 2^-34
  frame[4] = 1.0 / frame[3];
}

// Exact sums of each cluster's points: every coordinate rounded to a
// multiple of the quantum q above the box corner (at most 2^34 quanta) and
// added in 64-bit integers, which makes the sums independent of the order of
// the additions; point counts likewise. A warp first adds up the quanta of
// its lanes that share a cluster (consecutive points mostly do), so one lane
// per cluster and warp adds them on; for k <= KM_SMEM_SUMS a block gathers
// those in shared memory first.
__global__ void __launch_bounds__(FMM_TPB) k_km_sums(const double* __restrict__ X,
                                                     const int* __restrict__ lab, int64_t N,
                                                     const double* __restrict__ frame, int k,
                                                     unsigned long long* __restrict__ sums,
                                                     unsigned int* __restrict__ cnt) {
  __shared__ unsigned long long ss[KM_SMEM_SUMS][3];
  __shared__ unsigned int sn[KM_SMEM_SUMS];
  const bool local = k <= KM_SMEM_SUMS;
  if (local) {
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
      ss[j][0] = ss[j][1] = ss[j][2] = 0ull;
      sn[j] = 0u;
    }
    __syncthreads();
  }
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int l = i < N ? lab[i] : -1;
  unsigned long long q[3] = {0ull, 0ull, 0ull};
  if (l >= 0) {
    const double inv = frame[4];
    for (int a = 0; a < 3; ++a)
      q[a] = (unsigned long long)llrint(fmax(X[3 * i + a] - frame[a], 0.0) * inv);
  }
  // lanes of the same cluster (points without one form their own group)
  const unsigned grp = __match_any_sync(0xffffffffu, l);
  unsigned long long s[3] = {0ull, 0ull, 0ull};
  for (int r = 0; r < 32; ++r) {
    const unsigned long long a0 = __shfl_sync(0xffffffffu, q[0], r);
    const unsigned long long a1 = __shfl_sync(0xffffffffu, q[1], r);
    const unsigned long long a2 = __shfl_sync(0xffffffffu, q[2], r);
    if ((grp >> r) & 1u) {
      s[0] += a0;
      s[1] += a1;
      s[2] += a2;
    }
  }
  if (l >= 0 && lane == __ffs(grp) - 1) {
    const unsigned n = (unsigned)__popc(grp);
    if (local) {
      for (int a = 0; a < 3; ++a) atomicAdd(&ss[l][a], s[a]);
      atomicAdd(&sn[l], n);
    } else {
      for (int a = 0; a < 3; ++a) atomicAdd(&sums[3 * l + a], s[a]);
      atomicAdd(&cnt[l], n);
    }
  }
  if (local) {
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x)
      if (sn[j]) {
        for (int a = 0; a < 3; ++a) atomicAdd(&sums[3 * j + a], ss[j][a]);
        atomicAdd(&cnt[j], sn[j]);
      }
  }
}

// Thread per cluster: the centre moves to the mean of its points (an empty
// cluster keeps its centre); the FP32 copy is refreshed.
__global__ void k_km_centres(const unsigned long long* __restrict__ sums,
                             const unsigned int* __restrict__ cnt,
                             const double* __restrict__ frame, int k, double* __restrict__ C,
                             float4* __restrict__ C32) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  if (cnt[j] != 0u)
    for (int a = 0; a < 3; ++a)
      C[3 * j + a] = frame[a] + ((double)sums[3 * j + a] / (double)cnt[j]) * frame[3];
  const float x = (float)C[3 * j], y = (float)C[3 * j + 1], z = (float)C[3 * j + 2];
  C32[j] = make_float4(x, y, z, fmaxf(fabsf(x), fmaxf(fabsf(y), fabsf(z))));
}

// Sort keys of the labelled points in a given order (identity if null):
// key = label, or k for a zero-weight point, so a stable sort by key lists
// each cluster's points in that order.
__global__ void k_km_keys(const int* __restrict__ lab, const int* __restrict__ order, int64_t n,
                          int k, uint32_t* __restrict__ keys, int* __restrict__ vals) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int j = order ? order[i] : (int)i;
  const int l = lab[j];
  keys[i] = l < 0 ? (uint32_t)k : (uint32_t)l;
  vals[i] = j;
}

// Thread per cluster c: offs[c] = first position of key c in the sorted keys
// (offs[k] = points with a label), count[c] = offs[c + 1] - offs[c].
__global__ void k_km_offsets_sorted(const uint32_t* __restrict__ keys, int64_t n, int k,
                                    int* __restrict__ offs, int* __restrict__ count) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c > k) return;
  auto lower = [&](uint32_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
      const int64_t mid = (lo + hi) / 2;
      if (keys[mid] < v) lo = mid + 1; else hi = mid;
    }
    return (int)lo;
  };
  const int a = lower((uint32_t)c);
  offs[c] = a;
  if (c < k) count[c] = lower((uint32_t)c + 1) - a;
}

// block per cluster: cube centre and half width
__global__ void k_km_box(const double* __restrict__ X, const int* __restrict__ off,
                         const int* __restrict__ list, double* __restrict__ box) {
  __shared__ double s[6][FMM_TPB];
  const int c = blockIdx.x, t = threadIdx.x;
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int q = off[c] + t; q < off[c + 1]; q += FMM_TPB) {
    const int64_t i = list[q];
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
    const int64_t i = list[q];
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
      const int64_t i = list[q];
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
  const int64_t t = tlist[q];
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
        const int64_t i = list[qq];
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

// ---- FP32C path ---------------------------------------------------------------
// The neighbouring clusters' points go through the FP32-compensated pair
// kernel of the direct sum (same regimes, same FP64 near lists), and the far
// clusters' equivalent sources through its far loop: one list of source
// tiles per target block, split into work items. The check potentials are
// FP32 sums (their rounding moves the far field by ~1e-9 of |u|); the
// equivalent densities stay FP64, because the Tikhonov operator's large
// entries cancel.

constexpr int FMM_ITEM_TILES = 8;  // source tiles per work item of the pair kernel

constexpr int FMM_CHECK_SPLIT = 8;  // blocks per cluster for the check potentials

// Block (cluster c, part sp of FMM_CHECK_SPLIT): the plain-Stokeslet
// potential, at c's check points, of the sp-th contiguous share of c's
// points (g = w f), in FP32 relative to the cluster centre with compensated
// sums; stored FP64 per part, summed in part order by k_fmm_phi.
__global__ void __launch_bounds__(FMM_TPB) k_fmm_check32(
    const double* __restrict__ X, const double* __restrict__ w, const double* __restrict__ f,
    const int* __restrict__ off, const int* __restrict__ list, const double* __restrict__ box,
    const double* __restrict__ unit, int Np, double* __restrict__ ucheck_part) {
  __shared__ float4 sp[FMM_TPB], sg[FMM_TPB];
  const int c = blockIdx.x, part = blockIdx.y, t = threadIdx.x;
  const double cx = box[4 * c], cy = box[4 * c + 1], cz = box[4 * c + 2], a = box[4 * c + 3];
  const int n = off[c + 1] - off[c];
  const int p0 = off[c] + (int)((int64_t)part * n / FMM_CHECK_SPLIT);
  const int p1 = off[c] + (int)((int64_t)(part + 1) * n / FMM_CHECK_SPLIT);
  for (int q0 = 0; q0 < Np; q0 += FMM_TPB) {
    const int q = min(q0 + t, Np - 1);
    const float px = (float)(R_CHECK * a * unit[3 * q]), py = (float)(R_CHECK * a * unit[3 * q + 1]),
                pz = (float)(R_CHECK * a * unit[3 * q + 2]);
    float u[3] = {0.f, 0.f, 0.f}, hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f};
    for (int b0 = p0; b0 < p1; b0 += FMM_TPB) {
      __syncthreads();
      if (b0 + t < p1) {
        const int64_t i = list[b0 + t];
        sp[t] = make_float4((float)(X[3 * i] - cx), (float)(X[3 * i + 1] - cy),
                            (float)(X[3 * i + 2] - cz), 0.f);
        sg[t] = make_float4((float)(w[i] * f[3 * i]), (float)(w[i] * f[3 * i + 1]),
                            (float)(w[i] * f[3 * i + 2]), 0.f);
      }
      __syncthreads();
      const int nb = min(FMM_TPB, p1 - b0);
      for (int j = 0; j < nb; ++j) {
        const float4 y = sp[j], g = sg[j];
        const float dx = px - y.x, dy = py - y.y, dz = pz - y.z;
        const float r2 = dx * dx + dy * dy + dz * dz;
        const float ri = rsqrtf(r2);
        const float gd = (g.x * dx + g.y * dy + g.z * dz) * ri * ri;
        u[0] += (g.x + gd * dx) * ri;
        u[1] += (g.y + gd * dy) * ri;
        u[2] += (g.z + gd * dz) * ri;
        if ((j & 31) == 31 || j == nb - 1) {  // two-sum merge every 32 points
          for (int d = 0; d < 3; ++d) {
            const float s = hi[d] + u[d], bp = s - hi[d];
            lo[d] += (hi[d] - (s - bp)) + (u[d] - bp);
            hi[d] = s;
            u[d] = 0.f;
          }
        }
      }
    }
    if (q0 + t < Np)
      for (int d = 0; d < 3; ++d)
        ucheck_part[(((int64_t)c * FMM_CHECK_SPLIT + part) * Np + q) * 3 + d] =
            (double)hi[d] + (double)lo[d];
  }
}

// phi[c][r] = a_c sum_j P1[r][j] u_check[c][j] (FP64), u_check the parts of
// k_fmm_check32 summed in part order: 64 rows x 4 clusters per block.
__global__ void __launch_bounds__(256) k_fmm_phi(const double* __restrict__ P1T,
                                                 const double* __restrict__ ucheck_part,
                                                 const double* __restrict__ box, int k, int n3,
                                                 double* __restrict__ phi) {
  __shared__ double su[4][FMM_MAX_N3];
  const int r = blockIdx.x * 64 + (threadIdx.x & 63), cl = threadIdx.x >> 6;
  const int c = blockIdx.y * 4 + cl;
  if (c < k)
    for (int j = threadIdx.x & 63; j < n3; j += 64) {
      double v = 0.0;
      for (int sp = 0; sp < FMM_CHECK_SPLIT; ++sp)
        v += ucheck_part[((int64_t)c * FMM_CHECK_SPLIT + sp) * n3 + j];
      su[cl][j] = v;
    }
  __syncthreads();
  if (r >= n3 || c >= k) return;
  double s = 0.0;
  for (int j = 0; j < n3; ++j) s = fma(P1T[(int64_t)j * n3 + r], su[cl][j], s);
  phi[(int64_t)c * n3 + r] = box[4 * c + 3] * s;
}

// Neighbouring-cluster sources, packed cluster by cluster (each cluster's
// points in Morton order, padded to whole tiles): the FP32 records of the
// direct sum. Slot s belongs to cluster tile_cluster[s / TILE].
__global__ void k_fmm_pack_near(const double* __restrict__ X, const double* __restrict__ w,
                                const double* __restrict__ f, const int* __restrict__ list,
                                const int* __restrict__ off, const int* __restrict__ count,
                                const int* __restrict__ tile_cluster,
                                const int* __restrict__ src_first, int64_t n_slots, double scale,
                                float4* __restrict__ srcF, int* __restrict__ src_orig,
                                float4* __restrict__ segbox) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= n_slots) return;  // n_slots is a multiple of TILE: whole warps leave together
  const int j = tile_cluster[s / TILE];
  const int64_t q = s - src_first[j];
  const bool real = q < count[j];
  const int64_t i = real ? list[off[j] + q] : -1;
  float x = PAD_POS, y = PAD_POS, z = PAD_POS;
  if (real) {
    x = (float)X[3 * i];
    y = (float)X[3 * i + 1];
    z = (float)X[3 * i + 2];
  }
  const float3 c = warp_box(real, x, y, z, segbox + 2 * (s / SEG));
  float g0 = 0.f, g1 = 0.f, g2 = 0.f;
  if (real) {
    x = (float)(X[3 * i] - (double)c.x);
    y = (float)(X[3 * i + 1] - (double)c.y);
    z = (float)(X[3 * i + 2] - (double)c.z);
    const double ws = w[i] * scale;
    g0 = (float)(ws * f[3 * i]);
    g1 = (float)(ws * f[3 * i + 1]);
    g2 = (float)(ws * f[3 * i + 2]);
  }
  write_sl_record(srcF + s * V_SL, x, y, z, g0, g1, g2);
  src_orig[s] = (int)i;
}

// Equivalent sources, eqp slots per cluster (Np real ones, the rest padding),
// packed after the neighbouring-cluster sources (slot base + s).
__global__ void k_fmm_pack_eq(const double* __restrict__ box, const double* __restrict__ unit,
                              int Np, int eqp, const double* __restrict__ phi,
                              const int* __restrict__ count, int k, double scale, int64_t base,
                              float4* __restrict__ srcF, float4* __restrict__ segbox) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= (int64_t)k * eqp) return;  // k * eqp is a multiple of SEG
  const int j = (int)(s / eqp), q = (int)(s % eqp);
  const bool real = q < Np && count[j] > 0;
  double ex = PAD_POS, ey = PAD_POS, ez = PAD_POS;
  if (real) {
    const double a = box[4 * j + 3];
    ex = box[4 * j] + R_EQUIV * a * unit[3 * q];
    ey = box[4 * j + 1] + R_EQUIV * a * unit[3 * q + 1];
    ez = box[4 * j + 2] + R_EQUIV * a * unit[3 * q + 2];
  }
  const float3 c = warp_box(real, (float)ex, (float)ey, (float)ez, segbox + 2 * ((base + s) / SEG));
  float x = PAD_POS, y = PAD_POS, z = PAD_POS, g0 = 0.f, g1 = 0.f, g2 = 0.f;
  if (real) {
    x = (float)(ex - (double)c.x);
    y = (float)(ey - (double)c.y);
    z = (float)(ez - (double)c.z);
    const double* ph = phi + ((int64_t)j * Np + q) * 3;
    g0 = (float)(ph[0] * scale);
    g1 = (float)(ph[1] * scale);
    g2 = (float)(ph[2] * scale);
  }
  write_sl_record(srcF + (base + s) * V_SL, x, y, z, g0, g1, g2);
}

// Targets box by box (each box's targets in Morton order, padded to whole
// target blocks): slot t is in block t / tb, which belongs to box
// block_box[t / tb]. Padding slots repeat one of the box's targets and are
// dead (negative thresholds, perm = -1).
__global__ void k_fmm_pack_tgt(const double* __restrict__ Y, const double* __restrict__ delta,
                               int64_t n_delta, const int* __restrict__ tlist,
                               const int* __restrict__ toff, const int* __restrict__ tcount,
                               const int* __restrict__ block_box, const int* __restrict__ box_first,
                               int tb, int64_t n_slots, double rho_T, double rho_c,
                               float4* __restrict__ tgtF, double4_32a* __restrict__ tgt64,
                               int* __restrict__ perm) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n_slots) return;
  const int i = block_box[t / tb];
  const int64_t q = t - box_first[i];
  const bool real = q < tcount[i];
  const int64_t j = tlist[toff[i] + (real ? q : 0)];
  const double x = Y[3 * j], y = Y[3 * j + 1], z = Y[3 * j + 2];
  const double d = delta[n_delta == 1 ? 0 : j];
  const double rc = rho_c * d, rt = rho_T * d;
  tgtF[2 * t] = make_float4((float)x, (float)y, (float)z, (float)(1.0 / d));
  tgtF[2 * t + 1] = real ? make_float4((float)(rc * rc), (float)(rt * rt), 0.f, 0.f)
                         : make_float4(-1.f, -1.f, 0.f, 0.f);
  tgt64[t] = make_double4_32a(x, y, z, d);
  perm[t] = real ? (int)j : -1;
}

// One work item per CTA: (target block, first tile descriptor, tiles,
// partial slot); the block's partials go to slot * TB.
template <int NP, int MINB>
__global__ void __launch_bounds__(TPB32, MINB)
    k_pair32_fmm(p32::PairArgs a, const int4* __restrict__ items, const int2* __restrict__ desc) {
  extern __shared__ __align__(128) float4 sm[];
  __shared__ p32::PipeSmem<p32::pair_stages<p32::SLayer, NP>()> ps;
  if (threadIdx.x == 0) ps.initialized = 0;
  constexpr int TB = TPB32 * 2 * NP;
  const int4 it = items[blockIdx.x];
  p32::pair_item<p32::SLayer, NP>(
      a, it.x, p32::TileList{desc + it.y, it.z, it.w, TB, (int64_t)it.x * TB}, sm, ps);
}

// One CTA of G threads per target group of G targets (a thread per target):
// each target's item partials in item order plus its FP64 near sum (the
// near-sum scratch in dynamic shared memory); u at the target's original
// index.
template <int G>
__global__ void __launch_bounds__(G)
    k_fmm_finish32(p32::OverflowArgs oa, p32::FinishArgs fa, const int* __restrict__ item_first,
                   int tb) {
  extern __shared__ unsigned fsm[];
  int cnt = p32::near_group<p32::SLayer, G>(
      oa, fa, blockIdx.x, fsm, threadIdx.x, [&](int64_t t, double n0, double n1, double n2) {
        const int64_t j = fa.perm[t];
        if (j < 0) return;
        const int64_t b = t / tb, l = t - b * tb;
        double u0 = 0.0, u1 = 0.0, u2 = 0.0;
        for (int it = item_first[b]; it < item_first[b + 1]; ++it) {
          const double* p = fa.part + ((size_t)it * tb + l) * 3;
          u0 += p[0];
          u1 += p[1];
          u2 += p[2];
        }
        fa.u[3 * j] = u0 + n0;
        fa.u[3 * j + 1] = u1 + n1;
        fa.u[3 * j + 2] = u2 + n2;
      });
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt)
    atomicAdd(fa.flags + FLAG_NEAR_PAIRS, (unsigned long long)cnt);
}

template <int NP>
void launch_pair32_fmm(const p32::PairArgs& a, const int4* items, const int2* desc, int n_items,
                       cudaStream_t st) {
  constexpr int MINB = NP == 2 ? PAIR32_MINB_NP2 : PAIR32_MINB_NP1;
  const size_t smem = p32::pair_smem_bytes<p32::SLayer, NP>();
  cudaFuncSetAttribute(k_pair32_fmm<NP, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  k_pair32_fmm<NP, MINB><<<(unsigned)n_items, TPB32, smem, st>>>(a, items, desc);
}

// k_overflow32 of the direct path, for the FMM's targets.
__global__ void k_fmm_overflow32(p32::OverflowArgs a, int64_t M) {
  if (a.flags[FLAG_OVERFLOW] == 0ull) return;
  const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (t >= M) return;
  p32::overflow_target<p32::SLayer>(a, t);
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
    cudaFree(kv.second->P1T);
    delete kv.second;
  }
  ctx->fmm_ops.clear();
}

}  // namespace sk

using namespace sk;

extern "C" {

int stokes_sl_eval_fmm(sk_ctx* ctx, int precision, int mem, int64_t n_src,
                       const double* src_xyz, const double* src_w, const double* f,
                       int64_t n_tgt, const double* tgt_xyz, const double* delta,
                       int64_t n_delta, double mu, int k, const double* centers0,
                       int lloyd_iters, int p, double* u_out, void* stream) {
  if (!ctx) return SK_EINVAL;
  if (n_src < 1 || n_tgt < 1 || n_src > (1LL << 30) || n_tgt > (1LL << 30) || !src_xyz ||
      !src_w || !f || !tgt_xyz || !delta || !u_out || !centers0 || k < 1 || k > 65536 ||
      lloyd_iters < 0 || p < 3 || p > 10 || !(n_delta == 1 || n_delta == n_tgt) ||
      !(mu > 0.0 && mu < INFINITY) || (mem != SK_HOST && mem != SK_DEVICE) ||
      (precision != SK_FP64 && precision != SK_FP32C)) {
    ctx->err = "stokes_sl_eval_fmm: invalid argument (sizes, pointers, 1 <= k <= 65536, "
               "3 <= p <= 10, n_delta in {1, n_tgt}, mu > 0, mem, precision)";
    return SK_EINVAL;
  }
  if (precision == SK_FP32C && n_src > FP32C_MAX_SOURCES) {
    ctx->err = "stokes_sl_eval_fmm: more than 2^25 sources in SK_FP32C";
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
  const bool fp32 = precision == SK_FP32C;
  const int Np = op->Np, n3 = 3 * Np;
  // FP32C layout: target blocks of tb targets; equivalent sources padded to
  // whole segments; the bounds below size the workspace before the plan
  const int np32 = pair32_np(n_tgt);
  const int tb = TPB32 * 2 * np32;
  const int eqp = (int)align_up((size_t)Np, SEG);
  const int64_t near_slots_max = (int64_t)align_up((size_t)n_src, TILE) + (int64_t)k * TILE;
  const int64_t src_slots_max = near_slots_max + (int64_t)k * eqp;
  const int64_t m_slots_max = (int64_t)align_up((size_t)n_tgt, tb) + (int64_t)k * tb;
  const int64_t n_blocks_max = m_slots_max / tb;
  const int eq_tiles = (eqp + TILE - 1) / TILE;  // tiles of one cluster's equivalent sources
  const int64_t box_tiles_max = near_slots_max / TILE + (int64_t)k * eq_tiles;  // one box's list
  // tiles per work item: 8 unless the bound on the items' partials exceeds 512 MB
  const double part_bound = (double)n_blocks_max * (double)box_tiles_max * tb * 24.0;
  const int item_tiles = (int)std::max<double>(FMM_ITEM_TILES, std::ceil(part_bound / 536870912.0));
  const int64_t n_items_max = n_blocks_max * ((box_tiles_max + item_tiles - 1) / item_tiles);
  const int64_t n_desc_max = (int64_t)k * box_tiles_max;
  const int64_t nsort = std::max(n_src, n_tgt);
  const int sort_blocks = sort_grid_blocks(nsort);
  // workspace: inputs and output (host calls), clustering, target boxes,
  // densities, and (FP32C) the sort scratch, packed sources and targets, the
  // plan, partials and near lists
  struct Carve {
    double *tX = nullptr, *tW = nullptr, *tF = nullptr, *tY = nullptr, *tD = nullptr, *U = nullptr;
    int *lab = nullptr, *count = nullptr, *offs = nullptr, *list = nullptr;
    int *tlab = nullptr, *tcount = nullptr, *toffs = nullptr, *tlist = nullptr;
    double *C = nullptr, *box = nullptr, *tbox = nullptr, *ucheck = nullptr, *phi = nullptr;
    unsigned char* near = nullptr;
    double* frame = nullptr;            // k-means fixed-point frame: lo[3], quantum
    double* frame_part = nullptr;       // per-block partial boxes
    float4* C32 = nullptr;              // FP32 centres
    unsigned long long* sums = nullptr;  // [k][3] fixed-point coordinate sums
    unsigned int* cnt = nullptr;         // [k] points per cluster
    uint32_t *keys_a = nullptr, *keys_b = nullptr, *hist = nullptr;
    // FP32C
    int *vals_a = nullptr, *vals_b = nullptr, *meta = nullptr, *src_order = nullptr,
        *tgt_order = nullptr;
    float *bbox_part = nullptr, *bbox = nullptr;
    float4 *srcF = nullptr, *segbox = nullptr, *tgtF = nullptr;
    int *src_orig = nullptr, *perm = nullptr, *near_cnt = nullptr;
    unsigned* near_idx = nullptr;
    double4_32a* tgt64 = nullptr;
    double *near_ovf = nullptr, *part = nullptr;
    int* plan = nullptr;  // tile_cluster, src_first, block_box, box_first, item_first, items, desc
    unsigned long long* flags = nullptr;
  };
  const int64_t plan_ints = near_slots_max / TILE + k + n_blocks_max + k + (n_blocks_max + 1) +
                            4 * n_items_max + 2 * n_desc_max + 64;
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
    c.ucheck = b.take<double>((size_t)k * n3 * (fp32 ? FMM_CHECK_SPLIT : 1));
    c.phi = b.take<double>((size_t)k * n3);
    c.frame = b.take<double>(5);  // corner, quantum q, 1 / q
    c.frame_part = b.take<double>(6 * 128);
    c.C32 = b.take<float4>(k);
    c.sums = b.take<unsigned long long>(3 * (size_t)k);
    c.cnt = b.take<unsigned int>(k);
    c.keys_a = b.take<uint32_t>(nsort);
    c.keys_b = b.take<uint32_t>(nsort);
    c.vals_a = b.take<int>(nsort);
    c.vals_b = b.take<int>(nsort);
    c.hist = b.take<uint32_t>(256 * (size_t)sort_blocks + 256);
    if (!fp32) return;
    c.bbox_part = b.take<float>(128 * 6);
    c.bbox = b.take<float>(8);
    c.meta = b.take<int>(N_META);
    c.src_order = b.take<int>(n_src);
    c.tgt_order = b.take<int>(n_tgt);
    c.srcF = b.take<float4>((size_t)src_slots_max * V_SL);
    c.segbox = b.take<float4>((size_t)(src_slots_max / SEG) * 2);
    c.src_orig = b.take<int>(near_slots_max);
    c.tgtF = b.take<float4>((size_t)m_slots_max * 2);
    c.tgt64 = b.take<double4_32a>(m_slots_max);
    c.perm = b.take<int>(m_slots_max);
    c.near_cnt = b.take<int>(m_slots_max / NEAR_GROUP_MIN);
    c.near_idx = b.take<unsigned>((size_t)m_slots_max * NEAR_K);
    c.near_ovf = b.take<double>((size_t)m_slots_max * 3);
    c.part = b.take<double>((size_t)n_items_max * tb * 3);
    c.plan = b.take<int>(plan_ints);
    c.flags = b.take<unsigned long long>(N_FLAGS);
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
  cudaMemcpyAsync(C, centers0, 3 * (size_t)k * sizeof(double),
                  mem == SK_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st);
  // 1. k-means of the active sources: FP64 decisions, exact (fixed-point) sums
  const int frame_blocks = (int)std::min<int64_t>(128, (n_src + FMM_TPB - 1) / FMM_TPB);
  k_km_frame_part<<<frame_blocks, FMM_TPB, 0, st>>>(X, W, n_src, cv.frame_part);
  k_km_frame<<<1, 32, 0, st>>>(cv.frame_part, frame_blocks, cv.frame);
  k_km_centres32<<<nblk(k), FMM_TPB, 0, st>>>(C, k, cv.C32);
  for (int it = 0; it < lloyd_iters; ++it) {
    k_km_assign32<<<nblk(n_src), FMM_TPB, 0, st>>>(X, W, n_src, C, cv.C32, k, lab);
    cudaMemsetAsync(cv.sums, 0, 3 * (size_t)k * sizeof(unsigned long long), st);
    cudaMemsetAsync(cv.cnt, 0, (size_t)k * sizeof(unsigned int), st);
    k_km_sums<<<nblk(n_src), FMM_TPB, 0, st>>>(X, lab, n_src, cv.frame, k, cv.sums, cv.cnt);
    k_km_centres<<<nblk(k), FMM_TPB, 0, st>>>(cv.sums, cv.cnt, cv.frame, k, C, cv.C32);
  }
  k_km_assign32<<<nblk(n_src), FMM_TPB, 0, st>>>(X, W, n_src, C, cv.C32, k, lab);
  // each cluster's points listed in index order (FP64) or Morton order (FP32C,
  // the order of the direct sum): a stable sort of the points by label
  int key_bits = 1;
  while ((1ll << key_bits) <= (long long)k) ++key_bits;  // keys 0 .. k
  auto lists = [&](const int* lb, const int* order, int64_t n, int* off_out, int* cnt_out,
                   int* list_out) {
    k_km_keys<<<nblk(n), FMM_TPB, 0, st>>>(lb, order, n, k, cv.keys_a, cv.vals_a);
    const int r = launch_sort_pairs(cv.keys_a, cv.keys_b, cv.vals_a, cv.vals_b, n, key_bits,
                                    cv.hist, st);
    k_km_offsets_sorted<<<nblk(k + 1), FMM_TPB, 0, st>>>(r ? cv.keys_b : cv.keys_a, n, k,
                                                          off_out, cnt_out);
    cudaMemcpyAsync(list_out, r ? cv.vals_b : cv.vals_a, n * sizeof(int),
                    cudaMemcpyDeviceToDevice, st);
  };
  if (fp32) {
    launch_sort_points(X, W, n_src, cv.keys_a, cv.keys_b, cv.vals_a, cv.vals_b, cv.hist,
                       cv.bbox_part, cv.bbox, cv.meta + META_SCRATCH, ctx->small_sort_points, st);
    cudaMemcpyAsync(cv.src_order, cv.vals_a, n_src * sizeof(int), cudaMemcpyDeviceToDevice, st);
  }
  lists(lab, fp32 ? cv.src_order : nullptr, n_src, offs, count, list);
  k_km_box<<<k, FMM_TPB, 0, st>>>(X, offs, list, box);
  // 2. target boxes: nearest final centre, ordered lists, boxes, neighbour matrix
  k_km_assign32<<<nblk(n_tgt), FMM_TPB, 0, st>>>(Y, nullptr, n_tgt, C, cv.C32, k, cv.tlab);
  if (fp32) {
    launch_sort_points(Y, nullptr, n_tgt, cv.keys_a, cv.keys_b, cv.vals_a, cv.vals_b, cv.hist,
                       cv.bbox_part, cv.bbox, cv.meta + META_SCRATCH, ctx->small_sort_points, st);
    cudaMemcpyAsync(cv.tgt_order, cv.vals_a, n_tgt * sizeof(int), cudaMemcpyDeviceToDevice, st);
  }
  lists(cv.tlab, fp32 ? cv.tgt_order : nullptr, n_tgt, cv.toffs, cv.tcount, cv.tlist);
  k_tgt_box<<<k, FMM_TPB, 0, st>>>(Y, D, n_delta, cv.toffs, cv.tlist, cv.tbox);
  k_fmm_neighbours<<<nblk((int64_t)k * k), FMM_TPB, 0, st>>>(cv.tbox, cv.toffs, box, offs, k,
                                                              cv.near);
  const double scale = 1.0 / (8.0 * PI_CONST * mu);
  cudaError_t e;
  if (!fp32) {
    // 3. upward pass (FP64) and the evaluation, one thread per target
    k_fmm_upward<<<k, FMM_TPB, 0, st>>>(X, W, F, offs, list, box, op->unit, Np, op->P1,
                                        cv.ucheck, cv.phi);
    k_fmm_eval<<<nblk(n_tgt, 128), 128, 0, st>>>(Y, D, n_delta, n_tgt, k, box, offs, list,
                                                 cv.tlab, cv.tlist, cv.near, op->unit, Np,
                                                 cv.phi, X, W, F, scale, U);
    e = cudaGetLastError();
  } else {
    // 3. upward pass: FP32 check potentials, FP64 equivalent densities
    k_fmm_check32<<<dim3((unsigned)k, FMM_CHECK_SPLIT), FMM_TPB, 0, st>>>(
        X, W, F, offs, list, box, op->unit, Np, cv.ucheck);
    k_fmm_phi<<<dim3((unsigned)((n3 + 63) / 64), (unsigned)((k + 3) / 4)), 256, 0, st>>>(
        op->P1T, cv.ucheck, box, k, n3, cv.phi);
    // 4. the plan, on the host: cluster sizes, box sizes and the neighbour matrix
    std::vector<int> h_count(k), h_tcount(k);
    std::vector<unsigned char> h_near((size_t)k * k);
    cudaMemcpyAsync(h_count.data(), count, k * sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(h_tcount.data(), cv.tcount, k * sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(h_near.data(), cv.near, (size_t)k * k, cudaMemcpyDeviceToHost, st);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) {
      ctx->err = std::string("stokes_sl_eval_fmm: ") + cudaGetErrorString(e);
      return SK_ECUDA;
    }
    std::vector<int> src_first(k), box_first(k, 0), tile_cluster, block_box, item_first, items,
        desc;
    int64_t near_slots = 0;
    for (int j = 0; j < k; ++j) {
      src_first[j] = (int)near_slots;
      const int64_t tiles = (h_count[j] + TILE - 1) / TILE;
      for (int64_t t = 0; t < tiles; ++t) tile_cluster.push_back(j);
      near_slots += tiles * TILE;
    }
    if (near_slots == 0) {  // every weight is zero: u = 0
      cudaMemsetAsync(U, 0, 3 * n_tgt * sizeof(double), st);
    }
    int64_t m_slots = 0;
    for (int i = 0; i < k; ++i) {
      if (h_tcount[i] == 0 || near_slots == 0) continue;
      box_first[i] = (int)m_slots;
      const int nb = (h_tcount[i] + tb - 1) / tb;
      // the box's tile list: its neighbouring clusters' tiles (the last tile of
      // a cluster trimmed to whole segments), then the far clusters'
      // equivalent sources
      const int d0 = (int)(desc.size() / 2);
      for (int j = 0; j < k; ++j) {
        if (h_count[j] == 0) continue;
        if (h_near[(size_t)i * k + j]) {
          for (int64_t t = 0; t * TILE < h_count[j]; ++t) {
            const int64_t rem = h_count[j] - t * TILE;
            const int nseg = (int)std::min<int64_t>(TILE_SEGS, (rem + SEG - 1) / SEG);
            desc.push_back((int)(src_first[j] + t * TILE));
            desc.push_back(nseg);
          }
        } else {
          for (int s0 = 0; s0 < eqp / SEG; s0 += TILE_SEGS) {
            desc.push_back((int)(near_slots + (int64_t)j * eqp + (int64_t)s0 * SEG));
            desc.push_back(std::min(TILE_SEGS, eqp / SEG - s0));
          }
        }
      }
      const int nt = (int)(desc.size() / 2) - d0;
      for (int bb = 0; bb < nb; ++bb) {
        const int blk = (int)(m_slots / tb) + bb;
        block_box.push_back(i);
        item_first.push_back((int)(items.size() / 4));
        for (int c0 = 0; c0 < nt; c0 += item_tiles)
          items.insert(items.end(), {blk, d0 + c0, std::min(item_tiles, nt - c0),
                                     (int)(items.size() / 4)});
      }
      m_slots += (int64_t)nb * tb;
    }
    item_first.push_back((int)(items.size() / 4));
    const int n_blocks = (int)(m_slots / tb), n_items = (int)(items.size() / 4);
    {
      // launch order: most segments first (items keep their partial slots,
      // so the order changes nothing but the tail of the launch)
      std::vector<int> work(n_items), order(n_items);
      for (int q = 0; q < n_items; ++q) {
        int nseg = 0;
        for (int t = 0; t < items[4 * q + 2]; ++t) nseg += desc[2 * (items[4 * q + 1] + t) + 1];
        work[q] = nseg;
        order[q] = q;
      }
      std::stable_sort(order.begin(), order.end(),
                       [&](int a, int b) { return work[a] > work[b]; });
      std::vector<int> sorted(items.size());
      for (int q = 0; q < n_items; ++q)
        for (int c = 0; c < 4; ++c) sorted[4 * q + c] = items[4 * order[q] + c];
      items.swap(sorted);
    }
    if (n_items > 0) {
      // upload the plan: tile_cluster, src_first, block_box, box_first, item_first, items, desc
      std::vector<int> h_plan;
      auto put = [&](const std::vector<int>& v) {
        const size_t at = h_plan.size();
        h_plan.insert(h_plan.end(), v.begin(), v.end());
        while (h_plan.size() % 4) h_plan.push_back(0);  // 16-byte aligned sections
        return at;
      };
      const size_t o_tc = put(tile_cluster), o_sf = put(src_first), o_bb = put(block_box),
                   o_bf = put(box_first), o_if = put(item_first), o_it = put(items),
                   o_de = put(desc);
      if ((int64_t)h_plan.size() > plan_ints || m_slots > m_slots_max ||
          near_slots > near_slots_max || n_items > n_items_max) {
        ctx->err = "stokes_sl_eval_fmm: plan exceeds its bounds";
        return SK_ECUDA;
      }
      cudaMemcpyAsync(cv.plan, h_plan.data(), h_plan.size() * sizeof(int),
                      cudaMemcpyHostToDevice, st);
      int meta[N_META] = {};
      meta[META_NS] = (int)near_slots;  // the overflow rescan's range
      cudaMemcpyAsync(cv.meta, meta, sizeof(meta), cudaMemcpyHostToDevice, st);
      cudaMemsetAsync(cv.flags, 0, N_FLAGS * sizeof(unsigned long long), st);
      cudaMemsetAsync(cv.near_cnt, 0, (m_slots / NEAR_GROUP_MIN) * sizeof(int), st);
      const int* d_tc = cv.plan + o_tc;
      const int* d_sf = cv.plan + o_sf;
      const int* d_bb = cv.plan + o_bb;
      const int* d_bf = cv.plan + o_bf;
      const int* d_if = cv.plan + o_if;
      const int4* d_it = reinterpret_cast<const int4*>(cv.plan + o_it);
      const int2* d_de = reinterpret_cast<const int2*>(cv.plan + o_de);
      // 5. packed sources (neighbouring clusters, then equivalent sources) and targets
      k_fmm_pack_near<<<nblk(near_slots), FMM_TPB, 0, st>>>(X, W, F, list, offs, count, d_tc,
                                                            d_sf, near_slots, scale, cv.srcF,
                                                            cv.src_orig, cv.segbox);
      k_fmm_pack_eq<<<nblk((int64_t)k * eqp), FMM_TPB, 0, st>>>(
          box, op->unit, Np, eqp, cv.phi, count, k, scale, near_slots, cv.srcF, cv.segbox);
      k_fmm_pack_tgt<<<nblk(m_slots), FMM_TPB, 0, st>>>(Y, D, n_delta, cv.tlist, cv.toffs,
                                                        cv.tcount, d_bb, d_bf, tb, m_slots,
                                                        ctx->rho_T, ctx->rho_c, cv.tgtF,
                                                        cv.tgt64, cv.perm);
      // 6. the pair sums of every item, the overflow rescans and the finish
      p32::PairArgs a{cv.srcF, cv.segbox, cv.src_orig, cv.meta, cv.tgtF, cv.tgt64, m_slots, 1,
                      cv.part, cv.near_cnt, cv.near_idx, cv.flags, (float)ctx->rho_T, 8.0f,
                      nullptr};
      if (np32 == 2)
        launch_pair32_fmm<2>(a, d_it, d_de, n_items, st);
      else
        launch_pair32_fmm<1>(a, d_it, d_de, n_items, st);
      p32::OverflowArgs oa{cv.srcF,   cv.segbox, cv.src_orig, cv.meta, cv.tgtF,  cv.tgt64,
                           cv.near_cnt, X,        W,           F,       nullptr, scale,
                           cv.flags,  cv.near_ovf};
      oa.group = 64 * np32;
      k_fmm_overflow32<<<(unsigned)((m_slots * 32 + 255) / 256), 256, 0, st>>>(oa, m_slots);
      p32::FinishArgs fa{cv.tgt64, cv.perm, m_slots, 1, cv.part, cv.near_cnt, cv.near_idx,
                         cv.near_ovf, X, W, F, nullptr, scale, U, cv.flags};
      fa.group = 64 * np32;
      const size_t fsmem = (size_t)p32::near_warp_words(fa.group) * 4;
      if (np32 == 2)
        k_fmm_finish32<128><<<(unsigned)(m_slots / 128), 128, fsmem, st>>>(oa, fa, d_if, tb);
      else
        k_fmm_finish32<64><<<(unsigned)(m_slots / 64), 64, fsmem, st>>>(oa, fa, d_if, tb);
      ctx->stats = sk_eval_stats{};
      ctx->stats.n_tgt = n_tgt;
      ctx->stats.n_chunks = n_items;
      ctx->stats.precision = precision;
      (void)n_blocks;
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && mem == SK_HOST)
    e = cudaMemcpyAsync(u_out, U, 3 * n_tgt * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && (mem == SK_HOST || !stream || fp32)) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    ctx->err = std::string("stokes_sl_eval_fmm: ") + cudaGetErrorString(e);
    return SK_ECUDA;
  }
  if (fp32) {
    unsigned long long flags[N_FLAGS] = {};
    if (cudaMemcpy(flags, cv.flags, sizeof(flags), cudaMemcpyDeviceToHost) == cudaSuccess &&
        flags[FLAG_TIMEOUT]) {
      ctx->err = "stokes_sl_eval_fmm: a bounded device wait expired";
      return SK_ETIMEOUT;
    }
  }
  return SK_OK;
}

}  // extern "C"
