// sk_membrane.cu -- overset finite-difference surface derivatives and the
// Skalak membrane force on the six-patch grid (Sec. 3.5; Sec. 2.1, Eqs.
// tensor and intf; formulas of the Appendix).
//
// The derivative scheme is a fixed linear operator on node values that
// depends only on m (the transition maps and partition of unity live on the
// unit sphere), so it is built once per m on the host, in FP64, and cached in
// the context:
//   * ghost taps: for every ghost point of the extended grid that a 7-point
//     stencil touches, the patches q with psi_q > 0 there, the point's (u, v)
//     in patch q and psi_q (Eq. ext);
//   * blend taps: for every node, psi of its own patch and, for the other
//     patches q with psi_q > 0, (u, v) in q, psi_q and the Jacobian of the
//     transition map (Eqs. blendu / blendv).
// On the device, per batch of F fields (SoA [F][6][m-1][m-1], FP64):
//   1. spline slopes: each patch grid function becomes the tensor-product
//      not-a-knot cubic spline, stored as a bicubic Hermite interpolant
//      (g, g_u, g_v, g_uv at the nodes; one tridiagonal solve per grid line);
//   2. patch extension: ghost value = sum_q psi_q * spline_q(u_q, v_q);
//   3. 7-point central differences on the extended grid (Eq. fdm);
//   4. splines of the FD derivatives, then blending.
// Skalak: tangents of the current and reference nodes by the scheme; Lambda
// of Eq. tensor from the closed-form invariants of V^2 (tr V^2 and
// det = (W / W_r)^2); f = div_gamma Lambda column by column.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <cmath>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "sk_internal.h"

namespace sk {

constexpr int MEM_FMAX = 9;  // fields per pass (Lambda has 6, positions 3)
constexpr int MEM_SCRATCH_SETS = 4;  // scratch copies for concurrent streams (serving)

struct MembraneOp {
  int m = 0, n = 0, E = 0;  // E = m + 5: extended grid (indices -2..m+2)
  bool slope_staging = true;  // stage slope-solve lines in shared memory when they fit
  int64_t N = 0;
  double h = 0.0, ih = 0.0;
  int G = 0;  // ghost points used by the stencils, per field
  // operator tables (device). A tap is a spline evaluation at a fixed point
  // of one patch: its cell (node index p n^2 + a n + b of the cell's first
  // corner) and the eight Hermite basis values there (u: value left/right,
  // slope left/right; v likewise), followed by the tap's weights.
  int* ghost_dst = nullptr;    // [G] offset in a field's extended block (6 E^2)
  int* gtap_ptr = nullptr;     // [G + 1]
  int* gtap_cell = nullptr;    // [taps]
  double* gtap_w = nullptr;    // [taps][9]: basis[8], psi
  double* psi_own = nullptr;   // [N]
  int* btap_ptr = nullptr;     // [N + 1]
  int* btap_cell = nullptr;
  double* btap_w = nullptr;    // [taps][13]: basis[8], psi, dtau1/du, dtau2/du, dtau1/dv, dtau2/dv
  double* thomas = nullptr;    // slope-solve table (see k_slopes): c', 1/den, run products, 3/h 1/den
  // scratch for up to MEM_FMAX fields
  double *g = nullptr, *sg = nullptr;    // values, spline data [3][F][N] (u, v, uv slopes)
  double* ext = nullptr;                 // [F][6][E][E]
  double *du = nullptr, *dv = nullptr;   // FD derivatives [F][N]
  double *sdu = nullptr, *sdv = nullptr; // their spline data [3][F][N]
  double *gu = nullptr, *gv = nullptr;   // blended derivatives [F][N]
  double* cur_t = nullptr;               // current tangents [6][N]
  double* red = nullptr;                 // reduction partials
  // four-times upsampled single layer (built on first use)
  int nf = 0;                    // fine nodes per line, 4m - 1
  int64_t Nup = 0;               // 6 nf^2
  int* ucell1 = nullptr;         // [nf] cell of fine index J (both directions)
  double* ubasis1 = nullptr;     // [nf][4] Hermite bases there
  double* psi_up = nullptr;      // [Nup] POU of each fine node's patch
  double *Xu = nullptr, *Fu = nullptr, *wu = nullptr;   // fine sources
  double *Xc = nullptr, *Wc = nullptr, *fc = nullptr, *uc = nullptr;  // coarse staging
  double* dtgt = nullptr;        // [N] delta per coarse target
  unsigned long long* pmax = nullptr;  // [8] delta_u per patch (double bits)
  // copies that share the tables above and own their scratch, so that
  // their kernels may run on different streams at once (built on demand)
  MembraneOp* sets[MEM_SCRATCH_SETS] = {};
  bool owns_tables = true;
};

namespace {

// ---------------------------------------------------------------------------
// Host geometry of the six charts (Sec. 3.1, Eq. param_maps) and the POU.
struct D3 {
  double x, y, z;
};
inline double dot3(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

D3 h_chart(int p, double u, double v) {
  const double su = std::sin(u), cu = std::cos(u), sv = std::sin(v), cv = std::cos(v);
  switch (p) {
    case 0: return {su * cv, su * sv, cu};
    case 1: return {-su * cv, -su * sv, cu};
    case 2: return {su * sv, -su * cv, cu};
    case 3: return {-su * sv, su * cv, cu};
    case 4: return {su * cv, -cu, su * sv};
    default: return {su * cv, cu, -su * sv};
  }
}

void h_chart_tangents(int p, double u, double v, D3& tu, D3& tv) {
  const double su = std::sin(u), cu = std::cos(u), sv = std::sin(v), cv = std::cos(v);
  switch (p) {
    case 0: tu = {cu * cv, cu * sv, -su}; tv = {-su * sv, su * cv, 0.0}; break;
    case 1: tu = {-cu * cv, -cu * sv, -su}; tv = {su * sv, -su * cv, 0.0}; break;
    case 2: tu = {cu * sv, -cu * cv, -su}; tv = {su * cv, su * sv, 0.0}; break;
    case 3: tu = {-cu * sv, cu * cv, -su}; tv = {-su * cv, -su * sv, 0.0}; break;
    case 4: tu = {cu * cv, su, cu * sv}; tv = {-su * sv, 0.0, su * cv}; break;
    default: tu = {cu * cv, -su, -cu * sv}; tv = {-su * sv, 0.0, -su * cv}; break;
  }
}

// (u, v) of a unit vector in patch p: u from the chart's cos-u component,
// v from its (sin u cos v, sin u sin v) components.
void h_inverse_chart(int p, D3 x, double& u, double& v) {
  double cu, a, b;
  switch (p) {
    case 0: cu = x.z; a = x.x; b = x.y; break;
    case 1: cu = x.z; a = -x.x; b = -x.y; break;
    case 2: cu = x.z; a = -x.y; b = x.x; break;
    case 3: cu = x.z; a = x.y; b = -x.x; break;
    case 4: cu = -x.y; a = x.x; b = x.z; break;
    default: cu = x.y; a = x.x; b = -x.z; break;
  }
  u = std::acos(std::fmin(1.0, std::fmax(-1.0, cu)));
  v = std::atan2(b, a);
}

// psi_q(x0) for all patches (Eq. pou0): bump of the great-circle distance to
// the patch centre eta_q^0(pi/2, pi/2) over r0 = 5 pi / 12, normalized.
void h_pou(D3 x0, double psi[6]) {
  const double r0 = 5.0 * PI_CONST / 12.0;
  double s = 0.0;
  for (int q = 0; q < 6; ++q) {
    const D3 c = h_chart(q, 0.5 * PI_CONST, 0.5 * PI_CONST);
    const double d = std::acos(std::fmin(1.0, std::fmax(-1.0, dot3(x0, c)))) / r0;
    double b = 0.0;
    if (d < 1.0) b = std::exp(2.0 * (d > 0.0 ? std::exp(-1.0 / d) : 0.0) / (d - 1.0));
    psi[q] = b;
    s += b;
  }
  for (int q = 0; q < 6; ++q) psi[q] /= s;
}

// Jacobian of tau_pq at (u, v) in the layout of Eq. jacobian_diff:
// J = (dtau1/du, dtau2/du, dtau1/dv, dtau2/dv), from the chain rule
// eta_p,u = eta_q,u' dtau1/du + eta_q,v' dtau2/du (same for v).
void h_transition_jacobian(int p, int q, double u, double v, double uq, double vq, double J[4]) {
  D3 pu, pv, qu, qv;
  h_chart_tangents(p, u, v, pu, pv);
  h_chart_tangents(q, uq, vq, qu, qv);
  const double a = dot3(qu, qu), b = dot3(qu, qv), c = dot3(qv, qv);
  const double det = a * c - b * b;
  auto solve = [&](D3 t, double& x, double& y) {
    const double r1 = dot3(qu, t), r2 = dot3(qv, t);
    x = (c * r1 - b * r2) / det;
    y = (a * r2 - b * r1) / det;
  };
  solve(pu, J[0], J[1]);
  solve(pv, J[2], J[3]);
}

// Cell and cubic Hermite bases of the point (u, v) on a patch grid with n
// nodes per line at u = h, 2h, ..: the cell is clamped to the first/last one,
// so points beyond the nodes continue the end pieces.
int h_cell_basis(int p, int n, double h, double u, double v, double basis[8]) {
  const double tu = u / h - 1.0, tv = v / h - 1.0;
  int a = (int)std::floor(tu), b = (int)std::floor(tv);
  a = a < 0 ? 0 : (a > n - 2 ? n - 2 : a);
  b = b < 0 ? 0 : (b > n - 2 ? n - 2 : b);
  const double t = tu - a, s = tv - b;
  basis[0] = (1.0 + 2.0 * t) * (1.0 - t) * (1.0 - t);  // value at the left node
  basis[1] = t * t * (3.0 - 2.0 * t);                  // value at the right node
  basis[2] = t * (1.0 - t) * (1.0 - t) * h;            // slope at the left node
  basis[3] = t * t * (t - 1.0) * h;                    // slope at the right node
  basis[4] = (1.0 + 2.0 * s) * (1.0 - s) * (1.0 - s);
  basis[5] = s * s * (3.0 - 2.0 * s);
  basis[6] = s * (1.0 - s) * (1.0 - s) * h;
  basis[7] = s * s * (s - 1.0) * h;
  return (p * n + a) * n + b;
}

// ---------------------------------------------------------------------------
// Device kernels.
inline unsigned blocks_of(int64_t n) { return (unsigned)((n + 255) / 256); }

// Not-a-knot cubic-spline slopes, L lanes per grid line. Lines: for
// dir 0 the u-lines (fixed k, stride n), for dir 1 the v-lines (fixed j).
// With uniform spacing the end conditions read s0 + 2 s1 = (-5 g0 + 4 g1 +
// g2)/2h and 2 s_{n-2} + s_{n-1} = (5 g_{n-1} - 4 g_{n-2} - g_{n-3})/2h;
// eliminating s0 and s_{n-1} leaves a diagonally dominant tridiagonal system
// in s1..s_{n-2} whose factorization (c'_q, 1/den_q) is shared by all lines.
// Both sweeps of the solve are affine recurrences,
//   forward   d_q = -(1/den_q) d_{q-1} + v_q,   v_q = rhs_q / den_q,
//   backward  s_q = -c'_q s_{q+1} + d_q,
// each with |multiplier| <= 1/2. Each lane takes a run of consecutive terms
// and composes their maps ((a2, b2) o (a1, b1) = (a2 a1, a2 b1 + b2)); the
// product of a run's multipliers does not depend on the data and comes from
// the table. A scan over the line's lanes gives each lane its incoming value,
// and the lane replays its run. v_q is computed once (stored in s, then
// overwritten by d_q and s_q).
// L = 8, 16 or 32 lanes per line: fewer lanes cost fewer scan steps, more
// lanes give short lines and small grids enough threads (slope_lanes).
// Table (thomas): [c' (n) | 1/den (n) | 3/h * 1/den (n) | for L = 8, 16, 32:
// forward then backward run products (L each)].
constexpr int SLOPE_LPL_MIN = 8, SLOPE_LPL_MAX = 32;
__host__ __device__ constexpr int slope_products_offset(int n, int L) {
  return 3 * n + 2 * (L - SLOPE_LPL_MIN);  // L = 8: 0, 16: 16, 32: 48
}
constexpr int SLOPE_TABLE_EXTRA = 2 * (8 + 16 + 32);
constexpr int SLOPE_LINES = 8;  // grid lines per CTA

template <int L>
__device__ __forceinline__ void affine_scan_lines(double& a, double& b, int sub) {
#pragma unroll
  for (int o = 1; o < L; o <<= 1) {
    const double pa = __shfl_up_sync(0xffffffffu, a, o, L);
    const double pb = __shfl_up_sync(0xffffffffu, b, o, L);
    if (sub >= o) {
      b = fma(a, pb, b);
      a = a * pa;
    }
  }
}

// Padded shared-memory index of term q of a line: one spare double per 8, so
// that the run starts of 16 lanes (stride K = 8) fall in distinct banks.
__device__ __forceinline__ int spad(int q) { return q + (q >> 3); }

// First node of grid line `line` (patch-field fp = line / n, index r):
// u-lines (dir 0) start at column r, v-lines (dir 1) at row r.
__device__ __forceinline__ int64_t slope_line_base(int64_t line, int n, int dir) {
  const int64_t fp = line / n;
  const int r = (int)(line % n);
  return fp * n * n + (dir == 0 ? r : (int64_t)r * n);
}

// Term q of one line: staged in shared memory (padded) or in global memory
// (stride st).
struct StagedLine {
  double* p;
  __device__ __forceinline__ double& operator[](int q) const { return p[spad(q)]; }
};
struct GlobalLine {
  double* p;
  int64_t st;
  __device__ __forceinline__ double& operator[](int q) const { return p[q * st]; }
};

// Both sweeps of one line by its L lanes; g: values, s: output slopes (also
// the scratch of v and d). `live` lanes store; the others only take part in
// the shuffles.
template <int L, class Acc>
__device__ __forceinline__ void slope_sweeps(const Acc& g, const Acc& s, bool live, int n, int sub,
                                             double ih, const double* __restrict__ thomas) {
  const double* cp = thomas;
  const double* iden = thomas + n;
  const double* i3d = thomas + 2 * n;
  const double* afw = thomas + slope_products_offset(n, L);
  const double* abw = afw + L;
  const double i2h = 0.5 * ih;
  const int K = (n - 2 + L - 1) / L;  // terms per lane
  const int qa = 1 + sub * K;         // this lane's run [qa, qb) of q = 1..n-2
  const int qb = min(qa + K, n - 1);
  const double r0 = (-5.0 * g[0] + 4.0 * g[1] + g[2]) * i2h;
  const double rN = (5.0 * g[n - 1] - 4.0 * g[n - 2] - g[n - 3]) * i2h;
  const double c1 = r0 * iden[1], cN = rN * iden[n - 2];  // end-condition terms of v_1, v_{n-2}
  // forward sweep
  double B = 0.0;
  for (int q = qa; q < qb; ++q) {
    const double cq = q == 1 ? c1 : (q == n - 2 ? cN : 0.0);
    const double v = fma(i3d[q], g[q + 1] - g[q - 1], -cq);
    B = fma(q == 1 ? 0.0 : -iden[q], B, v);
    if (live) s[q] = v;
  }
  double A = afw[sub];
  affine_scan_lines<L>(A, B, sub);
  double x = __shfl_up_sync(0xffffffffu, B, 1, L);
  if (sub == 0) x = 0.0;
  for (int q = qa; q < qb; ++q) {
    x = fma(q == 1 ? 0.0 : -iden[q], x, s[q]);
    if (live) s[q] = x;
  }
  __syncwarp();
  // backward sweep over p = 1..n-2, q = n-1-p (s_{n-2} = d_{n-2})
  B = 0.0;
  for (int p = qa; p < qb; ++p) {
    const int q = n - 1 - p;
    B = fma(q == n - 2 ? 0.0 : -cp[q], B, s[q]);
  }
  A = abw[sub];
  affine_scan_lines<L>(A, B, sub);
  x = __shfl_up_sync(0xffffffffu, B, 1, L);
  if (sub == 0) x = 0.0;
  for (int p = qa; p < qb; ++p) {
    const int q = n - 1 - p;
    x = fma(q == n - 2 ? 0.0 : -cp[q], x, s[q]);
    if (live) s[q] = x;
  }
  __syncwarp();
  if (sub == 0 && live) {
    s[0] = r0 - 2.0 * s[1];
    s[n - 1] = rN - 2.0 * s[n - 2];
  }
}

// SLOPE_LINES lines per CTA (8 L threads). Staged: the lines' values and
// slopes sit in shared memory (dynamic, 2 x SLOPE_LINES x spad(n) doubles),
// loaded and stored coalesced (for dir 0 the CTA's lines are adjacent
// columns). Unstaged (long lines): the sweeps work in global memory.
template <int L, bool STAGED>
__global__ void __launch_bounds__(SLOPE_LINES * L)
    k_slopes(const double* __restrict__ g, double* __restrict__ s, int64_t n_lines, int n,
             int dir, double ih, const double* __restrict__ thomas) {
  constexpr int T = SLOPE_LINES * L;
  const int tid = threadIdx.x, l = tid / L, sub = tid % L;
  const int64_t line0 = (int64_t)blockIdx.x * SLOPE_LINES;
  const int64_t st = dir == 0 ? n : 1;
  if (!STAGED) {
    // lanes past the last line compute a copy of it and store nothing
    const bool live = line0 + l < n_lines;
    const int64_t b = slope_line_base(live ? line0 + l : n_lines - 1, n, dir);
    slope_sweeps<L>(GlobalLine{const_cast<double*>(g) + b, st}, GlobalLine{s + b, st}, live, n, sub,
                    ih, thomas);
    return;
  }
  extern __shared__ double sm_lines[];
  __shared__ int64_t base_sh[SLOPE_LINES];  // first node of each line (-1: past the last)
  const int stride = spad(n);
  double* gsh = sm_lines;
  double* ssh = sm_lines + SLOPE_LINES * stride;
  if (tid < SLOPE_LINES)
    base_sh[tid] = line0 + tid < n_lines ? slope_line_base(line0 + tid, n, dir) : -1;
  __syncthreads();
  // coalesced load: for dir 0 the line index runs fastest (adjacent columns),
  // for dir 1 the term index (contiguous rows)
  for (int idx = tid; idx < SLOPE_LINES * n; idx += T) {
    const int li = dir == 0 ? idx % SLOPE_LINES : idx / n;
    const int q = dir == 0 ? idx / SLOPE_LINES : idx % n;
    const int64_t b = base_sh[li];
    if (b >= 0) gsh[li * stride + spad(q)] = g[b + q * st];
  }
  __syncthreads();
  slope_sweeps<L>(StagedLine{gsh + l * stride}, StagedLine{ssh + l * stride}, true, n, sub, ih,
                  thomas);
  __syncthreads();
  for (int idx = tid; idx < SLOPE_LINES * n; idx += T) {
    const int li = dir == 0 ? idx % SLOPE_LINES : idx / n;
    const int q = dir == 0 ? idx / SLOPE_LINES : idx % n;
    const int64_t b = base_sh[li];
    if (b >= 0) s[b + q * st] = ssh[li * stride + spad(q)];
  }
}

// Bicubic Hermite evaluation of one field's spline at a tap: node values g,
// spline data sd (u, v, uv slopes at plane strides), field offset fo, the
// tap's cell (index of the cell's first corner) and bases w[0..7].
__device__ __forceinline__ double spline_tap(const double* __restrict__ g,
                                             const double* __restrict__ sd, int64_t plane,
                                             int64_t fo, int cell, int n,
                                             const double* __restrict__ w) {
  const double* su = sd;
  const double* sv = sd + plane;
  const double* suv = sd + 2 * plane;
  const int64_t i00 = fo + cell, i10 = i00 + n, i01 = i00 + 1, i11 = i00 + n + 1;
  const double A0 = w[0], A1 = w[1], B0 = w[2], B1 = w[3];
  const double C0 = w[4], C1 = w[5], D0 = w[6], D1 = w[7];
  return A0 * (C0 * g[i00] + C1 * g[i01] + D0 * sv[i00] + D1 * sv[i01]) +
         A1 * (C0 * g[i10] + C1 * g[i11] + D0 * sv[i10] + D1 * sv[i11]) +
         B0 * (C0 * su[i00] + C1 * su[i01] + D0 * suv[i00] + D1 * suv[i01]) +
         B1 * (C0 * su[i10] + C1 * su[i11] + D0 * suv[i10] + D1 * suv[i11]);
}

// Extended values: nodes copied, ghost points by patch extension (Eq. ext).
__global__ void k_extend(const MembraneOp op, int F) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t N = op.N, blk = 6LL * op.E * op.E, plane = (int64_t)F * N;
  if (i < F * N) {
    const int f = (int)(i / N);
    const int64_t node = i % N;
    const int p = (int)(node / ((int64_t)op.n * op.n));
    const int r = (int)(node % ((int64_t)op.n * op.n));
    const int j = r / op.n, k = r % op.n;
    op.ext[f * blk + ((int64_t)p * op.E + j + 3) * op.E + k + 3] = op.g[i];
    return;
  }
  const int64_t gi = i - F * N;
  if (gi >= (int64_t)F * op.G) return;
  const int f = (int)(gi / op.G);
  const int q = (int)(gi % op.G);
  double val = 0.0;
  for (int t = op.gtap_ptr[q]; t < op.gtap_ptr[q + 1]; ++t) {
    const double* w = op.gtap_w + 9 * t;
    val += w[8] * spline_tap(op.g, op.sg, plane, (int64_t)f * N, op.gtap_cell[t], op.n, w);
  }
  op.ext[f * blk + op.ghost_dst[q]] = val;
}

// Eq. fdm: 7-point central differences (-1, 9, -45, 0, 45, -9, 1) / 60h.
__global__ void k_fd(const MembraneOp op, int F) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t N = op.N;
  if (i >= F * N) return;
  const int f = (int)(i / N);
  const int64_t node = i % N;
  const int p = (int)(node / ((int64_t)op.n * op.n));
  const int r = (int)(node % ((int64_t)op.n * op.n));
  const int j = r / op.n, k = r % op.n;
  const int E = op.E;
  const double* e = op.ext + (int64_t)f * 6 * E * E + ((int64_t)p * E + j + 3) * E + k + 3;
  const double c1 = 45.0 / 60.0, c2 = -9.0 / 60.0, c3 = 1.0 / 60.0;
  op.du[i] = (c1 * (e[E] - e[-E]) + c2 * (e[2 * E] - e[-2 * E]) + c3 * (e[3 * E] - e[-3 * E])) * op.ih;
  op.dv[i] = (c1 * (e[1] - e[-1]) + c2 * (e[2] - e[-2]) + c3 * (e[3] - e[-3])) * op.ih;
}

// Eqs. blendu / blendv.
__global__ void k_blend(const MembraneOp op, int F) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t N = op.N, plane = (int64_t)F * N;
  if (i >= F * N) return;
  const int f = (int)(i / N);
  const int64_t node = i % N;
  const double po = op.psi_own[node];
  double ou = po * op.du[i], ov = po * op.dv[i];
  for (int t = op.btap_ptr[node]; t < op.btap_ptr[node + 1]; ++t) {
    const double* w = op.btap_w + 13 * t;
    const int cell = op.btap_cell[t];
    const double eu = spline_tap(op.du, op.sdu, plane, (int64_t)f * N, cell, op.n, w);
    const double ev = spline_tap(op.dv, op.sdv, plane, (int64_t)f * N, cell, op.n, w);
    ou += w[8] * (eu * w[9] + ev * w[10]);
    ov += w[8] * (eu * w[11] + ev * w[12]);
  }
  op.gu[i] = ou;
  op.gv[i] = ov;
}

// [N][ld] column block c0..c0+F  <->  [F][N]
__global__ void k_gather(const double* __restrict__ aos, int64_t N, int ld, int c0, int F,
                         double* __restrict__ soa) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= F * N) return;
  const int f = (int)(i / N);
  const int64_t node = i % N;
  soa[i] = aos[node * ld + c0 + f];
}
__global__ void k_scatter(const double* __restrict__ soa, int64_t N, int ld, int c0, int F,
                          double* __restrict__ aos) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= F * N) return;
  const int f = (int)(i / N);
  const int64_t node = i % N;
  aos[node * ld + c0 + f] = soa[i];
}

struct Frame {
  double a1[3], a2[3], E, F, G, W, n[3];
};
__device__ __forceinline__ Frame frame_at(const double* __restrict__ t6, int64_t N, int64_t i) {
  Frame fr;
  for (int c = 0; c < 3; ++c) {
    fr.a1[c] = t6[c * N + i];
    fr.a2[c] = t6[(3 + c) * N + i];
  }
  fr.E = fr.a1[0] * fr.a1[0] + fr.a1[1] * fr.a1[1] + fr.a1[2] * fr.a1[2];
  fr.F = fr.a1[0] * fr.a2[0] + fr.a1[1] * fr.a2[1] + fr.a1[2] * fr.a2[2];
  fr.G = fr.a2[0] * fr.a2[0] + fr.a2[1] * fr.a2[1] + fr.a2[2] * fr.a2[2];
  fr.W = sqrt(fr.E * fr.G - fr.F * fr.F);
  fr.n[0] = (fr.a1[1] * fr.a2[2] - fr.a1[2] * fr.a2[1]) / fr.W;
  fr.n[1] = (fr.a1[2] * fr.a2[0] - fr.a1[0] * fr.a2[2]) / fr.W;
  fr.n[2] = (fr.a1[0] * fr.a2[1] - fr.a1[1] * fr.a2[0]) / fr.W;
  return fr;
}

// Tangents of the last F = 3 pass (positions) -> t6 [6][N]; optional
// quadrature weights psi W h^2 (Sec. 3.3, Eq. smoothint).
__global__ void k_tangents(const MembraneOp op, double* __restrict__ t6, double* __restrict__ w,
                           double* __restrict__ Wraw) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t N = op.N;
  if (i >= N) return;
  for (int c = 0; c < 3; ++c) {
    t6[c * N + i] = op.gu[c * N + i];
    t6[(3 + c) * N + i] = op.gv[c * N + i];
  }
  if (w || Wraw) {
    const Frame fr = frame_at(t6, N, i);
    if (w) w[i] = op.psi_own[i] * fr.W * op.h * op.h;
    if (Wraw) Wraw[i] = fr.W;
  }
}

// Lambda of Eq. tensor into op.g as 6 fields (xx, yy, zz, xy, xz, yz).
// V^2 = F_s F_s^T = (G_r a1 a1^T - F_r (a1 a2^T + a2 a1^T) + E_r a2 a2^T) / W_r^2
// (F_s = a1 (x) a^1_r + a2 (x) a^2_r with the dual reference basis), so
// I1 = tr V^2 - 2, I2 = (W / W_r)^2 - 1, J_s = W / W_r.
__global__ void k_tension(const MembraneOp op, const double* __restrict__ cur,
                          const double* __restrict__ ref, double Es, double ED) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t N = op.N;
  if (i >= N) return;
  const Frame c = frame_at(cur, N, i), r = frame_at(ref, N, i);
  const double iw2 = 1.0 / (r.W * r.W);
  const double tr = (r.G * c.E - 2.0 * r.F * c.F + r.E * c.G) * iw2;
  const double Js = c.W / r.W;
  const double I1 = tr - 2.0, I2 = Js * Js - 1.0;
  const double k1 = Es / (2.0 * Js) * (I1 + 1.0), k2 = 0.5 * Js * (ED * I2 - Es);
  const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
  for (int q = 0; q < 6; ++q) {
    const int a = ia[q], b = ib[q];
    const double V2 = (r.G * c.a1[a] * c.a1[b] - r.F * (c.a1[a] * c.a2[b] + c.a2[a] * c.a1[b]) +
                       r.E * c.a2[a] * c.a2[b]) *
                      iw2;
    const double P = (a == b ? 1.0 : 0.0) - c.n[a] * c.n[b];
    op.g[q * N + i] = k1 * V2 + k2 * P;
  }
}

// f_k = div_gamma Lambda[:, k] = sum_i ((G L_u - F L_v)/W^2 a1 + (E L_v - F L_u)/W^2 a2)_i
// (Appendix, Table diff_formulas; Eq. intf), from the F = 6 pass on Lambda.
__global__ void k_divergence(const MembraneOp op, const double* __restrict__ cur,
                             double* __restrict__ f) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t N = op.N;
  if (i >= N) return;
  const Frame c = frame_at(cur, N, i);
  const double iw2 = 1.0 / (c.W * c.W);
  const int comp[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
  for (int k = 0; k < 3; ++k) {
    double acc = 0.0;
    for (int a = 0; a < 3; ++a) {
      const int q = comp[a][k];
      const double lu = op.gu[q * N + i], lv = op.gv[q * N + i];
      acc += ((c.G * lu - c.F * lv) * c.a1[a] + (c.E * lv - c.F * lu) * c.a2[a]) * iw2;
    }
    f[3 * i + k] = acc;
  }
}

// Area and volume terms (Sec. 4.1): w = psi W h^2, w and w x n_x, summed per
// block in a fixed order.
__global__ void k_area_volume(const MembraneOp op, const double* __restrict__ X,
                              const double* __restrict__ cur, double* __restrict__ part) {
  __shared__ double sa[256], sv[256];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double a = 0.0, v = 0.0;
  if (i < op.N) {
    const Frame c = frame_at(cur, op.N, i);
    const double w = op.psi_own[i] * c.W * op.h * op.h;
    a = w;
    v = w * X[3 * i] * c.n[0];
  }
  sa[threadIdx.x] = a;
  sv[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sa[threadIdx.x] += sa[threadIdx.x + o];
      sv[threadIdx.x] += sv[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sa[0];
    part[2 * blockIdx.x + 1] = sv[0];
  }
}

// Shape moments by the divergence theorem, POU quadrature (Sec. 3.3), with
// x taken relative to an origin o near the body (the node mean): A = int 1,
// V = int x n_x (Sec. 4.1), int_V x_i = (1/4) int x_i (x.n),
// int_V x_i x_j = (1/5) int x_i x_j (x.n); per block, fixed order, 13 sums.
// (About the coordinate origin, the central second moments of a body far from
// it would cancel catastrophically.)
constexpr int N_MOM = 13;
__global__ void k_node_mean(const double* __restrict__ X, int64_t N, double* __restrict__ o) {
  __shared__ double sm[3][256];
  const int t = threadIdx.x;
  double v[3] = {0.0, 0.0, 0.0};
  for (int64_t i = t; i < N; i += 256)
    for (int a = 0; a < 3; ++a) v[a] += X[3 * i + a];
  for (int a = 0; a < 3; ++a) sm[a][t] = v[a];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (t < s)
      for (int a = 0; a < 3; ++a) sm[a][t] += sm[a][t + s];
    __syncthreads();
  }
  if (t == 0)
    for (int a = 0; a < 3; ++a) o[a] = sm[a][0] / (double)N;
}

__global__ void k_moments(const MembraneOp op, const double* __restrict__ X,
                          const double* __restrict__ cur, const double* __restrict__ o,
                          double* __restrict__ part) {
  __shared__ double sm[N_MOM][128];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double v[N_MOM] = {};
  if (i < op.N) {
    const Frame c = frame_at(cur, op.N, i);
    const double w = op.psi_own[i] * c.W * op.h * op.h;
    const double x[3] = {X[3 * i] - o[0], X[3 * i + 1] - o[1], X[3 * i + 2] - o[2]};
    const double xn = x[0] * c.n[0] + x[1] * c.n[1] + x[2] * c.n[2];
    v[0] = w;
    v[1] = w * x[0] * c.n[0];
    for (int a = 0; a < 3; ++a) v[2 + a] = 0.25 * w * x[a] * xn;
    int q = 5;
    for (int a = 0; a < 3; ++a)
      for (int b = a; b < 3; ++b) v[q++] = 0.2 * w * x[a] * x[b] * xn;
  }
  for (int q = 0; q < N_MOM; ++q) sm[q][threadIdx.x] = v[q];
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int q = 0; q < N_MOM; ++q) sm[q][threadIdx.x] += sm[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < N_MOM; ++q) part[(int64_t)blockIdx.x * N_MOM + q] = sm[q][0];
}

__global__ void k_sum_moments(const double* __restrict__ part, int nb, double* __restrict__ out) {
  const int q = threadIdx.x;
  if (q >= N_MOM || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[(int64_t)b * N_MOM + q];
  out[q] = s;
}

__global__ void k_sum_pairs(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double a = 0.0, v = 0.0;
  for (int b = 0; b < n; ++b) {
    a += part[2 * b];
    v += part[2 * b + 1];
  }
  out[0] = a;
  out[1] = v;
}

// Upsampling I_u (Sec. 3.4): the patch splines of the 7 fields in op.g
// (x, y, z, f_x, f_y, f_z, W) at the fine nodes; writes fine positions and
// densities [Nup][3] and weights psi_u W_u h_u^2.
__global__ void k_upsample(const MembraneOp op, double hu2) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= op.Nup) return;
  const int64_t nf2 = (int64_t)op.nf * op.nf;
  const int p = (int)(i / nf2);
  const int r = (int)(i % nf2);
  const int J = r / op.nf, K = r % op.nf;
  double w[8];
  for (int c = 0; c < 4; ++c) {
    w[c] = op.ubasis1[4 * J + c];
    w[4 + c] = op.ubasis1[4 * K + c];
  }
  const int cell = (p * op.n + op.ucell1[J]) * op.n + op.ucell1[K];
  const int64_t plane = 7 * op.N;
  double v[7];
  for (int f = 0; f < 7; ++f) v[f] = spline_tap(op.g, op.sg, plane, (int64_t)f * op.N, cell, op.n, w);
  for (int c = 0; c < 3; ++c) {
    op.Xu[3 * i + c] = v[c];
    op.Fu[3 * i + c] = v[3 + c];
  }
  op.wu[i] = op.psi_up[i] * v[6] * hu2;
}

// delta_u per patch: Eq. regparam on the fine grid (largest distance from a
// node to an existing grid neighbour, maximized over the patch).
__global__ void k_fine_delta(const MembraneOp op) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= op.Nup) return;
  const int nf = op.nf;
  const int p = (int)(i / ((int64_t)nf * nf));
  const int r = (int)(i % ((int64_t)nf * nf));
  const int j = r / nf, k = r % nf;
  const double x = op.Xu[3 * i], y = op.Xu[3 * i + 1], z = op.Xu[3 * i + 2];
  double best = 0.0;
  for (int a = -1; a <= 1; ++a)
    for (int b = -1; b <= 1; ++b) {
      const int jj = j + a, kk = k + b;
      if ((a == 0 && b == 0) || jj < 0 || jj >= nf || kk < 0 || kk >= nf) continue;
      const int64_t q = ((int64_t)p * nf + jj) * nf + kk;
      const double dx = x - op.Xu[3 * q], dy = y - op.Xu[3 * q + 1], dz = z - op.Xu[3 * q + 2];
      best = fmax(best, sqrt(dx * dx + dy * dy + dz * dz));
    }
  // nonnegative doubles order like their bit patterns
  atomicMax(op.pmax + p, (unsigned long long)__double_as_longlong(best));
}

__global__ void k_delta_targets(const MembraneOp op) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < op.N) op.dtgt[i] = __longlong_as_double((long long)op.pmax[i / ((int64_t)op.n * op.n)]);
}

void free_op(MembraneOp* op) {
  if (!op) return;
  for (MembraneOp* c : op->sets) free_op(c);
  for (void* p : {(void*)op->g, (void*)op->sg, (void*)op->ext, (void*)op->du, (void*)op->dv,
                  (void*)op->sdu, (void*)op->sdv, (void*)op->gu, (void*)op->gv, (void*)op->cur_t,
                  (void*)op->red})
    if (p) cudaFree(p);
  if (op->owns_tables)
    for (void* p : {(void*)op->ghost_dst, (void*)op->gtap_ptr, (void*)op->gtap_cell,
                    (void*)op->gtap_w, (void*)op->psi_own, (void*)op->btap_ptr,
                    (void*)op->btap_cell, (void*)op->btap_w, (void*)op->thomas, (void*)op->ucell1,
                    (void*)op->ubasis1, (void*)op->psi_up, (void*)op->Xu, (void*)op->Fu,
                    (void*)op->wu, (void*)op->Xc, (void*)op->Wc, (void*)op->fc, (void*)op->uc,
                    (void*)op->dtgt, (void*)op->pmax})
      if (p) cudaFree(p);
  delete op;
}

// The scratch of up to MEM_FMAX fields (values, spline data, extended
// blocks, derivatives, tangents, reduction partials).
cudaError_t alloc_scratch(MembraneOp* op) {
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  const int E = op->E;
  const size_t fn = (size_t)MEM_FMAX * op->N * sizeof(double);
  ok(cudaMalloc(&op->g, fn));
  ok(cudaMalloc(&op->sg, 3 * fn));
  ok(cudaMalloc(&op->ext, (size_t)MEM_FMAX * 6 * E * E * sizeof(double)));
  ok(cudaMalloc(&op->du, fn));
  ok(cudaMalloc(&op->dv, fn));
  ok(cudaMalloc(&op->sdu, 3 * fn));
  ok(cudaMalloc(&op->sdv, 3 * fn));
  ok(cudaMalloc(&op->gu, fn));
  ok(cudaMalloc(&op->gv, fn));
  ok(cudaMalloc(&op->cur_t, 6 * op->N * sizeof(double)));
  ok(cudaMalloc(&op->red, (13 * (((size_t)op->N + 127) / 128) + 16) * sizeof(double)));
  return e;
}

template <class T>
cudaError_t upload(T** dst, const std::vector<T>& v) {
  cudaError_t e = cudaMalloc(dst, (v.empty() ? 1 : v.size()) * sizeof(T));
  if (e == cudaSuccess && !v.empty())
    e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

// Host construction of the operator tables for grid order m.
int build_op(int m, MembraneOp** out, std::string& err) {
  MembraneOp* op = new (std::nothrow) MembraneOp();
  if (!op) return SK_ENOMEM;
  op->m = m;
  op->n = m - 1;
  op->E = m + 5;
  op->N = 6LL * op->n * op->n;
  op->h = PI_CONST / m;
  op->ih = m / PI_CONST;
  const int n = op->n, E = op->E;
  const double h = op->h;
  // ghost taps (Eq. ext): ghost points with exactly one index outside 1..m-1
  std::vector<int> gdst, gptr{0}, gcell;
  std::vector<double> gw;
  for (int p = 0; p < 6; ++p)
    for (int j = -2; j <= m + 2; ++j)
      for (int k = -2; k <= m + 2; ++k) {
        const bool ij = j >= 1 && j <= m - 1, ik = k >= 1 && k <= m - 1;
        if (ij == ik) continue;  // interior node or corner block (no stencil uses it)
        const D3 x1 = h_chart(p, j * h, k * h);
        double psi[6];
        h_pou(x1, psi);
        for (int q = 0; q < 6; ++q) {
          if (!(psi[q] > 0.0)) continue;
          double uq, vq, bs[8];
          h_inverse_chart(q, x1, uq, vq);
          gcell.push_back(h_cell_basis(q, n, h, uq, vq, bs));
          gw.insert(gw.end(), bs, bs + 8);
          gw.push_back(psi[q]);
        }
        gptr.push_back((int)gcell.size());
        gdst.push_back((p * E + j + 2) * E + k + 2);
      }
  op->G = (int)gdst.size();
  // blend taps (Eqs. blendu / blendv)
  std::vector<double> pown(op->N), bw;
  std::vector<int> bptr{0}, bcell;
  for (int p = 0; p < 6; ++p)
    for (int j = 1; j <= m - 1; ++j)
      for (int k = 1; k <= m - 1; ++k) {
        const double u = j * h, v = k * h;
        const D3 x0 = h_chart(p, u, v);
        double psi[6];
        h_pou(x0, psi);
        pown[((int64_t)p * n + j - 1) * n + k - 1] = psi[p];
        for (int q = 0; q < 6; ++q) {
          if (q == p || !(psi[q] > 0.0)) continue;
          double uq, vq, J[4], bs[8];
          h_inverse_chart(q, x0, uq, vq);
          h_transition_jacobian(p, q, u, v, uq, vq, J);
          bcell.push_back(h_cell_basis(q, n, h, uq, vq, bs));
          bw.insert(bw.end(), bs, bs + 8);
          bw.insert(bw.end(), {psi[q], J[0], J[1], J[2], J[3]});
        }
        bptr.push_back((int)bcell.size());
      }
  // factorization of the reduced slope system: rows q = 1..n-2 with
  // (sub, diag, super) = (-, 2, 1), (1, 4, 1) ..., (1, 2, -); then the
  // 3/h * 1/den and the products of each lane run's multipliers (k_slopes)
  std::vector<double> th(3 * n + SLOPE_TABLE_EXTRA, 0.0);
  for (int q = 1; q <= n - 2; ++q) {
    const double b = (q == 1 || q == n - 2) ? 2.0 : 4.0;
    const double a = q == 1 ? 0.0 : 1.0;
    const double c = q == n - 2 ? 0.0 : 1.0;
    const double den = b - a * (q > 1 ? th[q - 1] : 0.0);
    th[q] = c / den;
    th[n + q] = 1.0 / den;
  }
  {
    const double i3h = 3.0 / h;
    for (int q = 1; q <= n - 2; ++q) th[2 * n + q] = i3h * th[n + q];
    for (int L = SLOPE_LPL_MIN; L <= SLOPE_LPL_MAX; L *= 2) {
      const int K = (n - 2 + L - 1) / L, off = slope_products_offset(n, L);
      for (int r = 0; r < L; ++r) {
        const int qa = 1 + r * K, qb = std::min(qa + K, n - 1);
        double pf = 1.0, pb = 1.0;
        for (int q = qa; q < qb; ++q) pf *= q == 1 ? 0.0 : -th[n + q];
        for (int p = qa; p < qb; ++p) {
          const int q = n - 1 - p;
          pb *= q == n - 2 ? 0.0 : -th[q];
        }
        th[off + r] = pf;
        th[off + L + r] = pb;
      }
    }
  }
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (x != cudaSuccess && e == cudaSuccess) e = x;
  };
  ok(upload(&op->ghost_dst, gdst));
  ok(upload(&op->gtap_ptr, gptr));
  ok(upload(&op->gtap_cell, gcell));
  ok(upload(&op->gtap_w, gw));
  ok(upload(&op->psi_own, pown));
  ok(upload(&op->btap_ptr, bptr));
  ok(upload(&op->btap_cell, bcell));
  ok(upload(&op->btap_w, bw));
  ok(upload(&op->thomas, th));
  ok(alloc_scratch(op));
  if (e != cudaSuccess) {
    err = std::string("membrane operator: ") + cudaGetErrorString(e);
    free_op(op);
    return e == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA;
  }
  *out = op;
  return SK_OK;
}

// Tables and buffers of the upsampled single layer (host work: the POU at
// every fine node, one thread per patch).
int ensure_upsampling(MembraneOp* op, std::string& err) {
  if (op->Xu) return SK_OK;
  const int m = op->m, n = op->n, nf = 4 * m - 1;
  const double h = op->h, hf = PI_CONST / (4.0 * m);
  std::vector<int> cell(nf);
  std::vector<double> basis(4 * (size_t)nf);
  for (int J = 0; J < nf; ++J) {
    double bs[8];
    const double u = (J + 1) * hf;
    cell[J] = h_cell_basis(0, n, h, u, u, bs) / n;  // a of the cell (patch 0, b = a)
    for (int c = 0; c < 4; ++c) basis[4 * J + c] = bs[c];
  }
  const int64_t nf2 = (int64_t)nf * nf, Nup = 6 * nf2;
  std::vector<double> psi(Nup);
  std::vector<std::thread> th;
  for (int p = 0; p < 6; ++p)
    th.emplace_back([&, p] {
      for (int J = 0; J < nf; ++J)
        for (int K = 0; K < nf; ++K) {
          double ps[6];
          h_pou(h_chart(p, (J + 1) * hf, (K + 1) * hf), ps);
          psi[p * nf2 + (int64_t)J * nf + K] = ps[p];
        }
    });
  for (auto& t : th) t.join();
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (x != cudaSuccess && e == cudaSuccess) e = x;
  };
  ok(upload(&op->ucell1, cell));
  ok(upload(&op->ubasis1, basis));
  ok(upload(&op->psi_up, psi));
  ok(cudaMalloc(&op->Xu, 3 * Nup * sizeof(double)));
  ok(cudaMalloc(&op->Fu, 3 * Nup * sizeof(double)));
  ok(cudaMalloc(&op->wu, Nup * sizeof(double)));
  ok(cudaMalloc(&op->Xc, 3 * op->N * sizeof(double)));
  ok(cudaMalloc(&op->Wc, op->N * sizeof(double)));
  ok(cudaMalloc(&op->fc, 3 * op->N * sizeof(double)));
  ok(cudaMalloc(&op->uc, 3 * op->N * sizeof(double)));
  ok(cudaMalloc(&op->dtgt, op->N * sizeof(double)));
  ok(cudaMalloc(&op->pmax, 8 * sizeof(unsigned long long)));
  if (e != cudaSuccess) {
    err = std::string("upsampled single layer: ") + cudaGetErrorString(e);
    for (double** q : {&op->Xu, &op->Fu, &op->wu, &op->Xc, &op->Wc, &op->fc, &op->uc, &op->dtgt})
      if (*q) {
        cudaFree(*q);
        *q = nullptr;
      }
    return e == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA;
  }
  op->nf = nf;
  op->Nup = Nup;
  return SK_OK;
}

#ifndef SK_SLOPE_LANES
#define SK_SLOPE_LANES 0  // 0: by size (below); 8, 16 or 32: fixed
#endif
// Lanes per line by line length n, as measured for the membrane force (8 /
// 16 / 32 lanes): m = 65: 0.54 / 0.46 / 0.50 ms; m = 129: 1.00 / 0.95 /
// 1.09 ms; m = 257: 2.71 / 3.24 / 2.97 ms (32 lanes was the earlier kernel's
// layout: 0.55, 1.30, 3.62 ms with its redundant arithmetic).
inline int slope_lanes(int n) {
  if (SK_SLOPE_LANES) return SK_SLOPE_LANES;
  return n <= 160 ? 16 : 8;
}

// Spline data (u, v, uv slopes) of F fields in `val` into `sd` ([3][F][N]).
void enqueue_splines(const MembraneOp& op, int F, const double* val, double* sd, cudaStream_t st) {
  const int64_t plane = (int64_t)F * op.N;
  const int64_t lines = (int64_t)F * 6 * op.n;
  const int L = slope_lanes(op.n);
  const unsigned nb = (unsigned)((lines + SLOPE_LINES - 1) / SLOPE_LINES);
  // staged lines: 2 arrays x SLOPE_LINES lines x spad(n) doubles, within the
  // default 48 KB of dynamic shared memory (lines up to n = 341)
  const size_t smem = 2 * (size_t)SLOPE_LINES * (op.n + (op.n >> 3)) * sizeof(double);
  const bool staged = op.slope_staging && smem <= 48 * 1024;
  auto run = [&](const double* in, double* out, int dir) {
    const unsigned T = (unsigned)(SLOPE_LINES * L);
    if (staged) {
      if (L == 8)
        k_slopes<8, true><<<nb, T, smem, st>>>(in, out, lines, op.n, dir, op.ih, op.thomas);
      else if (L == 16)
        k_slopes<16, true><<<nb, T, smem, st>>>(in, out, lines, op.n, dir, op.ih, op.thomas);
      else
        k_slopes<32, true><<<nb, T, smem, st>>>(in, out, lines, op.n, dir, op.ih, op.thomas);
    } else {
      if (L == 8)
        k_slopes<8, false><<<nb, T, 0, st>>>(in, out, lines, op.n, dir, op.ih, op.thomas);
      else if (L == 16)
        k_slopes<16, false><<<nb, T, 0, st>>>(in, out, lines, op.n, dir, op.ih, op.thomas);
      else
        k_slopes<32, false><<<nb, T, 0, st>>>(in, out, lines, op.n, dir, op.ih, op.thomas);
    }
  };
  run(val, sd, 0);
  run(val, sd + plane, 1);
  run(sd, sd + 2 * plane, 1);
}

}  // namespace

// The scheme of Sec. 3.5 on F <= MEM_FMAX fields already in op->g ([F][N]);
// blended derivatives land in op->gu, op->gv.
void enqueue_derivatives(const MembraneOp& op, int F, cudaStream_t st) {
  enqueue_splines(op, F, op.g, op.sg, st);
  k_extend<<<blocks_of((int64_t)F * (op.N + op.G)), 256, 0, st>>>(op, F);
  k_fd<<<blocks_of((int64_t)F * op.N), 256, 0, st>>>(op, F);
  enqueue_splines(op, F, op.du, op.sdu, st);
  enqueue_splines(op, F, op.dv, op.sdv, st);
  k_blend<<<blocks_of((int64_t)F * op.N), 256, 0, st>>>(op, F);
}

// Tangents of the nodes X ([N][3], device) into t6 ([6][N]; the operator's
// own buffer when null); weights psi W h^2 into w when w != nullptr.
void enqueue_tangents(const MembraneOp& op, const double* X, double* t6, double* w,
                      cudaStream_t st, double* Wraw) {
  if (!t6) t6 = op.cur_t;
  k_gather<<<blocks_of(3 * op.N), 256, 0, st>>>(X, op.N, 3, 0, 3, op.g);
  enqueue_derivatives(op, 3, st);
  k_tangents<<<blocks_of(op.N), 256, 0, st>>>(op, t6, w, Wraw);
}

// Skalak force f ([N][3]) at X given reference tangents ref6 ([6][N]).
void enqueue_skalak(const MembraneOp& op, const double* X, const double* ref6, double Es,
                    double ED, double* f, double* w, cudaStream_t st, double* Wraw) {
  enqueue_tangents(op, X, op.cur_t, w, st, Wraw);
  k_tension<<<blocks_of(op.N), 256, 0, st>>>(op, op.cur_t, ref6, Es, ED);
  enqueue_derivatives(op, 6, st);
  k_divergence<<<blocks_of(op.N), 256, 0, st>>>(op, op.cur_t, f);
}

// Area and volume of the nodes X into out2 (device, 2 doubles).
void enqueue_area_volume(const MembraneOp& op, const double* X, double* out2, cudaStream_t st) {
  enqueue_tangents(op, X, op.cur_t, nullptr, st);
  const unsigned nb = blocks_of(op.N);
  k_area_volume<<<nb, 256, 0, st>>>(op, X, op.cur_t, op.red);
  k_sum_pairs<<<1, 32, 0, st>>>(op.red, (int)nb, out2);
}

int64_t membrane_nodes(const MembraneOp& op) { return op.N; }

// Origin o (node mean, 3) followed by A, V, int_V x (3), int_V x_a x_b
// (a <= b, 6), x relative to o, of the nodes X into out16.
void enqueue_moments(const MembraneOp& op, const double* X, double* out16, cudaStream_t st) {
  enqueue_tangents(op, X, op.cur_t, nullptr, st);
  const unsigned nb = (unsigned)((op.N + 127) / 128);
  k_node_mean<<<1, 256, 0, st>>>(X, op.N, out16);
  k_moments<<<nb, 128, 0, st>>>(op, X, op.cur_t, out16, op.red);
  k_sum_moments<<<1, 32, 0, st>>>(op.red, (int)nb, out16 + 3);
}

int membrane_upsampling(sk_ctx* ctx, MembraneOp* op) { return ensure_upsampling(op, ctx->err); }

// I_u of the nodes X, area elements W and densities f (device) into the
// operator's fine sources, and delta_u per coarse target (Sec. 3.4).
void enqueue_upsample(const MembraneOp& op, const double* X, const double* W, const double* f,
                      cudaStream_t st) {
  const int64_t N = op.N;
  k_gather<<<blocks_of(3 * N), 256, 0, st>>>(X, N, 3, 0, 3, op.g);
  k_gather<<<blocks_of(3 * N), 256, 0, st>>>(f, N, 3, 0, 3, op.g + 3 * N);
  k_gather<<<blocks_of(N), 256, 0, st>>>(W, N, 1, 0, 1, op.g + 6 * N);
  enqueue_splines(op, 7, op.g, op.sg, st);
  const double hu = PI_CONST / (4.0 * op.m);
  k_upsample<<<blocks_of(op.Nup), 256, 0, st>>>(op, hu * hu);
  cudaMemsetAsync(op.pmax, 0, 8 * sizeof(unsigned long long), st);
  k_fine_delta<<<blocks_of(op.Nup), 256, 0, st>>>(op);
  k_delta_targets<<<blocks_of(N), 256, 0, st>>>(op);
}

UpsampledSources upsampled_sources(const MembraneOp& op) {
  return {op.Nup, op.Xu, op.wu, op.Fu, op.dtgt, op.Wc};
}

// The context's operator for grid order m (built on first use).
int membrane_op(sk_ctx* ctx, int m, MembraneOp** out) {
  for (auto& kv : ctx->membrane_ops)
    if (kv.first == m) {
      *out = kv.second;
      return SK_OK;
    }
  if (m < 6 || m > 4097) {
    ctx->err = "membrane: need 6 <= m <= 4097";
    return SK_EINVAL;
  }
  cudaSetDevice(ctx->device);
  MembraneOp* op = nullptr;
  const int rc = build_op(m, &op, ctx->err);
  if (rc != SK_OK) return rc;
  // SK_SLOPE_STAGING=0 in the environment keeps the slope solves in global
  // memory (same arithmetic, same results: a test compares the two)
  if (const char* v = std::getenv("SK_SLOPE_STAGING")) op->slope_staging = std::strcmp(v, "0") != 0;
  ctx->membrane_ops.push_back({m, op});
  *out = op;
  return SK_OK;
}

// Scratch copy i (0 <= i < MEM_SCRATCH_SETS) of op: op's tables, its own
// scratch. Built on first use; the copies live as long as op.
int membrane_scratch_set(sk_ctx* ctx, MembraneOp* op, int i, MembraneOp** out) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  if (i < 0 || i >= MEM_SCRATCH_SETS) return SK_EINVAL;
  if (!op->sets[i]) {
    MembraneOp* c = new (std::nothrow) MembraneOp(*op);
    if (!c) return SK_ENOMEM;
    c->owns_tables = false;
    for (MembraneOp*& q : c->sets) q = nullptr;
    c->g = c->sg = c->ext = c->du = c->dv = c->sdu = c->sdv = c->gu = c->gv = c->cur_t =
        c->red = nullptr;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    const cudaError_t e = alloc_scratch(c);
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    if (e != cudaSuccess) {
      free_op(c);
      ctx->err = std::string("membrane scratch: ") + cudaGetErrorString(e);
      return e == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA;
    }
    op->sets[i] = c;
  }
  *out = op->sets[i];
  return SK_OK;
}

void free_membrane_ops(sk_ctx* ctx) {
  for (auto& kv : ctx->membrane_ops) free_op(kv.second);
  ctx->membrane_ops.clear();
}

}  // namespace sk

using namespace sk;

extern "C" {

int surface_derivatives(sk_ctx* ctx, int m, int mem, int64_t n_fields, const double* g,
                        double* g_u, double* g_v, void* stream) {
  if (!ctx) return SK_EINVAL;
  if (n_fields < 1 || n_fields > (1 << 20) || !g || !g_u || !g_v ||
      (mem != SK_HOST && mem != SK_DEVICE)) {
    ctx->err = "surface_derivatives: need n_fields >= 1, g, g_u, g_v and mem SK_HOST or SK_DEVICE";
    return SK_EINVAL;
  }
  MembraneOp* op = nullptr;
  int rc = membrane_op(ctx, m, &op);
  if (rc != SK_OK) return rc;
  cudaSetDevice(ctx->device);
  cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
  const int64_t N = op->N;
  const size_t bytes = (size_t)N * n_fields * sizeof(double);
  const double* dg = g;
  double *du = g_u, *dv = g_v;
  if (mem == SK_HOST) {
    rc = ensure_workspace(ctx, 3 * bytes + 1024);
    if (rc != SK_OK) return rc;
    double* w = (double*)ctx->ws;
    const size_t off = (bytes + 255) / 256 * 256 / sizeof(double);
    cudaMemcpyAsync(w, g, bytes, cudaMemcpyHostToDevice, st);
    dg = w;
    du = w + off;
    dv = w + 2 * off;
  }
  for (int64_t c0 = 0; c0 < n_fields; c0 += MEM_FMAX) {
    const int F = (int)std::min<int64_t>(MEM_FMAX, n_fields - c0);
    k_gather<<<blocks_of(F * N), 256, 0, st>>>(dg, N, (int)n_fields, (int)c0, F, op->g);
    enqueue_derivatives(*op, F, st);
    k_scatter<<<blocks_of(F * N), 256, 0, st>>>(op->gu, N, (int)n_fields, (int)c0, F, du);
    k_scatter<<<blocks_of(F * N), 256, 0, st>>>(op->gv, N, (int)n_fields, (int)c0, F, dv);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && mem == SK_HOST) {
    cudaMemcpyAsync(g_u, du, bytes, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(g_v, dv, bytes, cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess && (mem == SK_HOST || !stream)) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    ctx->err = std::string("surface_derivatives: ") + cudaGetErrorString(e);
    return SK_ECUDA;
  }
  return SK_OK;
}

int membrane_force(sk_ctx* ctx, int m, int mem, const double* X, const double* X_ref, double Es,
                   double ED, double* f_out, double* w_out, void* stream) {
  if (!ctx) return SK_EINVAL;
  if (!X || !X_ref || !f_out || (mem != SK_HOST && mem != SK_DEVICE) ||
      !(Es >= 0.0 && Es < INFINITY) || !(ED >= 0.0 && ED < INFINITY)) {
    ctx->err = "membrane_force: need X, X_ref, f_out, finite Es, ED >= 0 and mem SK_HOST or SK_DEVICE";
    return SK_EINVAL;
  }
  MembraneOp* op = nullptr;
  int rc = membrane_op(ctx, m, &op);
  if (rc != SK_OK) return rc;
  cudaSetDevice(ctx->device);
  cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
  const int64_t N = op->N;
  const size_t b3 = 3 * (size_t)N * sizeof(double), b1 = (size_t)N * sizeof(double);
  const size_t pad = 256;
  rc = ensure_workspace(ctx, 3 * (b3 + pad) + 6 * b1 + b1 + 4 * pad);
  if (rc != SK_OK) return rc;
  Bump bp;
  bp.base = ctx->ws;
  double* ref6 = bp.take<double>(6 * (size_t)N);
  const double* dX = X;
  const double* dXr = X_ref;
  double* df = f_out;
  double* dw = w_out;
  if (mem == SK_HOST) {
    double* tX = bp.take<double>(3 * (size_t)N);
    double* tXr = bp.take<double>(3 * (size_t)N);
    df = bp.take<double>(3 * (size_t)N);
    dw = w_out ? bp.take<double>((size_t)N) : nullptr;
    cudaMemcpyAsync(tX, X, b3, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(tXr, X_ref, b3, cudaMemcpyHostToDevice, st);
    dX = tX;
    dXr = tXr;
  }
  enqueue_tangents(*op, dXr, ref6, nullptr, st);
  enqueue_skalak(*op, dX, ref6, Es, ED, df, dw, st);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && mem == SK_HOST) {
    cudaMemcpyAsync(f_out, df, b3, cudaMemcpyDeviceToHost, st);
    if (w_out) cudaMemcpyAsync(w_out, dw, b1, cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess && (mem == SK_HOST || !stream)) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    ctx->err = std::string("membrane_force: ") + cudaGetErrorString(e);
    return SK_ECUDA;
  }
  return SK_OK;
}

int stokes_sl_eval_upsampled(sk_ctx* ctx, int precision, int mem, int m, const double* X,
                             const double* W, const double* f, double mu, double* u_out,
                             void* stream) {
  if (!ctx) return SK_EINVAL;
  if (!X || !W || !f || !u_out || (mem != SK_HOST && mem != SK_DEVICE) ||
      (precision != SK_FP64 && precision != SK_FP32C) || !(mu > 0.0 && mu < INFINITY)) {
    ctx->err = "stokes_sl_eval_upsampled: need X, W, f, u_out, mu > 0, precision SK_FP64 or "
               "SK_FP32C and mem SK_HOST or SK_DEVICE";
    return SK_EINVAL;
  }
  MembraneOp* op = nullptr;
  int rc = membrane_op(ctx, m, &op);
  if (rc == SK_OK) rc = ensure_upsampling(op, ctx->err);
  if (rc != SK_OK) return rc;
  cudaSetDevice(ctx->device);
  cudaStream_t st = (mem == SK_DEVICE && stream) ? (cudaStream_t)stream : ctx->stream;
  const int64_t N = op->N;
  const double *dX = X, *dW = W, *df = f;
  if (mem == SK_HOST) {
    cudaMemcpyAsync(op->Xc, X, 3 * N * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(op->Wc, W, N * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(op->fc, f, 3 * N * sizeof(double), cudaMemcpyHostToDevice, st);
    dX = op->Xc;
    dW = op->Wc;
    df = op->fc;
  }
  // I_u of positions, densities and area element
  enqueue_upsample(*op, dX, dW, df, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    ctx->err = std::string("stokes_sl_eval_upsampled: ") + cudaGetErrorString(e);
    return SK_ECUDA;
  }
  // the sum at the coarse nodes over the fine sources; I_d is the identity
  // there (every coarse node is a fine node)
  double* du = mem == SK_HOST ? op->uc : u_out;
  rc = eval_call(ctx, LAYER_SL, precision, SK_DEVICE, op->Nup, op->Xu, op->wu, op->Fu, nullptr, N,
                 dX, op->dtgt, N, mu, du, mem == SK_DEVICE ? (void*)stream : nullptr);
  if (rc != SK_OK) return rc;
  if (mem == SK_HOST) {
    e = cudaMemcpy(u_out, op->uc, 3 * N * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      ctx->err = std::string("stokes_sl_eval_upsampled: ") + cudaGetErrorString(e);
      return SK_ECUDA;
    }
  }
  return SK_OK;
}

}  // extern "C"
