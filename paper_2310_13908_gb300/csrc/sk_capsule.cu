// sk_capsule.cu -- explicit Euler time stepping of a capsule's surface nodes
// (Sec. 3.6, Eq. bi_combined) with the regularized single layer.
//
// The nodes stay resident in device memory. One step is: with a membrane
// (capsule_set_membrane), the quadrature weights psi W h^2 from the current
// tangents and, when no force is supplied, the Skalak force f = div_gamma
// Lambda (Sec. 2.1, Eqs. tensor and intf, by the overset finite differences
// of Sec. 3.5); (optionally) the patch-dependent regularization parameter
// delta* of Eq. regparam; the full single-layer evaluation at all nodes; and
// the update X += dt (S[f](X) + u_inf(X)). The step is captured once into a
// CUDA graph and replayed n_steps times, so a step costs one graph launch on
// the host.
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>

#include "sk_decomp.h"
#include "sk_internal.h"

struct sk_capsule {
  sk_ctx* ctx = nullptr;
  int m = 0;
  int64_t N = 0;
  double* X = nullptr;
  double* w = nullptr;
  double* f = nullptr;
  double* u = nullptr;
  double* delta = nullptr;
  int64_t n_delta = 0;
  bool auto_delta = false;
  unsigned long long* patch_max = nullptr;  // [6] delta* per patch (double bits)
  unsigned long long* sticky = nullptr;     // [N_FLAGS] flags of all steps since the last call
  double mu = 1.0;
  int precision = SK_FP32C;
  // membrane (capsule_set_membrane): reference tangents [6][N] and moduli
  sk::MembraneOp* mop = nullptr;
  double* ref6 = nullptr;
  double Es = 0.0, ED = 0.0;
  double* av = nullptr;  // [2] area, volume (device)
  // four-times upsampled single layer (capsule_set_upsampling)
  int up = 1;
  sk::MembraneOp* uop = nullptr;
  // RKF45 (capsule_integrate_rkf45): stage positions, stage slopes, reductions
  double* Y = nullptr;    // [N][3]
  double* K = nullptr;    // [6][N][3]
  double* red = nullptr;  // block maxima, then [2] (error, |x4|)
  cudaGraphExec_t rhs_exec = nullptr;  // u = u_inf(Y) + S[f(Y)](Y)
  sk_flow r_flow{};
  char* r_ws = nullptr;
  size_t r_ws_bytes = 0;
  double r_rho_T = 0.0, r_rho_c = 0.0;
  int r_mode = -1;
  int r_up = 0;
  // captured step graph and the state it was captured for
  int g_mode = -1;  // 0: supplied f; 1: supplied f, membrane weights; 2: Skalak force
  int g_up = 0;
  cudaGraphExec_t exec = nullptr;
  double g_dt = 0.0;
  sk_flow g_flow{};
  char* g_ws = nullptr;
  size_t g_ws_bytes = 0;
  double g_rho_T = 0.0, g_rho_c = 0.0;
  // held by a served request (serve_submit with this capsule) until it completes
  std::atomic<bool> served{false};
};

namespace sk {
namespace {

inline unsigned blocks(int64_t n) { return (unsigned)((n + 255) / 256); }

// delta*_p = max over the nodes of patch p of the largest distance to an
// existing grid neighbour (offsets a, b in {-1, 0, 1}) (Eq. regparam).
__global__ void k_delta_star_patch(const double* __restrict__ X, int m,
                                   unsigned long long* __restrict__ pmax) {
  const int n = m - 1;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double best = 0.0;
  int p = -1;
  if (i < 6 * (int64_t)n * n) {
    p = (int)(i / ((int64_t)n * n));
    const int r = (int)(i % ((int64_t)n * n));
    const int j = r / n, k = r % n;
    const double x = X[3 * i], y = X[3 * i + 1], z = X[3 * i + 2];
    for (int a = -1; a <= 1; ++a)
      for (int b = -1; b <= 1; ++b) {
        const int jj = j - a, kk = k - b;
        if ((a == 0 && b == 0) || jj < 0 || jj >= n || kk < 0 || kk >= n) continue;
        const int64_t q = (int64_t)p * n * n + (int64_t)jj * n + kk;
        const double dx = x - X[3 * q], dy = y - X[3 * q + 1], dz = z - X[3 * q + 2];
        best = fmax(best, sqrt(dx * dx + dy * dy + dz * dz));
      }
  }
  // nonnegative doubles order like their bit patterns
  if (p >= 0) atomicMax(pmax + p, (unsigned long long)__double_as_longlong(best));
}

__global__ void k_delta_fill(const unsigned long long* __restrict__ pmax, int m, double C,
                             double* __restrict__ delta) {
  const int n = m - 1;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < 6 * (int64_t)n * n) delta[i] = C * __longlong_as_double((long long)pmax[i / ((int64_t)n * n)]);
}

// X += dt (u + u_inf(X)); background flows of Eqs. shear_flow, poiseuille_flow.
__global__ void k_euler(double* __restrict__ X, const double* __restrict__ u, int64_t N, double dt,
                        sk_flow fl) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double x = X[3 * i], y = X[3 * i + 1], z = X[3 * i + 2];
  double ux = u[3 * i], uy = u[3 * i + 1], uz = u[3 * i + 2];
  if (fl.kind == SK_FLOW_SHEAR) ux += fl.rate * y;
  if (fl.kind == SK_FLOW_POISEUILLE) ux += fl.alpha * (fl.R0 * fl.R0 - y * y - z * z);
  X[3 * i] = x + dt * ux;
  X[3 * i + 1] = y + dt * uy;
  X[3 * i + 2] = z + dt * uz;
}

__global__ void k_sticky(const unsigned long long* __restrict__ flags,
                         unsigned long long* __restrict__ sticky) {
  const int i = threadIdx.x;
  if (i < N_FLAGS && flags[i]) atomicOr(sticky + i, flags[i]);
}

// Fehlberg's RK4(5) tableau (Sec. 3.6 names the scheme): stage coefficients,
// fourth-order weights (propagated) and fifth-order weights (error estimate).
__constant__ double RK_A[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0 / 4, 0, 0, 0, 0},
    {3.0 / 32, 9.0 / 32, 0, 0, 0},
    {1932.0 / 2197, -7200.0 / 2197, 7296.0 / 2197, 0, 0},
    {439.0 / 216, -8.0, 3680.0 / 513, -845.0 / 4104, 0},
    {-8.0 / 27, 2.0, -3544.0 / 2565, 1859.0 / 4104, -11.0 / 40}};
__constant__ double RK_B4[6] = {25.0 / 216, 0, 1408.0 / 2565, 2197.0 / 4104, -1.0 / 5, 0};
__constant__ double RK_B5[6] = {16.0 / 135, 0, 6656.0 / 12825, 28561.0 / 56430, -9.0 / 50,
                                2.0 / 55};

// Y = X + dt sum_{j < s} a_sj K_j
__global__ void k_rk_stage(const double* __restrict__ X, const double* __restrict__ K, int s,
                           double dt, int64_t n3, double* __restrict__ Y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n3) return;
  double acc = 0.0;
  for (int j = 0; j < s; ++j) acc += RK_A[s][j] * K[j * n3 + i];
  Y[i] = X[i] + dt * acc;
}

// u += u_inf(Y) (Eqs. shear_flow, poiseuille_flow)
__global__ void k_add_uinf(double* __restrict__ u, const double* __restrict__ Y, int64_t N,
                           sk_flow fl) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double y = Y[3 * i + 1], z = Y[3 * i + 2];
  if (fl.kind == SK_FLOW_SHEAR) u[3 * i] += fl.rate * y;
  if (fl.kind == SK_FLOW_POISEUILLE) u[3 * i] += fl.alpha * (fl.R0 * fl.R0 - y * y - z * z);
}

// Y = X + dt sum b4_j K_j; per block: max |dt sum (b5_j - b4_j) K_j| and max |Y|.
__global__ void k_rk_finish(const double* __restrict__ X, const double* __restrict__ K, double dt,
                            int64_t n3, double* __restrict__ Y, double* __restrict__ part) {
  __shared__ double se[256], sy[256];
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double e = 0.0, a = 0.0;
  if (i < n3) {
    double y4 = 0.0, d = 0.0;
    for (int j = 0; j < 6; ++j) {
      const double k = K[j * n3 + i];
      y4 += RK_B4[j] * k;
      d += (RK_B5[j] - RK_B4[j]) * k;
    }
    const double y = X[i] + dt * y4;
    Y[i] = y;
    e = fabs(dt * d);
    a = fabs(y);
  }
  se[threadIdx.x] = e;
  sy[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      se[threadIdx.x] = fmax(se[threadIdx.x], se[threadIdx.x + o]);
      sy[threadIdx.x] = fmax(sy[threadIdx.x], sy[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = se[0];
    part[2 * blockIdx.x + 1] = sy[0];
  }
}

__global__ void k_max_pairs(const double* __restrict__ part, int n, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double e = 0.0, a = 0.0;
  for (int b = 0; b < n; ++b) {
    e = fmax(e, part[2 * b]);
    a = fmax(a, part[2 * b + 1]);
  }
  out[0] = e;
  out[1] = a;
}

// Shape of the capsule's single-layer evaluation: targets are the nodes;
// sources the nodes, or the fine nodes of the upsampled grid.
EvalShape capsule_shape(const sk_capsule* c) {
  EvalShape s;
  s.layer = LAYER_SL;
  s.precision = c->precision;
  s.mu = c->mu;
  s.copy_inputs = false;
  s.M = c->N;
  if (c->up == 4) {
    s.N = upsampled_sources(*c->uop).Nup;
    s.n_delta = c->N;
  } else {
    s.N = c->N;
    s.n_delta = c->n_delta;
  }
  s.small_sort_points = c->ctx->small_sort_points;
  s.split_sorts = true;  // the step graphs fork the target sort onto a second stream
  choose_decomposition(s, c->ctx->sm_count);
  return s;
}

// Enqueue u = S[f](P) at nodes P (device [N][3]) into c->u: membrane force
// and weights per mode (0: supplied f; 1: supplied f, membrane weights;
// 2: Skalak force), then delta* and the sum, or the upsampled sum.
void enqueue_velocity(sk_capsule* c, const double* P, int mode, const EvalShape& s,
                      cudaStream_t st) {
  sk_ctx* ctx = c->ctx;
  EvalBufs b;
  Bump bp;
  bp.base = ctx->ws;
  carve_eval_buffers(bp, s, b);
  const bool upsampled = c->up == 4;
  double* Wraw = upsampled ? upsampled_sources(*c->uop).W : nullptr;
  if (mode == 1) enqueue_tangents(*c->mop, P, nullptr, c->w, st, Wraw);
  if (mode == 2) enqueue_skalak(*c->mop, P, c->ref6, c->Es, c->ED, c->f, c->w, st, Wraw);
  if (mode == 0 && upsampled) enqueue_tangents(*c->uop, P, nullptr, nullptr, st, Wraw);
  if (upsampled) {
    enqueue_upsample(*c->uop, P, Wraw, c->f, st);
    const UpsampledSources us = upsampled_sources(*c->uop);
    b.src_xyz = us.X;
    b.src_w = us.w;
    b.dens = us.f;
    b.delta = us.delta;
  } else {
    if (c->auto_delta) {
      cudaMemsetAsync(c->patch_max, 0, 8 * sizeof(unsigned long long), st);
      k_delta_star_patch<<<blocks(c->N), 256, 0, st>>>(P, c->m, c->patch_max);
      k_delta_fill<<<blocks(c->N), 256, 0, st>>>(c->patch_max, c->m, 1.0, c->delta);
    }
    b.src_xyz = P;
    b.src_w = c->w;
    b.dens = c->f;
    b.delta = c->delta;
  }
  b.tgt_xyz = P;
  b.u = c->u;
  const PrepFork pf{ctx->aux_stream, ctx->fork_ev, ctx->join_ev};
  enqueue_eval(s, b, ctx->rho_T, ctx->rho_c, st, nullptr, &pf);
  k_sticky<<<1, 32, 0, st>>>(b.flags, c->sticky);
}

}  // namespace

// ---- steps run by the server (sk_serve.cu) ----------------------------------
bool capsule_try_acquire(sk_capsule* c) {
  bool expect = false;
  return c->served.compare_exchange_strong(expect, true);
}
void capsule_release(sk_capsule* c) { c->served = false; }
sk_ctx* capsule_ctx(const sk_capsule* c) { return c->ctx; }
bool capsule_servable(const sk_capsule* c) { return c->precision == SK_FP32C && c->up == 1; }
int64_t capsule_node_count(const sk_capsule* c) { return c->N; }
EvalShape capsule_step_shape(const sk_capsule* c) { return capsule_shape(c); }
const double* capsule_nodes(const sk_capsule* c) { return c->X; }
const unsigned long long* capsule_sticky(const sk_capsule* c) { return c->sticky; }

// The inputs of one step's single layer, enqueued on st: with a membrane the
// weights psi W h^2 and the Skalak force at the current nodes (else the
// capsule's f), delta* when it is automatic; b's inputs and output are
// pointed at the capsule's arrays. The same operations as a capsule_step, with
// the membrane operator's scratch copy `set`, so that the steps of capsules
// of one grid order can be prepared on different streams at once.
int capsule_prepare_sets(sk_capsule* c, int n_sets) {
  if (!c->mop) return SK_OK;
  for (int i = 0; i < n_sets; ++i) {
    MembraneOp* op = nullptr;
    const int rc = membrane_scratch_set(c->ctx, c->mop, i, &op);
    if (rc != SK_OK) return rc;
  }
  return SK_OK;
}

void capsule_enqueue_step_inputs(sk_capsule* c, EvalBufs& b, cudaStream_t st, int set) {
  if (c->mop) {
    MembraneOp* op = nullptr;
    membrane_scratch_set(c->ctx, c->mop, set, &op);  // built by capsule_prepare_sets
    enqueue_skalak(*op, c->X, c->ref6, c->Es, c->ED, c->f, c->w, st);
  }
  if (c->auto_delta) {
    cudaMemsetAsync(c->patch_max, 0, 8 * sizeof(unsigned long long), st);
    k_delta_star_patch<<<blocks(c->N), 256, 0, st>>>(c->X, c->m, c->patch_max);
    k_delta_fill<<<blocks(c->N), 256, 0, st>>>(c->patch_max, c->m, 1.0, c->delta);
  }
  b.src_xyz = c->X;
  b.src_w = c->w;
  b.dens = c->f;
  b.delta = c->delta;
  b.tgt_xyz = c->X;
  b.u = c->u;
}

// After a step's sum: its flags into the capsule's sticky flags, and the
// Euler update X += dt (u + u_inf(X)).
void capsule_enqueue_step_update(sk_capsule* c, const unsigned long long* flags, double dt,
                                 const sk_flow& fl, cudaStream_t st) {
  k_sticky<<<1, 32, 0, st>>>(flags, c->sticky);
  k_euler<<<blocks(c->N), 256, 0, st>>>(c->X, c->u, c->N, dt, fl);
}

void capsule_clear_sticky(sk_capsule* c, cudaStream_t st) {
  cudaMemsetAsync(c->sticky, 0, N_FLAGS * sizeof(unsigned long long), st);
}

namespace {

void free_capsule(sk_capsule* c) {
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->rhs_exec) cudaGraphExecDestroy(c->rhs_exec);
  for (double* p : {c->X, c->w, c->f, c->u, c->delta, c->ref6, c->av, c->Y, c->K, c->red})
    if (p) cudaFree(p);
  if (c->patch_max) cudaFree(c->patch_max);
  if (c->sticky) cudaFree(c->sticky);
  delete c;
}

}  // namespace
}  // namespace sk

using namespace sk;

extern "C" {

int capsule_create(sk_ctx* ctx, sk_capsule** out, int m, const double* X, const double* w,
                   const double* delta, int64_t n_delta, double mu, int precision) {
  if (!ctx || !out) return SK_EINVAL;
  *out = nullptr;
  if (m < 3 || m > 16385 || !X || !w || !(mu > 0.0 && mu < INFINITY) ||
      (precision != SK_FP64 && precision != SK_FP32C)) {
    ctx->err = "capsule_create: need m >= 3, X and w, mu > 0, precision SK_FP64 or SK_FP32C";
    return SK_EINVAL;
  }
  const int64_t N = 6 * (int64_t)(m - 1) * (m - 1);
  if (precision == SK_FP32C && N > FP32C_MAX_SOURCES) {
    ctx->err = "capsule_create: more than 2^25 nodes in SK_FP32C";
    return SK_EINVAL;
  }
  if (N > MAX_POINTS) {
    ctx->err = "capsule_create: more than 2^30 nodes";
    return SK_EINVAL;
  }
  if (delta) {
    if (!(n_delta == 1 || n_delta == N)) {
      ctx->err = "capsule_create: n_delta must be 1 or 6 (m-1)^2";
      return SK_EINVAL;
    }
    for (int64_t i = 0; i < n_delta; ++i)
      if (!(delta[i] > 0.0 && delta[i] < INFINITY)) {
        ctx->err = "capsule_create: delta must be positive and finite";
        return SK_EINVAL;
      }
  }
  cudaSetDevice(ctx->device);
  sk_capsule* c = new (std::nothrow) sk_capsule();
  if (!c) return SK_ENOMEM;
  c->ctx = ctx;
  c->m = m;
  c->N = N;
  c->auto_delta = delta == nullptr;
  c->n_delta = delta ? n_delta : N;
  c->mu = mu;
  c->precision = precision;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (x != cudaSuccess && e == cudaSuccess) e = x;
  };
  ok(cudaMalloc(&c->X, 3 * N * sizeof(double)));
  ok(cudaMalloc(&c->w, N * sizeof(double)));
  ok(cudaMalloc(&c->f, 3 * N * sizeof(double)));
  ok(cudaMalloc(&c->u, 3 * N * sizeof(double)));
  ok(cudaMalloc(&c->delta, c->n_delta * sizeof(double)));
  ok(cudaMalloc(&c->patch_max, 8 * sizeof(unsigned long long)));
  ok(cudaMalloc(&c->sticky, N_FLAGS * sizeof(unsigned long long)));
  if (e == cudaSuccess) {
    ok(cudaMemcpy(c->X, X, 3 * N * sizeof(double), cudaMemcpyHostToDevice));
    ok(cudaMemcpy(c->w, w, N * sizeof(double), cudaMemcpyHostToDevice));
    if (delta) ok(cudaMemcpy(c->delta, delta, n_delta * sizeof(double), cudaMemcpyHostToDevice));
    ok(cudaMemset(c->f, 0, 3 * N * sizeof(double)));
  }
  if (e != cudaSuccess) {
    ctx->err = std::string("capsule_create: ") + cudaGetErrorString(e);
    free_capsule(c);
    return e == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA;
  }
  *out = c;
  return SK_OK;
}

int capsule_step(sk_capsule* c, int n_steps, double dt, const sk_flow* flow, const double* f) {
  if (!c) return SK_EINVAL;
  sk_ctx* ctx = c->ctx;
  if (n_steps < 0 || !(dt > 0.0 && dt < INFINITY) ||
      (flow && (flow->kind < SK_FLOW_NONE || flow->kind > SK_FLOW_POISEUILLE))) {
    ctx->err = "capsule_step: need n_steps >= 0, dt > 0 and a known flow kind";
    return SK_EINVAL;
  }
  if (!f && !c->mop) {
    ctx->err = "capsule_step: f = NULL takes the Skalak force, which needs capsule_set_membrane";
    return SK_ENOTIMPL;
  }
  const int mode = c->mop ? (f ? 1 : 2) : 0;
  if (n_steps == 0) return SK_OK;
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  const sk_flow fl = flow ? *flow : sk_flow{SK_FLOW_NONE, 0.0, 0.0, 0.0};
  cudaError_t e = cudaSuccess;
  if (f) e = cudaMemcpyAsync(c->f, f, 3 * c->N * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return SK_ECUDA;
  const EvalShape s = capsule_shape(c);
  int rc = ensure_workspace(ctx, eval_workspace_bytes(s));
  if (rc != SK_OK) return rc;
  const bool stale = !c->exec || c->g_dt != dt || std::memcmp(&c->g_flow, &fl, sizeof(fl)) != 0 ||
                     c->g_ws != ctx->ws || c->g_ws_bytes != ctx->ws_bytes ||
                     c->g_rho_T != ctx->rho_T || c->g_rho_c != ctx->rho_c || c->g_mode != mode ||
                     c->g_up != c->up;
  if (stale) {
    if (c->exec) cudaGraphExecDestroy(c->exec);
    c->exec = nullptr;
    cudaGraph_t g = nullptr;
    if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
      ctx->err = std::string("capsule_step: capture: ") + cudaGetErrorString(e);
      return SK_ECUDA;
    }
    enqueue_velocity(c, c->X, mode, s, st);
    k_euler<<<blocks(c->N), 256, 0, st>>>(c->X, c->u, c->N, dt, fl);
    e = cudaStreamEndCapture(st, &g);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      c->exec = nullptr;
      ctx->err = std::string("capsule_step: graph: ") + cudaGetErrorString(e);
      return SK_ECUDA;
    }
    c->g_dt = dt;
    c->g_flow = fl;
    c->g_ws = ctx->ws;
    c->g_ws_bytes = ctx->ws_bytes;
    c->g_rho_T = ctx->rho_T;
    c->g_rho_c = ctx->rho_c;
    c->g_mode = mode;
    c->g_up = c->up;
  }
  cudaMemsetAsync(c->sticky, 0, N_FLAGS * sizeof(unsigned long long), st);
  for (int i = 0; i < n_steps; ++i)
    if ((e = cudaGraphLaunch(c->exec, st)) != cudaSuccess) break;
  unsigned long long flags[N_FLAGS] = {};
  if (e == cudaSuccess) e = cudaMemcpyAsync(flags, c->sticky, sizeof(flags), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    ctx->err = std::string("capsule_step: ") + cudaGetErrorString(e);
    return SK_ECUDA;
  }
  ctx->last_stream = st;
  if (flags[FLAG_TIMEOUT]) {
    ctx->err = "capsule_step: a bounded device wait expired";
    return SK_ETIMEOUT;
  }
  if (flags[FLAG_BAD_DELTA]) {
    ctx->err = "capsule_step: delta must be positive and finite";
    return SK_EINVAL;
  }
  return SK_OK;
}

int capsule_integrate_rkf45(sk_capsule* c, double t_end, double* dt_inout, double tol,
                            const sk_flow* flow, const double* f, int64_t max_steps,
                            int64_t* stats_out) {
  if (!c) return SK_EINVAL;
  sk_ctx* ctx = c->ctx;
  if (!dt_inout || !(t_end > 0.0 && t_end < INFINITY) || !(*dt_inout > 0.0 && *dt_inout < INFINITY) ||
      !(tol > 0.0 && tol < 1.0) || max_steps < 1 ||
      (flow && (flow->kind < SK_FLOW_NONE || flow->kind > SK_FLOW_POISEUILLE))) {
    ctx->err = "capsule_integrate_rkf45: need t_end > 0, *dt_inout > 0, 0 < tol < 1, "
               "max_steps >= 1 and a known flow kind";
    return SK_EINVAL;
  }
  if (!f && !c->mop) {
    ctx->err = "capsule_integrate_rkf45: f = NULL takes the Skalak force, which needs "
               "capsule_set_membrane";
    return SK_ENOTIMPL;
  }
  const int mode = c->mop ? (f ? 1 : 2) : 0;
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  const sk_flow fl = flow ? *flow : sk_flow{SK_FLOW_NONE, 0.0, 0.0, 0.0};
  const int64_t n3 = 3 * c->N;
  const unsigned nb = blocks(n3);
  cudaError_t e = cudaSuccess;
  if (!c->Y) e = cudaMalloc(&c->Y, n3 * sizeof(double));
  if (e == cudaSuccess && !c->K) e = cudaMalloc(&c->K, 6 * n3 * sizeof(double));
  if (e == cudaSuccess && !c->red) e = cudaMalloc(&c->red, (2 * (size_t)nb + 2) * sizeof(double));
  if (e == cudaSuccess && f) e = cudaMemcpyAsync(c->f, f, n3 * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    ctx->err = std::string("capsule_integrate_rkf45: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA;
  }
  const EvalShape s = capsule_shape(c);
  int rc = ensure_workspace(ctx, eval_workspace_bytes(s));
  if (rc != SK_OK) return rc;
  // right-hand side graph on the stage positions Y: u = u_inf(Y) + S[f(Y)](Y)
  const bool stale = !c->rhs_exec || std::memcmp(&c->r_flow, &fl, sizeof(fl)) != 0 ||
                     c->r_ws != ctx->ws || c->r_ws_bytes != ctx->ws_bytes ||
                     c->r_rho_T != ctx->rho_T || c->r_rho_c != ctx->rho_c || c->r_mode != mode ||
                     c->r_up != c->up;
  if (stale) {
    if (c->rhs_exec) cudaGraphExecDestroy(c->rhs_exec);
    c->rhs_exec = nullptr;
    cudaGraph_t g = nullptr;
    if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
      ctx->err = std::string("capsule_integrate_rkf45: capture: ") + cudaGetErrorString(e);
      return SK_ECUDA;
    }
    enqueue_velocity(c, c->Y, mode, s, st);
    k_add_uinf<<<blocks(c->N), 256, 0, st>>>(c->u, c->Y, c->N, fl);
    e = cudaStreamEndCapture(st, &g);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->rhs_exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      c->rhs_exec = nullptr;
      ctx->err = std::string("capsule_integrate_rkf45: graph: ") + cudaGetErrorString(e);
      return SK_ECUDA;
    }
    c->r_flow = fl;
    c->r_ws = ctx->ws;
    c->r_ws_bytes = ctx->ws_bytes;
    c->r_rho_T = ctx->rho_T;
    c->r_rho_c = ctx->rho_c;
    c->r_mode = mode;
    c->r_up = c->up;
  }
  // adaptive loop: accept when max|x5 - x4| / max|x4| <= tol, then
  // dt <- dt min(5, max(0.2, 0.9 (tol / err)^(1/5))); the last step lands on t_end
  cudaMemsetAsync(c->sticky, 0, N_FLAGS * sizeof(unsigned long long), st);
  double t = 0.0, dt = *dt_inout;
  int64_t acc = 0, rej = 0;
  while (t < t_end && acc + rej < max_steps) {
    const double hstep = std::fmin(dt, t_end - t);
    for (int sidx = 0; sidx < 6 && e == cudaSuccess; ++sidx) {
      k_rk_stage<<<nb, 256, 0, st>>>(c->X, c->K, sidx, hstep, n3, c->Y);
      if ((e = cudaGraphLaunch(c->rhs_exec, st)) != cudaSuccess) break;
      e = cudaMemcpyAsync(c->K + sidx * n3, c->u, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
    }
    if (e != cudaSuccess) break;
    k_rk_finish<<<nb, 256, 0, st>>>(c->X, c->K, hstep, n3, c->Y, c->red);
    k_max_pairs<<<1, 32, 0, st>>>(c->red, (int)nb, c->red + 2 * nb);
    double h2[2];
    e = cudaMemcpyAsync(h2, c->red + 2 * nb, sizeof(h2), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) break;
    const double err = h2[0] / std::fmax(h2[1], 1e-300);
    if (!(err == err)) {  // NaN: the step blew up
      ctx->err = "capsule_integrate_rkf45: non-finite step";
      return SK_EINVAL;
    }
    if (err <= tol) {
      e = cudaMemcpyAsync(c->X, c->Y, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
      t += hstep;
      ++acc;
    } else {
      ++rej;
    }
    dt = err == 0.0 ? hstep * 5.0 : hstep * std::fmin(5.0, std::fmax(0.2, 0.9 * std::pow(tol / err, 0.2)));
  }
  unsigned long long flags[N_FLAGS] = {};
  if (e == cudaSuccess) e = cudaMemcpyAsync(flags, c->sticky, sizeof(flags), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    ctx->err = std::string("capsule_integrate_rkf45: ") + cudaGetErrorString(e);
    return SK_ECUDA;
  }
  *dt_inout = dt;
  if (stats_out) {
    stats_out[0] = acc;
    stats_out[1] = rej;
  }
  if (flags[FLAG_TIMEOUT]) {
    ctx->err = "capsule_integrate_rkf45: a bounded device wait expired";
    return SK_ETIMEOUT;
  }
  if (flags[FLAG_BAD_DELTA]) {
    ctx->err = "capsule_integrate_rkf45: delta must be positive and finite";
    return SK_EINVAL;
  }
  if (t < t_end) {
    ctx->err = "capsule_integrate_rkf45: max_steps reached before t_end";
    return SK_EAGAIN;
  }
  return SK_OK;
}

int capsule_set_upsampling(sk_capsule* c, int factor) {
  if (!c) return SK_EINVAL;
  sk_ctx* ctx = c->ctx;
  if (factor != 1 && factor != 4) {
    ctx->err = "capsule_set_upsampling: factor must be 1 or 4";
    return SK_EINVAL;
  }
  if (factor == 4) {
    const int64_t n_up = 6 * (int64_t)(4 * c->m - 1) * (4 * c->m - 1);
    if (c->precision == SK_FP32C && n_up > FP32C_MAX_SOURCES) {
      ctx->err = "capsule_set_upsampling: more than 2^25 fine nodes in SK_FP32C";
      return SK_EINVAL;
    }
    if (n_up > MAX_POINTS) {
      ctx->err = "capsule_set_upsampling: more than 2^30 fine nodes";
      return SK_EINVAL;
    }
    MembraneOp* op = nullptr;
    int rc = membrane_op(ctx, c->m, &op);
    if (rc == SK_OK) rc = membrane_upsampling(ctx, op);
    if (rc != SK_OK) return rc;
    c->uop = op;
  }
  c->up = factor;
  return SK_OK;
}

int capsule_set_membrane(sk_capsule* c, const double* X_ref, double Es, double ED) {
  if (!c) return SK_EINVAL;
  sk_ctx* ctx = c->ctx;
  if (!X_ref || !(Es >= 0.0 && Es < INFINITY) || !(ED >= 0.0 && ED < INFINITY)) {
    ctx->err = "capsule_set_membrane: need X_ref and finite Es, ED >= 0";
    return SK_EINVAL;
  }
  MembraneOp* op = nullptr;
  int rc = membrane_op(ctx, c->m, &op);
  if (rc != SK_OK) return rc;
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaSuccess;
  if (!c->ref6) e = cudaMalloc(&c->ref6, 6 * c->N * sizeof(double));
  if (e == cudaSuccess && !c->av) e = cudaMalloc(&c->av, 2 * sizeof(double));
  // the reference nodes pass through u (free between steps)
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->u, X_ref, 3 * c->N * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    enqueue_tangents(*op, c->u, c->ref6, nullptr, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    ctx->err = std::string("capsule_set_membrane: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA;
  }
  c->mop = op;
  c->Es = Es;
  c->ED = ED;
  c->g_mode = -1;  // recapture the step graphs
  c->r_mode = -1;
  return SK_OK;
}

int capsule_area_volume(sk_capsule* c, double* area, double* volume) {
  if (!c || !area || !volume) return SK_EINVAL;
  sk_ctx* ctx = c->ctx;
  MembraneOp* op = nullptr;
  int rc = membrane_op(ctx, c->m, &op);
  if (rc != SK_OK) return rc;
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaSuccess;
  if (!c->av) e = cudaMalloc(&c->av, 2 * sizeof(double));
  double h[2] = {0.0, 0.0};
  if (e == cudaSuccess) {
    enqueue_area_volume(*op, c->X, c->av, st);
    e = cudaMemcpyAsync(h, c->av, sizeof(h), cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    ctx->err = std::string("capsule_area_volume: ") + cudaGetErrorString(e);
    return SK_ECUDA;
  }
  *area = h[0];
  *volume = h[1];
  return SK_OK;
}

int capsule_shape_moments(sk_capsule* c, double* out) {
  if (!c || !out) return SK_EINVAL;
  sk_ctx* ctx = c->ctx;
  MembraneOp* op = nullptr;
  int rc = membrane_op(ctx, c->m, &op);
  if (rc != SK_OK) return rc;
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  double* d = nullptr;
  cudaError_t e = cudaMallocAsync(&d, 16 * sizeof(double), st);
  double mo[16] = {};
  if (e == cudaSuccess) {
    enqueue_moments(*op, c->X, d, st);
    e = cudaMemcpyAsync(mo, d, sizeof(mo), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    ctx->err = std::string("capsule_shape_moments: ") + cudaGetErrorString(e);
    return SK_ECUDA;
  }
  // out: A, V, centroid (3), inertia tensor about the centroid (3 x 3); the
  // moments mo[3..] are about the node mean o = mo[0..2]
  const double* o = mo;
  const double* m = mo + 3;
  const double A = m[0], V = m[1];
  const double cx[3] = {m[2] / V, m[3] / V, m[4] / V};  // centroid - o
  double S[3][3];
  int q = 5;
  for (int a = 0; a < 3; ++a)
    for (int b = a; b < 3; ++b) S[a][b] = S[b][a] = m[q++];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) S[a][b] -= V * cx[a] * cx[b];  // central second moments
  const double tr = S[0][0] + S[1][1] + S[2][2];
  out[0] = A;
  out[1] = V;
  for (int a = 0; a < 3; ++a) out[2 + a] = o[a] + cx[a];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) out[5 + 3 * a + b] = (a == b ? tr : 0.0) - S[a][b];
  return SK_OK;
}

int capsule_get(sk_capsule* c, double* X_out) {
  if (!c || !X_out) return SK_EINVAL;
  cudaSetDevice(c->ctx->device);
  cudaError_t e = cudaMemcpy(X_out, c->X, 3 * c->N * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    c->ctx->err = std::string("capsule_get: ") + cudaGetErrorString(e);
    return SK_ECUDA;
  }
  return SK_OK;
}

void capsule_destroy(sk_capsule* c) {
  if (!c) return;
  cudaSetDevice(c->ctx->device);
  cudaStreamSynchronize(c->ctx->stream);
  free_capsule(c);
}

}  // extern "C"
