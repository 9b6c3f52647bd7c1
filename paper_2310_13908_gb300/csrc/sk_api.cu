// sk_api.cu -- host side of the C ABI: contexts, validation, workspace and
// the launch sequence of one evaluation.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "sk_decomp.h"
#include "sk_internal.h"

namespace {

const char* g_create_error = "";
thread_local std::string g_create_error_buf;

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int fail(sk_ctx* ctx, int code, const char* fmt, const char* detail = "") {
  char buf[512];
  std::snprintf(buf, sizeof(buf), fmt, detail);
  if (ctx) ctx->err = buf;
  return code;
}

int cuda_fail(sk_ctx* ctx, cudaError_t e, const char* where) {
  char buf[512];
  std::snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  ctx->err = buf;
  return e == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA;
}

}  // namespace

namespace sk {

size_t eval_workspace_bytes(const EvalShape& s) {
  EvalBufs b;
  Bump bp;
  carve_eval_buffers(bp, s, b);
  return bp.off;
}

void carve_eval_buffers(Bump& bp, const EvalShape& s, EvalBufs& b) {
  const bool dl = s.layer == LAYER_DL;
  const bool fp32 = s.precision == SK_FP32C;
  b.N = s.N;
  b.M = s.M;
  b.N_pad = (int64_t)align_up((size_t)s.N, TILE);
  b.M_pad = (int64_t)align_up((size_t)s.M, fp32 ? TGT_CTA32 : TGT_CTA64);
  b.n_chunks = s.n_chunks;
  b.pair_np = pair32_np(s.M);
  b.threads64 = s.threads64;
  b.fuse_finish = fp32 && s.fuse_finish;
  const int64_t nsort = s.N > s.M ? s.N : s.M;
  b.sort_blocks = sort_grid_blocks(nsort > 0 ? nsort : 1);
  if (s.copy_inputs) {
    b.src_xyz = bp.take<double>(3 * s.N);
    b.src_w = bp.take<double>(s.N);
    b.dens = bp.take<double>(3 * s.N);
    if (dl) b.nrm = bp.take<double>(3 * s.N);
    b.tgt_xyz = bp.take<double>(3 * s.M);
    b.delta = bp.take<double>(s.n_delta);
    b.u = bp.take<double>(3 * s.M);
  }
  b.keys_a = bp.take<uint32_t>(nsort);
  b.keys_b = bp.take<uint32_t>(nsort);
  b.vals_a = bp.take<int>(nsort);
  b.vals_b = bp.take<int>(nsort);
  b.hist = bp.take<uint32_t>(256 * (size_t)b.sort_blocks + 256);  // + the 256 row totals
  b.bbox_part = bp.take<float>(128 * 6);
  b.bbox = bp.take<float>(8);
  b.meta = bp.take<int>(N_META);
  b.src_orig = bp.take<int>(b.N_pad);
  if (fp32) {
    b.srcF = bp.take<float4>((size_t)b.N_pad * (dl ? V_DL : V_SL));
    if (dl) b.srcLo = bp.take<float4>(b.N_pad);
  } else {
    b.src64 = bp.take<double4_32a>((size_t)b.N_pad * 2);
    if (dl) b.nrm64 = bp.take<double4_32a>(b.N_pad);
  }
  b.segbox = bp.take<float4>((size_t)(b.N_pad / SEG) * 2);
  b.tgt_perm = bp.take<int>(b.M_pad);
  if (fp32) b.tgtF = bp.take<float4>((size_t)b.M_pad * 2);
  b.tgt64 = bp.take<double4_32a>(b.M_pad);
  b.part = bp.take<double>((size_t)s.n_chunks * b.M_pad * 3);
  if (fp32) {
    b.near_cnt = bp.take<int>(b.M_pad / NEAR_GROUP_MIN);
    b.tb_done = bp.take<int>(b.M_pad / 512 + 1);  // blocks of >= 512 targets
    b.near_idx = bp.take<unsigned>((size_t)b.M_pad * NEAR_K);
    b.near_ovf = bp.take<double>((size_t)b.M_pad * 3);
  }
  b.flags = bp.take<unsigned long long>(N_FLAGS);
  // the target sort's own scratch last, so that the buffers above keep the
  // offsets they have without it
  if (s.split_sorts && s.N > 0) {
    const int64_t mt = s.M > 0 ? s.M : 1;
    b.tkeys_a = bp.take<uint32_t>(mt);
    b.tkeys_b = bp.take<uint32_t>(mt);
    b.tvals_a = bp.take<int>(mt);
    b.tvals_b = bp.take<int>(mt);
    b.thist = bp.take<uint32_t>(256 * (size_t)sort_grid_blocks(mt) + 256);
    b.tbbox_part = bp.take<float>(128 * 6);
    b.tbbox = bp.take<float>(8);
  } else {
    b.tkeys_a = b.keys_a;
    b.tkeys_b = b.keys_b;
    b.tvals_a = b.vals_a;
    b.tvals_b = b.vals_b;
    b.thist = b.hist;
    b.tbbox_part = b.bbox_part;
    b.tbbox = b.bbox;
  }
}

double layer_scale(const EvalShape& s) {
  return s.layer == LAYER_SL ? 1.0 / (8.0 * PI_CONST * s.mu) : -6.0 / (8.0 * PI_CONST);
}

__global__ void k_check_delta(const double* __restrict__ d, int64_t n,
                              unsigned long long* __restrict__ flags) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && !(d[i] > 0.0 && d[i] < INFINITY)) atomicExch(flags + FLAG_BAD_DELTA, 1ull);
}

// Preparation of one evaluation on `st`: clear the counters, check delta,
// sort and pack sources and targets. With split sorts and a fork, the target
// sort and pack run on pf->aux beside the source sort and pack (the two touch
// disjoint buffers; the result does not change), and `st` waits for them.
// Returns the number of kernels launched.
int enqueue_prep(const EvalShape& s, const EvalBufs& b, double rho_T, double rho_c,
                 cudaStream_t st, const PrepFork* pf) {
  const bool fp32 = s.precision == SK_FP32C;
  const double scale = layer_scale(s);
  // bbox (2) + keys + 4 radix passes x 3 (hist, row scan, scatter), or the single-block sort
  auto sort_launches = [&](int64_t n) { return n <= s.small_sort_points ? 1 : 3 + 4 * 3; };
  int launches = 0;
  cudaMemsetAsync(b.flags, 0, N_FLAGS * sizeof(unsigned long long), st);
  cudaMemsetAsync(b.meta, 0, N_META * sizeof(int), st);
  if (fp32) {
    cudaMemsetAsync(b.near_cnt, 0, (b.M_pad / NEAR_GROUP_MIN) * sizeof(int), st);
    cudaMemsetAsync(b.tb_done, 0, (b.M_pad / 512 + 1) * sizeof(int), st);
  }
  k_check_delta<<<(unsigned)((s.n_delta + 255) / 256), 256, 0, st>>>(b.delta, s.n_delta, b.flags);
  launches += 1;
  const bool fork = pf && pf->aux && s.split_sorts && s.N > 0;
  cudaStream_t tst = st;
  if (fork) {
    cudaEventRecord(pf->fork, st);
    cudaStreamWaitEvent(pf->aux, pf->fork, 0);
    tst = pf->aux;
  }
  launch_sort_points(b.tgt_xyz, nullptr, s.M, b.tkeys_a, b.tkeys_b, b.tvals_a, b.tvals_b, b.thist,
                     b.tbbox_part, b.tbbox, b.meta + META_SCRATCH, s.small_sort_points, tst);
  launches += sort_launches(s.M);
  if (fp32)
    launch_pack_targets32(b, s.n_delta, rho_T, rho_c, tst);
  else
    launch_pack_targets64(b, s.n_delta, tst);
  if (s.N > 0) {
    launch_sort_points(b.src_xyz, b.src_w, s.N, b.keys_a, b.keys_b, b.vals_a, b.vals_b, b.hist,
                       b.bbox_part, b.bbox, b.meta + META_NS, s.small_sort_points, st);
    if (fp32)
      launch_pack_sources32(s.layer, b, scale, st);
    else
      launch_pack_sources64(s.layer, b, scale, st);
    launches += sort_launches(s.N) + 1;
  }
  if (fork) {
    cudaEventRecord(pf->join, pf->aux);
    cudaStreamWaitEvent(st, pf->join, 0);
  }
  return launches + 1;
}

// Enqueue one evaluation on `st`; inputs and output are device pointers in b.
int enqueue_eval(const EvalShape& s, const EvalBufs& b, double rho_T, double rho_c,
                 cudaStream_t st, cudaEvent_t* ev, const PrepFork* pf) {
  const bool fp32 = s.precision == SK_FP32C;
  const double scale = layer_scale(s);
  if (ev) cudaEventRecord(ev[0], st);
  int launches = enqueue_prep(s, b, rho_T, rho_c, st, pf);
  if (ev) cudaEventRecord(ev[1], st);
  if (fp32) {
    launch_pair32(s.layer, b, rho_T, scale, st, ev ? ev[2] : nullptr);  // with the finish
    launches += b.fuse_finish ? 1 : 3;
  } else {
    launch_pair64(s.layer, b, scale, st);
    if (ev) cudaEventRecord(ev[2], st);
    launch_finish64(b, st);
    launches += 1 + 1;
  }
  if (ev) cudaEventRecord(ev[3], st);
  return launches;
}

}  // namespace sk

using namespace sk;

extern "C" {

int sk_version(void) { return 100; }

int sk_create(sk_ctx** out, int device, size_t workspace_bytes) {
  if (!out) return SK_EINVAL;
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    g_create_error_buf = std::string("no CUDA device: ") + cudaGetErrorString(e);
    g_create_error = g_create_error_buf.c_str();
    return SK_ECUDA;
  }
  if (device < 0 || device >= ndev) {
    g_create_error = "device index out of range";
    return SK_EINVAL;
  }
  sk_ctx* ctx = new (std::nothrow) sk_ctx();
  if (!ctx) return SK_ENOMEM;
  ctx->device = device;
  DeviceGuard g(device);
  int code = SK_OK;
  if ((e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device)) !=
          cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaMallocHost(&ctx->h_flags, 256)) != cudaSuccess) {
    code = e == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA;
  } else if (workspace_bytes > 0) {
    if ((e = cudaMalloc(&ctx->ws, workspace_bytes)) != cudaSuccess)
      code = SK_ENOMEM;
    else {
      ctx->ws_bytes = workspace_bytes;
      ctx->ws_fixed = true;
    }
  }
  if (code != SK_OK) {
    g_create_error_buf = std::string("sk_create: ") + cudaGetErrorString(e);
    g_create_error = g_create_error_buf.c_str();
    sk_destroy(ctx);
    return code;
  }
  std::memset(ctx->h_flags, 0, 256);
  ctx->last_stream = ctx->stream;
  ctx->small_sort_points = SMALL_SORT_POINTS;
  if (const char* v = std::getenv("SK_SMALL_SORT_POINTS")) {
    char* end = nullptr;
    const long long k = std::strtoll(v, &end, 10);
    if (end != v && *end == '\0' && k >= 0 && k <= (1LL << 24)) ctx->small_sort_points = k;
  }
  *out = ctx;
  return SK_OK;
}

void sk_destroy(sk_ctx* ctx) {
  if (!ctx) return;
  if (ctx->server) serve_destroy(ctx->server);
  DeviceGuard g(ctx->device);
  cudaDeviceSynchronize();
  free_membrane_ops(ctx);
  free_fmm_ops(ctx);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->h_flags) cudaFreeHost(ctx->h_flags);
  for (int i = 0; i < 4; ++i)
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
  if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
  if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char* sk_last_error(const sk_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error; }

int sk_set_fp32c_thresholds(sk_ctx* ctx, double rho_T, double rho_c) {
  if (!ctx) return SK_EINVAL;
  if (!(rho_T > 0.0 && rho_T <= 2.0 && rho_c > rho_T && rho_c <= 8.0))
    return fail(ctx, SK_EINVAL, "sk_set_fp32c_thresholds: need 0 < rho_T <= 2, rho_T < rho_c <= 8");
  ctx->rho_T = rho_T;
  ctx->rho_c = rho_c;
  return SK_OK;
}

int sk_set_profiling(sk_ctx* ctx, int enable) {
  if (!ctx) return SK_EINVAL;
  DeviceGuard g(ctx->device);
  if (enable && !ctx->ev[0]) {
    for (int i = 0; i < 4; ++i) {
      cudaError_t e = cudaEventCreate(&ctx->ev[i]);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "sk_set_profiling");
    }
  }
  ctx->profile = enable != 0;
  return SK_OK;
}

int sk_last_eval_stats(const sk_ctx* ctx, sk_eval_stats* out) {
  if (!ctx || !out) return SK_EINVAL;
  DeviceGuard g(ctx->device);
  cudaStreamSynchronize(ctx->last_stream);
  *out = ctx->stats;
  out->pair_ms = out->eval_ms = -1.0;
  if (ctx->stats.pair_ms == 0.0 && ctx->profile && ctx->ev[0]) {
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, ctx->ev[1], ctx->ev[2]) == cudaSuccess &&
        cudaEventElapsedTime(&b, ctx->ev[0], ctx->ev[3]) == cudaSuccess) {
      out->pair_ms = a;
      out->eval_ms = b;
    }
  }
  const unsigned long long* f = ctx->h_flags;
  const int* meta = reinterpret_cast<const int*>(ctx->h_flags + N_FLAGS);
  out->n_src_active = meta[META_NS];
  out->near_pairs = (int64_t)f[FLAG_NEAR_PAIRS];
  out->overflow_targets = (int64_t)f[FLAG_OVERFLOW];
  return SK_OK;
}

}  // extern "C"

namespace sk {

int ensure_workspace(sk_ctx* ctx, size_t need) {
  if (need <= ctx->ws_bytes) return SK_OK;
  if (ctx->ws_fixed) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "workspace of %zu bytes too small: this call needs %zu",
                  ctx->ws_bytes, need);
    ctx->err = buf;
    return SK_ENOMEM;
  }
  cudaError_t e = cudaDeviceSynchronize();  // older work may still use the workspace
  if (e != cudaSuccess) return cuda_fail(ctx, e, "workspace grow (synchronize)");
  if (ctx->ws) cudaFree(ctx->ws);
  ctx->ws = nullptr;
  ctx->ws_bytes = 0;
  const size_t want = need + need / 4;
  if ((e = cudaMalloc(&ctx->ws, want)) != cudaSuccess) return cuda_fail(ctx, e, "workspace cudaMalloc");
  ctx->ws_bytes = want;
  return SK_OK;
}

}  // namespace sk

namespace {

int eval_entry(sk_ctx* ctx, int layer, int precision, int mem, int64_t N, const double* xyz,
               const double* w, const double* dens, const double* nrm, int64_t M,
               const double* txyz, const double* delta, int64_t n_delta, double mu, double* u_out,
               void* stream_v) {
  const char* fn = layer == LAYER_SL ? "stokes_sl_eval" : "stokes_dl_eval";
  if (!ctx) return SK_EINVAL;
  ctx->err.clear();
  if (precision != SK_FP64 && precision != SK_FP32C)
    return fail(ctx, SK_EINVAL, "%s: precision must be SK_FP64 or SK_FP32C", fn);
  if (mem != SK_HOST && mem != SK_DEVICE)
    return fail(ctx, SK_EINVAL, "%s: mem must be SK_HOST or SK_DEVICE", fn);
  if (N < 0 || M < 0) return fail(ctx, SK_EINVAL, "%s: negative size", fn);
  if (N > MAX_POINTS || M > MAX_POINTS)
    return fail(ctx, SK_EINVAL, "%s: more than 2^30 sources or targets", fn);
  if (precision == SK_FP32C && N > FP32C_MAX_SOURCES)
    return fail(ctx, SK_EINVAL, "%s: more than 2^25 sources in SK_FP32C", fn);
  if (M == 0) return SK_OK;
  if (N > 0 && (!xyz || !w || !dens || (layer == LAYER_DL && !nrm)))
    return fail(ctx, SK_EINVAL, "%s: NULL source array", fn);
  if (!txyz || !delta || !u_out) return fail(ctx, SK_EINVAL, "%s: NULL target/delta/output array", fn);
  if (!(n_delta == 1 || n_delta == M))
    return fail(ctx, SK_EINVAL, "%s: n_delta must be 1 or n_tgt", fn);
  if (layer == LAYER_SL && !(mu > 0.0 && std::isfinite(mu)))
    return fail(ctx, SK_EINVAL, "%s: mu must be positive and finite", fn);
  if (mem == SK_HOST)
    for (int64_t i = 0; i < n_delta; ++i)
      if (!(delta[i] > 0.0 && std::isfinite(delta[i])))
        return fail(ctx, SK_EINVAL, "%s: delta must be positive and finite", fn);

  DeviceGuard g(ctx->device);
  cudaStream_t st = stream_v ? (cudaStream_t)stream_v : ctx->stream;
  EvalShape s;
  s.layer = layer;
  s.precision = precision;
  s.N = N;
  s.M = M;
  s.n_delta = n_delta;
  s.mu = mu;
  s.copy_inputs = mem == SK_HOST;
  s.small_sort_points = ctx->small_sort_points;
  s.split_sorts = true;
  choose_decomposition(s, ctx->sm_count);
  const size_t need = eval_workspace_bytes(s);
  int rc = ensure_workspace(ctx, need);
  if (rc != SK_OK) return rc;
  EvalBufs b;
  Bump bp;
  bp.base = ctx->ws;
  carve_eval_buffers(bp, s, b);
  cudaError_t e;
  if (mem == SK_HOST) {
    if (N > 0) {
      cudaMemcpyAsync((void*)b.src_xyz, xyz, 3 * N * sizeof(double), cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync((void*)b.src_w, w, N * sizeof(double), cudaMemcpyHostToDevice, st);
      cudaMemcpyAsync((void*)b.dens, dens, 3 * N * sizeof(double), cudaMemcpyHostToDevice, st);
      if (layer == LAYER_DL)
        cudaMemcpyAsync((void*)b.nrm, nrm, 3 * N * sizeof(double), cudaMemcpyHostToDevice, st);
    }
    cudaMemcpyAsync((void*)b.tgt_xyz, txyz, 3 * M * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync((void*)b.delta, delta, n_delta * sizeof(double), cudaMemcpyHostToDevice, st);
  } else {
    b.src_xyz = xyz;
    b.src_w = w;
    b.dens = dens;
    b.nrm = nrm;
    b.tgt_xyz = txyz;
    b.delta = delta;
    b.u = u_out;
  }
  const PrepFork pf{ctx->aux_stream, ctx->fork_ev, ctx->join_ev};
  const int launches =
      enqueue_eval(s, b, ctx->rho_T, ctx->rho_c, st, ctx->profile ? ctx->ev : nullptr, &pf);
  if (mem == SK_HOST)
    cudaMemcpyAsync(u_out, b.u, 3 * M * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(ctx->h_flags, b.flags, N_FLAGS * sizeof(unsigned long long),
                  cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(ctx->h_flags + N_FLAGS, b.meta, N_META * sizeof(int), cudaMemcpyDeviceToHost,
                  st);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, fn);
  ctx->last_stream = st;
  ctx->stats = sk_eval_stats{};
  ctx->stats.n_tgt = M;
  ctx->stats.n_chunks = s.n_chunks;
  ctx->stats.finish_fused = b.fuse_finish ? 1 : 0;
  ctx->stats.kernel_launches = launches;
  ctx->stats.precision = precision;
  if (stream_v) return SK_OK;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(ctx, e, fn);
  if (ctx->h_flags[FLAG_TIMEOUT]) return fail(ctx, SK_ETIMEOUT, "%s: a bounded device wait expired", fn);
  if (ctx->h_flags[FLAG_BAD_DELTA])
    return fail(ctx, SK_EINVAL, "%s: delta must be positive and finite", fn);
  return SK_OK;
}

}  // namespace

namespace sk {
int eval_call(sk_ctx* ctx, int layer, int precision, int mem, int64_t N, const double* xyz,
              const double* w, const double* dens, const double* nrm, int64_t M,
              const double* txyz, const double* delta, int64_t n_delta, double mu,
              double* u_out, void* stream) {
  return eval_entry(ctx, layer, precision, mem, N, xyz, w, dens, nrm, M, txyz, delta, n_delta, mu,
                    u_out, stream);
}
}  // namespace sk

extern "C" {

int stokes_sl_eval(sk_ctx* ctx, int precision, int mem, int64_t n_src, const double* src_xyz,
                   const double* src_w, const double* f, int64_t n_tgt, const double* tgt_xyz,
                   const double* delta, int64_t n_delta, double mu, double* u_out,
                   void* cuda_stream) {
  return eval_entry(ctx, LAYER_SL, precision, mem, n_src, src_xyz, src_w, f, nullptr, n_tgt,
                    tgt_xyz, delta, n_delta, mu, u_out, cuda_stream);
}

int stokes_dl_eval(sk_ctx* ctx, int precision, int mem, int64_t n_src, const double* src_xyz,
                   const double* src_w, const double* src_n, const double* q, int64_t n_tgt,
                   const double* tgt_xyz, const double* delta, int64_t n_delta, double* u_out,
                   void* cuda_stream) {
  return eval_entry(ctx, LAYER_DL, precision, mem, n_src, src_xyz, src_w, q, src_n, n_tgt,
                    tgt_xyz, delta, n_delta, 1.0, u_out, cuda_stream);
}

}  // extern "C"
