// sk_noalloc.cu -- single-layer evaluation that allocates no memory.
//
// Some callers cannot let a library allocate: code that runs under a fixed
// device-memory budget owned by a framework allocator (a stray cudaMalloc
// can fail there, or fragment the pool), latency-critical loops in which a
// cudaMalloc/cudaFree would stall the device, and callers that must not hold
// a library context. stokes_sl_eval_noalloc serves them. It takes device
// pointers for all inputs and the output, creates no context or stream, and
// does its work in one scratch array that is part of the library image: a
// file-scope static __device__ array of NOALLOC_SCRATCH_BYTES. The paper has
// no counterpart of this entry point.
#include <mutex>

#include "sk_decomp.h"
#include "sk_internal.h"

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;  // 32 MiB
constexpr int NOALLOC_MAX_DEVICES = 64;

// Scratch of every call on a device. Host code must not use this name as an
// address: it is a host-side stand-in. The device address comes from
// cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

void* g_scratch_addr[NOALLOC_MAX_DEVICES] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (set-up on the
// first call on that device). Returns nullptr on failure.
void* scratch_address(int dev) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
    g_scratch_addr[dev] = p;
  }
  return g_scratch_addr[dev];
}

}  // namespace

extern "C" int stokes_sl_eval_noalloc(int64_t n_src, const double* src_xyz, const double* src_w,
                                      const double* f, int64_t n_tgt, const double* tgt_xyz,
                                      const double* delta, int64_t n_delta, double mu,
                                      double* u_out, void* cuda_stream) {
  using namespace sk;
  if (n_src < 0 || n_tgt < 0) return SK_EINVAL;
  if (n_tgt == 0) return SK_OK;
  if (n_src > 0 && (!src_xyz || !src_w || !f)) return SK_EINVAL;
  if (!tgt_xyz || !delta || !u_out) return SK_EINVAL;
  if (!(n_delta == 1 || n_delta == n_tgt)) return SK_EINVAL;
  if (!(mu > 0.0 && mu < INFINITY)) return SK_EINVAL;
  if (n_src > FP32C_MAX_SOURCES || n_tgt > (int64_t(1) << 30)) return SK_EINVAL;

  int dev = -1, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES)
    return SK_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SK_ECUDA;

  EvalShape s;
  s.layer = LAYER_SL;
  s.precision = SK_FP32C;
  s.N = n_src;
  s.M = n_tgt;
  s.n_delta = n_delta;
  s.mu = mu;
  s.copy_inputs = false;
  // the decomposition of stokes_sl_eval (chunks, fused or separate finish);
  // the single-block and multi-block sorts give the same order, so the sort
  // limit does not matter for the result
  choose_decomposition(s, sms);
  // fewer source chunks need less scratch; reject what does not fit at one chunk
  while (s.n_chunks > 1 && eval_workspace_bytes(s) > NOALLOC_SCRATCH_BYTES) s.n_chunks /= 2;
  if (eval_workspace_bytes(s) > NOALLOC_SCRATCH_BYTES) return SK_EINVAL;

  void* base = scratch_address(dev);
  if (!base) return SK_ECUDA;

  EvalBufs b;
  Bump bp;
  bp.base = static_cast<char*>(base);
  carve_eval_buffers(bp, s, b);
  b.src_xyz = src_xyz;
  b.src_w = src_w;
  b.dens = f;
  b.nrm = nullptr;
  b.tgt_xyz = tgt_xyz;
  b.delta = delta;
  b.u = u_out;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // enqueue_eval clears the flags, counters and near-pair counts it relies on;
  // every other scratch word is written before it is read. cudaGetLastError
  // reports a failure of any runtime call made since the last check on this
  // thread: the launches, and the memsets and attribute calls among them.
  enqueue_eval(s, b, 0.5, 5.0, st);
  if (cudaGetLastError() != cudaSuccess) return SK_ECUDA;
  if (cuda_stream) return SK_OK;
  unsigned long long flags[N_FLAGS] = {};
  if (cudaMemcpyAsync(flags, b.flags, sizeof(flags), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SK_ECUDA;
  if (flags[FLAG_TIMEOUT]) return SK_ETIMEOUT;
  if (flags[FLAG_BAD_DELTA]) return SK_EINVAL;
  return SK_OK;
}
