// sk_probe.cu -- microbenchmarks of the ceilings the pair kernels are
// measured against: packed FP32 FMA (FFMA2), FP64 FMA (DFMA), and the
// single-layer far-field pair loop itself with its sources in shared memory
// (no global-memory traffic, no near/far test, no compensated merge), at the
// C3 kernel's shape: 256 threads, two f32x2 target pairs per lane, two CTAs
// per SM. Every loop has a fixed trip count (no waits).
#include "sk_pair32.cuh"

namespace sk {
namespace {

using namespace p32;

constexpr int PROBE_TPB = 256;
constexpr int PROBE_ILP = 8;  // independent FMA chains per thread
constexpr int PROBE_FMA_ITERS = 100000;
constexpr int PROBE_DFMA_ITERS = 4000;
constexpr int PROBE_PAIR_ITERS = 400;  // passes over a 256-source tile

__global__ void __launch_bounds__(PROBE_TPB) k_probe_ffma2(int iters, float* sink) {
  const float2 b = make_float2(0.999999f, 0.999998f), c = make_float2(1e-7f, 2e-7f);
  float2 acc[PROBE_ILP];
#pragma unroll
  for (int k = 0; k < PROBE_ILP; ++k) acc[k] = make_float2(threadIdx.x * 1e-3f + k, 0.5f * k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < PROBE_ILP; ++k) acc[k] = fma2(acc[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < PROBE_ILP; ++k) s += acc[k].x + acc[k].y;
  if (s == -1.f) sink[0] = s;  // never true; keeps the chains live
}

__global__ void __launch_bounds__(PROBE_TPB) k_probe_dfma(int iters, double* sink) {
  const double b = 0.9999999, c = 1e-9;
  double acc[PROBE_ILP];
#pragma unroll
  for (int k = 0; k < PROBE_ILP; ++k) acc[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < PROBE_ILP; ++k) acc[k] = fma(acc[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < PROBE_ILP; ++k) s += acc[k];
  if (s == -1.0) sink[0] = s;
}

// The far loop of k_pair32<SLayer, 2, 2> over one shared-memory tile of 256
// synthetic sources, `iters` times: SLayer::far per source and target pair.
__global__ void __launch_bounds__(TPB32, 2) k_probe_pairs(int iters, float* sink) {
  constexpr int NP = 2, V = SLayer::V;
  __shared__ float4 S[TILE * V];
  for (int j = threadIdx.x; j < TILE; j += blockDim.x) {
    const float x = 0.01f * (j % 16), y = 0.01f * ((j / 16) % 16), z = 0.3f + 1e-3f * j;
    const float g0 = 1e-3f * (1 + j % 7), g1 = -1e-3f * (1 + j % 5), g2 = 1e-3f * (1 + j % 3);
    S[j * V] = make_float4(-x, -x, -y, -y);
    S[j * V + 1] = make_float4(-z, -z, g0, g0);
    S[j * V + 2] = make_float4(g1, g1, g2, g2);
  }
  __syncthreads();
  Tgt2 T[NP];
  float2 U[NP][3];
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const float t = 1e-4f * (threadIdx.x + 64 * p);
    T[p].x = make_float2(t, t + 1e-5f);
    T[p].y = make_float2(-t, 0.5f * t);
    T[p].z = make_float2(2.f * t, -t);
#pragma unroll
    for (int c = 0; c < 3; ++c) U[p][c] = make_float2(0.f, 0.f);
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll 1
    for (int s = 0; s < TILE_SEGS; ++s) {
      const float4* SS = S + s * SEG * V;
#pragma unroll kFarUnroll
      for (int j = 0; j < SEG; ++j) {
        const SLayer::Src src = SLayer::load(SS + j * V);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          float2 dx, dy, dz, r2;
          pair_d(T[p], src.nx, src.ny, src.nz, dx, dy, dz, r2);
          SLayer::far(src, dx, dy, dz, r2, U[p]);
        }
      }
    }
  }
  float s = 0.f;
#pragma unroll
  for (int p = 0; p < NP; ++p)
#pragma unroll
    for (int c = 0; c < 3; ++c) s += U[p][c].x + U[p][c].y;
  if (s == -1.f) sink[0] = s;
}

template <class F>
int time_launch(sk_ctx* ctx, F launch, float* ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) {
    launch();  // warm-up
    cudaEventRecord(a, ctx->stream);
    launch();
    cudaEventRecord(b, ctx->stream);
    e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  return e == cudaSuccess ? SK_OK : SK_ECUDA;
}

}  // namespace
}  // namespace sk

using namespace sk;

extern "C" int sk_probe_peaks(sk_ctx* ctx, sk_peaks* out) {
  if (!ctx || !out) return SK_EINVAL;
  cudaSetDevice(ctx->device);
  void* sink = nullptr;
  if (cudaMalloc(&sink, 64) != cudaSuccess) {
    ctx->err = "sk_probe_peaks: cudaMalloc failed";
    return SK_ENOMEM;
  }
  const int sms = ctx->sm_count;
  const unsigned full_grid = (unsigned)sms * (2048 / PROBE_TPB);  // 2048 resident threads per SM
  float ms_f = 0.f, ms_d = 0.f, ms_p = 0.f;
  int rc = time_launch(ctx, [&] {
    k_probe_ffma2<<<full_grid, PROBE_TPB, 0, ctx->stream>>>(PROBE_FMA_ITERS, (float*)sink);
  }, &ms_f);
  if (rc == SK_OK)
    rc = time_launch(ctx, [&] {
      k_probe_dfma<<<full_grid, PROBE_TPB, 0, ctx->stream>>>(PROBE_DFMA_ITERS, (double*)sink);
    }, &ms_d);
  if (rc == SK_OK)
    rc = time_launch(ctx, [&] {
      k_probe_pairs<<<(unsigned)sms * 2, TPB32, 0, ctx->stream>>>(PROBE_PAIR_ITERS, (float*)sink);
    }, &ms_p);
  cudaFree(sink);
  if (rc != SK_OK) {
    ctx->err = "sk_probe_peaks: a probe launch failed";
    return rc;
  }
  const double threads = (double)full_grid * PROBE_TPB;
  out->ffma2_tflops = threads * PROBE_FMA_ITERS * PROBE_ILP * 4.0 / (ms_f * 1e-3) / 1e12;
  out->dfma_tflops = threads * PROBE_DFMA_ITERS * PROBE_ILP * 2.0 / (ms_d * 1e-3) / 1e12;
  const double pairs = (double)sms * 2 * TPB32 * 4.0 * TILE * PROBE_PAIR_ITERS;  // 4 targets/lane
  out->far_pairs_per_s = pairs / (ms_p * 1e-3);
  out->sm_count = sms;
  return SK_OK;
}
