// sk_pair64.cu -- FP64 pair sums (single and double layer).
//
// Same work decomposition as the FP32 kernels (sorted targets, chunks of
// source tiles staged by bulk async copies, per-segment near/far test), all
// arithmetic in FP64:
//   rho >= 7          plain Stokeslet / stresslet (s_i = 1 to double precision)
//   2.2 <= rho < 7    closed-form s_i with erf/exp (Sec. 3.4)
//   rho < 2.2         power series of s_i / rho^k (sk_series.cuh), incl. r = 0
// Two targets per lane; plain FP64 accumulation per chunk; the finish
// kernel adds the chunks of a target in fixed order.
#include <cfloat>

#include "sk_internal.h"
#include "sk_series.cuh"

namespace sk {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int SEGS64 = TILE64 / SEG;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, "
        "p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
}

template <int LAYER>
__device__ __forceinline__ void far64(const double4_32a& P, const double4_32a& G, const double4_32a& Nn,
                                      double tx, double ty, double tz, double& u0, double& u1,
                                      double& u2) {
  const double dx = tx - P.x, dy = ty - P.y, dz = tz - P.z;
  const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
  const double ri = rsqrt(r2);
  const double ri2 = ri * ri;
  if (LAYER == LAYER_SL) {
    const double gd = fma(G.z, dz, fma(G.y, dy, G.x * dx));
    const double a = gd * ri2;
    u0 = fma(fma(dx, a, G.x), ri, u0);
    u1 = fma(fma(dy, a, G.y), ri, u1);
    u2 = fma(fma(dz, a, G.z), ri, u2);
  } else {
    const double dq = fma(G.z, dz, fma(G.y, dy, G.x * dx));
    const double dn = fma(Nn.z, dz, fma(Nn.y, dy, Nn.x * dx));
    const double c = dq * dn * (ri2 * ri2 * ri);
    u0 = fma(c, dx, u0);
    u1 = fma(c, dy, u1);
    u2 = fma(c, dz, u2);
  }
}

template <int LAYER>
__global__ void __launch_bounds__(TPB64, 2)
    k_pair64(const double4_32a* __restrict__ src64, const double4_32a* __restrict__ nrm64,
             const float4* __restrict__ segbox, const int* __restrict__ meta,
             const double4_32a* __restrict__ tgt64, int64_t M_pad, int n_chunks,
             double* __restrict__ part, unsigned long long* __restrict__ flags) {
  constexpr int REC = 2;  // double4_32a records per source in src64
  constexpr uint32_t SRC_BYTES = TILE64 * REC * sizeof(double4_32a);
  constexpr uint32_t NRM_BYTES = LAYER == LAYER_DL ? TILE64 * sizeof(double4_32a) : 0;
  constexpr uint32_t BUF_D4 = TILE64 * (REC + (LAYER == LAYER_DL ? 1 : 0));
  extern __shared__ __align__(128) double4_32a sm64[];
  __shared__ __align__(8) uint64_t mbar[2];

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int tb = blockIdx.x / n_chunks, ch = blockIdx.x % n_chunks;
  const int n_tiles = meta[META_NS_PAD] / TILE64;
  const int k0 = (int)((long long)ch * n_tiles / n_chunks);
  const int k1 = (int)((long long)(ch + 1) * n_tiles / n_chunks);

  const int64_t wbase = (int64_t)tb * (blockDim.x * TPL64) + wid * TGT_WARP64;
  double tx[2], ty[2], tz[2], invd[2], rc2[2];
  float blo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, bhi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
  float rc2max = -1.f, amax = 0.f;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const double4_32a x = tgt64[wbase + 32 * h + lane];
    tx[h] = x.x;
    ty[h] = x.y;
    tz[h] = x.z;
    const bool real = x.w > 0.0;
    invd[h] = real ? 1.0 / x.w : 1.0;
    rc2[h] = real ? (RHO_C64 * x.w) * (RHO_C64 * x.w) : -1.0;
    if (real) {
      const float fx = (float)x.x, fy = (float)x.y, fz = (float)x.z;
      blo[0] = fminf(blo[0], fx); bhi[0] = fmaxf(bhi[0], fx);
      blo[1] = fminf(blo[1], fy); bhi[1] = fmaxf(bhi[1], fy);
      blo[2] = fminf(blo[2], fz); bhi[2] = fmaxf(bhi[2], fz);
      rc2max = fmaxf(rc2max, (float)rc2[h]);
      amax = fmaxf(amax, fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz))));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      blo[c] = fminf(blo[c], __shfl_xor_sync(FULL, blo[c], o));
      bhi[c] = fmaxf(bhi[c], __shfl_xor_sync(FULL, bhi[c], o));
    }
    rc2max = fmaxf(rc2max, __shfl_xor_sync(FULL, rc2max, o));
    amax = fmaxf(amax, __shfl_xor_sync(FULL, amax, o));
  }
  const bool warp_live = rc2max >= 0.f;
  const float pad = 4e-7f * amax;  // covers FP64 -> FP32 rounding of both boxes
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    blo[c] -= pad;
    bhi[c] += pad;
  }
  const float rc2test = rc2max * 1.0001f;

  double u[2][3] = {{0, 0, 0}, {0, 0, 0}};

  if (tid == 0) {
    mbar_init(&mbar[0]);
    mbar_init(&mbar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  int issued[2] = {0, 0}, consumed[2] = {0, 0};
  auto issue = [&](int b, int k) {
    double4_32a* dst = sm64 + (size_t)b * BUF_D4;
    expect_tx(&mbar[b], SRC_BYTES + NRM_BYTES);
    bulk_copy(dst, src64 + (size_t)k * TILE64 * REC, SRC_BYTES, &mbar[b]);
    if (LAYER == LAYER_DL) bulk_copy(dst + TILE64 * REC, nrm64 + (size_t)k * TILE64, NRM_BYTES, &mbar[b]);
    issued[b]++;
  };
  if (tid == 0)
    for (int b = 0; b < 2; ++b)
      if (k0 + b < k1) issue(b, k0 + b);

  bool timed_out = false;
  for (int k = k0, it = 0; k < k1; ++k, ++it) {
    const int buf = it & 1;
    const bool ok = mbar_wait_bounded(&mbar[buf], (uint32_t)(consumed[buf] & 1));
    consumed[buf]++;
    if (__syncthreads_or(!ok)) {
      timed_out = true;
      break;
    }
    if (warp_live) {
      const double4_32a* S = sm64 + (size_t)buf * BUF_D4;
      const double4_32a* SN = S + TILE64 * REC;
      bool nb = false;
      if (lane < SEGS64) {
        const float4 lo = segbox[2 * ((size_t)k * SEGS64 + lane)];
        const float4 hi = segbox[2 * ((size_t)k * SEGS64 + lane) + 1];
        const float dx = fmaxf(0.f, fmaxf(lo.x - bhi[0], blo[0] - hi.x));
        const float dy = fmaxf(0.f, fmaxf(lo.y - bhi[1], blo[1] - hi.y));
        const float dz = fmaxf(0.f, fmaxf(lo.z - bhi[2], blo[2] - hi.z));
        nb = dx * dx + dy * dy + dz * dz < rc2test;
      }
      const unsigned nm = __ballot_sync(FULL, nb);
#pragma unroll 1
      for (int s = 0; s < SEGS64; ++s) {
        if (!((nm >> s) & 1u)) {
#pragma unroll 2
          for (int j = s * SEG; j < (s + 1) * SEG; ++j) {
            const double4_32a P = S[REC * j], G = S[REC * j + 1];
            const double4_32a Nn = LAYER == LAYER_DL ? SN[j] : make_double4_32a(0, 0, 0, 0);
#pragma unroll
            for (int h = 0; h < 2; ++h) far64<LAYER>(P, G, Nn, tx[h], ty[h], tz[h], u[h][0], u[h][1], u[h][2]);
          }
        } else {
#pragma unroll 1
          for (int j = s * SEG; j < (s + 1) * SEG; ++j) {
            const double4_32a P = S[REC * j], G = S[REC * j + 1];
            const double4_32a Nn = LAYER == LAYER_DL ? SN[j] : make_double4_32a(0, 0, 0, 0);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const double dx = tx[h] - P.x, dy = ty[h] - P.y, dz = tz[h] - P.z;
              const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
              if (r2 < rc2[h]) {
                if (LAYER == LAYER_SL)
                  sl_pair64(dx, dy, dz, G.x, G.y, G.z, 1.0, invd[h], u[h][0], u[h][1], u[h][2]);
                else
                  dl_pair64(dx, dy, dz, G.x, G.y, G.z, Nn.x, Nn.y, Nn.z, 1.0, invd[h], u[h][0],
                            u[h][1], u[h][2]);
              } else {
                far64<LAYER>(P, G, Nn, tx[h], ty[h], tz[h], u[h][0], u[h][1], u[h][2]);
              }
            }
          }
        }
      }
    }
    __syncthreads();
    if (tid == 0 && k + 2 < k1) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(buf, k + 2);
    }
  }
  if (timed_out) {
    if (tid == 0) {
      atomicExch(flags + FLAG_TIMEOUT, 1ull);
      for (int b = 0; b < 2; ++b)
        while (consumed[b] < issued[b]) {
          if (!mbar_wait_bounded(&mbar[b], (uint32_t)(consumed[b] & 1))) break;
          consumed[b]++;
        }
    }
    return;
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    double* o = part + ((size_t)ch * M_pad + wbase + 32 * h + lane) * 3;
    o[0] = u[h][0];
    o[1] = u[h][1];
    o[2] = u[h][2];
  }
}

__global__ void k_finish64(const int* __restrict__ perm, int64_t M, int64_t M_pad, int n_chunks,
                           const double* __restrict__ part, double* __restrict__ u_out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= M) return;
  double u0 = 0, u1 = 0, u2 = 0;
  for (int c = 0; c < n_chunks; ++c) {
    const double* p = part + ((size_t)c * M_pad + t) * 3;
    u0 += p[0];
    u1 += p[1];
    u2 += p[2];
  }
  const int64_t j = perm[t];
  u_out[3 * j] = u0;
  u_out[3 * j + 1] = u1;
  u_out[3 * j + 2] = u2;
}

}  // namespace

void launch_pair64(int layer, const EvalBufs& b, double /*scale*/, cudaStream_t st) {
  // M_pad is a multiple of TGT_CTA64, hence of the smaller CTA's targets too
  const int tpb = b.threads64;
  const unsigned grid = (unsigned)((b.M_pad / ((int64_t)tpb * TPL64)) * b.n_chunks);
  if (layer == LAYER_SL) {
    const size_t smem = 2 * TILE64 * 2 * sizeof(double4_32a);
    k_pair64<LAYER_SL><<<grid, tpb, smem, st>>>(b.src64, b.nrm64, b.segbox, b.meta, b.tgt64,
                                                 b.M_pad, b.n_chunks, b.part, b.flags);
  } else {
    const size_t smem = 2 * TILE64 * 3 * sizeof(double4_32a);
    k_pair64<LAYER_DL><<<grid, tpb, smem, st>>>(b.src64, b.nrm64, b.segbox, b.meta, b.tgt64,
                                                 b.M_pad, b.n_chunks, b.part, b.flags);
  }
}

void launch_finish64(const EvalBufs& b, cudaStream_t st) {
  k_finish64<<<(unsigned)((b.M + 127) / 128), 128, 0, st>>>(b.tgt_perm, b.M, b.M_pad, b.n_chunks,
                                                            b.part, b.u);
}

}  // namespace sk
