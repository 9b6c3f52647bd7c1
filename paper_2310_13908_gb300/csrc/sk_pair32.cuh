// sk_pair32.cuh -- device code of the FP32-compensated pair sums, shared by
// the standalone evaluation kernels (sk_pair32.cu) and the persistent
// serving kernel (sk_serve.cu).
//
// Regimes per pair, rho = r/delta_x (delta of the target, Eq. regparam):
//   rho >= rho_c          plain Stokeslet / stresslet (s_i = 1), FP32 f32x2
//   rho_T <= rho < rho_c  closed-form s_i with erf/exp, FP32 (Sec. 3.4)
//   rho < rho_T           recorded in a per-target list and summed in FP64
//                         by power series (finish step), incl. r = 0
//
// Work item = (block of sorted targets, chunk of source tiles). A CTA streams
// its chunk through shared memory in tiles of 256 sources with a 3-4 stage
// pipeline of bulk async copies (cp.async.bulk + mbarrier); a stage is
// released per warp, and the last warp to release it issues its next copy, so
// no CTA-wide barrier sits in the tile loop. Per warp and per 32-source
// segment a bounding-box test decides whether any pair can be closer than
// rho_c delta; if not, the segment runs the branch-free far loop. Each lane
// owns NP f32x2 target pairs, so every arithmetic instruction of the far loop
// is a packed FFMA2/FADD2/FMUL2.
//
// Coordinates: a source is stored relative to its segment's frame (the FP32
// midpoint of the segment's box, differenced in FP64 when packed); a target
// keeps an FP32 (hi, lo) split and is moved into each segment's frame once per
// segment. A pair difference x - y then carries FP32 rounding of |x - c| and
// |y - c| instead of |x| and |y|: for the stresslet's (x - y) . n, which
// cancels to O(r^2) on the surface, this removes an error that grew like
// 1/delta with absolute FP32 coordinates.
//
// Accumulation (a4): plain FP32 inside 128-source groups, two-sum merge into
// a (hi, lo) FP32 pair per target component, hi + lo written in FP64 per
// chunk; the finish step adds the chunks in fixed order and the FP64 near
// sum. The result of a target does not depend on which warp, CTA or chunk
// order it landed in: the far formula is bit-identical in both loops.
#pragma once

#include <cfloat>

#include "sk_internal.h"
#include "sk_erfc_scaled.h"
#include "sk_series.cuh"

// unroll factor of the far loop over the 32 sources of a segment
#ifndef SK_FAR_UNROLL
#define SK_FAR_UNROLL 8
#endif


namespace sk {
namespace p32 {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kFarUnroll = SK_FAR_UNROLL;

__device__ __forceinline__ float rsq(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// Fresh loads of an evaluation's prepared data inside a pair item (kFresh).
// The server's persistent kernel outlives the evaluations it serves: the
// memory of a finished one is rewritten for the next while the kernel runs,
// and an SM may still hold lines of the old contents in L1 or in the
// read-only path. ld.global.cg goes to L2, which every write reaches. A
// kernel launched per evaluation starts with clean L1 and keeps its ordinary
// loads.
__device__ __forceinline__ double4_32a ldcg4d(const double4_32a* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  const double2 a = __ldcg(q), b = __ldcg(q + 1);
  return make_double4_32a(a.x, a.y, b.x, b.y);
}

// ---- bulk async copy + mbarrier helpers (bounded waits) --------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try(bar, parity)) {
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
  return true;
}

// ---- per-lane target state --------------------------------------------------
// x, y, z: the pair's targets relative to the current segment's frame,
// recomputed per segment from the targets' FP32 (hi, lo) splits.
struct Tgt2 {
  float2 x, y, z, idl, rc2, rt2;
};

// A target coordinate x = hi + lo (hi = fl32(x), lo = fl32(x - hi)) relative
// to a segment frame c: (hi - c) is exact for close pairs (Sterbenz), so the
// result carries one rounding of |x - c|. It depends on the target and the
// segment only, not on which warp or CTA holds the target. The pair kernel
// (f32x2) and the overflow rescan (scalar) perform the same two roundings.
__device__ __forceinline__ float shift_to_segment(float hi, float lo, float c) {
  return __fadd_rn(__fsub_rn(hi, c), lo);
}
__device__ __forceinline__ float2 shift_to_segment2(float2 hi, float2 lo, float c) {
  return __fadd2_rn(__ffma2_rn(make_float2(c, c), make_float2(-1.f, -1.f), hi), lo);
}

// Rounding error of s = fl(a + b), exactly (Knuth's TwoSum).
__device__ __forceinline__ float2 two_sum_err2(float2 a, float2 b, float2 s) {
  const float2 bp = sub2(s, a);
  const float2 ap = sub2(s, bp);
  return add2(sub2(a, ap), sub2(b, bp));
}

// What shift_to_segment2 dropped: (hi + lo - c) - t for t = its result, to
// FP32 rounding of this small residual. With the source's residual (srcLo) it
// turns the FP32 difference of a pair into the exact one.
__device__ __forceinline__ float2 shift_residual2(float2 hi, float2 lo, float c, float2 t) {
  const float2 nc = make_float2(-c, -c);
  const float2 a = add2(hi, nc);  // fl(hi - c), the first rounding of shift_to_segment2
  return add2(two_sum_err2(hi, nc, a), two_sum_err2(a, lo, t));
}

// Margin added to rho_c delta in the segment-versus-warp box test: the boxes
// hold absolute FP32 coordinates, while pair distances come from frame-
// relative coordinates; the two differ by a few FP32 roundings of the
// coordinates' magnitude.
__device__ __forceinline__ float box_margin(float coord_max, float rc) {
  return 1.0e-6f * (coord_max + rc);
}

// Near pairs (rho < rho_T) are listed per target group: the 64 * NP targets
// of one warp of the pair kernel (group g = first target / (64 * NP)). An
// entry is (k << NEAR_SRC_BITS) | jo, k the target's place in the group and
// jo the source's original index. The warp appends the near pairs of one
// source together: one atomic per warp and source, and consecutive slots, so
// the group's list fills whole 32-byte sectors. (Entries appended one by one
// to per-target lists leave a partly written sector per target, which L2
// completes from DRAM when the finish reads it.) near_bits holds bit 2p + h
// for the lane's target 64p + 32h + lane. A list longer than NEAR_K * 64 * NP
// entries keeps counting but stores no more; the group's targets then take
// the rescan of overflow_target.
template <int NP, bool kFresh>
__device__ __noinline__ void near_append_list(unsigned near_bits, int lane, int64_t g,
                                              const int* jo_at, int* __restrict__ cnt,
                                              unsigned* __restrict__ idx,
                                              unsigned long long* __restrict__ flags) {
  constexpr int CAP = NEAR_K * 64 * NP;
  const unsigned jo = (unsigned)(kFresh ? __ldcg(jo_at) : *jo_at);
  const unsigned lt = (1u << lane) - 1u;
  int total = 0;
#pragma unroll
  for (int b = 0; b < 2 * NP; ++b) total += __popc(__ballot_sync(FULL, (near_bits >> b) & 1u));
  int base = 0;
  if (lane == 0) {
    base = atomicAdd(cnt + g, total);
    // the group's targets will be rescanned: count them
    if (base <= CAP && base + total > CAP) atomicAdd(flags + FLAG_OVERFLOW, 64ull * NP);
  }
  base = __shfl_sync(FULL, base, 0);
  unsigned* __restrict__ list = idx + (size_t)g * CAP;
  // slots in (bit, lane) order: the ballots again, so that no offsets stay live
#pragma unroll
  for (int b = 0; b < 2 * NP; ++b) {
    const unsigned m = __ballot_sync(FULL, (near_bits >> b) & 1u);
    const int slot = base + __popc(m & lt);
    if (((near_bits >> b) & 1u) && slot < CAP)
      list[slot] = ((unsigned)(64 * (b >> 1) + 32 * (b & 1) + lane) << NEAR_SRC_BITS) | jo;
    base += __popc(m);
  }
}

// Out of line beyond the vote: few general-path sources have a near pair,
// and the append's registers then do not weigh on the pair loop.
template <int NP, bool kFresh>
__device__ __forceinline__ void near_append_warp(unsigned near_bits, int lane, int64_t g,
                                                 const int* jo_at, int* __restrict__ cnt,
                                                 unsigned* __restrict__ idx,
                                                 unsigned long long* __restrict__ flags) {
  if (__any_sync(FULL, near_bits))
    near_append_list<NP, kFresh>(near_bits, lane, g, jo_at, cnt, idx, flags);
}

// ---- layer policies ---------------------------------------------------------
// Source record s (V float4) is read from shared memory; d and r2 of both
// targets of a pair are computed by the caller.
struct SLayer {
  static constexpr int V = V_SL;
  static constexpr int STAGES = 4;
  // no exact differences needed: the Stokeslet has no cancelling factor
  static constexpr bool kExactNear = false;
  struct Src {
    float2 nx, ny, nz, gx, gy, gz;
  };
  __device__ __forceinline__ static Src load(const float4* s) {
    const float4 a = s[0], b = s[1], c = s[2];
    return {lo2(a), hi2(a), lo2(b), hi2(b), lo2(c), hi2(c)};
  }
  // far: s1 = s2 = 1
  __device__ __forceinline__ static void far(const Src& S, float2 dx, float2 dy, float2 dz,
                                             float2 r2, float2* U) {
    const float2 ri = make_float2(rsq(r2.x), rsq(r2.y));
    const float2 ri2 = mul2(ri, ri);
    const float2 gd = fma2(S.gz, dz, fma2(S.gy, dy, mul2(S.gx, dx)));
    const float2 a = mul2(gd, ri2);
    U[0] = fma2(fma2(dx, a, S.gx), ri, U[0]);
    U[1] = fma2(fma2(dy, a, S.gy), ri, U[1]);
    U[2] = fma2(fma2(dz, a, S.gz), ri, U[2]);
  }
  // general: ri may be 0 (pair excluded), s1/s2 == 1 reproduces far() bit for bit
  __device__ __forceinline__ static void general(const Src& S, float2 dx, float2 dy, float2 dz,
                                                 float2 ri, float2 s1, float2 s2, float2* U) {
    const float2 ri2 = mul2(ri, ri);
    const float2 gd = fma2(S.gz, dz, fma2(S.gy, dy, mul2(S.gx, dx)));
    const float2 a = mul2(mul2(gd, ri2), s2);
    U[0] = fma2(fma2(dx, a, mul2(S.gx, s1)), ri, U[0]);
    U[1] = fma2(fma2(dy, a, mul2(S.gy, s1)), ri, U[1]);
    U[2] = fma2(fma2(dz, a, mul2(S.gz, s1)), ri, U[2]);
  }
  // FP32 closed forms at rho (Sec. 3.4), with erf(rho) = 1 - exp(-rho^2) E(rho):
  // s = 1 - exp(-rho^2) (E(rho) + (2 / (3 sqrt(pi))) rho q(rho)), q the
  // factor's polynomial; one exponential and the fitted E (sk_erfc_scaled.h)
  // instead of erff and an exponential. The caller clamps rho into range.
  __device__ __forceinline__ static void smooth(float rho, float& s1, float& s2) {
    const float p2 = rho * rho;
    const float e = __expf(-p2);
    const float E = erfc_scaled(rho);
    const float cr = (float)(2.0 / 3.0 * INV_SQRT_PI) * rho;
    s1 = 1.f - e * fmaf(cr, 2.f * p2 - 5.f, E);
    s2 = 1.f - e * fmaf(cr, fmaf(4.f * p2 - 14.f, p2, 3.f), E);
  }
};

struct DLayer {
  static constexpr int V = V_DL;
  static constexpr int STAGES = 3;
  // (x - y) . n cancels to O(r^2) on the surface: pairs inside rho_c delta take
  // the exact difference (FP32 residuals of the frame shifts added back),
  // which FP32 rounding of |x - c| and |y - c| would otherwise swamp when the
  // segment spans more than a few delta (sparse or irregular sources)
  static constexpr bool kExactNear = true;
  struct Src {
    float2 nx, ny, nz, qx, qy, qz, mx, my, mz;  // m: surface normal
  };
  __device__ __forceinline__ static Src load(const float4* s) {
    const float4 a = s[0], b = s[1], c = s[2], d = s[3], e = s[4];
    return {lo2(a), hi2(a), lo2(b), hi2(b), lo2(c), hi2(c), lo2(d), hi2(d), lo2(e)};
  }
  __device__ __forceinline__ static void far(const Src& S, float2 dx, float2 dy, float2 dz,
                                             float2 r2, float2* U) {
    const float2 ri = make_float2(rsq(r2.x), rsq(r2.y));
    const float2 ri2 = mul2(ri, ri);
    const float2 ri5 = mul2(mul2(ri2, ri2), ri);
    const float2 dq = fma2(S.qz, dz, fma2(S.qy, dy, mul2(S.qx, dx)));
    const float2 dn = fma2(S.mz, dz, fma2(S.my, dy, mul2(S.mx, dx)));
    const float2 c = mul2(mul2(dq, dn), ri5);
    U[0] = fma2(c, dx, U[0]);
    U[1] = fma2(c, dy, U[1]);
    U[2] = fma2(c, dz, U[2]);
  }
  __device__ __forceinline__ static void general(const Src& S, float2 dx, float2 dy, float2 dz,
                                                 float2 ri, float2 s3, float2 /*unused*/,
                                                 float2* U) {
    const float2 ri2 = mul2(ri, ri);
    const float2 ri5 = mul2(mul2(ri2, ri2), ri);
    const float2 dq = fma2(S.qz, dz, fma2(S.qy, dy, mul2(S.qx, dx)));
    const float2 dn = fma2(S.mz, dz, fma2(S.my, dy, mul2(S.mx, dx)));
    const float2 c = mul2(mul2(mul2(dq, dn), ri5), s3);
    U[0] = fma2(c, dx, U[0]);
    U[1] = fma2(c, dy, U[1]);
    U[2] = fma2(c, dz, U[2]);
  }
  // as SLayer::smooth: s3 = 1 - exp(-rho^2) (E(rho) + (2 / (9 sqrt(pi))) rho q3(rho))
  __device__ __forceinline__ static void smooth(float rho, float& s3, float& unused) {
    const float p2 = rho * rho;
    const float e = __expf(-p2);
    const float E = erfc_scaled(rho);
    const float cr = (float)(2.0 / 9.0 * INV_SQRT_PI) * rho;
    s3 = 1.f - e * fmaf(cr, fmaf(fmaf(8.f * p2 - 36.f, p2, 6.f), p2, 9.f), E);
    unused = 1.f;
  }
};

__device__ __forceinline__ void pair_d(const Tgt2& T, float2 nx, float2 ny, float2 nz, float2& dx,
                                       float2& dy, float2& dz, float2& r2) {
  dx = add2(T.x, nx);
  dy = add2(T.y, ny);
  dz = add2(T.z, nz);
  r2 = fma2(dz, dz, fma2(dy, dy, mul2(dx, dx)));
}

// Slow path of one target pair for one source: regime per lane component,
// decided on the FP32 difference r2 (the test of the far loop and of the
// overflow rescan). rho and the kernel use (dx, dy, dz) and r2k, which equal
// the FP32 difference and r2 except where pair_general corrected them.
template <class L>
__device__ __forceinline__ unsigned pair_general_regimes(const typename L::Src& S, const Tgt2& T,
                                                         float2 dx, float2 dy, float2 dz,
                                                         float2 r2, float2 r2k, float2* U,
                                                         float rho_lo, float rho_hi) {
  float2 ri = make_float2(rsq(r2k.x), rsq(r2k.y));
  float2 sa = make_float2(1.f, 1.f), sb = make_float2(1.f, 1.f);
  unsigned near_bits = 0;
  // component x
  {
    const bool vn = r2.x < T.rt2.x;
    const bool in = !vn && r2.x < T.rc2.x;
    if (vn) {
      near_bits |= 1u;
      ri.x = 0.f;
    }
    float rho = fminf(fmaxf(r2k.x * ri.x * T.idl.x, rho_lo), rho_hi);
    float a, b;
    L::smooth(rho, a, b);
    if (in) {
      sa.x = a;
      sb.x = b;
    }
  }
  {
    const bool vn = r2.y < T.rt2.y;
    const bool in = !vn && r2.y < T.rc2.y;
    if (vn) {
      near_bits |= 2u;
      ri.y = 0.f;
    }
    float rho = fminf(fmaxf(r2k.y * ri.y * T.idl.y, rho_lo), rho_hi);
    float a, b;
    L::smooth(rho, a, b);
    if (in) {
      sa.y = a;
      sb.y = b;
    }
  }
  L::general(S, dx, dy, dz, ri, sa, sb, U);
  return near_bits;
}

// For L::kExactNear, (cx, cy, cz) is the residual that makes the FP32
// difference exact: pairs with rho_T <= rho < rho_c take the corrected
// difference; the others keep the FP32 one, so a pair at or beyond rho_c
// still reproduces the far formula bit for bit.
// Returns the pair's near bits (x component: 1, y component: 2).
template <class L>
__device__ __forceinline__ unsigned pair_general(const typename L::Src& S, const Tgt2& T,
                                                 float2 dx, float2 dy, float2 dz, float2 r2,
                                                 float2* U, float rho_lo, float rho_hi,
                                                 float2 cx = float2{}, float2 cy = float2{},
                                                 float2 cz = float2{}) {
  if constexpr (L::kExactNear) {
    const bool in0 = r2.x >= T.rt2.x && r2.x < T.rc2.x;
    const bool in1 = r2.y >= T.rt2.y && r2.y < T.rc2.y;
    const float2 ex = add2(dx, cx), ey = add2(dy, cy), ez = add2(dz, cz);
    const float2 er2 = fma2(ez, ez, fma2(ey, ey, mul2(ex, ex)));
    dx = make_float2(in0 ? ex.x : dx.x, in1 ? ex.y : dx.y);
    dy = make_float2(in0 ? ey.x : dy.x, in1 ? ey.y : dy.y);
    dz = make_float2(in0 ? ez.x : dz.x, in1 ? ez.y : dz.y);
    const float2 r2k = make_float2(in0 ? er2.x : r2.x, in1 ? er2.y : r2.y);
    return pair_general_regimes<L>(S, T, dx, dy, dz, r2, r2k, U, rho_lo, rho_hi);
  } else {
    return pair_general_regimes<L>(S, T, dx, dy, dz, r2, r2, U, rho_lo, rho_hi);
  }
}

__device__ __forceinline__ void two_sum_merge(float2* U, float2* HI, float2* LO) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float2 s = add2(HI[c], U[c]);
    const float2 bp = sub2(s, HI[c]);
    const float2 e = add2(sub2(HI[c], sub2(s, bp)), sub2(U[c], bp));
    LO[c] = add2(LO[c], e);
    HI[c] = s;
    U[c] = make_float2(0.f, 0.f);
  }
}

// per-thread target state: TGT_SLOTS float4 per f32x2 pair (see pair_smem_bytes)
constexpr int TGT_SLOTS = 5;
// A segment is wide for a target when its frame's half extent exceeds this
// many of the target's delta (see pair_item's general branch).
constexpr float WIDE_FRAME = 4.0f;

// A lane's accumulators and target pairs, passed by value in and out of the
// out-of-line exact loop below.
template <int NP>
struct LaneAcc {
  float2 u[NP][3];
};
template <int NP>
struct LaneTgt {
  Tgt2 t[NP];
};

// The general loop over the 32 sources of one segment near the warp's
// targets: per source and target pair p, the far formula unless some lane's
// pair p lies inside rho_c delta, then the regimes (which give the far
// formula's bits for pairs beyond rho_c, so the choice per pair changes no
// result) and the warp's near-pair append. Out of line:
// its registers do not weigh on the far loop, and such segments are few (the
// ones within rho_c delta of the warp's box).
template <class L, int NP, bool kFresh>
__device__ __noinline__ LaneAcc<NP> general_segment(LaneAcc<NP> acc, LaneTgt<NP> tg,
                                                    const float4* SS, const int* orig,
                                                    int64_t group, int* near_cnt,
                                                    unsigned* near_idx,
                                                    unsigned long long* flags, float rho_lo,
                                                    float rho_hi) {
  constexpr int V = L::V;
  const int lane = threadIdx.x & 31;
#pragma unroll 1
  for (int j = 0; j < SEG; ++j) {
    const typename L::Src src = L::load(SS + j * V);
    float2 dx[NP], dy[NP], dz[NP], r2[NP];
    unsigned inr = 0;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      pair_d(tg.t[p], src.nx, src.ny, src.nz, dx[p], dy[p], dz[p], r2[p]);
      inr |= (__any_sync(FULL, (r2[p].x < tg.t[p].rc2.x) | (r2[p].y < tg.t[p].rc2.y)) ? 1u : 0u)
             << p;
    }
    if (inr) {
      unsigned near_bits = 0;
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        if ((inr >> p) & 1u)
          near_bits |= pair_general<L>(src, tg.t[p], dx[p], dy[p], dz[p], r2[p], acc.u[p],
                                       rho_lo, rho_hi)
                       << (2 * p);
        else
          L::far(src, dx[p], dy[p], dz[p], r2[p], acc.u[p]);
      }
      near_append_warp<NP, kFresh>(near_bits, lane, group, orig + j, near_cnt, near_idx, flags);
    } else {
#pragma unroll
      for (int p = 0; p < NP; ++p) L::far(src, dx[p], dy[p], dz[p], r2[p], acc.u[p]);
    }
  }
  return acc;
}

// The general loop over the 32 sources of one segment that is wide for some
// target of the warp (L::kExactNear): pairs with rho_T <= rho < rho_c on a
// target for which the segment is wide take the exact difference (the
// target's frame-shift residual, recomputed from its (hi, lo) column ts, minus
// the source's residual ylo[j]); every other pair computes what the inline
// general loop computes, in the same order, so the accumulators come out bit
// for bit as there. Out of line: its registers do not weigh on the pair loop,
// and wide segments are rare on dense surfaces.
template <class L, int NP, bool kFresh>
__device__ __noinline__ LaneAcc<NP> exact_segment(
    LaneAcc<NP> acc, LaneTgt<NP> tg, const float4* SS, const float4* __restrict__ ylo,
    const int* orig, const float4* ts, float sx, float sy, float sz, float hs, int64_t group,
    int* near_cnt, unsigned* near_idx, unsigned long long* flags, float rho_lo, float rho_hi) {
  constexpr int V = L::V;
  const int lane = threadIdx.x & 31;
#pragma unroll 1
  for (int j = 0; j < SEG; ++j) {
    const typename L::Src src = L::load(SS + j * V);
    float2 dx[NP], dy[NP], dz[NP], r2[NP];
    bool any = false;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      pair_d(tg.t[p], src.nx, src.ny, src.nz, dx[p], dy[p], dz[p], r2[p]);
      any |= (r2[p].x < tg.t[p].rc2.x) | (r2[p].y < tg.t[p].rc2.y);
    }
    if (__any_sync(FULL, any)) {
      const float4 yl = kFresh ? __ldcg(ylo + j) : ylo[j];
      unsigned near_bits = 0;
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const float4 hx = ts[(p * TGT_SLOTS) * TPB32], hy = ts[(p * TGT_SLOTS + 1) * TPB32],
                     hz = ts[(p * TGT_SLOTS + 2) * TPB32];
        const float2 wd = make_float2(hs * tg.t[p].idl.x > WIDE_FRAME ? 1.f : 0.f,
                                      hs * tg.t[p].idl.y > WIDE_FRAME ? 1.f : 0.f);
        near_bits |= pair_general<L>(
                         src, tg.t[p], dx[p], dy[p], dz[p], r2[p], acc.u[p], rho_lo, rho_hi,
                         mul2(wd, sub2(shift_residual2(lo2(hx), hi2(hx), sx, tg.t[p].x),
                                       make_float2(yl.x, yl.x))),
                         mul2(wd, sub2(shift_residual2(lo2(hy), hi2(hy), sy, tg.t[p].y),
                                       make_float2(yl.y, yl.y))),
                         mul2(wd, sub2(shift_residual2(lo2(hz), hi2(hz), sz, tg.t[p].z),
                                       make_float2(yl.z, yl.z))))
                     << (2 * p);
      }
      near_append_warp<NP, kFresh>(near_bits, lane, group, orig + j, near_cnt, near_idx, flags);
    } else {
#pragma unroll
      for (int p = 0; p < NP; ++p) L::far(src, dx[p], dy[p], dz[p], r2[p], acc.u[p]);
    }
  }
  return acc;
}

// Shared memory of a pair item: the source stages; the per-thread target
// state (TGT_SLOTS float4 per f32x2 pair: (hi, lo) of x, y, z, then
// (1/delta, rho_c^2 delta^2), (rho_T^2 delta^2, -)), read once per segment;
// and, for one pair per lane, the compensated accumulators. With one pair per
// lane three CTAs share an SM, so that configuration runs one stage fewer.
template <class L>
__host__ __device__ constexpr bool hilo_in_smem(int np) {
  // one pair per lane: the freed registers buy the third CTA per SM; two
  // pairs, single layer: still two CTAs per SM in shared memory, and the
  // freed registers measured 1% faster (the stresslet's larger records would
  // drop it to one CTA per SM, so it keeps them in registers)
  return np == 1 || (np == 2 && L::V == V_SL);
}
template <class L, int NP>
__host__ __device__ constexpr int pair_stages() {
  return NP == 1 ? L::STAGES - 1 : L::STAGES;
}

template <class L, int NP>
constexpr size_t pair_smem_bytes() {
  return (size_t)pair_stages<L, NP>() * TILE * L::V * sizeof(float4) +
         (size_t)NP * TGT_SLOTS * TPB32 * sizeof(float4) +
         (hilo_in_smem<L>(NP) ? (size_t)NP * 6 * TPB32 * sizeof(float2) : 0);
}

// Shared-memory state of the source pipeline of one CTA.
template <int STAGES>
struct PipeSmem {
  uint64_t full[STAGES];  // stage b's bulk copy landed (transaction count)
  int rel[STAGES];        // warps that released stage b so far (monotonic)
  int issued[STAGES];     // copies issued into stage b (for the drain after a timeout)
  int timed_out;
  int initialized;
};

// Arguments of the FP32 pair sums of one evaluation (or one served request).
struct PairArgs {
  const float4* srcF;
  const float4* segbox;
  const int* src_orig;
  const int* meta;
  const float4* tgtF;
  const double4_32a* tgt64;
  int64_t M_pad;
  int n_chunks;
  double* part;
  int* near_cnt;       // per target group (64 * NP targets)
  unsigned* near_idx;  // per target group: NEAR_K * 64 * NP entries
  unsigned long long* flags;
  float rho_lo, rho_hi;
  const float4* srcLo = nullptr;  // double layer: residuals of the packed positions
};

// The source tiles of one work item: n tiles, each (first packed source,
// segments of SEG sources, at most TILE_SEGS). With desc == nullptr they are
// the full tiles k0 .. k0 + n - 1 of the packed array; a list serves work
// whose tiles are scattered (the FMM's neighbouring clusters and
// equivalent sources).
// out(a, t): where the item writes target t's partial. A list's item
// writes its block's partials to slot * tb (t - t_sub indexes the block).
struct TileList {
  static constexpr bool kFull = false;  // tiles may have fewer than TILE_SEGS segments
  const int2* desc;
  int n;
  int slot, tb;
  int64_t t_sub;
  __device__ __forceinline__ int2 tile(int it) const { return desc[it]; }
  __device__ __forceinline__ size_t first_segment(int, int src0) const {
    return (size_t)(src0 / SEG);
  }
  __device__ __forceinline__ double* out(const PairArgs& a, int64_t t) const {
    return a.part + ((size_t)slot * tb + (size_t)(t - t_sub)) * 3;
  }
};
// A contiguous range of full tiles k0 .. k0 + n - 1 of source chunk ch
// (known to be full at compile time, so the direct evaluation's loops keep
// their fixed shape); partials at [ch][M_pad][3].
struct TileRange {
  static constexpr bool kFull = true;
  int k0, n, ch;
  __device__ __forceinline__ int2 tile(int it) const {
    return make_int2((k0 + it) * TILE, TILE_SEGS);
  }
  __device__ __forceinline__ size_t first_segment(int it, int) const {
    return (size_t)(k0 + it) * TILE_SEGS;
  }
  __device__ __forceinline__ double* out(const PairArgs& a, int64_t t) const {
    return a.part + ((size_t)ch * a.M_pad + t) * 3;
  }
};

// Tiles of source chunk ch of a direct evaluation: an even split of the
// padded sources into a.n_chunks contiguous ranges.
template <bool kFresh = false>
__device__ __forceinline__ TileRange chunk_tiles(const PairArgs& a, int ch) {
  const int n_tiles = (kFresh ? __ldcg(a.meta + META_NS_PAD) : a.meta[META_NS_PAD]) / TILE;
  const int k0 = (int)((long long)ch * n_tiles / a.n_chunks);
  const int k1 = (int)((long long)(ch + 1) * n_tiles / a.n_chunks);
  return TileRange{k0, k1 - k0, ch};
}

// One work item: target block tb (TPB32 * 2 * NP sorted targets) against
// the source tiles tl. Writes the block's partials (target t at
// tl.out(a, t)); returns false if a bounded wait expired (the flag is set,
// nothing is written).
// kFresh: the evaluation's data is read with fresh loads (ld.global.cg), for
// the server's persistent kernel.
template <class L, int NP, bool kFresh = false, class TL>
__device__ __forceinline__ bool pair_item(const PairArgs& a, int tb, const TL& tl, float4* sm,
                                          PipeSmem<pair_stages<L, NP>()>& ps) {
  constexpr int V = L::V;
  constexpr int STAGES = pair_stages<L, NP>();
  constexpr int WARPS = TPB32 / 32;
  constexpr uint32_t SEG_BYTES = SEG * V * sizeof(float4);
  const float4* __restrict__ srcF = a.srcF;
  const float4* __restrict__ segbox = a.segbox;
  const int* __restrict__ src_orig = a.src_orig;
  const float4* __restrict__ tgtF = a.tgtF;
  const double4_32a* __restrict__ tgt64 = a.tgt64;
  int* __restrict__ near_cnt = a.near_cnt;
  unsigned* __restrict__ near_idx = a.near_idx;
  unsigned long long* __restrict__ flags = a.flags;
  const float rho_lo = a.rho_lo, rho_hi = a.rho_hi;
  uint64_t* full = ps.full;
  int* rel = ps.rel;
  int* issued = ps.issued;

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int n_it = tl.n;

  // ---- targets of this lane: pair p holds targets (base + 64p + lane, base + 64p + 32 + lane)
  const int64_t wbase = (int64_t)tb * (TPB32 * 2 * NP) + wid * (64 * NP) + lane;
  // this warp's target group (its near-pair list)
  const int64_t group = (int64_t)tb * (TPB32 / 32) + wid;
  // per-thread target state: [(p * TGT_SLOTS + slot) * TPB32 + tid]
  float4* const ts = sm + STAGES * TILE * V + tid;
  Tgt2 T[NP];
  float blo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, bhi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
  float rc2max = -1.f;
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    float4 a[2], b[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t t = wbase + 64 * p + 32 * h;
      a[h] = kFresh ? __ldcg(tgtF + 2 * t) : tgtF[2 * t];
      b[h] = kFresh ? __ldcg(tgtF + 2 * t + 1) : tgtF[2 * t + 1];
      if (b[h].x >= 0.f) {
        blo[0] = fminf(blo[0], a[h].x); bhi[0] = fmaxf(bhi[0], a[h].x);
        blo[1] = fminf(blo[1], a[h].y); bhi[1] = fmaxf(bhi[1], a[h].y);
        blo[2] = fminf(blo[2], a[h].z); bhi[2] = fmaxf(bhi[2], a[h].z);
        rc2max = fmaxf(rc2max, b[h].x);
      }
    }
    ts[(p * TGT_SLOTS + 3) * TPB32] = make_float4(a[0].w, a[1].w, b[0].x, b[1].x);
    ts[(p * TGT_SLOTS + 4) * TPB32] = make_float4(b[0].y, b[1].y, 0.f, 0.f);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      blo[c] = fminf(blo[c], __shfl_xor_sync(FULL, blo[c], o));
      bhi[c] = fmaxf(bhi[c], __shfl_xor_sync(FULL, bhi[c], o));
    }
    rc2max = fmaxf(rc2max, __shfl_xor_sync(FULL, rc2max, o));
  }
  const bool warp_live = rc2max >= 0.f;
  // FP32 (hi, lo) split of the targets' FP64 coordinates
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const double4_32a x0 = kFresh ? ldcg4d(tgt64 + wbase + 64 * p) : tgt64[wbase + 64 * p],
                      x1 = kFresh ? ldcg4d(tgt64 + wbase + 64 * p + 32)
                                  : tgt64[wbase + 64 * p + 32];
    const double a0[3] = {x0.x, x0.y, x0.z}, a1[3] = {x1.x, x1.y, x1.z};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float h0 = (float)a0[c], h1 = (float)a1[c];
      ts[(p * TGT_SLOTS + c) * TPB32] =
          make_float4(h0, h1, (float)(a0[c] - (double)h0), (float)(a1[c] - (double)h1));
    }
  }
  float rc2test;
  {
    const float rc = sqrtf(fmaxf(rc2max, 0.f));
    const float cmax = fmaxf(fmaxf(fmaxf(fabsf(blo[0]), fabsf(bhi[0])),
                                   fmaxf(fabsf(blo[1]), fabsf(bhi[1]))),
                             fmaxf(fabsf(blo[2]), fabsf(bhi[2])));
    const float rm = rc * 1.00005f + box_margin(cmax, rc);
    rc2test = rm * rm;
  }

  // Compensated accumulators (hi, lo): in shared memory, touched once per 128
  // sources, or in registers (hilo_in_smem gives the measured choice).
  constexpr bool kHiLoSmem = hilo_in_smem<L>(NP);
  float2 U[NP][3], HI[NP][3], LO[NP][3];
  // [(p * 3 + c) * 2 + {0: hi, 1: lo}][thread]: one float2 column per thread
  float2* acc = reinterpret_cast<float2*>(sm + STAGES * TILE * V + NP * TGT_SLOTS * TPB32);
#pragma unroll
  for (int p = 0; p < NP; ++p)
#pragma unroll
    for (int c = 0; c < 3; ++c) U[p][c] = HI[p][c] = LO[p][c] = make_float2(0.f, 0.f);
  if constexpr (kHiLoSmem) {
#pragma unroll
    for (int i = 0; i < NP * 6; ++i) acc[i * TPB32 + tid] = make_float2(0.f, 0.f);
  }

  // ---- source pipeline: no CTA-wide barrier inside the loop; the last warp
  // to release a stage issues the next bulk copy into it.
  __syncthreads();  // the previous item (if any) no longer uses the stages
  if (tid == 0) {
    for (int b = 0; b < STAGES; ++b) {
      if (ps.initialized) mbar_inval(&full[b]);
      mbar_init(&full[b]);
      rel[b] = 0;
      issued[b] = 0;
    }
    ps.initialized = 1;
    ps.timed_out = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    for (int b = 0; b < STAGES; ++b)
      if (b < n_it) {
        if constexpr (TL::kFull) {
          bulk_load(sm + b * TILE * V, srcF + (size_t)(tl.k0 + b) * TILE * V, TILE * V * 16u,
                    &full[b]);
        } else {
          const int2 t = tl.tile(b);
          bulk_load(sm + b * TILE * V, srcF + (size_t)t.x * V, t.y * SEG_BYTES, &full[b]);
        }
        issued[b] = 1;
      }
  }
  for (int it = 0; it < n_it; ++it) {
    // first packed source and segments of this tile
    int src0, nseg;
    if constexpr (TL::kFull) {
      src0 = (tl.k0 + it) * TILE;
      nseg = TILE_SEGS;
    } else {
      const int2 tile = tl.tile(it);
      src0 = tile.x;
      nseg = tile.y;
    }
    const int buf = it % STAGES;
    const int use = it / STAGES;
    const bool ok = __all_sync(FULL, mbar_wait_bounded(&full[buf], (uint32_t)(use & 1)));
    if (!ok) {
      if (lane == 0) atomicExch(&ps.timed_out, 1);
      break;
    }
    if (warp_live) {
      const float4* S = sm + buf * TILE * V;
      bool nb = false;
      float csx = 0.f, csy = 0.f, csz = 0.f;  // lane s < nseg: segment s's frame
      float chs = 0.f;                        // ... and the half extent of its box
      if (lane < nseg) {
        const size_t sg = tl.first_segment(it, src0);
        const float4 lo = kFresh ? __ldcg(segbox + 2 * (sg + lane)) : segbox[2 * (sg + lane)];
        const float4 hi =
            kFresh ? __ldcg(segbox + 2 * (sg + lane) + 1) : segbox[2 * (sg + lane) + 1];
        const float dx = fmaxf(0.f, fmaxf(lo.x - bhi[0], blo[0] - hi.x));
        const float dy = fmaxf(0.f, fmaxf(lo.y - bhi[1], blo[1] - hi.y));
        const float dz = fmaxf(0.f, fmaxf(lo.z - bhi[2], blo[2] - hi.z));
        nb = dx * dx + dy * dy + dz * dz < rc2test;
        csx = frame_mid(lo.x, hi.x);
        csy = frame_mid(lo.y, hi.y);
        csz = frame_mid(lo.z, hi.z);
        if constexpr (L::kExactNear)
          chs = 0.5f * fmaxf(fmaxf(hi.x - lo.x, hi.y - lo.y), hi.z - lo.z);
      }
      const unsigned nm = __ballot_sync(FULL, nb);
#pragma unroll 1
      for (int s = 0; s < nseg; ++s) {
        const float4* SS = S + s * SEG * V;
        const float sx = __shfl_sync(FULL, csx, s), sy = __shfl_sync(FULL, csy, s),
                    sz = __shfl_sync(FULL, csz, s);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          const float4 hx = ts[(p * TGT_SLOTS) * TPB32], hy = ts[(p * TGT_SLOTS + 1) * TPB32],
                       hz = ts[(p * TGT_SLOTS + 2) * TPB32];
          T[p].x = shift_to_segment2(lo2(hx), hi2(hx), sx);
          T[p].y = shift_to_segment2(lo2(hy), hi2(hy), sy);
          T[p].z = shift_to_segment2(lo2(hz), hi2(hz), sz);
        }
        if (!((nm >> s) & 1u)) {
#pragma unroll kFarUnroll
          for (int j = 0; j < SEG; ++j) {
            const typename L::Src src = L::load(SS + j * V);
#pragma unroll
            for (int p = 0; p < NP; ++p) {
              float2 dx, dy, dz, r2;
              pair_d(T[p], src.nx, src.ny, src.nz, dx, dy, dz, r2);
              L::far(src, dx, dy, dz, r2, U[p]);
            }
          }
        } else {
          const int* orig = src_orig + (size_t)src0 + s * SEG;
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            const float4 q = ts[(p * TGT_SLOTS + 3) * TPB32], r = ts[(p * TGT_SLOTS + 4) * TPB32];
            T[p].idl = lo2(q);
            T[p].rc2 = hi2(q);
            T[p].rt2 = lo2(r);
          }
          // Exact differences (L::kExactNear) where the segment is wide for a
          // target: its frame half extent above WIDE_FRAME target deltas, so
          // that FP32 rounding of |x - c| and |y - c| could swamp an O(r^2)
          // (x - y) . n. Decided per target and segment, so a target's result
          // does not depend on the warp it landed in.
          bool wide = false;
          const float hs = __shfl_sync(FULL, chs, s);
          if constexpr (L::kExactNear) {
#pragma unroll
            for (int p = 0; p < NP; ++p)
              wide |= (hs * T[p].idl.x > WIDE_FRAME) | (hs * T[p].idl.y > WIDE_FRAME);
            wide = __any_sync(FULL, wide);
          }
          if (!wide) {
            LaneAcc<NP> acc;
            LaneTgt<NP> tg;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
              tg.t[p] = T[p];
#pragma unroll
              for (int c = 0; c < 3; ++c) acc.u[p][c] = U[p][c];
            }
            acc = general_segment<L, NP, kFresh>(acc, tg, SS, orig, group, near_cnt, near_idx, flags,
                                         rho_lo, rho_hi);
#pragma unroll
            for (int p = 0; p < NP; ++p)
#pragma unroll
              for (int c = 0; c < 3; ++c) U[p][c] = acc.u[p][c];
          } else if constexpr (L::kExactNear) {
            LaneAcc<NP> acc;
            LaneTgt<NP> tg;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
              tg.t[p] = T[p];
#pragma unroll
              for (int c = 0; c < 3; ++c) acc.u[p][c] = U[p][c];
            }
            acc = exact_segment<L, NP, kFresh>(acc, tg, SS, a.srcLo + (size_t)src0 + s * SEG,
                                       orig, ts, sx, sy, sz, hs, group, near_cnt, near_idx,
                                       flags, rho_lo, rho_hi);
#pragma unroll
            for (int p = 0; p < NP; ++p)
#pragma unroll
              for (int c = 0; c < 3; ++c) U[p][c] = acc.u[p][c];
          }
        }
        // at most 128 sources in plain FP32 (a full tile ends on a merge)
        if ((s & 3) == 3 || (!TL::kFull && s == nseg - 1)) {
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            if constexpr (kHiLoSmem) {
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                HI[p][c] = acc[((p * 3 + c) * 2) * TPB32 + tid];
                LO[p][c] = acc[((p * 3 + c) * 2 + 1) * TPB32 + tid];
              }
            }
            two_sum_merge(U[p], HI[p], LO[p]);
            if constexpr (kHiLoSmem) {
#pragma unroll
              for (int c = 0; c < 3; ++c) {
                acc[((p * 3 + c) * 2) * TPB32 + tid] = HI[p][c];
                acc[((p * 3 + c) * 2 + 1) * TPB32 + tid] = LO[p][c];
              }
            }
          }
        }
      }
    }
    // release the stage; the last of the WARPS releases refills it
    __syncwarp();
    if (lane == 0) {
      __threadfence_block();
      const int prev = atomicAdd(&rel[buf], 1);
      if (prev == (use + 1) * WARPS - 1 && it + STAGES < n_it) {
        __threadfence_block();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if constexpr (TL::kFull) {
          bulk_load(sm + buf * TILE * V, srcF + (size_t)(tl.k0 + it + STAGES) * TILE * V,
                    TILE * V * 16u, &full[buf]);
        } else {
          const int2 t = tl.tile(it + STAGES);
          bulk_load(sm + buf * TILE * V, srcF + (size_t)t.x * V, t.y * SEG_BYTES, &full[buf]);
        }
        atomicAdd(&issued[buf], 1);
      }
    }
  }
  __syncthreads();
  if (ps.timed_out) {
    if (tid == 0) {
      atomicExch(flags + FLAG_TIMEOUT, 1ull);
      // wait (bounded) for the last copy issued into each stage before leaving
      for (int b = 0; b < STAGES; ++b)
        if (issued[b] > 0) mbar_wait_bounded(&full[b], (uint32_t)((issued[b] - 1) & 1));
    }
    return false;
  }
#pragma unroll
  for (int p = 0; p < NP; ++p)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t t = wbase + 64 * p + 32 * h;
      double* o = tl.out(a, t);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float2 H2 = kHiLoSmem ? acc[((p * 3 + c) * 2) * TPB32 + tid] : HI[p][c];
        const float2 L2 = kHiLoSmem ? acc[((p * 3 + c) * 2 + 1) * TPB32 + tid] : LO[p][c];
        const float hv = h ? H2.y : H2.x;
        const float lv = h ? L2.y : L2.x;
        o[c] = (double)hv + (double)lv;
      }
    }
  return true;
}

// FP64 near pair of the finish/overflow kernels, by layer.
template <class L>
struct Near64;

template <>
struct Near64<SLayer> {
  __device__ __forceinline__ static void eval(double4_32a x, const double* xyz, const double* w,
                                              const double* f, const double* /*nrm*/, int64_t j,
                                              double scale, double invd, double& u0, double& u1,
                                              double& u2) {
    sl_pair64(x.x - xyz[3 * j], x.y - xyz[3 * j + 1], x.z - xyz[3 * j + 2], f[3 * j], f[3 * j + 1],
              f[3 * j + 2], w[j] * scale, invd, u0, u1, u2);
  }
};

template <>
struct Near64<DLayer> {
  __device__ __forceinline__ static void eval(double4_32a x, const double* xyz, const double* w,
                                              const double* q, const double* nrm, int64_t j,
                                              double scale, double invd, double& u0, double& u1,
                                              double& u2) {
    dl_pair64(x.x - xyz[3 * j], x.y - xyz[3 * j + 1], x.z - xyz[3 * j + 2], q[3 * j], q[3 * j + 1],
              q[3 * j + 2], nrm[3 * j], nrm[3 * j + 1], nrm[3 * j + 2], w[j] * scale, invd, u0, u1,
              u2);
  }
};

// Arguments of the near-list overflow rescan and of the finish step.
struct OverflowArgs {
  const float4* srcF;
  const float4* segbox;
  const int* src_orig;
  const int* meta;
  const float4* tgtF;
  const double4_32a* tgt64;
  const int* near_cnt;  // per target group
  const double* xyz;
  const double* w;
  const double* dens;
  const double* nrm;
  double scale;
  const unsigned long long* flags;
  double* near_ovf;
  int group = 0;  // targets per group: 64 * (f32x2 pairs per lane) of the pair kernel
};

struct FinishArgs {
  const double4_32a* tgt64;
  const int* perm;
  int64_t M_pad;
  int n_chunks;
  const double* part;
  const int* near_cnt;       // per target group
  const unsigned* near_idx;  // per target group
  const double* near_ovf;
  const double* xyz;
  const double* w;
  const double* dens;
  const double* nrm;
  double scale;
  double* u;
  unsigned long long* flags;
  int group = 0;  // targets per group: 64 * (f32x2 pairs per lane) of the pair kernel
};

// FP64 near sum of target t by a rescan of all packed sources with exactly the
// FP32 test of the pair kernel, split over the calling warp's lanes and
// summed by a fixed butterfly (deterministic); every lane gets the sum.
template <class L>
__device__ __forceinline__ void rescan_target(const OverflowArgs& a, int64_t t, double& u0,
                                              double& u1, double& u2) {
  const int lane = threadIdx.x & 31;
  constexpr int V = L::V;
  const float rt2 = a.tgtF[2 * t + 1].y;
  const double4_32a x = a.tgt64[t];
  const double invd = 1.0 / x.w;
  const float hx = (float)x.x, hy = (float)x.y, hz = (float)x.z;
  const float lx = (float)(x.x - (double)hx), ly = (float)(x.y - (double)hy),
              lz = (float)(x.z - (double)hz);
  const int Ns = a.meta[META_NS];
  u0 = u1 = u2 = 0;
  for (int s = lane; s < Ns; s += 32) {
    const float4 blo = a.segbox[2 * (s / SEG)], bhi = a.segbox[2 * (s / SEG) + 1];
    const float tx = shift_to_segment(hx, lx, frame_mid(blo.x, bhi.x));
    const float ty = shift_to_segment(hy, ly, frame_mid(blo.y, bhi.y));
    const float tz = shift_to_segment(hz, lz, frame_mid(blo.z, bhi.z));
    const float4 p0 = a.srcF[(size_t)s * V], p1 = a.srcF[(size_t)s * V + 1];
    const float dx = __fadd_rn(tx, p0.x), dy = __fadd_rn(ty, p0.z), dz = __fadd_rn(tz, p1.x);
    const float r2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    if (r2 < rt2) Near64<L>::eval(x, a.xyz, a.w, a.dens, a.nrm, a.src_orig[s], a.scale, invd, u0, u1, u2);
  }
  for (int o = 16; o > 0; o >>= 1) {
    u0 += __shfl_xor_sync(FULL, u0, o);
    u1 += __shfl_xor_sync(FULL, u1, o);
    u2 += __shfl_xor_sync(FULL, u2, o);
  }
}

// Target t's group list overflowed: the calling warp rescans for it and
// stores the sum for the finish.
template <class L>
__device__ __forceinline__ void overflow_target(const OverflowArgs& a, int64_t t) {
  if (a.near_cnt[t / a.group] <= NEAR_K * a.group) return;
  double u0, u1, u2;
  rescan_target<L>(a, t, u0, u1, u2);
  if ((threadIdx.x & 31) == 0) {
    a.near_ovf[3 * t] = u0;
    a.near_ovf[3 * t + 1] = u1;
    a.near_ovf[3 * t + 2] = u2;
  }
}

// Finish one sorted target: chunk partials in fixed order plus the FP64 near
// sum (list sorted by source index, or the overflow rescan's sum); writes
// u at the target's original index. Returns the target's near-pair count.
// v[0 .. n) in ascending order, by one thread: insertion sort for short runs,
// heapsort for long ones (a group list may hold thousands of one target's
// entries).
__device__ __forceinline__ void sort_entries(unsigned* v, int n) {
  if (n <= 32) {
    for (int i = 1; i < n; ++i) {
      const unsigned x = v[i];
      int k = i;
      while (k > 0 && v[k - 1] > x) {
        v[k] = v[k - 1];
        --k;
      }
      v[k] = x;
    }
    return;
  }
  auto sift = [v](int root, int end) {
    for (int c = 2 * root + 1; c < end; c = 2 * root + 1) {
      if (c + 1 < end && v[c] < v[c + 1]) ++c;
      if (v[root] >= v[c]) return;
      const unsigned x = v[root];
      v[root] = v[c];
      v[c] = x;
      root = c;
    }
  };
  for (int i = n / 2 - 1; i >= 0; --i) sift(i, n);
  for (int e = n - 1; e > 0; --e) {
    const unsigned x = v[0];
    v[0] = v[e];
    v[e] = x;
    sift(0, e);
  }
}

// Shared 32-bit words of one warp's near-sum scratch for groups of G targets:
// the same in every kernel that finishes such groups, so that a target's sum
// never depends on which kernel finished it.
__host__ __device__ constexpr int near_warp_words(int G) { return G <= 64 ? 2048 : 3200; }

// Barrier of a team of TEAM threads: one warp, or the whole CTA.
template <int TEAM>
__device__ __forceinline__ void team_sync() {
  if constexpr (TEAM == 32) __syncwarp();
  else __syncthreads();
}

// FP64 near sums of target group g (G = a.group targets) by a team of TEAM
// threads (one warp, or a CTA of TEAM threads; tid = the thread's place in
// it) with the shared words R[0 .. near_warp_words(G)); fin(t, n0, n1, n2)
// then finishes target t (one thread per target). The group list is bucketed
// by target in R, in passes over target ranges whose entries fit, and each
// bucket sorted by source index: every target sums its near pairs in
// ascending source order, whatever the order of the appends. The targets of
// an overflowed group take their overflow rescan sums; a target with more
// near pairs than R holds is rescanned here. Returns the near pairs this
// thread counted.
template <class L, int TEAM, class Fin>
__device__ __forceinline__ int near_group(const OverflowArgs& oa, const FinishArgs& a, int64_t g,
                                          unsigned* R, int tid, Fin fin) {
  const int G = a.group, CAP = NEAR_K * G, lane = tid & 31;
  int* const cnt = reinterpret_cast<int*>(R);  // per target: count, then fill position
  int* const beg = cnt + G;                    // per target: first entry (exclusive scan)
  unsigned* const ent = R + 2 * G + 1;
  const int EW = near_warp_words(G) - (2 * G + 1);
  const int64_t tg0 = g * G;
  const int c = a.near_cnt[g];
  if (c > CAP) {
    for (int k = tid; k < G; k += TEAM) {
      const int64_t t = tg0 + k;
      fin(t, a.near_ovf[3 * t], a.near_ovf[3 * t + 1], a.near_ovf[3 * t + 2]);
    }
    return tid == 0 ? c : 0;
  }
  const unsigned* list = a.near_idx + (size_t)g * CAP;
  for (int k = tid; k < G; k += TEAM) cnt[k] = 0;
  team_sync<TEAM>();
  for (int i = tid; i < c; i += TEAM) atomicAdd(&cnt[list[i] >> NEAR_SRC_BITS], 1);
  team_sync<TEAM>();
  if (tid < 32) {
    int run = 0;
    for (int k0 = 0; k0 < G; k0 += 32) {
      const int v = cnt[k0 + lane];
      int x = v;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
      }
      beg[k0 + lane] = run + x - v;
      run += __shfl_sync(FULL, x, 31);
    }
    if (lane == 0) beg[G] = run;
  }
  team_sync<TEAM>();
  int pairs = 0;
  for (int ka = 0; ka < G;) {
    // the longest target range [ka, kb) whose entries fit (at least one target)
    int lo = ka + 1, hi = G;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (beg[mid] - beg[ka] <= EW) lo = mid;
      else hi = mid - 1;
    }
    const int kb = lo, base = beg[ka];
    if (beg[kb] - base <= EW) {
      for (int k = ka + tid; k < kb; k += TEAM) cnt[k] = beg[k] - base;
      team_sync<TEAM>();
      for (int i = tid; i < c; i += TEAM) {
        const unsigned e = list[i];
        const int k = (int)(e >> NEAR_SRC_BITS);
        if (k >= ka && k < kb) ent[atomicAdd(&cnt[k], 1)] = e & ((1u << NEAR_SRC_BITS) - 1u);
      }
      team_sync<TEAM>();
      for (int k = ka + tid; k < kb; k += TEAM) {
        const int64_t t = tg0 + k;
        const int b0 = beg[k] - base, b1 = beg[k + 1] - base;
        sort_entries(ent + b0, b1 - b0);
        const double4_32a x = a.tgt64[t];
        const double invd = 1.0 / x.w;
        double n0 = 0, n1 = 0, n2 = 0;
        for (int i = b0; i < b1; ++i)
          Near64<L>::eval(x, a.xyz, a.w, a.dens, a.nrm, (int)ent[i], a.scale, invd, n0, n1, n2);
        pairs += b1 - b0;
        fin(t, n0, n1, n2);
      }
    } else if (tid < 32) {
      // target ka alone has more near pairs than R holds: the team's first
      // warp rescans for it
      const int64_t t = tg0 + ka;
      double n0, n1, n2;
      rescan_target<L>(oa, t, n0, n1, n2);
      if (lane == 0) {
        pairs += beg[ka + 1] - base;
        fin(t, n0, n1, n2);
      }
    }
    team_sync<TEAM>();
    ka = kb;
  }
  return pairs;
}

// Near sums of targets t0 .. t0 + nt - 1 (whole groups) by the calling CTA:
// warp w takes groups w, w + warps, ...; R holds near_warp_words(group) shared
// words per warp.
template <class L, class Fin>
__device__ __forceinline__ int near_groups(const OverflowArgs& oa, const FinishArgs& a,
                                           int64_t t0, int nt, unsigned* R, Fin fin) {
  const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int W = near_warp_words(a.group);
  int pairs = 0;
  for (int q = wid; q < nt / a.group; q += nw)
    pairs += near_group<L, 32>(oa, a, t0 / a.group + q, R + (size_t)wid * W, threadIdx.x & 31,
                               fin);
  return pairs;
}

// Target t of a direct evaluation: its chunk partials in chunk order plus its
// FP64 near sum, written at the target's original index.
__device__ __forceinline__ void finish_merge(const FinishArgs& a, int64_t t, double n0, double n1,
                                             double n2) {
  double u0 = 0, u1 = 0, u2 = 0;
  for (int c = 0; c < a.n_chunks; ++c) {
    const double* p = a.part + ((size_t)c * a.M_pad + t) * 3;
    u0 += p[0];
    u1 += p[1];
    u2 += p[2];
  }
  const int64_t j = a.perm[t];
  a.u[3 * j] = u0 + n0;
  a.u[3 * j + 1] = u1 + n1;
  a.u[3 * j + 2] = u2 + n2;
}

// Drop from L2, without writing them back, the 128-byte lines lying wholly
// inside [begin, begin + bytes): scratch that has been read for the last
// time in this evaluation (chunk partials, near lists of a finished target
// block). Lines only partly inside are left alone, so no other block's data
// is touched. The calling threads (tid of n) split the lines.
__device__ __forceinline__ void discard_l2(const void* begin, size_t bytes, int tid, int n) {
  const size_t g = (size_t)__cvta_generic_to_global(begin);
  const size_t a = (g + 127) & ~(size_t)127, e = (g + bytes) & ~(size_t)127;
  for (size_t q = a + (size_t)tid * 128; q < e; q += (size_t)n * 128)
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(q) : "memory");
}

// The scratch of targets t0 .. t0 + nt - 1 after their finish: their chunk
// partials and near lists.
__device__ __forceinline__ void discard_block_scratch(const FinishArgs& fa, int64_t t0, int nt,
                                                      int tid, int n) {
  for (int c = 0; c < fa.n_chunks; ++c)
    discard_l2(fa.part + ((size_t)c * fa.M_pad + t0) * 3, (size_t)nt * 3 * sizeof(double), tid, n);
  discard_l2(fa.near_idx + (size_t)t0 * NEAR_K, (size_t)nt * NEAR_K * sizeof(int), tid, n);
}

// Finish targets t0 .. t0 + nt - 1 (of M real ones) of a target block whose
// chunks are all done: overflow rescans (if any list overflowed), FP64 near
// sums and chunk merge, and the near-pair count. Run by a whole CTA, with
// near_warp_words(group) free shared words per warp at sm; kept out of line
// so that the pair loop's register allocation does not carry it.
template <class L>
__device__ __noinline__ void finish_block(const OverflowArgs& oa, const FinishArgs& fa, int64_t M,
                                          int64_t t0, int nt, unsigned* sm) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  if (*(volatile const unsigned long long*)&fa.flags[FLAG_OVERFLOW] != 0ull) {
    for (int i = wid; i < nt; i += nw)
      if (t0 + i < M) overflow_target<L>(oa, t0 + i);
    __syncthreads();
    __threadfence_block();
  }
  int cnt = near_groups<L>(oa, fa, t0, nt, sm, [&](int64_t t, double n0, double n1, double n2) {
    if (t < M) finish_merge(fa, t, n0, n1, n2);
  });
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULL, cnt, o);
  if (lane == 0 && cnt) atomicAdd(fa.flags + FLAG_NEAR_PAIRS, (unsigned long long)cnt);
  __syncthreads();  // every read of the block's partials and near lists is done
  discard_block_scratch(fa, t0, nt, tid, blockDim.x);
}

}  // namespace p32
}  // namespace sk
