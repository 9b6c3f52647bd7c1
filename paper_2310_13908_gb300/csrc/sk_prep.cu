// sk_prep.cu -- preparation of one evaluation: spatial ordering and packing.
//
// Sources with nonzero weight and all targets are put in Morton (Z-curve)
// order of their position so that a warp's 128 targets and a segment's 32
// sources are compact in space; the near/far test of the pair kernels then
// touches few segments. Zero-weight sources get the largest key and fall
// behind the active ones, which compacts them away. The sort is a stable
// least-significant-digit radix sort (4 passes of 8 bits), so the order --
// and every result -- is deterministic.
#include "sk_internal.h"

#include <cfloat>

namespace sk {

namespace {

#ifndef SK_RS_ITEMS
#define SK_RS_ITEMS 4
#endif
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = SK_RS_ITEMS;  // keys per thread and radix tile (large sorts)
// Up to RS_FINE_MAX keys, tiles of one key per thread: four times the blocks
// for the same keys, which the short launches of mid-size sorts need.
constexpr int64_t RS_FINE_MAX = 65536;
inline int rs_items(int64_t n) { return n <= RS_FINE_MAX ? 1 : RS_ITEMS; }
inline int rs_tiles(int64_t n, int items) {
  return (int)((n + (int64_t)RS_THREADS * items - 1) / ((int64_t)RS_THREADS * items));
}
constexpr int BBOX_BLOCKS = 128;
constexpr unsigned FULL = 0xffffffffu;

// ---- bounding box of the (active) points -----------------------------------
// Min/max over points i = first, first + stride, ... of this block, reduced
// over the block; threads 0..5 return (lo x, y, z, hi x, y, z) in *out.
// (Min and max do not depend on the grouping, so one block or many give the
// same box.)
__device__ void bbox_block(const double* __restrict__ xyz, const double* __restrict__ w,
                           int64_t n, int64_t first, int64_t stride, float (*s)[RS_THREADS],
                           float* out) {
  float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
  for (int64_t i = first; i < n; i += stride) {
    if (w && w[i] == 0.0) continue;
    for (int c = 0; c < 3; ++c) {
      float v = (float)xyz[3 * i + c];
      lo[c] = fminf(lo[c], v);
      hi[c] = fmaxf(hi[c], v);
    }
  }
  for (int c = 0; c < 3; ++c) {
    s[c][threadIdx.x] = lo[c];
    s[3 + c][threadIdx.x] = hi[c];
  }
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      for (int c = 0; c < 3; ++c) {
        s[c][threadIdx.x] = fminf(s[c][threadIdx.x], s[c][threadIdx.x + k]);
        s[3 + c][threadIdx.x] = fmaxf(s[3 + c][threadIdx.x], s[3 + c][threadIdx.x + k]);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < 6) *out = s[threadIdx.x][0];
}

__global__ void k_bbox_partial(const double* __restrict__ xyz, const double* __restrict__ w,
                               int64_t n, float* __restrict__ part) {
  __shared__ float s[6][RS_THREADS];
  float v;
  bbox_block(xyz, w, n, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
             (int64_t)gridDim.x * blockDim.x, s, &v);
  if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = v;
}

// One warp per box component (6 warps): lanes stride over the partial boxes,
// then a shuffle reduction.
__global__ void k_bbox_final(const float* __restrict__ part, int nblk, float* __restrict__ bbox) {
  const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (c >= 6) return;  // whole warps
  float v = c < 3 ? FLT_MAX : -FLT_MAX;
  for (int b = lane; b < nblk; b += 32) v = c < 3 ? fminf(v, part[b * 6 + c]) : fmaxf(v, part[b * 6 + c]);
  for (int o = 16; o > 0; o >>= 1) {
    const float w = __shfl_xor_sync(FULL, v, o);
    v = c < 3 ? fminf(v, w) : fmaxf(v, w);
  }
  if (lane == 0) bbox[c] = v;
}

// Spread the low 10 bits of v so that bit i lands at bit 3i.
__device__ __forceinline__ uint32_t spread3(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// Morton key of point i (0xffffffff for a zero-weight source); true if active.
__device__ __forceinline__ bool morton_key(const double* __restrict__ xyz,
                                           const double* __restrict__ w, int64_t i,
                                           const float* bbox, uint32_t* key) {
  const bool active = !(w && w[i] == 0.0);
  *key = 0xffffffffu;
  if (active) {
    float ext = fmaxf(fmaxf(bbox[3] - bbox[0], bbox[4] - bbox[1]), bbox[5] - bbox[2]);
    float sc = ext > 0.f ? 1023.0f / ext : 0.f;
    uint32_t q[3];
    for (int c = 0; c < 3; ++c) {
      float v = ((float)xyz[3 * i + c] - bbox[c]) * sc;
      v = fminf(fmaxf(v, 0.f), 1023.f);
      q[c] = (uint32_t)v;
    }
    *key = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
  }
  return active;
}

__global__ void k_morton_keys(const double* __restrict__ xyz, const double* __restrict__ w,
                              int64_t n, const float* __restrict__ bbox,
                              uint32_t* __restrict__ keys, int* __restrict__ vals,
                              int* __restrict__ count) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  bool active = false;
  if (i < n) {
    uint32_t key;
    active = morton_key(xyz, w, i, bbox, &key);
    keys[i] = key;
    vals[i] = (int)i;
  }
  unsigned b = __ballot_sync(FULL, active);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(count, __popc(b));
}

// ---- radix sort: histogram, scan, stable scatter ----------------------------
// Digit counts of tile blk (of nblk; ITEMS keys per thread) into column blk
// of hist[digit][nblk].
template <int ITEMS>
__device__ void rs_hist_tile(const uint32_t* __restrict__ keys, int n, int shift,
                             uint32_t* __restrict__ hist, int blk, int nblk, uint32_t* h) {
  h[threadIdx.x] = 0;
  __syncthreads();
  int base = blk * RS_THREADS * ITEMS;
  for (int r = 0; r < ITEMS; ++r) {
    int i = base + r * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * nblk + blk] = h[threadIdx.x];
}

template <int ITEMS>
__global__ void k_rs_hist(const uint32_t* __restrict__ keys, int n, int shift,
                          uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[256];
  rs_hist_tile<ITEMS>(keys, n, shift, hist, blockIdx.x, gridDim.x, h);
}

// Exclusive scan of `total` counts by one block of THREADS threads: each
// thread sums its own contiguous run, one block scan of the run totals gives
// every run its offset, and the thread rewrites its run (exact integer sums).
template <int THREADS>
__device__ void rs_scan_block(uint32_t* __restrict__ a, int total, uint32_t* warp_sums) {
  static_assert(THREADS % 32 == 0 && THREADS <= 1024, "one block of whole warps");
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int K = (total + THREADS - 1) / THREADS;
  const int b = min(t * K, total), e = min(b + K, total);
  uint32_t v = 0;
  for (int i = b; i < e; ++i) v += a[i];
  uint32_t x = v;  // inclusive warp scan of the run totals
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t s = lane < THREADS / 32 ? warp_sums[lane] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, s, o);
      if (lane >= o) s += y;
    }
    warp_sums[lane] = s;  // inclusive over warps
  }
  __syncthreads();
  uint32_t run = (wid > 0 ? warp_sums[wid - 1] : 0u) + x - v;  // exclusive offset of this run
  for (int i = b; i < e; ++i) {
    const uint32_t c = a[i];
    a[i] = run;
    run += c;
  }
}

// Inclusive scan of one value per thread over a block of RS_THREADS threads;
// *total gets the block's sum. Ends with the block synchronized, so the
// warp_sums scratch can be reused at once.
__device__ __forceinline__ uint32_t block_scan_incl(uint32_t v, uint32_t* warp_sums,
                                                   uint32_t* total) {
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  uint32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(FULL, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t s = lane < RS_THREADS / 32 ? warp_sums[lane] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(FULL, s, o);
      if (lane >= o) s += y;
    }
    if (lane < RS_THREADS / 32) warp_sums[lane] = s;  // inclusive over warps
  }
  __syncthreads();
  const uint32_t r = (wid > 0 ? warp_sums[wid - 1] : 0u) + x;
  *total = warp_sums[RS_THREADS / 32 - 1];
  __syncthreads();
  return r;
}

// Per digit d = blockIdx.x (one block per digit): exclusive scan, in place,
// of row d of hist[256][nblk] (contiguous, so the loads are coalesced), and
// the row's total into tot[d]. With the exclusive scan of tot (done by each
// scatter block), offset(d, b) = sum of tot below d + row prefix (d, b): the
// same integers as one scan of the whole flattened array.
__global__ void __launch_bounds__(RS_THREADS) k_rs_rowscan(uint32_t* __restrict__ hist, int nblk,
                                                           uint32_t* __restrict__ tot) {
  __shared__ uint32_t warp_sums[RS_THREADS / 32];
  uint32_t* row = hist + (size_t)blockIdx.x * nblk;
  uint32_t carry = 0;
  for (int base = 0; base < nblk; base += RS_THREADS) {
    const int i = base + threadIdx.x;
    const uint32_t v = i < nblk ? row[i] : 0u;
    uint32_t sum;
    const uint32_t incl = block_scan_incl(v, warp_sums, &sum);
    if (i < nblk) row[i] = carry + incl - v;
    carry += sum;
  }
  if (threadIdx.x == 0) tot[blockIdx.x] = carry;
}

// Stable scatter of tile blk (of nblk; ITEMS keys per thread) to the offsets
// of column blk of offs, plus digit_base (this thread's digit) when offs holds
// row prefixes only.
template <int ITEMS>
__device__ void rs_scatter_tile(const uint32_t* __restrict__ kin, const int* __restrict__ vin,
                                uint32_t* __restrict__ kout, int* __restrict__ vout, int n,
                                int shift, const uint32_t* __restrict__ offs, uint32_t digit_base,
                                int blk, int nblk, uint32_t* base_d, uint32_t (*wcnt)[256]) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  base_d[tid] = offs[tid * nblk + blk] + digit_base;
  const unsigned lt = (1u << lane) - 1u;
  const int base = blk * RS_THREADS * ITEMS;
  for (int r = 0; r < ITEMS; ++r) {
    for (int w = 0; w < RS_THREADS / 32; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    int i = base + r * RS_THREADS + tid;
    bool valid = i < n;
    uint32_t key = valid ? kin[i] : 0u;
    uint32_t dig = (key >> shift) & 255u;
    unsigned peers = __match_any_sync(FULL, valid ? dig : (256u + lane));
    unsigned rank = __popc(peers & lt);
    if (valid && rank == 0) wcnt[wid][dig] = __popc(peers);
    __syncthreads();
    if (valid) {
      uint32_t off = 0;
      for (int w = 0; w < wid; ++w) off += wcnt[w][dig];
      uint32_t pos = base_d[dig] + off + rank;
      kout[pos] = key;
      vout[pos] = vin[i];
    }
    __syncthreads();
    uint32_t add = 0;
    for (int w = 0; w < RS_THREADS / 32; ++w) add += wcnt[w][tid];
    base_d[tid] += add;
    __syncthreads();
  }
}

// offs: row prefixes from k_rs_rowscan; tot: the rows' totals.
template <int ITEMS>
__global__ void __launch_bounds__(RS_THREADS)
    k_rs_scatter(const uint32_t* __restrict__ kin, const int* __restrict__ vin,
                 uint32_t* __restrict__ kout, int* __restrict__ vout, int n, int shift,
                 const uint32_t* __restrict__ offs, const uint32_t* __restrict__ tot) {
  static_assert(RS_THREADS == 256, "one thread per digit");
  __shared__ uint32_t base_d[256];
  __shared__ uint32_t wcnt[RS_THREADS / 32][256];
  __shared__ uint32_t warp_sums[RS_THREADS / 32];
  const uint32_t t = tot[threadIdx.x];
  uint32_t all;
  const uint32_t digit_base = block_scan_incl(t, warp_sums, &all) - t;
  rs_scatter_tile<ITEMS>(kin, vin, kout, vout, n, shift, offs, digit_base, blockIdx.x, gridDim.x,
                         base_d, wcnt);
}

// The whole ordering of a small point set in one block of RS_THREADS threads:
// box, Morton keys and the four radix passes, tile by tile, with the same
// device code as the multi-block launches, so the order is the same. Saves
// fourteen launches (and their gaps) per point set.
__global__ void __launch_bounds__(RS_THREADS)
    k_sort_small(const double* __restrict__ xyz, const double* __restrict__ w, int64_t n,
                 uint32_t* __restrict__ keys_a, uint32_t* __restrict__ keys_b,
                 int* __restrict__ vals_a, int* __restrict__ vals_b, uint32_t* __restrict__ hist,
                 float* __restrict__ bbox, int* __restrict__ count_out, int nblk) {
  __shared__ float sbox[6][RS_THREADS];
  __shared__ float box[6];
  __shared__ uint32_t h[256];
  __shared__ uint32_t warp_sums[32];
  __shared__ uint32_t base_d[256];
  __shared__ uint32_t wcnt[RS_THREADS / 32][256];
  __shared__ int active_total;
  const int tid = threadIdx.x;
  float v;
  bbox_block(xyz, w, n, tid, RS_THREADS, sbox, &v);
  if (tid < 6) {
    box[tid] = v;
    bbox[tid] = v;
  }
  if (tid == 0) active_total = 0;
  __syncthreads();
  int act = 0;
  for (int64_t i = tid; i < n; i += RS_THREADS) {
    uint32_t key;
    act += morton_key(xyz, w, i, box, &key) ? 1 : 0;
    keys_a[i] = key;
    vals_a[i] = (int)i;
  }
  atomicAdd(&active_total, act);
  uint32_t *ka = keys_a, *kb = keys_b;
  int *va = vals_a, *vb = vals_b;
  for (int shift = 0; shift < 32; shift += 8) {
    __syncthreads();  // the keys (or the previous pass's scatter) are complete
    for (int b = 0; b < nblk; ++b) rs_hist_tile<RS_ITEMS>(ka, (int)n, shift, hist, b, nblk, h);
    __syncthreads();
    rs_scan_block<RS_THREADS>(hist, 256 * nblk, warp_sums);
    __syncthreads();
    for (int b = 0; b < nblk; ++b)
      rs_scatter_tile<RS_ITEMS>(ka, va, kb, vb, (int)n, shift, hist, 0u, b, nblk, base_d, wcnt);
    uint32_t* tk = ka; ka = kb; kb = tk;
    int* tv = va; va = vb; vb = tv;
  }
  __syncthreads();
  if (tid == 0) atomicAdd(count_out, active_total);
}

// ---- packing ----------------------------------------------------------------
// FP32 packed layout (duplicated lanes for f32x2 arithmetic), x, y, z relative
// to the segment's frame (frame_mid of its box; padding keeps PAD_POS):
//   single layer: {-x,-x,-y,-y} {-z,-z,gx,gx} {gy,gy,gz,gz},  g = w f scale
//   double layer: {-x,-x,-y,-y} {-z,-z,qx,qx} {qy,qy,qz,qz} {nx,nx,ny,ny} {nz,nz,0,0},
//                 q = w q_in scale; and, in srcLo, the FP32 residuals of the
//                 frame-relative position, (y - c) - fl32(y - c) per axis, from
//                 which the stresslet forms exact differences for pairs inside
//                 rho_c delta
template <int LAYER>
__global__ void k_pack_src32(const double* __restrict__ xyz, const double* __restrict__ w,
                             const double* __restrict__ dens, const double* __restrict__ nrm,
                             const int* __restrict__ sorted, int* __restrict__ meta,
                             int64_t N_pad, double scale, float4* __restrict__ srcF,
                             float4* __restrict__ srcLo, int* __restrict__ src_orig,
                             float4* __restrict__ segbox) {
  constexpr int V = LAYER == LAYER_SL ? V_SL : V_DL;
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int Ns = meta[META_NS];
  const int Ns_pad = (int)align_up((size_t)Ns, TILE);
  if (s == 0) meta[META_NS_PAD] = Ns_pad;
  if (s >= Ns_pad || s >= N_pad) return;  // whole warps leave together (multiples of 32)
  const bool real = s < Ns;
  const int64_t j = real ? sorted[s] : -1;
  float x = PAD_POS, y = PAD_POS, z = PAD_POS;
  if (real) {
    x = (float)xyz[3 * j];
    y = (float)xyz[3 * j + 1];
    z = (float)xyz[3 * j + 2];
  }
  // the box holds absolute FP32 positions; the record holds positions
  // relative to the segment's frame, differenced in FP64
  const float3 c = warp_box(real, x, y, z, segbox + 2 * (s / SEG));
  float d0 = 0.f, d1 = 0.f, d2 = 0.f, n0 = 0.f, n1 = 0.f, n2 = 0.f;
  float4 res = make_float4(0.f, 0.f, 0.f, 0.f);
  if (real) {
    const double rx = xyz[3 * j] - (double)c.x, ry = xyz[3 * j + 1] - (double)c.y,
                 rz = xyz[3 * j + 2] - (double)c.z;
    x = (float)rx;
    y = (float)ry;
    z = (float)rz;
    res = make_float4((float)(rx - (double)x), (float)(ry - (double)y), (float)(rz - (double)z),
                      0.f);
    const double ws = w[j] * scale;
    d0 = (float)(ws * dens[3 * j]);
    d1 = (float)(ws * dens[3 * j + 1]);
    d2 = (float)(ws * dens[3 * j + 2]);
    if (LAYER == LAYER_DL) {
      n0 = (float)nrm[3 * j];
      n1 = (float)nrm[3 * j + 1];
      n2 = (float)nrm[3 * j + 2];
    }
  }
  float4* o = srcF + s * V;
  write_sl_record(o, x, y, z, d0, d1, d2);
  if (LAYER == LAYER_DL) {
    o[3] = make_float4(n0, n0, n1, n1);
    o[4] = make_float4(n2, n2, 0.f, 0.f);
    srcLo[s] = res;
  }
  src_orig[s] = (int)j;
}

// FP64 packed layout: src64[2s] = (x, y, z, 0), src64[2s+1] = (g or q scaled, 0);
// normals in nrm64[s]. Segment boxes are FP32 (the kernel adds a margin).
template <int LAYER>
__global__ void k_pack_src64(const double* __restrict__ xyz, const double* __restrict__ w,
                             const double* __restrict__ dens, const double* __restrict__ nrm,
                             const int* __restrict__ sorted, int* __restrict__ meta,
                             int64_t N_pad, double scale, double4_32a* __restrict__ src64,
                             double4_32a* __restrict__ nrm64, float4* __restrict__ segbox) {
  const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int Ns = meta[META_NS];
  const int Ns_pad = (int)align_up((size_t)Ns, TILE64);
  if (s == 0) meta[META_NS_PAD] = Ns_pad;
  if (s >= Ns_pad || s >= N_pad) return;
  const bool real = s < Ns;
  double x = PAD_POS, y = PAD_POS, z = PAD_POS, d0 = 0, d1 = 0, d2 = 0;
  double4_32a nn = make_double4_32a(0, 0, 0, 0);
  if (real) {
    const int64_t j = sorted[s];
    x = xyz[3 * j];
    y = xyz[3 * j + 1];
    z = xyz[3 * j + 2];
    const double ws = w[j] * scale;
    d0 = ws * dens[3 * j];
    d1 = ws * dens[3 * j + 1];
    d2 = ws * dens[3 * j + 2];
    if (LAYER == LAYER_DL) nn = make_double4_32a(nrm[3 * j], nrm[3 * j + 1], nrm[3 * j + 2], 0.0);
  }
  src64[2 * s] = make_double4_32a(x, y, z, 0.0);
  src64[2 * s + 1] = make_double4_32a(d0, d1, d2, 0.0);
  if (LAYER == LAYER_DL) nrm64[s] = nn;
  warp_box(real, (float)x, (float)y, (float)z, segbox + 2 * (s / SEG));
}

__global__ void k_pack_tgt32(const double* __restrict__ xyz, const double* __restrict__ delta,
                             int64_t n_delta, const int* __restrict__ sorted, int64_t M,
                             int64_t M_pad, double rho_T, double rho_c, float4* __restrict__ tgtF,
                             double4_32a* __restrict__ tgt64, int* __restrict__ perm) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= M_pad) return;
  const bool real = t < M;
  const int64_t j = sorted[real ? t : M - 1];
  const double x = xyz[3 * j], y = xyz[3 * j + 1], z = xyz[3 * j + 2];
  const double d = delta[n_delta == 1 ? 0 : j];
  const double rc = rho_c * d, rt = rho_T * d;
  tgtF[2 * t] = make_float4((float)x, (float)y, (float)z, (float)(1.0 / d));
  tgtF[2 * t + 1] = real ? make_float4((float)(rc * rc), (float)(rt * rt), 0.f, 0.f)
                         : make_float4(-1.f, -1.f, 0.f, 0.f);
  tgt64[t] = make_double4_32a(x, y, z, d);
  perm[t] = real ? (int)j : -1;
}

__global__ void k_pack_tgt64(const double* __restrict__ xyz, const double* __restrict__ delta,
                             int64_t n_delta, const int* __restrict__ sorted, int64_t M,
                             int64_t M_pad, double4_32a* __restrict__ tgt64, int* __restrict__ perm) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= M_pad) return;
  const bool real = t < M;
  const int64_t j = sorted[real ? t : M - 1];
  const double d = delta[n_delta == 1 ? 0 : j];
  // padding targets get a negative delta: the pair kernel skips them
  tgt64[t] = make_double4_32a(xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2], real ? d : -1.0);
  perm[t] = real ? (int)j : -1;
}

inline unsigned blocks_for(int64_t n, int tpb) { return (unsigned)((n + tpb - 1) / tpb); }

}  // namespace

// Blocks (tiles) whose digit counts a sort of up to n keys may need: the
// fine tiling holds more tiles than the coarse one for the same keys.
int sort_grid_blocks(int64_t n) {
  const int fine = rs_tiles(n < RS_FINE_MAX ? n : RS_FINE_MAX, 1);
  const int coarse = rs_tiles(n, RS_ITEMS);
  return fine > coarse ? fine : coarse;
}

// One radix pass (8 bits at shift) of n keys in nblk tiles of ITEMS keys per thread.
static void rs_pass(const uint32_t* ka, const int* va, uint32_t* kb, int* vb, int64_t n, int shift,
             uint32_t* hist, cudaStream_t st) {
  const int items = rs_items(n), nblk = rs_tiles(n, items);
  uint32_t* tot = hist + 256 * (size_t)nblk;  // row totals (hist holds 256 more words)
  if (items == 1)
    k_rs_hist<1><<<nblk, RS_THREADS, 0, st>>>(ka, (int)n, shift, hist);
  else
    k_rs_hist<RS_ITEMS><<<nblk, RS_THREADS, 0, st>>>(ka, (int)n, shift, hist);
  k_rs_rowscan<<<256, RS_THREADS, 0, st>>>(hist, nblk, tot);
  if (items == 1)
    k_rs_scatter<1><<<nblk, RS_THREADS, 0, st>>>(ka, va, kb, vb, (int)n, shift, hist, tot);
  else
    k_rs_scatter<RS_ITEMS><<<nblk, RS_THREADS, 0, st>>>(ka, va, kb, vb, (int)n, shift, hist, tot);
}

void launch_sort_points(const double* xyz, const double* w, int64_t n, uint32_t* keys_a,
                        uint32_t* keys_b, int* vals_a, int* vals_b, uint32_t* hist,
                        float* bbox_part, float* bbox, int* count_out, int64_t small_max_points,
                        cudaStream_t st) {
  if (n <= 0) return;
  // tiles of this point set (at most the sort_grid_blocks the buffers hold);
  // the stable order does not depend on the tiling or on the path
  if (n <= small_max_points) {
    k_sort_small<<<1, RS_THREADS, 0, st>>>(xyz, w, n, keys_a, keys_b, vals_a, vals_b, hist, bbox,
                                           count_out, rs_tiles(n, RS_ITEMS));
    return;  // four passes: the sorted data is in keys_a / vals_a
  }
  k_bbox_partial<<<BBOX_BLOCKS, RS_THREADS, 0, st>>>(xyz, w, n, bbox_part);
  k_bbox_final<<<1, 6 * 32, 0, st>>>(bbox_part, BBOX_BLOCKS, bbox);
  k_morton_keys<<<blocks_for(n, 256), 256, 0, st>>>(xyz, w, n, bbox, keys_a, vals_a, count_out);
  uint32_t *ka = keys_a, *kb = keys_b;
  int *va = vals_a, *vb = vals_b;
  for (int shift = 0; shift < 32; shift += 8) {
    rs_pass(ka, va, kb, vb, n, shift, hist, st);
    uint32_t* tk = ka; ka = kb; kb = tk;
    int* tv = va; va = vb; vb = tv;
  }
  // four passes: the sorted data is back in keys_a / vals_a
}

int launch_sort_pairs(uint32_t* keys_a, uint32_t* keys_b, int* vals_a, int* vals_b, int64_t n,
                      int bits, uint32_t* hist, cudaStream_t st) {
  if (n <= 0) return 0;
  uint32_t *ka = keys_a, *kb = keys_b;
  int *va = vals_a, *vb = vals_b;
  int passes = 0;
  for (int shift = 0; shift < bits; shift += 8, ++passes) {
    rs_pass(ka, va, kb, vb, n, shift, hist, st);
    uint32_t* tk = ka; ka = kb; kb = tk;
    int* tv = va; va = vb; vb = tv;
  }
  return passes & 1;
}

void launch_pack_sources32(int layer, const EvalBufs& b, double scale, cudaStream_t st) {
  unsigned g = blocks_for(b.N_pad, 256);
  if (layer == LAYER_SL)
    k_pack_src32<LAYER_SL><<<g, 256, 0, st>>>(b.src_xyz, b.src_w, b.dens, b.nrm, b.vals_a, b.meta,
                                              b.N_pad, scale, b.srcF, nullptr, b.src_orig,
                                              b.segbox);
  else
    k_pack_src32<LAYER_DL><<<g, 256, 0, st>>>(b.src_xyz, b.src_w, b.dens, b.nrm, b.vals_a, b.meta,
                                              b.N_pad, scale, b.srcF, b.srcLo, b.src_orig,
                                              b.segbox);
}

void launch_pack_sources64(int layer, const EvalBufs& b, double scale, cudaStream_t st) {
  unsigned g = blocks_for(b.N_pad, 256);
  if (layer == LAYER_SL)
    k_pack_src64<LAYER_SL><<<g, 256, 0, st>>>(b.src_xyz, b.src_w, b.dens, b.nrm, b.vals_a, b.meta,
                                              b.N_pad, scale, b.src64, b.nrm64, b.segbox);
  else
    k_pack_src64<LAYER_DL><<<g, 256, 0, st>>>(b.src_xyz, b.src_w, b.dens, b.nrm, b.vals_a, b.meta,
                                              b.N_pad, scale, b.src64, b.nrm64, b.segbox);
}

void launch_pack_targets32(const EvalBufs& b, int64_t n_delta, double rho_T, double rho_c,
                           cudaStream_t st) {
  k_pack_tgt32<<<blocks_for(b.M_pad, 256), 256, 0, st>>>(b.tgt_xyz, b.delta, n_delta, b.tvals_a,
                                                         b.M, b.M_pad, rho_T, rho_c, b.tgtF,
                                                         b.tgt64, b.tgt_perm);
}

void launch_pack_targets64(const EvalBufs& b, int64_t n_delta, cudaStream_t st) {
  k_pack_tgt64<<<blocks_for(b.M_pad, 256), 256, 0, st>>>(b.tgt_xyz, b.delta, n_delta, b.tvals_a,
                                                         b.M, b.M_pad, b.tgt64, b.tgt_perm);
}

}  // namespace sk
