// sk_internal.h -- shared declarations of libstokesreg (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cfloat>
#include <cstddef>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/stokesreg.h"

namespace sk {

// ---- work decomposition of the pair kernels --------------------------------
constexpr int SEG = 32;                 // sources per segment (near/far classification unit)
constexpr int TILE_SEGS = 8;
constexpr int TILE = SEG * TILE_SEGS;   // sources per shared-memory tile (FP32 kernels)
#ifndef SK_TPB32
#define SK_TPB32 256
#endif
constexpr int TPB32 = SK_TPB32;         // threads per CTA, FP32 kernels
constexpr int TPL32 = 4;                // targets per lane (two f32x2 pairs)
constexpr int TGT_WARP32 = 32 * TPL32;  // 128 targets per warp
constexpr int TGT_CTA32 = TPB32 * TPL32;
constexpr int TILE64 = 128;             // sources per tile, FP64 kernels
constexpr int TPB64 = 256;
constexpr int TPL64 = 2;
constexpr int TGT_WARP64 = 32 * TPL64;
constexpr int TGT_CTA64 = TPB64 * TPL64;
constexpr int NEAR_K = 96;              // FP64 near-pair slots per target (pooled per group)
constexpr int NEAR_GROUP_MIN = 64;      // targets per near-list group: 64 * (f32x2 pairs per lane)
constexpr int NEAR_SRC_BITS = 25;       // near-list entry: source index bits (the rest: target)
// SK_FP32C lists near pairs by the source's original index in NEAR_SRC_BITS bits
constexpr int64_t FP32C_MAX_SOURCES = int64_t(1) << NEAR_SRC_BITS;
// any precision: sources and targets of one evaluation (sorted indices are int)
constexpr int64_t MAX_POINTS = int64_t(1) << 30;
constexpr int RHO_C64 = 7;              // FP64 path: s_i == 1 to double precision beyond 7

// layer kinds
constexpr int LAYER_SL = 0;
constexpr int LAYER_DL = 1;

// float4 records per source in the packed FP32 layout
constexpr int V_SL = 3;
constexpr int V_DL = 5;

// device flag slots (unsigned long long)
constexpr int FLAG_TIMEOUT = 0;
constexpr int FLAG_OVERFLOW = 1;
constexpr int FLAG_NEAR_PAIRS = 2;
constexpr int FLAG_BAD_DELTA = 3;
constexpr int N_FLAGS = 8;

// meta ints written on the device by the preparation kernels
constexpr int META_NS = 0;       // active sources
constexpr int META_NS_PAD = 1;   // padded to a multiple of TILE (FP32) / TILE64 (FP64)
constexpr int META_SCRATCH = 2;  // count slot of the target sort (all targets are active)
constexpr int N_META = 8;

constexpr double PI_CONST = 3.14159265358979323846;

// bounded waits: about one second at 2 GHz
constexpr long long WAIT_CYCLES = 2000000000LL;

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

#ifdef __CUDACC__
// Local frame of a group of points (the 32 sources of a segment, the targets
// of a warp): the FP32 midpoint of the group's FP32 bounding box, 0 for an
// empty box (lo > hi). The FP32 pair kernels store coordinates relative to
// these frames, taken from the FP64 input, so a source-target difference is
// accurate to FP32 rounding of |x - y| plus the frames' extents rather than of
// |x| and |y|. That matters for the stresslet, whose (x - y) . n cancels to
// O(r^2) for close pairs on the surface. Pack, pair and rescan kernels all
// call this one definition, so they agree bit for bit.
__device__ __forceinline__ float frame_mid(float lo, float hi) {
  return lo <= hi ? __fmul_rn(__fadd_rn(lo, hi), 0.5f) : 0.f;
}

// Writes the FP32 box of the warp's real points (lane 0) and returns its
// midpoint frame to every lane. All 32 lanes call it (the packers run whole
// warps over slots padded to multiples of 32).
__device__ __forceinline__ float3 warp_box(bool real, float x, float y, float z, float4* out) {
  constexpr float BIG = FLT_MAX;
  float lx = real ? x : BIG, ly = real ? y : BIG, lz = real ? z : BIG;
  float hx = real ? x : -BIG, hy = real ? y : -BIG, hz = real ? z : -BIG;
  for (int o = 16; o > 0; o >>= 1) {
    lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
    ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
    lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
    hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, o));
    hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, o));
    hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, o));
  }
  if ((threadIdx.x & 31) == 0) {
    out[0] = make_float4(lx, ly, lz, 0.f);
    out[1] = make_float4(hx, hy, hz, 0.f);
  }
  return make_float3(frame_mid(lx, hx), frame_mid(ly, hy), frame_mid(lz, hz));
}

// Single-layer FP32 source record (duplicated lanes for f32x2 arithmetic):
// {-x,-x,-y,-y} {-z,-z,gx,gx} {gy,gy,gz,gz}, x relative to the segment frame.
__device__ __forceinline__ void write_sl_record(float4* o, float x, float y, float z, float g0,
                                                float g1, float g2) {
  o[0] = make_float4(-x, -x, -y, -y);
  o[1] = make_float4(-z, -z, g0, g0);
  o[2] = make_float4(g1, g1, g2, g2);
}
#endif

// Padding sources sit this far away, with zero density.
constexpr float PAD_POS = 1.0e15f;

// Bump allocator over one device buffer; a null base only measures.
struct Bump {
  char* base = nullptr;
  size_t off = 0;
  template <class T>
  T* take(size_t n) {
    off = align_up(off, 256);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
};

// Buffers of one evaluation, carved from the context workspace.
struct EvalBufs {
  // FP64 inputs on the device (caller's pointers or copies in the workspace)
  const double* src_xyz = nullptr;
  const double* src_w = nullptr;
  const double* dens = nullptr;   // f (single layer) or q (double layer)
  const double* nrm = nullptr;    // double layer only
  const double* tgt_xyz = nullptr;
  const double* delta = nullptr;
  double* u = nullptr;            // device result
  // sort scratch
  uint32_t* keys_a = nullptr;
  uint32_t* keys_b = nullptr;
  int* vals_a = nullptr;
  int* vals_b = nullptr;
  uint32_t* hist = nullptr;       // [256][sort_blocks] digit counts, then 256 row totals
  float* bbox_part = nullptr;
  float* bbox = nullptr;
  // scratch of the target sort: the sort scratch above, unless the shape
  // splits the sorts (then a set of its own, so that the two sorts can run at
  // the same time)
  uint32_t* tkeys_a = nullptr;
  uint32_t* tkeys_b = nullptr;
  int* tvals_a = nullptr;
  int* tvals_b = nullptr;
  uint32_t* thist = nullptr;
  float* tbbox_part = nullptr;
  float* tbbox = nullptr;
  // prepared sources / targets
  int* meta = nullptr;
  int* src_orig = nullptr;        // packed source -> original index (-1: padding)
  float4* srcF = nullptr;         // FP32 packed sources
  float4* srcLo = nullptr;        // double layer, FP32C: residual (y - c) - fl32(y - c) per source
  double4_32a* src64 = nullptr;       // FP64 packed sources (pos, density)
  double4_32a* nrm64 = nullptr;       // FP64 packed normals (double layer)
  float4* segbox = nullptr;       // per segment: lo, hi
  int* tgt_perm = nullptr;        // sorted target -> original index
  float4* tgtF = nullptr;         // FP32 sorted targets: (x, y, z, 1/delta), (rc2, rt2, 0, 0)
  double4_32a* tgt64 = nullptr;       // FP64 sorted targets: (x, y, z, delta)
  // accumulation
  double* part = nullptr;         // [n_chunks][M_pad][3]
  int* near_cnt = nullptr;        // [M_pad / NEAR_GROUP_MIN] entries per target group
  int* tb_done = nullptr;         // [M_pad / 512 + 1] chunks done per target block (FP32C)
  unsigned* near_idx = nullptr;   // [M_pad / group][NEAR_K * group] near-pair entries
  double* near_ovf = nullptr;     // [M_pad][3]
  unsigned long long* flags = nullptr;
  // sizes
  int64_t N = 0, M = 0, N_pad = 0, M_pad = 0;
  int n_chunks = 1;
  int pair_np = 2;  // FP32 pair kernel: f32x2 target pairs per lane (1 or 2)
  bool fuse_finish = false;  // FP32C: the pair kernel finishes the target blocks
  int threads64 = TPB64;  // FP64 pair kernel: threads per CTA
  int sort_blocks = 0;
};

// FP32 pair kernel configuration: two f32x2 target pairs per lane at two
// CTAs per SM for large target counts, one pair per lane at three CTAs per SM
// (more warps, smaller target blocks) otherwise.
#ifndef SK_NP1_MAX_TARGETS
#define SK_NP1_MAX_TARGETS 131072
#endif
constexpr int64_t PAIR32_NP1_MAX_TARGETS = SK_NP1_MAX_TARGETS;
inline int pair32_np(int64_t M) { return M > PAIR32_NP1_MAX_TARGETS ? 2 : 1; }
#ifndef SK_MINB_NP2
#define SK_MINB_NP2 (512 / SK_TPB32)
#endif
#ifndef SK_MINB_NP1
#define SK_MINB_NP1 (768 / SK_TPB32)
#endif
constexpr int PAIR32_MINB_NP2 = SK_MINB_NP2, PAIR32_MINB_NP1 = SK_MINB_NP1;
inline int pair32_ctas_per_sm(int np) { return np == 2 ? PAIR32_MINB_NP2 : PAIR32_MINB_NP1; }

}  // namespace sk

struct sk_server;

namespace sk {
struct MembraneOp;
struct FmmOp;
}

struct sk_ctx {
  int device = 0;
  sk_server* server = nullptr;  // at most one server per context
  cudaStream_t stream = nullptr;
  // second stream and fork/join events of the preparation (sk::PrepFork)
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t fork_ev = nullptr;
  cudaEvent_t join_ev = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_fixed = false;
  unsigned long long* h_flags = nullptr;  // pinned copy of the device flags
  cudaStream_t last_stream = nullptr;
  int sm_count = 0;
  double rho_T = 0.5;
  double rho_c = 5.0;
  bool profile = false;
  int64_t small_sort_points = 0;  // single-block sort limit (sk::SMALL_SORT_POINTS unless overridden)
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // eval begin, pair begin/end, eval end
  sk_eval_stats stats{};
  std::vector<std::pair<int, sk::MembraneOp*>> membrane_ops;  // derivative operators by m
  std::vector<std::pair<int, sk::FmmOp*>> fmm_ops;            // FMM operators by p
  std::string err;
};

namespace sk {

// Largest point set ordered by the single-block sort by default;
// SK_SMALL_SORT_POINTS in the environment of sk_create overrides it per
// context (0 turns it off). Measured: one block costs ~24 us more per extra
// 1024-point tile than the fifteen multi-block launches, and saves ~30 us at
// two tiles, so the break-even is near three tiles.
constexpr int64_t SMALL_SORT_POINTS = 3072;

// CTA size of the FP64 pair kernel for problems too small to fill the GPU
// with TPB64-thread CTAs (TPL64 targets per lane in both)
constexpr int TPB64_SMALL = 64;

// Shape of one evaluation.
struct EvalShape {
  int layer = LAYER_SL;
  int precision = SK_FP32C;
  int64_t N = 0, M = 0, n_delta = 1;
  double mu = 1.0;
  bool copy_inputs = false;  // inputs/outputs live in the workspace (host-memory calls)
  int n_chunks = 1;
  int threads64 = TPB64;  // CTA size of the FP64 pair kernel (TPB64 or TPB64_SMALL)
  bool fuse_finish = false;  // FP32C: finish target blocks inside the pair kernel
  // point sets of at most this many points are ordered by one single-block
  // kernel instead of fifteen launches (0: never)
  int64_t small_sort_points = SMALL_SORT_POINTS;
  // the target sort takes scratch of its own and runs beside the source sort
  // on a second stream (context evaluations, capsule steps, served requests;
  // the allocation-free call keeps one set)
  bool split_sorts = false;
};

// A second stream and two events that let the preparation run the target
// sort beside the source sort: fork is recorded on the evaluation's stream
// and waited for on aux; join the other way round.
struct PrepFork {
  cudaStream_t aux = nullptr;
  cudaEvent_t fork = nullptr;
  cudaEvent_t join = nullptr;
};

// sk_api.cu
// Grow the context workspace to `need` bytes (synchronizes the device when it
// reallocates); SK_ENOMEM for a fixed workspace that is too small.
int ensure_workspace(sk_ctx* ctx, size_t need);
size_t eval_workspace_bytes(const EvalShape& s);
void carve_eval_buffers(Bump& bp, const EvalShape& s, EvalBufs& b);
// choose_chunks and choose_decomposition (the split into work items): sk_decomp.h
double layer_scale(const EvalShape& s);  // 1/(8 pi mu) or -6/(8 pi)
// pf (optional) forks the target sort onto pf->aux when s.split_sorts.
int enqueue_prep(const EvalShape& s, const EvalBufs& b, double rho_T, double rho_c,
                 cudaStream_t st, const PrepFork* pf = nullptr);
// Returns the number of kernels launched. ev (optional, 4 events) brackets
// the whole evaluation (ev[0], ev[3]) and the pair kernel (ev[1], ev[2]).
int enqueue_eval(const EvalShape& s, const EvalBufs& b, double rho_T, double rho_c,
                 cudaStream_t st, cudaEvent_t* ev = nullptr, const PrepFork* pf = nullptr);

// launchers (sk_prep.cu)
void launch_sort_points(const double* xyz, const double* w, int64_t n, uint32_t* keys_a,
                        uint32_t* keys_b, int* vals_a, int* vals_b, uint32_t* hist,
                        float* bbox_part, float* bbox, int* count_out, int64_t small_max_points,
                        cudaStream_t st);
// Stable LSD radix sort of (key, value) pairs by the low `bits` bits of the
// keys, 8 bits per pass, in the buffers of launch_sort_points (hist holds
// 256 * sort_grid_blocks(n) + 256 words). Returns 0 when the sorted pairs are
// in (keys_a, vals_a), 1 when they are in (keys_b, vals_b).
int launch_sort_pairs(uint32_t* keys_a, uint32_t* keys_b, int* vals_a, int* vals_b, int64_t n,
                      int bits, uint32_t* hist, cudaStream_t st);
void launch_pack_sources32(int layer, const EvalBufs& b, double scale, cudaStream_t st);
void launch_pack_sources64(int layer, const EvalBufs& b, double scale, cudaStream_t st);
void launch_pack_targets32(const EvalBufs& b, int64_t n_delta, double rho_T, double rho_c,
                           cudaStream_t st);
void launch_pack_targets64(const EvalBufs& b, int64_t n_delta, cudaStream_t st);
int sort_grid_blocks(int64_t n);

// launchers (sk_pair32.cu / sk_pair64.cu)
// FP32C pair sums and the finish of every target block (overflow rescans,
// FP64 near sums, chunk merge, output write): fused into the pair kernel when
// b.fuse_finish, else two more launches. pair_end (optional) is recorded
// after the pair kernel, before any finish launch.
void launch_pair32(int layer, const EvalBufs& b, double rho_T, double scale, cudaStream_t st,
                   cudaEvent_t pair_end = nullptr);
void launch_pair64(int layer, const EvalBufs& b, double scale, cudaStream_t st);
void launch_finish64(const EvalBufs& b, cudaStream_t st);

// One evaluation with the argument checks, statistics and flags of the
// public entry points (stokes_sl_eval / stokes_dl_eval).
int eval_call(sk_ctx* ctx, int layer, int precision, int mem, int64_t N, const double* xyz,
              const double* w, const double* dens, const double* nrm, int64_t M,
              const double* txyz, const double* delta, int64_t n_delta, double mu,
              double* u_out, void* stream);

// sk_capsule.cu: capsule steps run by the server. A served request holds
// the capsule (try_acquire) until it completes; each step enqueues its sum's
// inputs (membrane force, weights, delta*), the sum, then the update.
bool capsule_try_acquire(sk_capsule* c);
void capsule_release(sk_capsule* c);
sk_ctx* capsule_ctx(const sk_capsule* c);
bool capsule_servable(const sk_capsule* c);  // SK_FP32C, no upsampling
int64_t capsule_node_count(const sk_capsule* c);
EvalShape capsule_step_shape(const sk_capsule* c);
const double* capsule_nodes(const sk_capsule* c);
const unsigned long long* capsule_sticky(const sk_capsule* c);
// set: the membrane operator's scratch copy used on st (see
// membrane_scratch_set; capsule_prepare_sets builds them beforehand).
int capsule_prepare_sets(sk_capsule* c, int n_sets);
void capsule_enqueue_step_inputs(sk_capsule* c, EvalBufs& b, cudaStream_t st, int set);
void capsule_enqueue_step_update(sk_capsule* c, const unsigned long long* flags, double dt,
                                 const sk_flow& fl, cudaStream_t st);
void capsule_clear_sticky(sk_capsule* c, cudaStream_t st);

// sk_fmm.cu: single-level FMM operators (cached per p in ctx)
void free_fmm_ops(sk_ctx* ctx);

// sk_membrane.cu: overset finite-difference derivatives and the Skalak force
// on the six-patch grid of order m (built once per m and cached in ctx).
int membrane_op(sk_ctx* ctx, int m, MembraneOp** out);
int membrane_scratch_set(sk_ctx* ctx, MembraneOp* op, int i, MembraneOp** out);
void free_membrane_ops(sk_ctx* ctx);
int64_t membrane_nodes(const MembraneOp& op);
// Wraw (optional): the area element W itself.
void enqueue_tangents(const MembraneOp& op, const double* X, double* t6, double* w,
                      cudaStream_t st, double* Wraw = nullptr);
void enqueue_skalak(const MembraneOp& op, const double* X, const double* ref6, double Es,
                    double ED, double* f, double* w, cudaStream_t st, double* Wraw = nullptr);
// Four-times upsampled single layer (Sec. 3.4): buffers built on first use;
// enqueue_upsample fills the fine sources and the coarse targets' delta.
struct UpsampledSources {
  int64_t Nup;
  const double *X, *w, *f, *delta;
  double* W;  // [N] staging for the coarse area element
};
int membrane_upsampling(sk_ctx* ctx, MembraneOp* op);
void enqueue_upsample(const MembraneOp& op, const double* X, const double* W, const double* f,
                      cudaStream_t st);
UpsampledSources upsampled_sources(const MembraneOp& op);
void enqueue_area_volume(const MembraneOp& op, const double* X, double* out2, cudaStream_t st);
void enqueue_moments(const MembraneOp& op, const double* X, double* out16, cudaStream_t st);

}  // namespace sk
