// sk_pair32.cu -- kernels and launchers of the FP32-compensated pair sums
// (device code in sk_pair32.cuh).
#include "sk_pair32.cuh"

namespace sk {
namespace {

using namespace p32;

// One work item (target block tb, source chunk ch) per CTA. In the fused
// kernel (many target blocks) the CTA that completes a block's last chunk
// finishes that block (FP64 near sums, chunk merge): that FP64 work then runs
// beside other CTAs' FP32 pair work instead of in kernels of its own. With
// few blocks a block's finish on one CTA would become the tail, so the plain
// kernel is followed by the finish kernels below.
template <class L, int NP, int MINB>
__global__ void __launch_bounds__(TPB32, MINB) k_pair32(PairArgs a) {
  extern __shared__ __align__(128) float4 sm[];
  __shared__ PipeSmem<pair_stages<L, NP>()> ps;
  if (threadIdx.x == 0) ps.initialized = 0;
  const int tb = blockIdx.x / a.n_chunks, ch = blockIdx.x % a.n_chunks;
  pair_item<L, NP>(a, tb, chunk_tiles(a, ch), sm, ps);
}

template <class L, int NP, int MINB>
__global__ void __launch_bounds__(TPB32, MINB)
    k_pair32_fused(PairArgs a, OverflowArgs oa, FinishArgs fa, int* __restrict__ tb_done,
                   int64_t M) {
  extern __shared__ __align__(128) float4 sm[];
  __shared__ PipeSmem<pair_stages<L, NP>()> ps;
  __shared__ int s_last;
  if (threadIdx.x == 0) ps.initialized = 0;
  const int tb = blockIdx.x / a.n_chunks, ch = blockIdx.x % a.n_chunks;
  pair_item<L, NP>(a, tb, chunk_tiles(a, ch), sm, ps);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // this chunk's partials and near-list entries before the count
    s_last = atomicAdd(&tb_done[tb], 1) == a.n_chunks - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  constexpr int TB = TPB32 * 2 * NP;  // targets per block
  // the source stages are free now: the finish buckets the near lists there
  static_assert(pair_smem_bytes<L, NP>() / 4 >= (size_t)(TPB32 / 32) * near_warp_words(64 * NP),
                "finish scratch");
  finish_block<L>(oa, fa, M, (int64_t)tb * TB, TB, reinterpret_cast<unsigned*>(sm));
}

template <class L>
__global__ void k_overflow32(OverflowArgs a, int64_t M) {
  if (a.flags[FLAG_OVERFLOW] == 0ull) return;
  const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (t >= M) return;
  overflow_target<L>(a, t);
}

// Separate finish for grids too small to fuse it: one CTA of G threads per
// target group of G targets (a thread per target), the near-sum scratch in
// dynamic shared memory.
template <class L, int G>
__global__ void __launch_bounds__(G) k_finish32(OverflowArgs oa, FinishArgs a, int64_t M) {
  extern __shared__ unsigned fsm[];
  const int64_t t0 = (int64_t)blockIdx.x * G;
  int cnt = near_group<L, G>(oa, a, blockIdx.x, fsm, threadIdx.x,
                             [&](int64_t t, double n0, double n1, double n2) {
                               if (t < M) finish_merge(a, t, n0, n1, n2);
                             });
  // count near pairs: one atomic per warp
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(FULL, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(a.flags + FLAG_NEAR_PAIRS, (unsigned long long)cnt);
  __syncthreads();  // this group's targets are finished: their scratch is dead
  discard_block_scratch(a, t0, G, threadIdx.x, blockDim.x);
}

}  // namespace

template <class L, int NP>
void launch_pair32_t(const EvalBufs& b, float rho_lo, float rho_hi, double scale, cudaStream_t st,
                     cudaEvent_t pair_end) {
  constexpr int MINB = NP == 2 ? PAIR32_MINB_NP2 : PAIR32_MINB_NP1;
  const unsigned grid = (unsigned)((b.M_pad / (TPB32 * 2 * NP)) * b.n_chunks);
  const size_t smem = pair_smem_bytes<L, NP>();
  PairArgs a{b.srcF,  b.segbox,   b.src_orig, b.meta,     b.tgtF,  b.tgt64, b.M_pad,
             b.n_chunks, b.part, b.near_cnt, b.near_idx, b.flags, rho_lo, rho_hi, b.srcLo};
  OverflowArgs oa{b.srcF, b.segbox, b.src_orig, b.meta,  b.tgtF,  b.tgt64,     b.near_cnt,
                  b.src_xyz, b.src_w, b.dens,   b.nrm, scale, b.flags, b.near_ovf};
  FinishArgs fa{b.tgt64, b.tgt_perm, b.M_pad, b.n_chunks, b.part, b.near_cnt, b.near_idx,
                b.near_ovf, b.src_xyz, b.src_w, b.dens, b.nrm, scale, b.u, b.flags};
  oa.group = fa.group = 64 * NP;
  if (b.fuse_finish) {
    cudaFuncSetAttribute(k_pair32_fused<L, NP, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    k_pair32_fused<L, NP, MINB><<<grid, TPB32, smem, st>>>(a, oa, fa, b.tb_done, b.M);
    if (pair_end) cudaEventRecord(pair_end, st);
  } else {
    cudaFuncSetAttribute(k_pair32<L, NP, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    k_pair32<L, NP, MINB><<<grid, TPB32, smem, st>>>(a);
    if (pair_end) cudaEventRecord(pair_end, st);
    k_overflow32<L><<<(unsigned)((b.M * 32 + 255) / 256), 256, 0, st>>>(oa, b.M);
    constexpr int G = 64 * NP;
    const size_t fsmem = (size_t)near_warp_words(G) * sizeof(unsigned);
    k_finish32<L, G><<<(unsigned)(b.M_pad / G), G, fsmem, st>>>(oa, fa, b.M);
  }
}

void launch_pair32(int layer, const EvalBufs& b, double rho_T, double scale, cudaStream_t st,
                   cudaEvent_t pair_end) {
  const float rho_lo = (float)rho_T, rho_hi = 8.0f;
  if (layer == LAYER_SL) {
    if (b.pair_np == 2)
      launch_pair32_t<SLayer, 2>(b, rho_lo, rho_hi, scale, st, pair_end);
    else
      launch_pair32_t<SLayer, 1>(b, rho_lo, rho_hi, scale, st, pair_end);
  } else {
    if (b.pair_np == 2)
      launch_pair32_t<DLayer, 2>(b, rho_lo, rho_hi, scale, st, pair_end);
    else
      launch_pair32_t<DLayer, 1>(b, rho_lo, rho_hi, scale, st, pair_end);
  }
}

}  // namespace sk
