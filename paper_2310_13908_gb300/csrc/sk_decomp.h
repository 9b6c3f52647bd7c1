// sk_decomp.h -- how an evaluation is split into work items: the number of
// source chunks per target block, the FP64 pair kernel's CTA size, and
// whether the FP32C pair kernel finishes its target blocks itself. Host code
// only (a CPU test compiles it with the host C++ compiler).
#pragma once

#include <cmath>
#include <cstdint>

#include "sk_internal.h"

namespace sk {

inline int choose_chunks(int precision, int64_t N, int64_t M, int sm_count) {
#ifdef SK_FORCE_CHUNKS
  if (SK_FORCE_CHUNKS > 0) return SK_FORCE_CHUNKS;
#endif
  // Split the source sum into chunks so that the grid (target blocks x
  // chunks) fills whole waves of resident CTAs: a partial last wave idles SMs.
  const bool fp32 = precision == SK_FP32C;
  const int np = pair32_np(M);
  const int64_t tgt_cta = fp32 ? (int64_t)TPB32 * 2 * np : TGT_CTA64;
  const int64_t tile = fp32 ? TILE : TILE64;
  const int64_t slots = (int64_t)sm_count * (fp32 ? pair32_ctas_per_sm(np) : 2);
  const int64_t n_tb = (int64_t)align_up((size_t)(M > 0 ? M : 1), tgt_cta) / tgt_cta;
  const int64_t tiles = (int64_t)align_up((size_t)(N > 0 ? N : 1), tile) / tile;
  int64_t cap = tiles / 2;
  if (cap < 1) cap = 1;
  if (cap > 64) cap = 64;
  // Many small items balance the ragged last wave better than partial-sum
  // traffic costs (measured at 493k targets: 5 chunks 71.0 ms, 13: 69.1,
  // 29: 68.7, 45: 68.4). Take the fewest chunks that give >= 32 waves filled
  // to >= 98%; if the problem is too small for that, see below (SK_FP32C),
  // or the fullest waves with at least four of them (SK_FP64).
  auto waves_of = [&](int64_t nc) { return (double)(n_tb * nc) / (double)slots; };
  for (int64_t nc = 1; nc <= cap; ++nc) {
    const double w = waves_of(nc);
    if (w >= 32.0 && w / std::ceil(w) >= 0.98) return (int)nc;
  }
  // A grid that cannot fill 32 waves: SK_FP32C takes the most chunks, down to
  // one source tile each (at most 64). Short items balance the uneven work of
  // the general (erf/exp) path better than full waves do (measured, evaluation
  // time by chunks: 24,576 x 15,384 single layer 38: 0.791, 57: 0.752,
  // 64: 0.740 ms; 98,304 x 60,504: 19: 4.95, 44: 4.71, 64: 4.71 ms).
  if (fp32) {
    int64_t many = tiles < 64 ? tiles : 64;
    return (int)(many < 1 ? 1 : many);
  }
  int best = (int)cap;
  double best_eff = -1.0;
  for (int64_t nc = 1; nc <= cap; ++nc) {
    const double w = waves_of(nc);
    if (w < 4.0 && nc < cap) continue;
    const double eff = w / std::ceil(w);
    if (eff > best_eff + 1e-3) {
      best_eff = eff;
      best = (int)nc;
    }
  }
  return best;
}

// The FP64 pipe issues a warp instruction per scheduler only every few dozen
// cycles, so about one warp per scheduler keeps it busy: for small problems
// the limit is how many SMs get work at all. When TPB64-thread CTAs cannot
// fill four waves even at the largest chunk count, the FP64 kernel runs
// TPB64_SMALL-thread CTAs (4x more target blocks) with one source tile per
// chunk. (Measured at 1944 x 1344: 32 CTAs left 120 SMs idle.)
inline void choose_decomposition(EvalShape& s, int sm_count) {
  s.n_chunks = choose_chunks(s.precision, s.N, s.M, sm_count);
  s.threads64 = TPB64;
  if (s.precision == SK_FP32C) {
    // The finish of a target block runs on the CTA that completes it: with at
    // least two blocks per SM those finishes overlap the pair work, and only
    // the last ones form a tail (measured: C3, 482 blocks: -1.5% per
    // evaluation; C2, 48 blocks: +25%, so smaller grids keep the finish
    // kernels).
    const int64_t tgt_cta = (int64_t)TPB32 * 2 * pair32_np(s.M);
    s.fuse_finish = (int64_t)align_up((size_t)(s.M > 0 ? s.M : 1), tgt_cta) / tgt_cta >=
                    2 * (int64_t)sm_count;
    return;
  }
  if (s.precision != SK_FP64) return;
  const int64_t n_tb = (int64_t)align_up((size_t)(s.M > 0 ? s.M : 1), TGT_CTA64) / TGT_CTA64;
  const int64_t slots = (int64_t)sm_count * 2;  // resident TPB64-thread CTAs
  if (n_tb * s.n_chunks >= 4 * slots) return;
  const int64_t tiles = (int64_t)align_up((size_t)(s.N > 0 ? s.N : 1), TILE64) / TILE64;
  s.threads64 = TPB64_SMALL;
  s.n_chunks = (int)(tiles < 64 ? tiles : 64);
}

}  // namespace sk
