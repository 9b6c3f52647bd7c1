// sk_serve.cu -- continuous batching of single-layer requests.
//
// Device side: one persistent kernel (k_serve) whose CTAs take work items
// from a table of resident requests ("slots"). An item is (target block,
// source chunk) of one request and runs the same pair_item code as the
// standalone evaluation. The CTA that completes the last chunk of a target
// block also finishes that block (FP64 near sums, chunk merge, output write);
// the CTA that finishes a request's last block raises the request's done flag
// in mapped host memory. Claims are a single 64-bit atomicAdd on the slot's
// claim word (items available in the high half, next item in the low half):
// a claim is valid iff item < n_items, so a request's descriptor is never
// rewritten while a CTA holds one of its items. All waits are bounded: the
// kernel exits after idle_exit_us without work and is relaunched on demand.
// The exit is collective: a CTA leaves on idleness only while no CTA holds
// an item, and it then raises a flag on which every other CTA leaves after
// its current item. (CTAs that left one by one could leave a few of them
// alive, busy with later arrivals, and the host relaunches only a kernel
// that has ended.)
//
// Host side: a scheduler thread admits queued requests when a slot and
// enough arena memory are free, prepares them (H2D copy from the pinned
// staging pool, sort and pack kernels on a preparation stream that runs
// beside the persistent kernel), publishes their items, returns results with
// D2H copies and relaunches the persistent kernel when it has exited.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "sk_decomp.h"
#include "sk_pair32.cuh"
#include "sk_range_alloc.h"

namespace sk {
namespace {

using namespace p32;

constexpr int SERVE_NP = 1;                           // target pairs per lane
constexpr int SERVE_MINB = 3;                         // CTAs per SM
constexpr int SERVE_TGT_CTA = TPB32 * 2 * SERVE_NP;  // targets per block (512)
constexpr int SERVE_RESERVE_CTAS = 24;  // CTA slots left free for the preparation kernels
constexpr int MAX_SLOTS = 256;
constexpr int SERVE_PREP_STREAMS = 4;
// device control words: host stop request, CTAs holding an item, exit raised
constexpr int CTL_STOP = 0, CTL_BUSY = 1, CTL_EXIT = 2, CTL_WORDS = 4;
#ifndef SK_SERVE_AGE
#define SK_SERVE_AGE 16
#endif
constexpr int SERVE_AGE_LIMIT = SK_SERVE_AGE;  // admissions that may overtake a request

// Device descriptor of one resident request.
struct SlotDesc {
  PairArgs pa;
  OverflowArgs oa;
  FinishArgs fa;
  int* tb_done;      // [n_tb] finished chunks per target block
  int* tb_finished;  // finished target blocks
  int64_t M;
  int n_tb;
  int n_chunks;
  unsigned seq;      // admission order (priority) and the done-flag value
  int pad;
};

struct alignas(64) SlotClaim {
  unsigned long long word;  // (n_items << 32) | next_item
  unsigned long long pad[7];
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(TPB32, SERVE_MINB)
    k_serve(const SlotDesc* __restrict__ desc, SlotClaim* __restrict__ claim, int n_slots,
            int* __restrict__ ctl, unsigned* __restrict__ done_host,
            unsigned long long idle_ns) {
  extern __shared__ __align__(128) float4 sm[];
  __shared__ PipeSmem<pair_stages<SLayer, SERVE_NP>()> ps;
  __shared__ SlotDesc d;
  __shared__ int s_slot, s_item, s_exit, s_finish;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) ps.initialized = 0;
  unsigned long long idle_since = gtimer();
  while (true) {
    if (wid == 0) {
      // pick the resident request with the fewest unclaimed items (shortest
      // remaining work first; the admission order breaks ties), so small
      // requests do not wait behind large ones admitted just before them;
      // a request that SERVE_AGE_LIMIT later admissions have passed is
      // overdue and goes first (oldest first), which bounds how long a large
      // request can be overtaken
      unsigned newest = 0;
      for (int s = lane; s < n_slots; s += 32) {
        const unsigned long long w = *(volatile const unsigned long long*)&claim[s].word;
        if ((unsigned)w < (unsigned)(w >> 32))
          newest = max(newest, *(volatile const unsigned*)&desc[s].seq);
      }
      for (int o = 16; o > 0; o >>= 1) newest = max(newest, __shfl_xor_sync(0xffffffffu, newest, o));
      unsigned long long best_key = ~0ull;
      int best = -1;
      for (int s = lane; s < n_slots; s += 32) {
        const unsigned long long w = *(volatile const unsigned long long*)&claim[s].word;
        const unsigned n_items = (unsigned)(w >> 32), next = (unsigned)w;
        if (next < n_items) {
          const unsigned q = *(volatile const unsigned*)&desc[s].seq;
          const bool overdue = newest - q >= (unsigned)SERVE_AGE_LIMIT;
          const unsigned long long key =
              ((unsigned long long)(overdue ? 0u : n_items - next) << 32) | q;
          if (key < best_key || best < 0) {
            best_key = key;
            best = s;
          }
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long q = __shfl_xor_sync(0xffffffffu, best_key, o);
        const int b = __shfl_xor_sync(0xffffffffu, best, o);
        if (b >= 0 && (best < 0 || q < best_key || (q == best_key && b < best))) {
          best_key = q;
          best = b;
        }
      }
      if (lane == 0) {
        s_slot = -1;
        s_exit = 0;
        volatile int* vctl = ctl;
        if (vctl[CTL_EXIT]) {
          s_exit = 1;  // another CTA has decided to leave: unclaimed items wait for the relaunch
        } else if (best >= 0) {
          const unsigned long long old = atomicAdd(&claim[best].word, 1ull);
          if ((unsigned)old < (unsigned)(old >> 32)) {
            atomicAdd(&ctl[CTL_BUSY], 1);
            s_slot = best;
            s_item = (int)(unsigned)old;
          }
        } else if (vctl[CTL_STOP]) {
          s_exit = 1;
        } else if (gtimer() - idle_since > idle_ns && vctl[CTL_BUSY] == 0) {
          atomicExch(&ctl[CTL_EXIT], 1);
          s_exit = 1;
        }
      }
    }
    __syncthreads();
    if (s_exit) break;
    const int slot = s_slot;
    if (slot < 0) {
      if (tid == 0) __nanosleep(2000);
      __syncthreads();
      continue;
    }
    idle_since = gtimer();
    // the descriptor of a slot with a valid claim is stable: copy it
    {
      const volatile int* src = reinterpret_cast<const volatile int*>(&desc[slot]);
      int* dst = reinterpret_cast<int*>(&d);
      for (int i = tid; i < (int)(sizeof(SlotDesc) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int item = s_item;
    const int tb = item / d.n_chunks, ch = item % d.n_chunks;
    // fresh loads: the arena block of an earlier request may have held other
    // data at these addresses while this kernel ran (a timeout sets the
    // request's flag)
    pair_item<SLayer, SERVE_NP, true>(d.pa, tb, chunk_tiles<true>(d.pa, ch), sm, ps);
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      s_finish = atomicAdd(&d.tb_done[tb], 1) == d.n_chunks - 1;
    }
    __syncthreads();
    if (s_finish) {
      // last chunk of this target block: finish the block's targets
      __threadfence();
      static_assert(pair_smem_bytes<SLayer, SERVE_NP>() / 4 >=
                        (size_t)(TPB32 / 32) * near_warp_words(64 * SERVE_NP),
                    "finish scratch");
      finish_block<SLayer>(d.oa, d.fa, d.M, (int64_t)tb * SERVE_TGT_CTA, SERVE_TGT_CTA,
                           reinterpret_cast<unsigned*>(sm));
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        if (atomicAdd(d.tb_finished, 1) == d.n_tb - 1) {
          __threadfence_system();
          *(volatile unsigned*)&done_host[slot] = d.seq;
        }
      }
    }
    if (tid == 0) atomicSub(&ctl[CTL_BUSY], 1);
  }
}

using Clock = std::chrono::steady_clock;

struct Req {
  uint64_t ticket = 0;
  EvalShape shape;
  size_t stage_off = 0, stage_len = 0;  // pinned staging block: inputs, then output
  double* h_xyz = nullptr;
  double* h_w = nullptr;
  double* h_f = nullptr;
  double* h_txyz = nullptr;
  double* h_delta = nullptr;
  double* h_u = nullptr;
  size_t footprint = 0;
  int64_t n_active = 0;
  int status = SK_EAGAIN;
  sk_req_stats st{};
  unsigned long long flags[N_FLAGS] = {};
  // capsule request: Euler steps of a resident capsule
  sk_capsule* cap = nullptr;
  int steps = 0, steps_done = 0;
  double dt = 0.0;
  sk_flow flow{};
};

enum class SlotState { Free, Prep, Running, Copying };

struct Slot {
  SlotState state = SlotState::Free;
  Req* req = nullptr;
  size_t arena_off = 0, arena_len = 0;
  EvalBufs b;
  int* tb_counters = nullptr;  // [n_tb + 1]
  unsigned seq = 0;
  cudaEvent_t prep_done = nullptr, copy_done = nullptr, update_done = nullptr;
  // fork and join of the target sort onto the preparation stream's partner
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  // pinned per-slot block (PIN_WORDS words): [0, 8) device flags, [8, 12)
  // meta ints, [12] claim word, [16, ...) descriptor being published
  unsigned long long* h_flags = nullptr;
};

constexpr int PIN_WORDS = 128;
constexpr int PIN_META = 8, PIN_CLAIM = 12, PIN_DESC = 16;
static_assert(sizeof(SlotDesc) <= (PIN_WORDS - PIN_DESC) * sizeof(unsigned long long),
              "slot descriptor does not fit the pinned block");

}  // namespace
}  // namespace sk

struct sk_server {
  sk_ctx* ctx = nullptr;
  sk_serve_cfg cfg{};
  int n_slots = 0;
  cudaStream_t s_kernel = nullptr, s_ctl = nullptr, s_copy = nullptr;
  // preparation streams: independent requests prepare concurrently (slot i
  // uses stream i mod SERVE_PREP_STREAMS), so a burst of admissions does not
  // queue behind one stream
  cudaStream_t s_prep[sk::SERVE_PREP_STREAMS] = {};
  // each preparation stream's partner: a request's target sort and pack run
  // there beside its source sort and pack
  cudaStream_t s_prep_aux[sk::SERVE_PREP_STREAMS] = {};
  sk::SlotDesc* d_desc = nullptr;
  sk::SlotClaim* d_claim = nullptr;
  int* d_ctl = nullptr;  // CTL_WORDS device control words
  unsigned* h_done = nullptr;  // mapped pinned page
  unsigned* d_done = nullptr;
  unsigned long long* h_flagbuf = nullptr;  // pinned, N_FLAGS per slot
  int* h_stop_one = nullptr;                // pinned constant 1
  char* arena = nullptr;
  size_t arena_bytes = 0;
  char* stage = nullptr;
  size_t stage_bytes = 0;
  sk::RangeAlloc arena_alloc, stage_alloc;
  std::vector<sk::Slot> slots;
  std::mutex mu;
  std::condition_variable cv_done;
  std::condition_variable cv_work;  // wakes an idle scheduler: a submit or shutdown
  std::deque<sk::Req*> queue;
  std::map<uint64_t, sk::Req*> reqs;
  std::thread thr;
  std::atomic<bool> shutting_down{false};
  std::atomic<bool> failed{false};
  cudaEvent_t kernel_done = nullptr;
  bool kernel_launched = false;
  uint64_t next_ticket = 1;
  unsigned next_seq = 1;
  sk::Clock::time_point t0;
  std::string err;
};

namespace sk {
namespace {

double now_us(const sk_server* s) {
  return std::chrono::duration<double, std::micro>(Clock::now() - s->t0).count();
}

size_t request_footprint(const EvalShape& s, int n_tb) {
  return eval_workspace_bytes(s) + align_up((size_t)(n_tb + 1) * sizeof(int), 256) + 1024;
}

bool kernel_running(sk_server* srv) {
  if (!srv->kernel_launched) return false;
  const cudaError_t e = cudaEventQuery(srv->kernel_done);
  if (e == cudaErrorNotReady) return true;
  srv->kernel_launched = false;
  return false;
}

// capsules: some resident request is a capsule's. Its steps prepare with
// FP64 membrane kernels between the sums, and those run only on the CTA
// slots the persistent kernel leaves free: then the kernel leaves one slot
// per SM (SERVE_MINB - 1 CTAs per SM) instead of SERVE_RESERVE_CTAS in all.
void launch_kernel(sk_server* srv, bool capsules) {
  const size_t smem = pair_smem_bytes<SLayer, SERVE_NP>();
  cudaFuncSetAttribute(k_serve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int grid = capsules ? srv->ctx->sm_count * (SERVE_MINB - 1)
                      : srv->ctx->sm_count * SERVE_MINB - SERVE_RESERVE_CTAS;
  if (grid < 1) grid = 1;
  // the previous instance has ended (stream order): clear its busy count and
  // exit flag, but not the host's stop word
  cudaMemsetAsync(srv->d_ctl + CTL_BUSY, 0, (CTL_WORDS - CTL_BUSY) * sizeof(int), srv->s_kernel);
  k_serve<<<grid, TPB32, smem, srv->s_kernel>>>(
      srv->d_desc, srv->d_claim, srv->n_slots, srv->d_ctl, srv->d_done,
      (unsigned long long)srv->cfg.idle_exit_us * 1000ull);
  cudaEventRecord(srv->kernel_done, srv->s_kernel);
  srv->kernel_launched = true;
}

// A capsule request's steps run on its slot's preparation stream, with that
// stream's scratch copy of the membrane operator: capsules of one grid order
// in different slots prepare at the same time, and the steps of one capsule
// follow one another on its stream.
int capsule_set(int slot) { return slot % SERVE_PREP_STREAMS; }

// One step of a capsule request, on st: the inputs of its sum (membrane
// force, weights, delta* at the current nodes), cleared counters and the
// preparation kernels; the step's items are published when st reaches
// prep_done.
void enqueue_capsule_step(sk_server* srv, Slot& sl, int slot, cudaStream_t st) {
  Req* r = sl.req;
  capsule_enqueue_step_inputs(r->cap, sl.b, st, capsule_set(slot));
  const int n_tb = (int)(sl.b.M_pad / SERVE_TGT_CTA);
  cudaMemsetAsync(sl.tb_counters, 0, (n_tb + 1) * sizeof(int), st);
  const PrepFork pf{srv->s_prep_aux[slot % SERVE_PREP_STREAMS], sl.fork_ev, sl.join_ev};
  enqueue_prep(r->shape, sl.b, srv->ctx->rho_T, srv->ctx->rho_c, st, &pf);
  cudaEventRecord(sl.prep_done, st);
}

// Admit: bind a queued request to a free slot and its arena block, enqueue
// the H2D copy and the preparation kernels.
bool admit_one(sk_server* srv, Req* r, Slot& sl, int slot) {
  size_t off = 0;
  if (!srv->arena_alloc.alloc(r->footprint, &off)) return false;
  sl.state = SlotState::Prep;
  sl.req = r;
  sl.arena_off = off;
  sl.arena_len = r->footprint;
  sl.seq = srv->next_seq++;
  EvalBufs& b = sl.b;
  b = EvalBufs{};
  Bump bp;
  bp.base = srv->arena + off;
  carve_eval_buffers(bp, r->shape, b);
  const int n_tb = (int)(b.M_pad / SERVE_TGT_CTA);
  sl.tb_counters = bp.take<int>(n_tb + 1);
  const EvalShape& s = r->shape;
  cudaStream_t st = srv->s_prep[slot % SERVE_PREP_STREAMS];
  if (r->cap) {  // the first step of a capsule request: its inputs are resident
    capsule_clear_sticky(r->cap, st);
    enqueue_capsule_step(srv, sl, slot, st);
    r->st.admit_us = now_us(srv);
    return true;
  }
  if (s.N > 0) {
    cudaMemcpyAsync((void*)b.src_xyz, r->h_xyz, 3 * s.N * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync((void*)b.src_w, r->h_w, s.N * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync((void*)b.dens, r->h_f, 3 * s.N * sizeof(double), cudaMemcpyHostToDevice, st);
  }
  cudaMemcpyAsync((void*)b.tgt_xyz, r->h_txyz, 3 * s.M * sizeof(double), cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync((void*)b.delta, r->h_delta, s.n_delta * sizeof(double), cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(sl.tb_counters, 0, (n_tb + 1) * sizeof(int), st);
  const PrepFork pf{srv->s_prep_aux[slot % SERVE_PREP_STREAMS], sl.fork_ev, sl.join_ev};
  enqueue_prep(s, b, srv->ctx->rho_T, srv->ctx->rho_c, st, &pf);
  cudaEventRecord(sl.prep_done, st);
  r->st.admit_us = now_us(srv);
  return true;
}

// Publish a prepared request: descriptor first, then its claim word.
void publish(sk_server* srv, int slot) {
  Slot& sl = srv->slots[slot];
  const EvalBufs& b = sl.b;
  const EvalShape& s = sl.req->shape;
  const double scale = layer_scale(s);
  const float rho_lo = (float)srv->ctx->rho_T, rho_hi = 8.0f;
  SlotDesc d{};
  d.pa = PairArgs{b.srcF, b.segbox, b.src_orig, b.meta, b.tgtF, b.tgt64, b.M_pad, b.n_chunks,
                  b.part, b.near_cnt, b.near_idx, b.flags, rho_lo, rho_hi};
  d.oa = OverflowArgs{b.srcF, b.segbox, b.src_orig, b.meta, b.tgtF, b.tgt64, b.near_cnt,
                      b.src_xyz, b.src_w, b.dens, b.nrm, scale, b.flags, b.near_ovf};
  d.fa = FinishArgs{b.tgt64, b.tgt_perm, b.M_pad, b.n_chunks, b.part, b.near_cnt, b.near_idx,
                    b.near_ovf, b.src_xyz, b.src_w, b.dens, b.nrm, scale, b.u, b.flags};
  d.oa.group = d.fa.group = 64 * SERVE_NP;
  d.n_tb = (int)(b.M_pad / SERVE_TGT_CTA);
  d.tb_done = sl.tb_counters;
  d.tb_finished = sl.tb_counters + d.n_tb;
  d.M = s.M;
  d.n_chunks = b.n_chunks;
  d.seq = sl.seq;
  // descriptor first, then the claim word that makes its items visible
  std::memcpy(sl.h_flags + PIN_DESC, &d, sizeof(d));
  unsigned long long* word = sl.h_flags + PIN_CLAIM;
  *word = ((unsigned long long)(unsigned)(d.n_tb * d.n_chunks) << 32);
  cudaMemcpyAsync(srv->d_desc + slot, sl.h_flags + PIN_DESC, sizeof(d), cudaMemcpyHostToDevice,
                  srv->s_ctl);
  // stream order lands the descriptor before the claim word; the pinned block
  // is rewritten only by this slot's next publish, after this request is done
  cudaMemcpyAsync(&srv->d_claim[slot].word, word, sizeof(*word), cudaMemcpyHostToDevice,
                  srv->s_ctl);
  sl.state = SlotState::Running;
  sl.req->st.publish_us = now_us(srv);
}

void scheduler(sk_server* srv) {
  cudaSetDevice(srv->ctx->device);
  while (true) {
    bool progress = false;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      // 1. admissions (oldest first)
      for (int i = 0; i < srv->n_slots && !srv->queue.empty(); ++i) {
        Slot& sl = srv->slots[i];
        if (sl.state != SlotState::Free) continue;
        Req* r = srv->queue.front();
        if (!admit_one(srv, r, sl, i)) break;  // not enough arena yet
        srv->queue.pop_front();
        progress = true;
      }
      if (srv->shutting_down && srv->queue.empty()) {
        bool busy = false;
        for (auto& sl : srv->slots) busy |= sl.state != SlotState::Free;
        if (!busy) break;
      }
    }
    bool any_running = false;
    for (int i = 0; i < srv->n_slots; ++i) {
      Slot& sl = srv->slots[i];
      if (sl.state == SlotState::Prep && cudaEventQuery(sl.prep_done) == cudaSuccess) {
        publish(srv, i);
        progress = true;
      }
      if (sl.state == SlotState::Running) {
        any_running = true;
        if (*(volatile unsigned*)&srv->h_done[i] == sl.seq && sl.req->cap) {
          // a capsule step's sum is done: update the nodes, then the next
          // step, or read the nodes back after the last one
          Req* r = sl.req;
          cudaStream_t st = srv->s_prep[i % SERVE_PREP_STREAMS];
          capsule_enqueue_step_update(r->cap, sl.b.flags, r->dt, r->flow, st);
          if (++r->steps_done < r->steps) {
            {
              std::unique_lock<std::mutex> lk(srv->mu);
              sl.seq = srv->next_seq++;
            }
            enqueue_capsule_step(srv, sl, i, st);
            sl.state = SlotState::Prep;
          } else {
            r->st.done_us = now_us(srv);
            cudaEventRecord(sl.update_done, st);
            cudaStreamWaitEvent(srv->s_copy, sl.update_done, 0);
            cudaMemcpyAsync(r->h_u, capsule_nodes(r->cap), 3 * r->shape.M * sizeof(double),
                            cudaMemcpyDeviceToHost, srv->s_copy);
            cudaMemcpyAsync(sl.h_flags, capsule_sticky(r->cap),
                            N_FLAGS * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                            srv->s_copy);
            cudaMemcpyAsync(sl.h_flags + PIN_META, sl.b.meta, N_META * sizeof(int),
                            cudaMemcpyDeviceToHost, srv->s_copy);
            cudaEventRecord(sl.copy_done, srv->s_copy);
            sl.state = SlotState::Copying;
          }
          progress = true;
        } else if (*(volatile unsigned*)&srv->h_done[i] == sl.seq) {
          Req* r = sl.req;
          r->st.done_us = now_us(srv);
          cudaMemcpyAsync(r->h_u, sl.b.u, 3 * r->shape.M * sizeof(double), cudaMemcpyDeviceToHost,
                          srv->s_copy);
          cudaMemcpyAsync(sl.h_flags, sl.b.flags, N_FLAGS * sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, srv->s_copy);
          cudaMemcpyAsync(sl.h_flags + PIN_META, sl.b.meta, N_META * sizeof(int),
                          cudaMemcpyDeviceToHost, srv->s_copy);
          cudaEventRecord(sl.copy_done, srv->s_copy);
          sl.state = SlotState::Copying;
          progress = true;
        }
      }
      if (sl.state == SlotState::Copying && cudaEventQuery(sl.copy_done) == cudaSuccess) {
        std::unique_lock<std::mutex> lk(srv->mu);
        Req* r = sl.req;
        std::memcpy(r->flags, sl.h_flags, sizeof(r->flags));
        r->n_active = reinterpret_cast<const int*>(sl.h_flags + PIN_META)[META_NS];
        r->status = r->flags[FLAG_TIMEOUT] ? SK_ETIMEOUT
                    : r->flags[FLAG_BAD_DELTA] ? SK_EINVAL : SK_OK;
        r->st.status = r->status;
        r->st.ready_us = now_us(srv);
        if (r->cap) capsule_release(r->cap);
        srv->arena_alloc.release(sl.arena_off, sl.arena_len);
        sl.state = SlotState::Free;
        sl.req = nullptr;
        srv->cv_done.notify_all();
        progress = true;
      }
    }
    if (any_running && !kernel_running(srv)) {
      bool capsules = false;
      for (int i = 0; i < srv->n_slots; ++i)
        capsules |= srv->slots[i].state != SlotState::Free && srv->slots[i].req &&
                    srv->slots[i].req->cap;
      launch_kernel(srv, capsules);
      progress = true;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      std::unique_lock<std::mutex> lk(srv->mu);
      srv->err = std::string("serving: ") + cudaGetErrorString(e);
      srv->failed = true;
      for (auto& kv : srv->reqs)
        if (kv.second->status == SK_EAGAIN) kv.second->status = SK_ECUDA;
      srv->cv_done.notify_all();
      break;
    }
    // While a request is in flight the thread only yields: every state change
    // it waits for (preparation done, done flag, copy done) is noticed within
    // microseconds. With nothing in flight it sleeps until a submit (or
    // shutdown) wakes it.
    bool in_flight = false;
    for (const auto& sl : srv->slots) in_flight |= sl.state != SlotState::Free;
    if (progress || in_flight) {
      std::this_thread::yield();
    } else {
      std::unique_lock<std::mutex> lk(srv->mu);
      if (srv->queue.empty() && !srv->shutting_down)
        srv->cv_work.wait_for(lk, std::chrono::milliseconds(10));
    }
  }
}

void free_server(sk_server* srv) {
  if (srv->d_desc) cudaFree(srv->d_desc);
  if (srv->d_claim) cudaFree(srv->d_claim);
  if (srv->d_ctl) cudaFree(srv->d_ctl);
  if (srv->h_done) cudaFreeHost(srv->h_done);
  if (srv->h_flagbuf) cudaFreeHost(srv->h_flagbuf);
  if (srv->h_stop_one) cudaFreeHost(srv->h_stop_one);
  if (srv->arena) cudaFree(srv->arena);
  if (srv->stage) cudaFreeHost(srv->stage);
  for (auto& sl : srv->slots) {
    if (sl.prep_done) cudaEventDestroy(sl.prep_done);
    if (sl.copy_done) cudaEventDestroy(sl.copy_done);
    if (sl.update_done) cudaEventDestroy(sl.update_done);
    if (sl.fork_ev) cudaEventDestroy(sl.fork_ev);
    if (sl.join_ev) cudaEventDestroy(sl.join_ev);
  }
  if (srv->kernel_done) cudaEventDestroy(srv->kernel_done);
  for (cudaStream_t s : {srv->s_kernel, srv->s_ctl, srv->s_copy})
    if (s) cudaStreamDestroy(s);
  for (cudaStream_t s : srv->s_prep)
    if (s) cudaStreamDestroy(s);
  for (cudaStream_t s : srv->s_prep_aux)
    if (s) cudaStreamDestroy(s);
  for (auto& kv : srv->reqs) {
    if (kv.second->cap) capsule_release(kv.second->cap);
    delete kv.second;
  }
  delete srv;
}

}  // namespace
}  // namespace sk

using namespace sk;

extern "C" {

int serve_create(sk_ctx* ctx, const sk_serve_cfg* cfg_in, sk_server** out) {
  if (!ctx || !out) return SK_EINVAL;
  *out = nullptr;
  if (ctx->server) {
    ctx->err = "serve_create: this context already has a server";
    return SK_EBUSY;
  }
  sk_serve_cfg cfg{};
  if (cfg_in) cfg = *cfg_in;
  if (cfg.max_slots == 0) cfg.max_slots = 32;
  if (cfg.queue_capacity == 0) cfg.queue_capacity = 4096;
  if (cfg.idle_exit_us == 0) cfg.idle_exit_us = 20000;
  if (cfg.host_staging_bytes == 0) cfg.host_staging_bytes = size_t(512) << 20;
  if (cfg.max_slots < 1 || cfg.max_slots > MAX_SLOTS || cfg.queue_capacity < 1 ||
      cfg.idle_exit_us < 0) {
    ctx->err = "serve_create: max_slots must be 1..256, queue_capacity >= 1, idle_exit_us >= 0";
    return SK_EINVAL;
  }
  cudaSetDevice(ctx->device);
  if (cfg.hbm_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    cfg.hbm_budget_bytes = std::min(fr / 4, size_t(16) << 30);
  }
  sk_server* srv = new (std::nothrow) sk_server();
  if (!srv) return SK_ENOMEM;
  srv->ctx = ctx;
  srv->cfg = cfg;
  srv->n_slots = cfg.max_slots;
  srv->t0 = Clock::now();
  srv->slots.resize(srv->n_slots);
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) {
    if (x != cudaSuccess && e == cudaSuccess) e = x;
    return x == cudaSuccess;
  };
  ok(cudaStreamCreateWithFlags(&srv->s_kernel, cudaStreamNonBlocking));
  for (cudaStream_t& s : srv->s_prep) ok(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  for (cudaStream_t& s : srv->s_prep_aux) ok(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  ok(cudaStreamCreateWithFlags(&srv->s_ctl, cudaStreamNonBlocking));
  ok(cudaStreamCreateWithFlags(&srv->s_copy, cudaStreamNonBlocking));
  ok(cudaMalloc(&srv->d_desc, MAX_SLOTS * sizeof(SlotDesc)));
  ok(cudaMalloc(&srv->d_claim, MAX_SLOTS * sizeof(SlotClaim)));
  ok(cudaMalloc(&srv->d_ctl, CTL_WORDS * sizeof(int)));
  ok(cudaHostAlloc(&srv->h_done, MAX_SLOTS * sizeof(unsigned), cudaHostAllocMapped));
  ok(cudaHostAlloc(&srv->h_flagbuf, (size_t)srv->n_slots * PIN_WORDS * sizeof(unsigned long long),
                   cudaHostAllocDefault));
  ok(cudaHostAlloc(&srv->h_stop_one, sizeof(int), cudaHostAllocDefault));
  ok(cudaMalloc(&srv->arena, cfg.hbm_budget_bytes));
  ok(cudaHostAlloc(&srv->stage, cfg.host_staging_bytes, cudaHostAllocDefault));
  ok(cudaEventCreateWithFlags(&srv->kernel_done, cudaEventDisableTiming));
  for (auto& sl : srv->slots) {
    ok(cudaEventCreateWithFlags(&sl.prep_done, cudaEventDisableTiming));
    ok(cudaEventCreateWithFlags(&sl.copy_done, cudaEventDisableTiming));
    ok(cudaEventCreateWithFlags(&sl.update_done, cudaEventDisableTiming));
    ok(cudaEventCreateWithFlags(&sl.fork_ev, cudaEventDisableTiming));
    ok(cudaEventCreateWithFlags(&sl.join_ev, cudaEventDisableTiming));
  }
  if (e == cudaSuccess) {
    ok(cudaHostGetDevicePointer((void**)&srv->d_done, srv->h_done, 0));
    ok(cudaMemset(srv->d_desc, 0, MAX_SLOTS * sizeof(SlotDesc)));
    ok(cudaMemset(srv->d_claim, 0, MAX_SLOTS * sizeof(SlotClaim)));
    ok(cudaMemset(srv->d_ctl, 0, CTL_WORDS * sizeof(int)));
  }
  if (e != cudaSuccess) {
    ctx->err = std::string("serve_create: ") + cudaGetErrorString(e);
    const int code = e == cudaErrorMemoryAllocation ? SK_ENOMEM : SK_ECUDA;
    free_server(srv);
    return code;
  }
  std::memset(srv->h_done, 0, MAX_SLOTS * sizeof(unsigned));
  *srv->h_stop_one = 1;
  for (int i = 0; i < srv->n_slots; ++i)
    srv->slots[i].h_flags = srv->h_flagbuf + PIN_WORDS * (size_t)i;
  srv->arena_bytes = cfg.hbm_budget_bytes;
  srv->stage_bytes = cfg.host_staging_bytes;
  srv->arena_alloc.reset(srv->arena_bytes);
  srv->stage_alloc.reset(srv->stage_bytes);
  srv->thr = std::thread(scheduler, srv);
  ctx->server = srv;
  *out = srv;
  return SK_OK;
}

namespace {

// A capsule request: n_steps Euler steps of a resident capsule; the result
// is its nodes after the last step.
int submit_capsule(sk_server* srv, const sk_request* q, uint64_t* ticket) {
  sk_capsule* c = q->capsule;
  if (capsule_ctx(c) != srv->ctx || !capsule_servable(c) || q->n_steps < 1 ||
      !(q->dt > 0.0 && q->dt < INFINITY) || q->flow.kind < SK_FLOW_NONE ||
      q->flow.kind > SK_FLOW_POISEUILLE)
    return SK_EINVAL;
  Req* r = new (std::nothrow) Req();
  if (!r) return SK_ENOMEM;
  r->cap = c;
  r->steps = q->n_steps;
  r->dt = q->dt;
  r->flow = q->flow;
  r->shape = capsule_step_shape(c);
  const int64_t M = r->shape.M;
  const int n_tb = (int)(align_up((size_t)M, TGT_CTA32) / SERVE_TGT_CTA);
  r->footprint = request_footprint(r->shape, n_tb);
  const size_t bytes = 3 * (size_t)M * sizeof(double) + 256;
  if (r->footprint > srv->arena_bytes || bytes > srv->stage_bytes) {
    delete r;
    return SK_ENOMEM;
  }
  // the membrane operator's scratch copies of the preparation streams
  const int rc = capsule_prepare_sets(c, SERVE_PREP_STREAMS);
  if (rc != SK_OK) {
    delete r;
    return rc;
  }
  std::unique_lock<std::mutex> lk(srv->mu);
  if ((int)srv->queue.size() >= srv->cfg.queue_capacity ||
      !srv->stage_alloc.alloc(bytes, &r->stage_off)) {
    delete r;
    return SK_EBUSY;
  }
  if (!capsule_try_acquire(c)) {  // one request per capsule at a time
    srv->stage_alloc.release(r->stage_off, bytes);
    delete r;
    return SK_EBUSY;
  }
  r->stage_len = bytes;
  r->h_u = reinterpret_cast<double*>(srv->stage + r->stage_off);
  r->ticket = srv->next_ticket++;
  r->st.submit_us = now_us(srv);
  r->st.n_chunks = r->shape.n_chunks;
  srv->reqs[r->ticket] = r;
  srv->queue.push_back(r);
  *ticket = r->ticket;
  srv->cv_work.notify_one();
  return SK_OK;
}

}  // namespace

int serve_submit(sk_server* srv, const sk_request* q, uint64_t* ticket) {
  if (!srv || !q || !ticket) return SK_EINVAL;
  if (srv->failed) return SK_ECUDA;
  if (q->capsule) return submit_capsule(srv, q, ticket);
  const int64_t N = q->n_src, M = q->n_tgt;
  if (N < 0 || M < 1 || N > FP32C_MAX_SOURCES || M > (int64_t(1) << 30)) return SK_EINVAL;
  if (N > 0 && (!q->src_xyz || !q->src_w || !q->f)) return SK_EINVAL;
  if (!q->tgt_xyz || !q->delta || !(q->n_delta == 1 || q->n_delta == M)) return SK_EINVAL;
  if (!(q->mu > 0.0 && q->mu < INFINITY)) return SK_EINVAL;
  for (int64_t i = 0; i < q->n_delta; ++i)
    if (!(q->delta[i] > 0.0 && q->delta[i] < INFINITY)) return SK_EINVAL;
  Req* r = new (std::nothrow) Req();
  if (!r) return SK_ENOMEM;
  EvalShape& s = r->shape;
  s.layer = LAYER_SL;
  s.precision = SK_FP32C;
  s.N = N;
  s.M = M;
  s.n_delta = q->n_delta;
  s.mu = q->mu;
  s.copy_inputs = true;
  s.small_sort_points = srv->ctx->small_sort_points;
  s.split_sorts = true;  // the target sort runs on the preparation stream's partner
  s.n_chunks = choose_chunks(SK_FP32C, N, M, srv->ctx->sm_count);
  const int n_tb = (int)(align_up((size_t)M, TGT_CTA32) / SERVE_TGT_CTA);
  r->footprint = request_footprint(s, n_tb);
  if (r->footprint > srv->arena_bytes) {
    delete r;
    return SK_ENOMEM;
  }
  const size_t in_doubles = (size_t)7 * N + 3 * M + q->n_delta;
  const size_t bytes = (in_doubles + 3 * (size_t)M) * sizeof(double) + 6 * 256;
  if (bytes > srv->stage_bytes) {
    delete r;
    return SK_ENOMEM;
  }
  std::unique_lock<std::mutex> lk(srv->mu);
  if ((int)srv->queue.size() >= srv->cfg.queue_capacity ||
      !srv->stage_alloc.alloc(bytes, &r->stage_off)) {
    delete r;
    return SK_EBUSY;
  }
  r->stage_len = bytes;
  char* p = srv->stage + r->stage_off;
  auto take = [&](size_t n) {
    double* d = reinterpret_cast<double*>(p);
    p += align_up(n * sizeof(double), 256);
    return d;
  };
  r->h_xyz = take(3 * N);
  r->h_w = take(N);
  r->h_f = take(3 * N);
  r->h_txyz = take(3 * M);
  r->h_delta = take(q->n_delta);
  r->h_u = take(3 * M);
  lk.unlock();
  if (N > 0) {
    std::memcpy(r->h_xyz, q->src_xyz, 3 * N * sizeof(double));
    std::memcpy(r->h_w, q->src_w, N * sizeof(double));
    std::memcpy(r->h_f, q->f, 3 * N * sizeof(double));
  }
  std::memcpy(r->h_txyz, q->tgt_xyz, 3 * M * sizeof(double));
  std::memcpy(r->h_delta, q->delta, q->n_delta * sizeof(double));
  lk.lock();
  r->ticket = srv->next_ticket++;
  r->st.submit_us = now_us(srv);
  r->st.n_chunks = s.n_chunks;
  srv->reqs[r->ticket] = r;
  srv->queue.push_back(r);
  *ticket = r->ticket;
  srv->cv_work.notify_one();
  return SK_OK;
}

int serve_poll(sk_server* srv, uint64_t ticket, double* u_out, sk_req_stats* st,
               int64_t timeout_us) {
  if (!srv) return SK_EINVAL;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) return SK_EINVAL;
  Req* r = it->second;
  auto ready = [&] { return r->status != SK_EAGAIN; };
  if (!ready()) {
    if (timeout_us == 0) return SK_EAGAIN;
    if (timeout_us < 0)
      srv->cv_done.wait(lk, ready);
    else if (!srv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
      return SK_EAGAIN;
  }
  const int status = r->status;
  if (status == SK_OK && u_out) std::memcpy(u_out, r->h_u, 3 * r->shape.M * sizeof(double));
  if (st) {
    *st = r->st;
    st->interactions = r->shape.M * r->n_active * (r->cap ? r->steps : 1);
  }
  srv->stage_alloc.release(r->stage_off, r->stage_len);
  srv->reqs.erase(it);
  lk.unlock();
  delete r;
  return status;
}

void serve_destroy(sk_server* srv) {
  if (!srv) return;
  {
    std::unique_lock<std::mutex> lk(srv->mu);
    srv->shutting_down = true;
    srv->cv_work.notify_one();
  }
  if (srv->thr.joinable()) srv->thr.join();
  cudaSetDevice(srv->ctx->device);
  cudaMemcpyAsync(srv->d_ctl + CTL_STOP, srv->h_stop_one, sizeof(int), cudaMemcpyHostToDevice,
                  srv->s_ctl);
  cudaStreamSynchronize(srv->s_ctl);
  cudaStreamSynchronize(srv->s_kernel);
  cudaDeviceSynchronize();
  srv->ctx->server = nullptr;
  free_server(srv);
}

}  // extern "C"
