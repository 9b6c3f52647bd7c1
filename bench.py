#!/usr/bin/env python3
"""Benchmark of the regularized Stokes layer sums (libstokesreg, GB300).

One step = one single-layer evaluation (SK_FP32C) of the high-resolution
ellipsoid workload: axes (1, 0.8, 0.5), m = 257 (256 x 256 nodes per patch,
N = 393,216, of which N_s = 239,880 carry nonzero weight), targets = the N
nodes followed by 100,000 exterior probes at 0.1h-5h, delta = 2h, mu = 1.
Interactions per step = targets x N_s. Inputs are resident in HBM when the
timed region starts; L2 is flushed (256 MB write) between timed steps.

Extra measurements on rank 0 (single GPU): the FP64 path on the same
workload, the double layer on the rotated Evans-Fung cell (m = 65), a delta
sweep {1.5, 2, 3}h, the end-to-end call with pinned host buffers, and the FP64
CPU oracle on a bounded sample (the CPU baseline, which also supplies the
relative errors).

--impl reference times that oracle alone (the reference arm of this metric).
Under torchrun every rank runs its own seeded copy of the workload (weak
scaling, no collective on the data path); timing is max over ranks.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("Ginteractions/s, FP32 vs FP64 at stated rel. error vs oracle; "
          "serving p50/p99 latency")
UNIT = "Ginteractions/s"
FLOPS_SL = 29  # flops credited per single-layer interaction (FMA = 2, MUFU = 1)
FLOPS_DL = 33  # per double-layer interaction
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
FP32_PEAK_TFLOPS = 2 * 128 * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12  # 80.55
FP64_PEAK_TFLOPS = 1.25  # nominal dense FP64 of GB300
CPU_SAMPLE_TARGETS = 24576  # about 10 s of the oracle on 16 host cores
SWEEP_SAMPLE_TARGETS = 8192  # oracle check of each delta of the sweep (about 3 s each)
SERVE_ORACLE_REQUESTS = 50   # served results checked against the oracle ...
SERVE_ORACLE_TARGETS = 256   # ... on this many seeded targets each
REF_STEP_TARGETS = 512


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--m", type=int, default=257, help="grid order (default 257)")
    ap.add_argument("--probes", type=int, default=100_000)
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--layer", choices=["sl", "dl"], default="sl",
                    help="timed step: single layer (default) or double layer (q = the SH "
                         "density); extras run only for the default sl/fp32c step")
    ap.add_argument("--precision", choices=["fp32c", "fp64"], default="fp32c")
    ap.add_argument("--fmm-only", action="store_true",
                    help="time only the single-level FMM (SK_FP32C, k = --fmm-k clusters, p = 6) "
                         "on the ellipsoid (1, 0.8, 0.5) nodes of grid order --m, delta = 2h, "
                         "and print that line")
    ap.add_argument("--fmm-k", type=int, default=64)
    ap.add_argument("--membrane-only", action="store_true",
                    help="time only the Skalak membrane force on the stress-free ellipsoid "
                         "(0.9, 1, 1) of grid order --m, and print that line")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def workload(m, n_probes, rank=0):
    import capsule_inputs as ci
    return ci.ellipsoid_hires_workload(m=m, n_probes=n_probes, seed=3000 + 17 * rank)


def workload_name(w, layer="sl"):
    s = w.surface
    kind = "single layer, delta=2h, mu=1" if layer == "sl" else \
        "double layer (q = the SH density), delta=2h"
    return (f"ellipsoid(1,0.8,0.5) m={s.m}: N={s.N} nodes (N_s={s.n_active} active) + "
            f"{w.targets.shape[0] - s.N} exterior probes (0.1h-5h), {kind}")


def sample_targets(w, n, seed=1234):
    rng = np.random.default_rng(seed)
    M = w.targets.shape[0]
    n_on = w.n_on_surface
    k_probe = min(n // 4, M - n_on)
    return np.concatenate([rng.choice(n_on, n - k_probe, replace=False),
                           n_on + rng.choice(M - n_on, k_probe, replace=False)])


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        with open(self.path) as fh:
            lines = fh.readlines()
        os.remove(self.path)
        return clock_summary(lines)


def clock_summary(lines):
    """Median SM clock, maximum SM clock and the throttle reasons seen, from
    lines of `nvidia-smi --query-gpu=<ClockSampler.QUERY> --format=csv,noheader,nounits`
    (None without a sample). Values nvidia-smi cannot report ("[N/A]") are skipped."""
    rows = []
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) >= 9:
            rows.append(parts)
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
            "samples": len(rows)}


# ----------------------------------------------------------------------------- reference arm

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    w = workload(args.m, args.probes)
    s = w.surface
    rng = np.random.default_rng(99)
    times = []
    n_src_active = s.n_active
    for it in range(args.warmup + args.steps):
        idx = rng.choice(w.targets.shape[0], REF_STEP_TARGETS, replace=False)
        t0 = time.perf_counter()
        oracle.sl(s.X, s.w, w.f, w.targets[idx], w.delta, w.mu)
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    per_step = float(np.mean(times))
    value = REF_STEP_TARGETS * n_src_active / per_step / 1e9
    cores = oracle.max_threads()
    sample = (f"{REF_STEP_TARGETS} random targets of the workload per step x all "
              f"{n_src_active} active sources")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": per_step * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(w), "targets_per_step": REF_STEP_TARGETS},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- ranks

def max_over_ranks(x, pg=None, device=None):
    """Largest x over all ranks (x itself without a process group)."""
    if pg is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, seconds):
    """Whole-job rate in G units/s: every rank processes its own copy of the
    workload (weak scaling), the job takes as long as its slowest rank."""
    return world * units_per_rank / seconds / 1e9


# ----------------------------------------------------------------------------- our arm

def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


PAIR32_SOURCES = ("sk_pair32.cuh", "sk_pair32.cu", "sk_series.cuh")


def pair32_source_hash():
    """Hash of what shapes the FP32 pair kernel's launch: its own sources, the
    chunk and decomposition policy (choose_chunks, choose_decomposition in
    sk_decomp.h) and the work-decomposition constants of sk_internal.h (up to
    the Bump allocator)."""
    csrc = os.path.join(ROOT, "paper_2310_13908_gb300", "csrc")
    h = hashlib.sha256()
    for name in PAIR32_SOURCES:
        h.update(open(os.path.join(csrc, name), "rb").read())
    api = open(os.path.join(csrc, "sk_decomp.h")).read()
    for fn in ("int choose_chunks(", "void choose_decomposition("):
        i = api.index(fn)
        h.update(api[i:api.index("\n}\n", i)].encode())
    hdr = open(os.path.join(csrc, "sk_internal.h")).read()
    h.update(hdr[hdr.index("namespace sk {"):hdr.index("// Bump allocator")].encode())
    return h.hexdigest()


def traffic_from_profile():
    """DRAM bytes per pair-kernel launch (full-size workload) from the committed
    ncu summary, if it was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "pair32_dram_traffic.txt")
    if not os.path.exists(path):
        return None
    rec = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            rec[k.strip()] = v.strip()
    try:
        if rec.get("source_sha256") != pair32_source_hash():
            return None
        return float(rec["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.membrane_only:
        return membrane_only(args)
    if args.fmm_only:
        return fmm_only(args)
    rank, world, local = dist_env()
    import torch
    import paper_2310_13908_gb300 as sk

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    serve_future = None
    default_step = args.layer == "sl" and args.precision == "fp32c"
    if rank == 0 and world == 1 and not args.no_extras and default_step:
        import concurrent.futures
        serve_future = concurrent.futures.ThreadPoolExecutor(1).submit(build_serving_mix)
    w = workload(args.m, args.probes, rank)
    s = w.surface
    if serve_future is not None:
        serve_future.result()  # keep the host idle (no GIL contention) while timing
    M = w.targets.shape[0]
    Ns = s.n_active
    inter = M * Ns

    def tdev(a):
        return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)

    X, W, F, Y, D = (tdev(a) for a in (s.X, s.w, w.f, w.targets, w.delta))
    dl = args.layer == "dl"
    NRM = tdev(s.n) if dl else None
    prec_main = sk.SK_FP64 if args.precision == "fp64" else sk.SK_FP32C
    out = torch.empty((M, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    ctx = sk.Context(local)
    h = ctx.handle
    sk.sk_set_profiling(h, True)
    stream = torch.cuda.current_stream(dev)

    def step(prec=prec_main, delta=D):
        if dl:
            sk.stokes_dl_eval(h, prec, sk.SK_DEVICE, X, W, NRM, F, Y, delta, u_out=out,
                              stream=stream)
        else:
            sk.stokes_sl_eval(h, prec, sk.SK_DEVICE, X, W, F, Y, delta, 1.0, u_out=out,
                              stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    pair_ms, launches = [], 0
    torch.cuda.synchronize(dev)
    t_wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        st = sk.sk_last_eval_stats(h)  # waits for this step
        pair_ms.append(st["pair_ms"])
        launches += st["kernel_launches"]
    torch.cuda.synchronize(dev)
    if pg:
        pg.barrier()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_step = max_over_ranks(np.mean(step_ms), pg, dev)
    value = job_throughput(world, inter, t_step * 1e-3)
    u_fp32 = out.cpu().numpy()
    stats = sk.sk_last_eval_stats(h)

    pair_avg = float(np.mean(pair_ms))
    flops = FLOPS_DL if dl else FLOPS_SL
    fp64 = prec_main == sk.SK_FP64
    peak = FP64_PEAK_TFLOPS if fp64 else FP32_PEAK_TFLOPS
    achieved = flops * inter / (pair_avg * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic_from_profile() if default_step else None,
                "kernel": ({(False, False): "k_pair32<SLayer>", (True, False): "k_pair32<DLayer>",
                            (False, True): "k_pair64<SL>", (True, True): "k_pair64<DL>"}[(dl, fp64)]
                           .replace("k_pair32", "k_pair32_fused" if stats["finish_fused"]
                                    else "k_pair32")),
                "kernel_includes_finish": bool(stats["finish_fused"]),
                "pair_ms": pair_avg, "flops_per_interaction": flops,
                "peak_basis": "nominal dense FP64 of GB300" if fp64 else
                              "2 x 128 FP32 lanes x 152 SMs x 2070 MHz (max SM clock)"}

    # ---- end to end through the C ABI with pinned host buffers (SK_HOST, synchronous)
    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    hX, hW, hF, hY, hD = (pinned(np.ascontiguousarray(a, dtype=np.float64))
                          for a in (s.X, s.w, w.f, w.targets, w.delta))
    hN = pinned(np.ascontiguousarray(s.n, dtype=np.float64)) if dl else None
    hU = pinned(np.zeros((M, 3)))

    def host_step():
        if dl:
            sk.stokes_dl_eval(h, prec_main, sk.SK_HOST, hX, hW, hN, hF, hY, hD, u_out=hU)
        else:
            sk.stokes_sl_eval(h, prec_main, sk.SK_HOST, hX, hW, hF, hY, hD, 1.0, u_out=hU)

    e2e_steps = max(3, min(args.steps, 10))
    for _ in range(2):
        host_step()
    e2e_t = []
    for _ in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        host_step()
        e2e_t.append(time.perf_counter() - t0)
    e2e_step = max_over_ranks(np.mean(e2e_t), pg, dev)
    h2d = (hX.nbytes + hW.nbytes + hF.nbytes + hY.nbytes + hD.nbytes +
           (hN.nbytes if dl else 0))
    e2e = {"value": job_throughput(world, inter, e2e_step), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(hU.nbytes), "ms_per_step": e2e_step * 1e3,
           "path": f"stokes_{args.layer}_eval(SK_{args.precision.upper()}, SK_HOST), pinned host "
                   "buffers, synchronous"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if fp64 else "f32 pairs + f64 near/final", "data": "synthetic",
            "config": {"workload": workload_name(w, args.layer), "targets": M,
                       "sources_active": Ns, "interactions_per_step": inter,
                       "sources_total": int(s.X.shape[0]),
                       "interactions_dense_per_step": int(M * s.X.shape[0]),
                       "interactions_basis": "value counts targets x active sources (w != 0); "
                                             "the dense count includes the zero-weight nodes",
                       "precision": f"SK_{args.precision.upper()}",
                       "rho_T": 0.5, "rho_c": 5.0,
                       "l2": "flushed between timed steps (256 MB write); inputs 58 MB",
                       "parallelism": f"replicas x{world} (independent workloads)"},
            "roofline": roofline, "e2e": e2e, "gpu_launches": int(launches),
            "clocks": clk, "wall_s_timed": wall,
            "near_pairs_per_step": stats["near_pairs"],
            "overflow_targets": stats["overflow_targets"]}

    if rank == 0 and world == 1 and not args.no_extras and default_step:
        line.update(extras(sk, h, w, X, W, F, Y, D, out, u_fp32, stream, dev, torch,
                           serve_future))
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if pg:
        pg.destroy_process_group()
    return 0


SERVE_REQUESTS = 1000
SERVE_LOADS = (0.3, 0.5, 0.7, 0.9)


def build_serving_mix(n=SERVE_REQUESTS):
    """The serving mix: n requests, ellipsoid or rotated cell, N = 6 n^2
    log-uniform in [1536, 98304], seeded; arrays ready to submit."""
    import capsule_inputs as ci
    from capsule_inputs.workloads import build_request
    out = []
    for spec in ci.serving_mix(n):
        surf, f, delta = build_request(spec)
        out.append((surf.X, surf.w, f, surf.X, np.array([delta]), surf.n_active))
    return out


def run_serving(sk, h, reqs, arrivals=None, keep=()):
    """Serve reqs (all at once if arrivals is None, else at those times in s).
    Returns (wall seconds, latencies in ms, interactions); the results of the
    requests whose indices are in keep go to run_serving.kept."""
    import collections
    srv = sk.serve_create(h, max_slots=32)
    n = len(reqs)
    lat = [None] * n
    phases = []
    inter = 0
    outstanding = collections.OrderedDict()
    kept = {}
    keep = set(keep)
    nxt = 0
    t0 = time.perf_counter()
    while nxt < n or outstanding:
        now = time.perf_counter() - t0
        while nxt < n and (arrivals is None or arrivals[nxt] <= now):
            X, W, F, Y, D, _ = reqs[nxt]
            try:
                tk = sk.serve_submit(srv, X, W, F, Y, D, 1.0)
            except sk.SkError as e:
                if e.code != sk.SK_EBUSY:
                    raise
                break
            late_ms = 0.0 if arrivals is None else (time.perf_counter() - t0 - arrivals[nxt]) * 1e3
            outstanding[tk] = (nxt, late_ms)
            nxt += 1
        progressed = False
        for tk in list(outstanding):
            i, late_ms = outstanding[tk]
            code, u, st = sk.serve_poll(srv, tk, reqs[i][3].shape[0], timeout_us=0)
            if code == sk.SK_EAGAIN:
                continue
            if code != sk.SK_OK:
                raise RuntimeError(f"served request failed: {code}")
            if i in keep:
                kept[i] = u
            lat[i] = late_ms + (st["ready_us"] - st["submit_us"]) * 1e-3
            phases.append((st["admit_us"] - st["submit_us"], st["publish_us"] - st["admit_us"],
                           st["done_us"] - st["publish_us"], st["ready_us"] - st["done_us"]))
            inter += st["interactions"]
            del outstanding[tk]
            progressed = True
        if not progressed:
            time.sleep(50e-6)
    wall = time.perf_counter() - t0
    sk.serve_destroy(srv)
    ph = np.mean(np.array(phases), axis=0) * 1e-3
    run_serving.last_phases_ms = {"queue": ph[0], "prepare": ph[1], "device": ph[2],
                                  "copy_back": ph[3]}
    run_serving.kept = kept
    return wall, lat, inter


def serving_oracle_check(reqs, check, kept, per_request=SERVE_ORACLE_TARGETS):
    """The served results of a seeded subsample of requests against the oracle
    on seeded targets of each: relative L2 per request and over all, and the
    oracle's own throughput on that sample (the CPU baseline of the mix)."""
    import oracle
    rng = np.random.default_rng(8)
    errs, num, den, pairs, secs = [], 0.0, 0.0, 0, 0.0
    for i in check:
        X, W, F, Y, D, n_active = reqs[i]
        tsel = rng.choice(Y.shape[0], min(per_request, Y.shape[0]), replace=False)
        t0 = time.perf_counter()
        ref = oracle.sl(X, W, F, Y[tsel], D, 1.0)
        secs += time.perf_counter() - t0
        pairs += len(tsel) * n_active
        d = kept[int(i)][tsel] - ref
        errs.append(float(np.linalg.norm(d) / np.linalg.norm(ref)))
        num += float(np.sum(d * d))
        den += float(np.sum(ref * ref))
    return {"requests": len(check), "targets_per_request": per_request,
            "rel_l2_vs_oracle": float(np.sqrt(num / den)), "max_request_rel_l2": max(errs),
            "cpu_oracle": {"value": pairs / secs / 1e9, "unit": UNIT,
                           "cores": oracle.max_threads(), "seconds": secs,
                           "sample": f"{len(check)} seeded requests x {per_request} seeded "
                                     "targets x all active sources, FP64, OpenMP"}}


def one_at_a_time(sk, h, reqs):
    """The same requests evaluated one by one (stokes_sl_eval, device memory,
    profiling on): the baseline continuous batching is measured against."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    tot = pair = whole = 0.0
    for X, W, F, Y, D, _ in reqs:
        args = [torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
                for a in (X, W, F, Y, D)]
        out = torch.empty((Y.shape[0], 3), dtype=torch.float64, device=dev)
        sk.stokes_sl_eval(h, sk.SK_FP32C, sk.SK_DEVICE, *args, 1.0, u_out=out)
        st = sk.sk_last_eval_stats(h)
        tot += Y.shape[0] * st["n_src_active"]
        pair += st["pair_ms"]
        whole += st["eval_ms"]
    return {"ginter_per_s_whole_evals": tot / (whole * 1e-3) / 1e9,
            "ginter_per_s_pair_kernel_only": tot / (pair * 1e-3) / 1e9,
            "note": "device time of each evaluation, one after another (the first "
                    "evaluation of each shape, cold)"}


def serving_bench(sk, h, reqs):
    n = len(reqs)
    run_serving(sk, h, reqs[:64])  # warm-up
    check = np.random.default_rng(7).choice(n, SERVE_ORACLE_REQUESTS, replace=False)
    wall, lat, inter = run_serving(sk, h, reqs, keep=check)
    cap = n / wall
    oracle_check = serving_oracle_check(reqs, check, run_serving.kept)
    res = {"requests": n, "mix": "ellipsoid (axes U[0.5,1]) or rotated Evans-Fung cell, "
                                 "N = 6n^2 log-uniform in [1536, 98304], SH density, delta=2h",
           "saturated": {"req_per_s": cap, "ginter_per_s": inter / wall / 1e9,
                         "wall_s": wall, "p50_ms": float(np.percentile(lat, 50)),
                         "p99_ms": float(np.percentile(lat, 99)),
                         "mean_phase_ms": run_serving.last_phases_ms},
           "oracle_check": oracle_check,
           "one_at_a_time": one_at_a_time(sk, h, reqs)}
    for frac in SERVE_LOADS:
        rng = np.random.default_rng(int(frac * 1000))
        arr = np.cumsum(rng.exponential(1.0 / (frac * cap), size=n))
        wall, lat, inter = run_serving(sk, h, reqs, arr)
        res[f"load_{frac}"] = {"lambda_req_per_s": frac * cap, "p50_ms": float(np.percentile(lat, 50)),
                               "p99_ms": float(np.percentile(lat, 99)),
                               "ginter_per_s": inter / wall / 1e9, "wall_s": wall,
                               "mean_phase_ms": run_serving.last_phases_ms}
    return res


def capsule_sweep_bench(sk, h, m=33, rates=(0.25, 0.5, 1.0, 2.0, 4.0, 8.0, 0.5, 1.0), steps=20,
                        dt=1e-3, Es=2.0, ED=20.0):
    """A shear-rate sweep of resident capsules served together: each request
    advances its capsule (stretched ellipsoid (0.9, 1, 1) with a Skalak
    membrane, delta* per step) by `steps` Euler steps; all are submitted at
    once. Against the same steps taken one capsule after another with
    capsule_step. The results agree bit for bit (checked here)."""
    import capsule_inputs as ci
    ref = ci.make_surface(ci.Ellipsoid(0.9, 1.0, 1.0), m)

    def make():
        cap = sk.Capsule(h, m, ref.X * np.array([1.04, 0.98, 1.0]), ref.w, delta=None, mu=1.0,
                         precision=sk.SK_FP32C)
        cap.set_membrane(ref.X, Es, ED)
        return cap

    flows = [(sk.SK_FLOW_SHEAR, r, 0.0, 0.0) for r in rates]
    seq = [make() for _ in flows]
    served = [make() for _ in flows]
    try:
        for cap, fl in zip(seq, flows):  # warm-up (captures the step graphs)
            cap.step(1, dt, None, fl)
        seq2 = [make() for _ in flows]
        t0 = time.perf_counter()
        for cap, fl in zip(seq2, flows):
            cap.step(steps, dt, None, fl)
        t_seq = time.perf_counter() - t0
        srv = sk.serve_create(h, max_slots=len(flows))
        try:
            warm = make()  # warm-up request
            w = sk.serve_submit_capsule(srv, warm, 2, dt, flows[0])
            sk.serve_poll(srv, w, warm.N, timeout_us=60_000_000)
            warm.close()
            t0 = time.perf_counter()
            tickets = [sk.serve_submit_capsule(srv, c, steps, dt, fl)
                       for c, fl in zip(served, flows)]
            lat, same = [], True
            for t, c, twin in zip(tickets, served, seq2):
                code, x, st = sk.serve_poll(srv, t, c.N, timeout_us=120_000_000)
                lat.append((st["ready_us"] - st["submit_us"]) * 1e-3)
                same &= code == sk.SK_OK and np.array_equal(x, twin.positions())
            t_srv = time.perf_counter() - t0
        finally:
            sk.serve_destroy(srv)
        inter = len(flows) * steps * ref.N * np.count_nonzero(ref.w)
        for c in seq2:
            c.close()
        return {"workload": f"{len(flows)} capsules m={m} (N={ref.N}), shear rates {list(rates)}, "
                            f"{steps} Euler steps each, dt={dt}, Skalak Es={Es} ED={ED}",
                "served_wall_s": t_srv, "served_ginter_per_s": inter / t_srv / 1e9,
                "served_p50_ms": float(np.percentile(lat, 50)),
                "served_max_ms": float(np.max(lat)),
                "one_after_another_wall_s": t_seq,
                "one_after_another_ginter_per_s": inter / t_seq / 1e9,
                "bitwise_equal_to_capsule_step": bool(same)}
    finally:
        for c in seq + served:
            c.close()


def fmm_only(args, iters=10, p=6):
    """stokes_sl_eval_fmm(SK_FP32C) on the ellipsoid (1, 0.8, 0.5) nodes of
    order args.m (sources and targets), delta = 2h, k = args.fmm_k clusters
    seeded from every (N_s / k)-th active node: args.warmup untimed calls,
    then args.steps calls timed with CUDA events; one JSON line."""
    import torch
    import capsule_inputs as ci
    import paper_2310_13908_gb300 as sk
    dev = torch.device("cuda", 0)
    s = ci.make_surface(ci.Ellipsoid(1.0, 0.8, 0.5), args.m)
    f = ci.sh_density(s.x0, np.random.default_rng(5), lmax=8)

    def td(a):
        return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)

    X, W, F, D = td(s.X), td(s.w), td(f), td(np.array([2 * s.h]))
    act = np.flatnonzero(s.w)
    k = args.fmm_k
    C0 = td(s.X[act[:: len(act) // k][:k]])
    with sk.Context(0) as c:
        def call():
            return sk.stokes_sl_eval_fmm(c.handle, sk.SK_DEVICE, X, W, F, X, D, 1.0, C0, iters,
                                         p, precision=sk.SK_FP32C)
        for _ in range(max(args.warmup, 1)):
            call()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            call()
        b.record()
        torch.cuda.synchronize(dev)
    inter = s.N * len(act)
    ms = a.elapsed_time(b) / args.steps
    print(json.dumps({"metric": METRIC, "value": inter / (ms * 1e-3) / 1e9, "unit": UNIT,
                      "ms_per_step": ms, "higher_is_better": True,
                      "config": {"workload": f"ellipsoid(1,0.8,0.5) m={args.m} nodes (N={s.N}, "
                                             f"N_s={len(act)}), delta=2h, single-level FMM "
                                             f"SK_FP32C, k={k}, p={p}, {iters} Lloyd steps"}}),
          flush=True)
    return 0


def membrane_only(args, Es=2.0, ED=20.0, reps=10):
    """membrane_force (overset FD derivatives + Skalak tension + divergence,
    FP64) on a deformed ellipsoid (0.9, 1, 1) of order args.m, device memory,
    CUDA events; one JSON line."""
    import torch
    import capsule_inputs as ci
    import paper_2310_13908_gb300 as sk
    dev = torch.device("cuda", 0)
    ref = ci.make_surface(ci.Ellipsoid(0.9, 1.0, 1.0), args.m)
    Xd = torch.as_tensor(ref.X * np.array([1.02, 0.99, 1.0]), device=dev)
    Xr = torch.as_tensor(ref.X, device=dev)
    with sk.Context(0) as c:
        for _ in range(max(args.warmup, 1)):
            sk.membrane_force(c.handle, args.m, sk.SK_DEVICE, Xd, Xr, Es, ED)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            sk.membrane_force(c.handle, args.m, sk.SK_DEVICE, Xd, Xr, Es, ED)
        b.record()
        torch.cuda.synchronize(dev)
    print(json.dumps({"metric": "membrane_force_ms", "value": a.elapsed_time(b) / reps,
                      "unit": "ms", "higher_is_better": False,
                      "config": {"workload": f"ellipsoid(0.9,1,1) m={args.m} (N={ref.N}) "
                                             f"stretched (1.02, 0.99, 1), Es={Es}, ED={ED}, FP64"}}),
          flush=True)
    return 0


def capsule_bench(sk, h, torch, dev, m=129, steps=100, dt=5e-4, Es=2.0, ED=20.0):
    """Capsule with a Skalak membrane in shear flow: stress-free ellipsoid
    (0.9, 1, 1), Es = 2, ED = 20, shear rate 1 (Sec. 4.3 setup), m = 129,
    explicit Euler steps with f = div_gamma Lambda, weights and delta* updated
    every step (Sec. 3.6). Both precisions run all `steps` steps at dt and are
    compared at the end: displacement, area and volume drift. The configured
    dt = 1e-3 is run as written too; explicit Euler is unstable there on this
    grid, so a sweep of dt gives the largest stable step."""
    import capsule_inputs as ci
    ref = ci.make_surface(ci.Ellipsoid(0.9, 1.0, 1.0), m)
    flow = (sk.SK_FLOW_SHEAR, 1.0, 0.0, 0.0)
    res = {"workload": f"ellipsoid(0.9,1,1) stress-free, m={m} (N={ref.N}), Es={Es}, ED={ED}, "
                       f"shear rate 1, explicit Euler, delta* per step",
           "steps": steps, "dt": dt}
    # the membrane force alone (device memory, CUDA events)
    Xd = torch.as_tensor(ref.X * np.array([1.02, 0.99, 1.0]), device=dev)
    Xr = torch.as_tensor(ref.X, device=dev)
    for _ in range(2):
        sk.membrane_force(h, m, sk.SK_DEVICE, Xd, Xr, Es, ED)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(10):
        sk.membrane_force(h, m, sk.SK_DEVICE, Xd, Xr, Es, ED)
    b.record()
    torch.cuda.synchronize(dev)
    res["membrane_force_ms"] = a.elapsed_time(b) / 10

    def run(prec, n, step_dt):
        cap = sk.Capsule(h, m, ref.X, ref.w, delta=None, mu=1.0, precision=prec)
        try:
            cap.set_membrane(ref.X, Es, ED)
            A0, V0 = cap.area_volume()
            cap.step(1, step_dt, None, flow)  # captures the step graph
            t0 = time.perf_counter()
            cap.step(n - 1, step_dt, None, flow)
            ms = (time.perf_counter() - t0) * 1e3 / max(n - 1, 1)
            A, V = cap.area_volume()
            X = cap.positions()
            return X, {"steps": n, "dt": step_dt, "ms_per_step": ms,
                       "area_change": A / A0 - 1.0, "volume_drift": V / V0 - 1.0,
                       "finite": bool(np.all(np.isfinite(X))),
                       "max_displacement": float(np.nanmax(np.linalg.norm(X - ref.X, axis=1)))}
        finally:
            cap.close()

    X32, res["fp32c"] = run(sk.SK_FP32C, steps, dt)
    X64, res["fp64"] = run(sk.SK_FP64, steps, dt)
    res["fp32c_vs_fp64_at_final_step"] = {
        "steps": steps,
        "displacement_rel_l2": rel_l2(X32 - ref.X, X64 - ref.X),
        "area_change_diff": res["fp32c"]["area_change"] - res["fp64"]["area_change"],
        "volume_drift_diff": res["fp32c"]["volume_drift"] - res["fp64"]["volume_drift"]}
    # as written: dt = 1e-3; and the stability sweep (a run counts as stable
    # when it stays finite with |area change| below 1e-2)
    sweep = {}
    for sdt in (6e-4, 7e-4, 8e-4, 9e-4, 1e-3):
        try:
            _, r = run(sk.SK_FP32C, steps, sdt)
            r["stable"] = bool(r["finite"] and abs(r["area_change"]) < 1e-2)
        except sk.SkError as e:  # e.g. delta* no longer finite once the shape has blown up
            r = {"steps": steps, "dt": sdt, "error": str(e), "stable": False}
        sweep[f"{sdt:g}"] = r
    res["fp32c_dt_1e-3_as_configured"] = sweep["0.001"]
    res["dt_stability_fp32c"] = sweep
    stable = [float(k) for k, v in sweep.items() if v["stable"]] + [dt]
    res["largest_stable_dt_of_sweep"] = max(stable)
    return res


def fmm_bench(sk, h, torch, dev):
    """Single-level FMM (Sec. 5) against the direct sums, on the ellipsoid
    (1, 0.8, 0.5) at delta = 2h: nodes as sources and targets at m = 129 and
    193, and the 4x upsampled setting of the paper's m = 96 (the 4m-th order
    nodes as sources, the m-th order nodes as targets, delta = 2 h_fine).
    FP32C FMM and direct FP32C are timed with CUDA events; both are checked
    against the oracle on 1024 seeded targets; the FP64 FMM is timed at
    m = 129 beside the direct FP64 sum."""
    import capsule_inputs as ci
    import oracle

    def td(a):
        return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            u = fn()
        b.record()
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps, u.cpu().numpy()

    shape = ci.Ellipsoid(1.0, 0.8, 0.5)
    out = {"paper_speedup_fmm_vs_direct": {"m32": 1.02, "m64": 1.57, "m96": 1.81},
           "p": 6, "lloyd_iters": 10}
    cases = [("m129", 129, None, (48, 64, 96)), ("m193", 193, None, (96, 128)),
             ("up4_m96", 96, 384, (96, 128))]
    for name, m, m_src, ks in cases:
        tgt_s = ci.make_surface(shape, m)
        src_s = tgt_s if m_src is None else ci.make_surface(shape, m_src)
        f = ci.sh_density(src_s.x0, np.random.default_rng(5), lmax=8)
        delta = 2 * src_s.h
        X, W, F, Y, D = td(src_s.X), td(src_s.w), td(f), td(tgt_s.X), td(np.array([delta]))
        act = np.flatnonzero(src_s.w)
        inter = tgt_s.N * len(act)
        t32, u32 = timed(lambda: sk.stokes_sl_eval(h, sk.SK_FP32C, sk.SK_DEVICE, X, W, F, Y, D,
                                                   1.0), 5)
        idx = np.random.default_rng(7).choice(tgt_s.N, 1024, replace=False)
        ref = oracle.sl(src_s.X, src_s.w, f, tgt_s.X[idx], delta, 1.0)
        row = {"targets": tgt_s.N, "sources_active": int(len(act)), "interactions": inter,
               "direct_fp32c_ms": t32, "direct_fp32c_rel_l2_vs_oracle": rel_l2(u32[idx], ref)}
        for k in ks:
            C0 = td(src_s.X[act[:: len(act) // k][:k]])
            tf, uf = timed(lambda: sk.stokes_sl_eval_fmm(h, sk.SK_DEVICE, X, W, F, Y, D, 1.0, C0,
                                                         10, 6, precision=sk.SK_FP32C), 5)
            row[f"fmm_fp32c_k{k}"] = {"ms": tf, "speedup_vs_direct_fp32c": t32 / tf,
                                      "rel_l2_vs_oracle": rel_l2(uf[idx], ref),
                                      "work_items": sk.sk_last_eval_stats(h)["n_chunks"]}
        if name == "m129":
            C0 = td(src_s.X[act[:: len(act) // 64][:64]])
            t64, u64 = timed(lambda: sk.stokes_sl_eval(h, sk.SK_FP64, sk.SK_DEVICE, X, W, F, Y, D,
                                                       1.0), 2)
            tf64, uf64 = timed(lambda: sk.stokes_sl_eval_fmm(h, sk.SK_DEVICE, X, W, F, Y, D, 1.0,
                                                             C0, 10, 6), 2)
            row["direct_fp64_ms"] = t64
            row["fmm_fp64_k64"] = {"ms": tf64, "speedup_vs_direct_fp64": t64 / tf64,
                                   "rel_l2_vs_oracle": rel_l2(uf64[idx], ref)}
        out[name] = row
    return out


def extras(sk, h, w, X, W, F, Y, D, out, u_fp32, stream, dev, torch, serve_future=None):
    import capsule_inputs as ci
    import oracle
    res = {}
    s = w.surface
    M = w.targets.shape[0]
    inter = M * s.n_active

    # FP64 path, same workload, one timed step
    sk.stokes_sl_eval(h, sk.SK_FP64, sk.SK_DEVICE, X, W, F, Y, D, 1.0, u_out=out, stream=stream)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sk.stokes_sl_eval(h, sk.SK_FP64, sk.SK_DEVICE, X, W, F, Y, D, 1.0, u_out=out, stream=stream)
    e1.record(stream)
    st64 = sk.sk_last_eval_stats(h)
    torch.cuda.synchronize(dev)
    ms64 = e0.elapsed_time(e1)
    u_fp64 = out.cpu().numpy()
    ach64 = FLOPS_SL * inter / (st64["pair_ms"] * 1e-3) / 1e12

    # CPU oracle on a bounded sample: the CPU baseline and the error reference
    idx = sample_targets(w, CPU_SAMPLE_TARGETS)
    t0 = time.perf_counter()
    ref = oracle.sl(s.X, s.w, w.f, w.targets[idx], w.delta, w.mu)
    t_cpu = time.perf_counter() - t0
    cpu_inter = len(idx) * s.n_active
    res["cpu_baseline"] = {"value": cpu_inter / t_cpu / 1e9, "unit": UNIT,
                           "cores": oracle.max_threads(), "kind": "oracle",
                           "sample": f"{len(idx)} seeded targets ({len(idx) - len(idx) // 4} "
                                     f"nodes + {len(idx) // 4} probes) x all {s.n_active} "
                                     "active sources, FP64, OpenMP",
                           "seconds": t_cpu}
    res["rel_l2_vs_oracle"] = {"fp32c": rel_l2(u_fp32[idx], ref),
                               "fp64": rel_l2(u_fp64[idx], ref),
                               "sample_targets": int(len(idx))}
    res["fp64"] = {"value": inter / (ms64 * 1e-3) / 1e9, "unit": UNIT, "ms_per_step": ms64,
                   "rel_l2_vs_oracle": res["rel_l2_vs_oracle"]["fp64"],
                   "roofline": {"bound": "alu", "achieved": ach64, "peak": FP64_PEAK_TFLOPS,
                                "unit": "TFLOP/s", "frac": ach64 / FP64_PEAK_TFLOPS,
                                "kernel": "k_pair64<SL>", "pair_ms": st64["pair_ms"],
                                "peak_basis": "nominal dense FP64 of GB300"}}

    # delta sweep (FP32C timed, one step each), both precisions checked against
    # the oracle on the same seeded sample of nodes and probes
    sweep = {}
    sidx = sample_targets(w, SWEEP_SAMPLE_TARGETS, seed=4321)
    for fac in (1.5, 2.0, 3.0):
        Dd = torch.tensor([fac * s.h], dtype=torch.float64, device=dev)
        sk.stokes_sl_eval(h, sk.SK_FP32C, sk.SK_DEVICE, X, W, F, Y, Dd, 1.0, u_out=out,
                          stream=stream)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sk.stokes_sl_eval(h, sk.SK_FP32C, sk.SK_DEVICE, X, W, F, Y, Dd, 1.0, u_out=out,
                          stream=stream)
        b.record(stream)
        st = sk.sk_last_eval_stats(h)
        torch.cuda.synchronize(dev)
        u32 = out.cpu().numpy()[sidx]
        sk.stokes_sl_eval(h, sk.SK_FP64, sk.SK_DEVICE, X, W, F, Y, Dd, 1.0, u_out=out,
                          stream=stream)
        torch.cuda.synchronize(dev)
        u64 = out.cpu().numpy()[sidx]
        dref = oracle.sl(s.X, s.w, w.f, w.targets[sidx], fac * s.h, w.mu)
        sweep[f"{fac}h"] = {"value": inter / (a.elapsed_time(b) * 1e-3) / 1e9,
                            "pair_ms": st["pair_ms"], "near_pairs": st["near_pairs"],
                            "overflow_targets": st["overflow_targets"],
                            "rel_l2_vs_oracle": {"fp32c": rel_l2(u32, dref),
                                                 "fp64": rel_l2(u64, dref),
                                                 "sample_targets": int(len(sidx))}}
    res["delta_sweep_fp32c"] = sweep

    # double layer on the rotated Evans-Fung cell (m = 65, N = 24,576)
    rw = ci.rbc_workload()
    rs = rw.surface

    def td(a):
        return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)

    RX, RW, RN, RQ, RF, RY, RD = (td(a) for a in (rs.X, rs.w, rs.n, rw.q, rw.f, rw.targets,
                                                  rw.delta))
    rout = torch.empty((rw.targets.shape[0], 3), dtype=torch.float64, device=dev)
    ridx = np.random.default_rng(5).choice(rs.N, 2048, replace=False)
    rinter = rw.targets.shape[0] * rs.n_active
    t0 = time.perf_counter()
    dref = oracle.dl(rs.X, rs.w, rs.n, rw.q, rw.targets[ridx], rw.delta)
    t_dl = time.perf_counter() - t0
    t0 = time.perf_counter()
    sref = oracle.sl(rs.X, rs.w, rw.f, rw.targets[ridx], rw.delta, rw.mu)
    t_sl = time.perf_counter() - t0

    def timed_c2(layer_eval, ref):
        r = {}
        for prec, name in ((sk.SK_FP32C, "fp32c"), (sk.SK_FP64, "fp64")):
            for _ in range(2):
                layer_eval(prec)
            torch.cuda.synchronize(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            reps = 5
            for _ in range(reps):
                layer_eval(prec)
            b.record(stream)
            torch.cuda.synchronize(dev)
            ms = a.elapsed_time(b) / reps
            r[name] = {"value": rinter / (ms * 1e-3) / 1e9, "ms": ms,
                       "rel_l2_vs_oracle": rel_l2(rout.cpu().numpy()[ridx], ref)}
        return r

    dl = timed_c2(lambda prec: sk.stokes_dl_eval(h, prec, sk.SK_DEVICE, RX, RW, RN, RQ, RY, RD,
                                                 u_out=rout, stream=stream), dref)
    sl = timed_c2(lambda prec: sk.stokes_sl_eval(h, prec, sk.SK_DEVICE, RX, RW, RF, RY, RD,
                                                 rw.mu, u_out=rout, stream=stream), sref)
    sample = f"{len(ridx)} seeded node targets x all {rs.n_active} active sources, FP64, OpenMP"
    res["dl_rbc_m65"] = {"workload": f"rotated Evans-Fung cell m=65 N={rs.N} "
                                     f"(N_s={rs.n_active}), double layer, delta=2h",
                         "interactions": rinter, "flops_per_interaction": FLOPS_DL, **dl,
                         "cpu_oracle": {"value": len(ridx) * rs.n_active / t_dl / 1e9,
                                        "unit": UNIT, "cores": oracle.max_threads(),
                                        "sample": sample, "seconds": t_dl}}
    res["sl_rbc_m65"] = {"workload": f"rotated Evans-Fung cell m=65 N={rs.N} "
                                     f"(N_s={rs.n_active}), single layer, delta=2h",
                         "interactions": rinter, "flops_per_interaction": FLOPS_SL, **sl,
                         "cpu_oracle": {"value": len(ridx) * rs.n_active / t_sl / 1e9,
                                        "unit": UNIT, "cores": oracle.max_threads(),
                                        "sample": sample, "seconds": t_sl}}
    # C1: unit sphere m = 19 with a noisy density, FP64 (and FP32C), all targets vs the oracle
    cw = ci.sphere_noise_workload()
    cs = cw.surface
    CX, CW, CF, CY, CD = (td(a) for a in (cs.X, cs.w, cw.f, cw.targets, cw.delta))
    cout = torch.empty((cw.targets.shape[0], 3), dtype=torch.float64, device=dev)
    t0 = time.perf_counter()
    cref = oracle.sl(cs.X, cs.w, cw.f, cw.targets, cw.delta, cw.mu)
    t_c1 = time.perf_counter() - t0
    cinter = cw.targets.shape[0] * cs.n_active
    c1 = {}
    for prec, name in ((sk.SK_FP64, "fp64"), (sk.SK_FP32C, "fp32c")):
        for _ in range(3):
            sk.stokes_sl_eval(h, prec, sk.SK_DEVICE, CX, CW, CF, CY, CD, cw.mu, u_out=cout,
                              stream=stream)
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        reps = 20
        for _ in range(reps):
            sk.stokes_sl_eval(h, prec, sk.SK_DEVICE, CX, CW, CF, CY, CD, cw.mu, u_out=cout,
                              stream=stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b) / reps
        c1[name] = {"value": cinter / (ms * 1e-3) / 1e9, "ms": ms,
                    "rel_l2_vs_oracle": rel_l2(cout.cpu().numpy(), cref)}
    res["sl_sphere_m19"] = {"workload": f"unit sphere m=19 N={cs.N} (N_s={cs.n_active}), "
                                        "f = (1,0,0) + N(0, 0.1^2), single layer, delta=2h, "
                                        "targets = nodes (launch-bound at this size)",
                            "interactions": cinter, **c1,
                            "cpu_oracle": {"value": cinter / t_c1 / 1e9, "unit": UNIT,
                                           "cores": oracle.max_threads(),
                                           "sample": "all targets, FP64, OpenMP",
                                           "seconds": t_c1}}

    # double layer at a size that fills the GPU: ellipsoid m=193 (221,184 nodes)
    try:
        ew = ci.ellipsoid_hires_workload(m=193, n_probes=0, seed=3300)
        es = ew.surface
        eq = ci.sh_density(es.x0, np.random.default_rng(33), lmax=8)
        EX, EW, EN, EQ, EY, ED = (td(a) for a in (es.X, es.w, es.n, eq, ew.targets, ew.delta))
        eout = torch.empty((ew.targets.shape[0], 3), dtype=torch.float64, device=dev)
        for _ in range(2):
            sk.stokes_dl_eval(h, sk.SK_FP32C, sk.SK_DEVICE, EX, EW, EN, EQ, EY, ED, u_out=eout,
                              stream=stream)
        pms = []
        for _ in range(3):
            sk.stokes_dl_eval(h, sk.SK_FP32C, sk.SK_DEVICE, EX, EW, EN, EQ, EY, ED, u_out=eout,
                              stream=stream)
            pms.append(sk.sk_last_eval_stats(h)["pair_ms"])
        einter = ew.targets.shape[0] * es.n_active
        eidx = np.random.default_rng(6).choice(ew.targets.shape[0], 512, replace=False)
        eref = oracle.dl(es.X, es.w, es.n, eq, ew.targets[eidx], ew.delta)
        ach = FLOPS_DL * einter / (np.mean(pms) * 1e-3) / 1e12
        res["dl_ellipsoid_m193"] = {
            "workload": f"ellipsoid(1,0.8,0.5) m=193 N={es.N} (N_s={es.n_active}), double layer, "
                        "delta=2h, targets = nodes",
            "value": einter / (np.mean(pms) * 1e-3) / 1e9, "unit": UNIT,
            "rel_l2_vs_oracle_512": rel_l2(eout.cpu().numpy()[eidx], eref),
            "roofline": {"bound": "alu", "achieved": ach, "peak": FP32_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": ach / FP32_PEAK_TFLOPS,
                         "kernel": "k_pair32<DLayer>", "pair_ms": float(np.mean(pms)),
                         "flops_per_interaction": FLOPS_DL}}
    except Exception as e:
        res["dl_ellipsoid_m193"] = {"error": repr(e)}
    try:
        pk = sk.sk_probe_peaks(h)
        res["peaks_probe"] = {
            "ffma2_tflops": pk["ffma2_tflops"], "dfma_tflops": pk["dfma_tflops"],
            "far_pairs_per_s": pk["far_pairs_per_s"],
            "far_loop_ceiling_tflops": pk["far_pairs_per_s"] * FLOPS_SL / 1e12,
            "note": "microbenchmarks (sk_probe_peaks): FFMA2 and DFMA over full occupancy; "
                    "the single-layer far pair loop with sources in shared memory at the C3 "
                    "kernel's shape (2 f32x2 pairs per lane, 2 CTAs/SM). The roofline peak "
                    "stays the unit-count figure."}
    except Exception as e:
        res["peaks_probe"] = {"error": repr(e)}
    try:
        res["capsule_skalak_m129"] = capsule_bench(sk, h, torch, dev)
    except Exception as e:
        res["capsule_skalak_m129"] = {"error": repr(e)}
    try:
        res["fmm"] = fmm_bench(sk, h, torch, dev)
    except Exception as e:
        res["fmm"] = {"error": repr(e)}
    if serve_future is not None:
        try:
            res["serving"] = serving_bench(sk, h, serve_future.result())
        except Exception as e:  # report, but keep the headline line
            res["serving"] = {"error": repr(e)}
    res["serving_capsule_sweep"] = {}
    for m in (33, 65):
        try:
            res["serving_capsule_sweep"][f"m{m}"] = capsule_sweep_bench(sk, h, m=m)
        except Exception as e:
            res["serving_capsule_sweep"][f"m{m}"] = {"error": repr(e)}
    return res


if __name__ == "__main__":
    sys.exit(main())
