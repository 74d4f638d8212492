#!/usr/bin/env python
"""Benchmark of the Monte-Carlo ELBO step (variational sparse phase search).

Workload: the K=50 single fit — 50 candidate phases with 5-80 peaks each,
N=4500 2-theta points (10-100 deg, 0.02 deg step), S=256 Monte-Carlo samples,
2000 SVI steps, seeded synthetic diffractogram with 4 planted phases.

One bench step = one complete fit on the resident problem: 2000 SVI steps
(sample -> profile/likelihood -> backward -> Adam -> ELBO) followed by the
posterior over phase combinations (4096 posterior draws).  The headline value
is ELBO evaluations per second, counted densely as S * sum_k M_k * N per SVI
step: every step computes the profile and its gradient as the full sum over
every (sample, peak, point) triple.  Peaks far from a 256-point tile reach it
only through a smooth Lorentzian tail, which is evaluated at 32 Chebyshev
nodes of the tile and interpolated (the same sums to below FP32 rounding), so
fewer evaluations are executed than counted; "executed_evals_per_step" gives
their number, and the roofline is taken on the executed work.  The step time
is the time-to-posterior.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank fits its own replica (no data-path
collective; weak scaling), and the timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import shutil
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ELBO evals/s (S·K·peaks·N) + time-to-posterior K=50; served p50/p99 latency"
S_POST = 4096
TOP_M = 16
PROFILE_STEPS = 64          # of the 2000 SVI steps, launched kernel by kernel between events
CPU_SAMPLE_STEPS = 4        # oracle cpu-baseline sample: 4 of the fit's 2000 SVI steps (S = 256)
REF_STEP_ITERS = 1          # reference-arm step: one oracle SVI step (S = 256)
# Algorithmic work of each profile kernel: FP32-pipe lane operations (an FMA
# counts once) and MUFU operations per evaluation of each kind, times the
# evaluations the step executed (counted from its peak ranges):
#   direct side-uniform, forward: t = fma(s, x - x0, b), 1 + t^2, I0 d1 + I1 d0 (2 for
#       two peaks), d0 d1, accumulate          -> 4 FP32 + 0.5 MUFU (rcp per two peaks)
#   direct side-uniform, backward: t, 1 + t^2, I L, sum I L, I L^2, sum I L^2 t,
#       sum I L^2                               -> 7 FP32 + 1 MUFU
#   mixed range, forward: x - p - mu (2), s t, t^2, 1 + t^2, two accumulations
#                                               -> 7 FP32 + 2 MUFU (rcp, ex2)
#   mixed range, backward: t (3), t^2, 1 + t^2, g I, q L, q L^2, q L^2 t, q L^2 t^2
#       and their five sums (Lorentzian part)   -> 14 FP32 + 1 MUFU; its Gaussian part,
#       on the 64-point blocks within the peak's reach: q G, q G t and five sums
#                                               -> 7 FP32 + 1 MUFU (ex2)
#   Gaussian reach beyond the mixed range: t (2), t^2, accumulate (forward, every
#       point: 4 FP32; backward, the blocks within reach: g I G, three sums: 9 FP32),
#       1 MUFU (ex2)
#   far field, per (peak, node): x_p - p, t, 1 + t^2, accumulate -> 4 FP32 + 1 MUFU
#       forward; backward t (2), 1 + t^2, I L, I L^2 and three sums -> 8 FP32 + 1 MUFU
#   likelihood: the far-field interpolation and node weights, 32 FMAs each per point
# FP32 pipe 128 lanes/clk/SM; MUFU 32 lanes/clk/SM (ex2.approx measured at 30).
OPS = {
    "direct": {"uniform": (4, 0.5), "mixed": (7, 2), "gauss_reach": (4, 1)},
    "far_fwd": {"far_nodes": (4, 1)},
    "bwd_uniform": {"uniform": (7, 1)},
    "bwd_near": {"mixed": (14, 1), "mixed_gauss_bwd": (7, 1), "gauss_reach_bwd": (9, 1)},
    "far_bwd": {"far_nodes": (8, 1)},
}
MUFU_LANES = 32
# The contract count of the work per executed evaluation (every (sample, peak,
# point) term and every far-field (peak, node) term): 8 FP32 lane operations +
# 2 MUFU in the forward profile kernel, 16 FP32 + 2 MUFU in the backward.
CONTRACT_OPS = {"k_fwd_direct": (8, 2), "k_bwd_direct": (16, 2)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--iters", type=int, default=None, help="SVI steps per fit (default: workload's 2000)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-enumeration", action="store_true", help="skip the K=8 exact-enumeration and estimator-variant legs")
    ap.add_argument("--variants-only", action="store_true",
                    help="run only the estimator/model-variant leg and print its JSON (profiling aid)")
    ap.add_argument("--batch-only", type=int, default=0, metavar="NFITS",
                    help="run only the batched-fits leg on this many serving-workload requests and print its JSON "
                         "(profiling aid)")
    ap.add_argument("--batch-iters", type=int, default=100, help="SVI steps of the batched-fits leg")
    ap.add_argument("--batch-samples", type=int, default=0,
                    help="Monte-Carlo samples per fit of the batched-fits leg (0: the requests' own, 256)")
    ap.add_argument("--serve-slots", type=int, default=SERVE_SLOTS, help="resident fits of the serving leg")
    ap.add_argument("--serve-requests", type=int, default=64,
                    help="requests of the serving leg (0: skip); the first is the K=50 fit")
    ap.add_argument("--serve-rate", type=float, default=SERVE_RATE,
                    help="Poisson arrival rate of the serving leg, requests/s (the workload's is 200)")
    ap.add_argument("--serve-only", action="store_true",
                    help="run only the serving leg (no overlap sub-leg) and print its JSON")
    return ap.parse_args()


def guarded(name, fn):
    """fn() or, if it raises, {"error": ...} (the message also on stderr)."""
    try:
        return fn()
    except Exception as e:   # noqa: BLE001 - any failure of an extra leg is reported, not raised
        msg = f"{type(e).__name__}: {e}"[:300]
        print(f"bench: {name} leg failed: {msg}", file=sys.stderr, flush=True)
        return {"error": msg}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, value):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def recorded_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu record of the
    K=50 step, or None when the kernel source changed since it was taken."""
    import hashlib
    rec = os.path.join(ROOT, "profiles", "dram_traffic_K50_N4500_S256.json")
    src = os.path.join(ROOT, "paper_2501_09308_gb300", "csrc", "xrdvi_kernels.cu")
    try:
        d = json.load(open(rec))
        if d.get("kernels_source_sha256") != hashlib.sha256(open(src, "rb").read()).hexdigest():
            return None
        return d["dram_bytes_per_launch"].get(kernel)
    except Exception:
        return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = None
        self.gpu = gpu_index
        exe = shutil.which("nvidia-smi")
        if exe:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen([exe, "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def l2_flush(buf):
    buf.add_(1.0)  # writes a buffer larger than L2 (129 MB) between timed steps


def cpu_baseline(inst, steps):
    """The FP64 oracle as it stands, on this host's cores: `steps` SVI steps
    (sample, ELBO + gradient at all S samples, Adam) of the same fit."""
    import oracle
    P = oracle.Problem.from_instance(inst)
    t0 = time.perf_counter()
    P.fit(inst.S, steps, 1000)
    dt = time.perf_counter() - t0
    evals = inst.evals_per_iter * steps
    return {"value": evals / dt, "unit": "evals/s", "cores": oracle.max_threads(), "kind": "oracle",
            "seconds": dt,
            "sample": f"{steps} of the {inst.iters} FP64 SVI steps (S={inst.S}) of the K={inst.K}, N={inst.N} "
                      f"fit ({evals:.3e} evals)"}


def run_reference(args, world, rank):
    """Reference arm: the FP64 oracle on the host cores, same metric and
    config; each step is a bounded sample of the fit: one SVI step at S=256."""
    if rank != 0:
        return
    import oracle
    from paper_2501_09308_gb300 import synth
    inst = synth.config(1)
    P = oracle.Problem.from_instance(inst)
    state = P.fit(inst.S, args.warmup, 1000) if args.warmup > 0 else None
    t0 = time.perf_counter()
    for i in range(args.steps):
        kw = {} if state is None else {"loc": state["loc"], "raw": state["raw"], "m": state["m"], "v": state["v"],
                                       "t0": args.warmup + i}
        state = P.fit(inst.S, REF_STEP_ITERS, 1000, **kw)
    dt = time.perf_counter() - t0
    evals = inst.evals_per_iter * REF_STEP_ITERS * args.steps
    v = evals / dt
    out = {
        "metric": METRIC, "value": v, "unit": "evals/s", "impl": "reference", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(inst, l2="host caches; no GPU"),
        "cpu_baseline": {"value": v, "unit": "evals/s", "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": f"per step {REF_STEP_ITERS} FP64 SVI step (S={inst.S}) of the {inst.iters}-step fit"},
        "e2e": {"value": v, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


SERVE_SLOTS = 4             # fits the server keeps resident (one batch); --serve-slots
SERVE_OVERLAP_FITS = 8      # requests timed alone and served together (device-side overlap)
SERVE_RATE = 200.0          # Poisson arrival rate of the serving workload, requests/s; --serve-rate


def serving_leg(n_requests, plain_ms, slots=SERVE_SLOTS, rate=None, overlap=True):
    """Continuous batching: the K=50 fit followed by serving-workload requests
    (K ~ U{10..200}, N ~ U{2000..9000}, 5-100 peaks per phase, S=256, 1000
    steps) arriving as a Poisson stream at `rate` requests/s (the workload's
    200 by default; a lower rate shows the latency without the queue), on a server with
    `slots` resident fits (4 by default: each of these fits fills the GPU by
    itself, so with the same throughput fewer resident fits finish the early
    requests sooner) and a 32 GB device-memory budget; every SVI step of the
    resident fits runs as one batched step.
    Reports time-to-posterior (completion - arrival) percentiles, fits/s, the
    aggregate evaluation rate (dense count) against the single fit's, and the
    K=50 request's served time-to-posterior beside the plain single-fit path's.
    Device-side overlap: SERVE_OVERLAP_FITS of the requests fitted one after
    another through standalone contexts, then the same requests served
    together (all submitted at once), wall-clock time of each."""
    import numpy as np
    from paper_2501_09308_gb300 import serving, synth, xrdvi
    rate = SERVE_RATE if rate is None else float(rate)
    reqs = [synth.config(1)] + [synth.config(4, instance=i) for i in range(1, n_requests)]
    arrivals = synth.arrival_times(n_requests, rate, seed=synth.SEED_BASE + 4000)
    srv = serving.Server(hbm_budget=32 << 30, max_slots=slots)
    res = serving.replay_arrivals(srv, reqs, arrivals, S_post=S_POST, post_seed=77, top_m=TOP_M)
    stats = srv.stats()
    srv.close()
    evals = [r_.evals_per_iter * r_.iters for r_ in reqs]
    out = serving.summarize(res, evals)
    single_rate = reqs[0].evals_per_iter * reqs[0].iters / (plain_ms / 1e3) if plain_ms else None
    out.update({
        "slots": slots, "hbm_budget_bytes": 32 << 30, "arrival_rate_per_s": rate,
        "peak_bytes_in_use": stats["peak_bytes"],
        "single_fit_evals_per_s": single_rate,
        "aggregate_over_single_fit": out["evals_per_s"] / single_rate if single_rate else None,
        "k50_served_time_to_posterior_s": res[0]["latency"],
        "k50_plain_time_to_posterior_s": plain_ms / 1e3 if plain_ms else None,
        "k50_top_combination": [int(k) for k in np.flatnonzero(res[0]["combos"][0])],
        "requests_K": [int(r_.K) for r_ in reqs], "requests_N": [int(r_.N) for r_ in reqs],
        "latency_s": [float(r["latency"]) for r in res],
        "note": f"the first {n_requests} requests of the 4096-request stream (at ~8e12 evaluations per fit the "
                "full stream is hours of work for one GPU; latency is queueing-dominated)" if rate >= 10 else
                f"the first {n_requests} requests of the stream at {rate} requests/s, below the server's throughput",
    })
    if not overlap:
        return out
    sub = reqs[1:1 + SERVE_OVERLAP_FITS]
    t0 = time.perf_counter()
    for r_ in sub:
        c = xrdvi.Context.from_instance(r_, S=r_.S)
        c.fit(r_.iters, trace=False)
        c.posterior(S_POST, 77, TOP_M)
        c.close()
    t_alone = time.perf_counter() - t0
    srv = serving.Server(hbm_budget=32 << 30, max_slots=SERVE_OVERLAP_FITS)
    t0 = time.perf_counter()
    ids = [srv.submit(r_, S_post=S_POST, post_seed=77, top_m=TOP_M) for r_ in sub]
    for i in ids:
        srv.wait(i)
    t_mix = time.perf_counter() - t0
    srv.close()
    out["overlap"] = {"fits": len(sub), "alone_one_after_another_s": t_alone, "served_together_s": t_mix,
                      "speedup": t_alone / t_mix}
    return out


def batch_leg(n_fits, iters, samples=0):
    """xrdvi_fit_batch against the same fits run one after another: n_fits
    serving-workload requests (contexts created up front, graphs warmed; with
    `samples` > 0 that many Monte-Carlo samples per fit instead of 256, which
    makes fits too small to fill the GPU alone), each set advanced by `iters`
    SVI steps; wall-clock times and whether every fit ends bit-identical."""
    import numpy as np
    import torch
    from paper_2501_09308_gb300 import synth, xrdvi
    reqs = [synth.config(4, instance=i) for i in range(1, n_fits + 1)]
    S = samples if samples > 0 else None
    A = [xrdvi.Context.from_instance(r, S=S or r.S) for r in reqs]
    B = [xrdvi.Context.from_instance(r, S=S or r.S) for r in reqs]
    for c in A:
        c.fit(16, trace=False)
    xrdvi.xrdvi_fit_batch([c.h for c in B], 16)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in A:
        c.fit(iters, trace=False)
    t_seq = time.perf_counter() - t0
    t0 = time.perf_counter()
    xrdvi.xrdvi_fit_batch([c.h for c in B], iters)
    t_bat = time.perf_counter() - t0
    same = all(np.array_equal(a.params()[0], b.params()[0]) and np.array_equal(a.params()[1], b.params()[1])
               for a, b in zip(A, B))
    for c in A + B:
        c.close()
    return {"fits": n_fits, "svi_steps": iters, "S": S or int(reqs[0].S), "K": [int(r.K) for r in reqs],
            "N": [int(r.N) for r in reqs],
            "one_after_another_s": t_seq, "batched_s": t_bat, "speedup": t_seq / t_bat, "bit_identical": same}


def enumeration_leg(iters=3000):
    """Exact posterior over all 2^8 - 1 phase combinations of the tiny
    workload (K = 8 candidates, 20 peaks each, N = 2000, S = 16): every
    sub-model fitted to convergence in sub-model batches, FP64 log-sum-exp.
    Timed with CUDA events around the call (host buffers in and out)."""
    import numpy as np
    import torch
    from paper_2501_09308_gb300 import serving, synth
    inst = synth.config(0)
    serving.enumerate_combinations(inst, iters=20)   # warm-up (library load, first contexts)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    masks, elbo, p = serving.enumerate_combinations(inst, iters=iters)
    ev1.record()
    torch.cuda.synchronize()
    sec = ev0.elapsed_time(ev1) / 1e3
    M = np.diff(inst.offsets)
    evals = sum(int(inst.S) * int(M[masks[i]].sum()) * int(inst.N) * iters for i in range(len(masks)))
    best = masks[int(np.argmax(p))]
    return {"K": inst.K, "sub_models": int(len(masks)), "svi_steps": iters, "S": inst.S, "N": inst.N,
            "seconds": sec, "sub_model_fits_per_s": len(masks) / sec, "evals_per_s": evals / sec,
            "best_combination": [int(k) for k in np.flatnonzero(best)], "p_best": float(p.max()),
            "planted": [int(k) for k in inst.planted]}


def kernel_slots(far_on):
    """The kernels behind the library's per-kernel timing slots on each path
    (slots without a kernel on a path are left out)."""
    if far_on:
        return {"sample": "k_sample", "ranges": "k_ranges", "direct": "k_fwd_direct", "lik": "k_lik",
                "bwd_uniform": "k_bwd_direct", "grad_adam": "k_grad", "elbo": "k_elbo"}
    return {"sample": "k_sample", "ranges": "k_ranges", "direct": "k_forward", "lik": "k_lik",
            "bwd_uniform": "k_bwd_uniform", "bwd_near": "k_bwd_near", "grad_adam": "k_grad", "elbo": "k_elbo"}


def named(kern, far_on):
    """{kernel name: mean ms per launch} of the kernels a step launches."""
    return {name: kern[slot] for slot, name in kernel_slots(far_on).items()}


def kernel_rooflines(kern, work, sms, clock_mhz):
    """Per profile kernel: FP32 and MUFU fractions of the peaks from the
    step's evaluation counts (OPS) and the kernels' mean times."""
    fp32_peak = sms * 128 * clock_mhz * 1e6 / 1e12
    mufu_peak = sms * MUFU_LANES * clock_mhz * 1e6 / 1e12
    ops_table = dict(OPS)
    if work["far_nodes"] > 0:   # far field on: node evaluations inside the two direct kernels
        ops_table = {"direct": dict(OPS["direct"], far_nodes=OPS["far_fwd"]["far_nodes"]),
                     "bwd_uniform": {"uniform": (7, 1), "mixed": (14, 1), "mixed_gauss_bwd": (7, 1),
                                     "gauss_reach_bwd": (9, 1),
                                     "far_nodes": OPS["far_bwd"]["far_nodes"]}}
    out = {}
    slots = kernel_slots(work["far_nodes"] > 0)
    for name, kinds in ops_table.items():
        if name not in slots or kern[name] <= 1e-4:
            continue
        ops = sum(work[kd] * o[0] for kd, o in kinds.items())
        mufu = sum(work[kd] * o[1] for kd, o in kinds.items())
        if ops == 0:
            continue
        ach = ops / (kern[name] * 1e-3) / 1e12
        row = {"ms": kern[name], "fp32_tops_per_kind": ach, "frac_per_kind": ach / fp32_peak,
               "mufu_frac_per_kind": mufu / (kern[name] * 1e-3) / 1e12 / mufu_peak}
        if slots[name] in CONTRACT_OPS:
            executed = work["uniform"] + work["mixed"] + work["gauss_reach"] + work["far_nodes"]
            c_ops, c_mufu = CONTRACT_OPS[slots[name]]
            c_ach = c_ops * executed / (kern[name] * 1e-3) / 1e12
            row.update({"executed_evals": executed, "fp32_tops": c_ach, "frac": c_ach / fp32_peak,
                        "mufu_frac": c_mufu * executed / (kern[name] * 1e-3) / 1e12 / mufu_peak})
        out[slots[name]] = row
    return out


def variants_leg(peaks, steps=32):
    """Estimator and model variants on the K=50 workload: per-kernel CUDA-event
    times of `steps` SVI steps with the Gaussian likelihood, the
    importance-weighted objective, the angle-dependent width, the all-direct
    evaluation (XRDVI_FLAG_DENSE, with its kernels' rooflines) and the
    shared-shape estimator; for the last also the whole fit
    + posterior (time-to-posterior, CUDA events) and the roofline of its
    backward contraction on the tensor cores."""
    import numpy as np
    import torch
    from paper_2501_09308_gb300 import synth, xrdvi
    inst = synth.config(1)
    out = {}
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    c = xrdvi.Context.from_instance(inst, S=inst.S, flags=xrdvi.FLAG_DENSE)
    c.fit(16, trace=False)
    km, work = c.profile_kernels(steps)
    c.close()
    kd = named(km, False)
    out["dense"] = {"kernel_ms_per_launch": kd, "svi_step_ms": sum(kd.values()), "work_counts_per_step": work,
                    "roofline": kernel_rooflines(km, work, sms, float(peaks.get("sm_max_mhz", 2070.0)))}
    for name, flags in (("gauss_lik", xrdvi.FLAG_GAUSS_LIK), ("iw_elbo", xrdvi.FLAG_IW_ELBO),
                        ("sec_width", xrdvi.FLAG_SEC_WIDTH), ("shared_shapes", xrdvi.FLAG_SHARED_SHAPES)):
        c = xrdvi.Context.from_instance(inst, S=inst.S, flags=flags)
        c.fit(16, trace=False)
        k = c.profile_steps(steps)
        out[name] = {"kernel_ms_per_launch": k, "svi_step_ms": sum(k.values())}
        if flags == xrdvi.FLAG_SHARED_SHAPES:
            c.close()
            c = xrdvi.Context.from_instance(inst, S=inst.S, flags=flags)
            init = c.state()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c.fit(inst.iters, trace=False)   # warm-up fit (graphs captured)
            c.set_state(init)
            torch.cuda.synchronize()
            ev0.record()
            c.fit(inst.iters, trace=False)
            post = c.posterior(S_POST, 77, TOP_M)
            ev1.record()
            torch.cuda.synchronize()
            ttp = ev0.elapsed_time(ev1) / 1e3
            Npad = (inst.N + 255) // 256 * 256
            flop = 2.0 * inst.S * 10 * inst.K * Npad          # backward contraction, FP32-equivalent
            tflops = flop / (k["backward"] * 1e-3) / 1e12
            tf32_peak = float(peaks.get("bf16_tflops", 1965.0)) * 1.1 / 2.25
            out[name].update({
                "time_to_posterior_s": ttp, "svi_steps": inst.iters,
                "top_combination": [int(v) for v in np.flatnonzero(post["combos"][0])],
                "backward_gemm": {"shape": [inst.S, 10 * inst.K, Npad], "achieved_tflops": tflops,
                                  "tensor_tflops_3xtf32": 3 * tflops, "tf32_peak_tflops": tf32_peak,
                                  "frac_of_tf32_peak": 3 * tflops / tf32_peak,
                                  "peak_source": "measured bf16 cuBLAS burst x nominal TF32/BF16 ratio 1.1/2.25"}})
        c.close()
    return out


def workload_config(inst, l2):
    return {"workload": f"single fit K={inst.K} (5-80 peaks, sum M={int(inst.offsets[-1])}), N={inst.N}, "
                        f"S={inst.S}, {inst.iters} SVI steps + posterior ({S_POST} draws)",
            "K": inst.K, "peaks_total": int(inst.offsets[-1]), "N": inst.N, "S": inst.S,
            "svi_steps": inst.iters, "posterior_draws": S_POST, "parallelism": "replicas",
            "l2": l2}


def main():
    args = parse()
    if args.variants_only:
        print(json.dumps({"variants": variants_leg(measured_peaks()[0])}), flush=True)
        return
    if args.batch_only > 0:
        print(json.dumps({"batch": batch_leg(args.batch_only, args.batch_iters, args.batch_samples)}), flush=True)
        return
    if args.serve_only:
        print(json.dumps({"serving": serving_leg(args.serve_requests, None, args.serve_slots, args.serve_rate,
                                                 overlap=False)}), flush=True)
        return
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import numpy as np
    import torch
    from paper_2501_09308_gb300 import synth, xrdvi

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the xrdvi library has no CPU path)")
    torch.cuda.set_device(local)
    xrdvi.lib()
    inst = synth.config(1, instance=rank)
    iters = args.iters or inst.iters
    evals_step = inst.evals_per_iter * iters
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    ctx = xrdvi.Context.from_instance(inst, seed=1000 + rank)
    ctx.set_stream(stream.cuda_stream)
    init_state = ctx.state()

    n_prof = max(1, min(PROFILE_STEPS, iters // 2))

    def one_step(prof):
        ctx.fit(iters - (n_prof if prof else 0), trace=False)
        k = ctx.profile_kernels(n_prof) if prof else None
        post = ctx.posterior(S_POST, 77, TOP_M)
        return k, post

    for _ in range(args.warmup):
        ctx.set_state(init_state)
        one_step(prof=False)
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    times = []
    kern = {k: 0.0 for k in xrdvi.PROFILE_KERNELS}
    work = None
    post = None
    barrier(world)
    torch.cuda.synchronize()
    for _ in range(args.steps):
        ctx.set_state(init_state)
        l2_flush(flush)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        (km, work), post = one_step(prof=True)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        for k, v in km.items():
            kern[k] += v / args.steps
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop() if clocks else None
    total_ms = max_over_ranks(world, float(sum(times)))
    ms_step = total_ms / args.steps
    value = sum_over_ranks(world, evals_step * args.steps) / (total_ms / 1e3)

    # end to end through the C ABI with host buffers: create (H2D) -> fit (trace D2H) -> posterior (D2H)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c2 = xrdvi.Context.from_instance(inst, seed=2000 + rank)
    trace = c2.fit(iters, trace=True)
    post2 = c2.posterior(S_POST, 77, TOP_M)
    c2.close()
    e2e_s = max_over_ranks(world, time.perf_counter() - t0)
    e2e_value = sum_over_ranks(world, evals_step) / e2e_s
    K, N, M = inst.K, inst.N, int(inst.offsets[-1])
    h2d = (K + 1) * 4 + 2 * M * 4 + 3 * N * 4
    d2h = iters * 8 + 8 + K * 8 + TOP_M * ((K + 63) // 64) * 8 + TOP_M * 8

    # the legs after the timed fits are reported beside the metric; one that fails
    # reports its error instead of taking the metric's line with it
    serve = None
    if rank == 0 and world == 1 and args.serve_requests > 0:
        serve = guarded("serving", lambda: serving_leg(args.serve_requests, ms_step, args.serve_slots,
                                                       args.serve_rate))
    enum = guarded("enumeration", enumeration_leg) if rank == 0 and world == 1 and not args.no_enumeration else None
    variants = (guarded("variants", lambda: variants_leg(measured_peaks()[0]))
                if rank == 0 and world == 1 and not args.no_enumeration else None)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = guarded("cpu_baseline", lambda: cpu_baseline(inst, CPU_SAMPLE_STEPS))

    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if rank != 0:
        return
    peaks, peak_src = measured_peaks()
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    clock_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = sms * 128 * clock_mhz * 1e6 / 1e12   # FP32 lane operations per second (Top/s)
    per_kernel = kernel_rooflines(kern, work, sms, clock_mhz)
    dom = max(per_kernel, key=lambda k: per_kernel[k]["ms"])
    executed = work["uniform"] + work["mixed"] + work["gauss_reach"] + work["far_nodes"]
    far_on = work["far_nodes"] > 0
    # per SVI step: sample, ranges, forward, lik, grad (whose extra block forms the ELBO) and
    # either bwd_uniform + bwd_near (dense) or bwd_direct (far field); posterior: sample,
    # ranges, forward, lik, post_sample, post_reduce, post_sort, post_topm
    launches_per_step = (6 if far_on else 7) * iters + 8
    kern_named = named(kern, far_on)
    share = {k: v / sum(kern_named.values()) for k, v in kern_named.items()}
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "evals/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": workload_config(inst, l2="256 MB buffer written between timed steps (L2 flush)"),
        "time_to_posterior_s": ms_step / 1e3,
        "svi_step_ms": ms_step / iters,
        "kernel_ms_per_launch": kern_named,
        "kernel_share": share,
        "executed_evals_per_step": executed,
        "work_counts_per_step": work,
        "roofline": {
            "bound": "alu",
            "kernel": dom,
            "achieved": per_kernel[dom]["fp32_tops"],
            "peak": fp32_peak,
            "unit": "Top/s (FP32 lane ops)",
            "frac": per_kernel[dom]["frac"],
            "traffic": recorded_traffic(dom),
            "peak_source": f"FP32 pipe: {sms} SMs x 128 lanes x {clock_mhz:.0f} MHz ({peak_src} sm_max_mhz, "
                           "nominal lane count; no measured FP32 peak exists for this pool)",
            "count": "contract: 8 FP32 + 2 MUFU per executed evaluation (forward), 16 + 2 (backward), times the "
                     "step's executed (sample, peak, point) and far-field (peak, node) terms; *_per_kind: the "
                     "builder's finer count of each kind of evaluation (OPS in bench.py)",
            "mufu_frac": per_kernel[dom]["mufu_frac"],
            "frac_per_kind": per_kernel[dom]["frac_per_kind"],
            "kernels": per_kernel,
        },
        "e2e": {"value": e2e_value, "unit": "evals/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "seconds": e2e_s},
        "gpu_launches": launches_per_step * args.steps,
        "posterior": {"top_combination": [int(k) for k in np.flatnonzero(post["combos"][0])],
                      "planted": [int(k) for k in inst.planted],
                      "pi_planted_min": float(min(post["pi"][inst.planted])),
                      "e2e_top_combination": [int(k) for k in np.flatnonzero(post2["combos"][0])],
                      "final_elbo": float(trace[-1])},
    }
    if serve:
        out["serving"] = serve
    if enum is not None:
        out["enumeration"] = enum
    if variants is not None:
        out["variants"] = variants
    if clk:
        out["clocks"] = clk
    if cpu:
        out["cpu_baseline"] = cpu
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
