"""Benchmark of the fast Slepian projection on GB300 (one JSON line on stdout).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload c65k|c1m|c4m|tiny]

A step is one fast projection of the whole batch (plan prebuilt): the FFT
convolution B y and the rank-r correction S_T (D o S_T^T y), i.e. every step of the
hot path.  Default workload: N = 65536, W = 1/8, eps = 1e-4, 1024 real FP32
signals (half N(0,1), half 256-tone band-limited), inputs resident in HBM.

  value         projected samples/s (sum of N over the batch, all ranks) / step time
  e2e           the same metric through fst_project_host with pinned HOST buffers:
                host->device copy, projection and device->host copy in the timed region
  roofline      dominant kernel: algorithmic bytes per launch (2 N s per signal read +
                written, plus S_T and the spectrum) / its CUDA-event launch time,
                against the measured HBM copy bandwidth
  cpu_baseline  the FP64 oracle's fast projection on the host cores, bounded sample
  clocks        nvidia-smi samples taken during the timed region

--impl reference times the oracle (the CPU reference of this build) on the same
workload, a bounded sample of signals per step, on rank 0 only.

Multi-GPU (torchrun): every rank projects its own batch (weak scaling, no
collective on the data path); barrier + max over ranks of the step time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "c65k": dict(desc="N=65536 W=1/8 eps=1e-4, 1024 real FP32 signals (512 N(0,1), 512 256-tone)",
                 batch=1024),
    "c1m": dict(desc="N=2^20 W=0.05 eps=1e-6, 64 complex64 signals (32 CN(0,1), 32 band-limited)",
                batch=64),
    "c4m": dict(desc="N=2^22 W=1/4 eps=1e-8, 16 real FP32 signals (8 N(0,1), 8 1024-tone)", batch=16),
    "tiny": dict(desc="N=4096 W=1/16 eps=1e-6, 2 real signals (N(0,1), 64-tone)", batch=2),
    "ragged": dict(desc="ragged batch of 4096 real FP32 signals, N log-uniform in [1000, 262144], "
                        "W ~ U[1/64, 1/4], eps in {1e-3, 1e-6, 1e-8}, N(0,1) entries; one plan per signal",
                   batch=4096),
}


def make_workload(name, device, batch=None, n=None):
    from paper_1611_04950_gb300 import workloads as WL
    if name == "c65k":
        return WL.c65k(batch=batch or 1024, device=device, **({"N": n} if n else {}))
    if name == "c1m":
        return WL.c1m(batch=batch or 64, device=device, **({"N": n} if n else {}))
    if name == "c4m":
        return WL.c4m(batch=batch or 16, device=device, **({"N": n} if n else {}))
    if name == "tiny":
        return WL.tiny(device=device)
    raise ValueError(name)


def max_over_ranks(x, world, device):
    """The largest of every rank's x (the whole job's time is the slowest rank's)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(samples_per_rank, world, seconds):
    """Weak scaling: every rank projects its own batch; value = all ranks' samples / time."""
    return samples_per_rank * world / seconds


def ncu_traffic(kernel, pairs_per_launch, M):
    """DRAM bytes (read + write) of one launch of `kernel`, from the ncu capture summarised in
    profiles/ncu_traffic.txt (lines: kernel, bytes, pairs per captured launch, FFT length M of
    the captured workload), scaled to this launch's pairs; None when that kernel has no capture
    at this FFT length."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        for line in f:
            parts = line.split()
            if len(parts) == 4 and not line.startswith("#") and parts[0] == kernel and int(parts[3]) == M:
                return float(parts[1]) * pairs_per_launch / float(parts[2])
    return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(wl_name, y_sample, plan, budget_s=10.0):
    """Oracle fast projection (FP64, numpy/scipy as written) on host cores, with its plan
    prebuilt; returns (samples/s, threads used, sample description)."""
    from oracle import fst_oracle as O
    import numpy as np
    N = y_sample.shape[1]
    y = np.ascontiguousarray(y_sample.T)
    O.fast_project(plan, y[:, :1])  # warm
    n_done, t0, c0 = 0, time.perf_counter(), time.process_time()
    while True:
        O.fast_project(plan, y)
        n_done += y.shape[1]
        if time.perf_counter() - t0 >= budget_s:
            break
    wall = time.perf_counter() - t0
    cpu = time.process_time() - c0
    threads = max(1, round(cpu / wall))
    return n_done * N / wall, threads, (f"{y.shape[1]} signals of the {wl_name} workload, repeated "
                                        f"{n_done // y.shape[1]}x over {wall:.1f} s, plan prebuilt")


def run_reference(args):
    """--impl reference: the oracle on the host cores, rank 0 only."""
    import numpy as np
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import fst_oracle as O
    wl = make_workload(args.workload, "cpu", batch=8 if args.workload == "c65k" else None)
    y = wl.y.numpy()
    if np.iscomplexobj(y):
        y = y.astype(np.complex128)
    else:
        y = y.astype(np.float64)
    sample = y[: min(8, y.shape[0])]
    N = sample.shape[1]
    K = O.default_K(N, wl.W)
    plan = O.make_plan(N, wl.W, K, wl.eps)
    ys = np.ascontiguousarray(sample.T)
    for _ in range(args.warmup):
        O.fast_project(plan, ys)
    times = []
    c0, t0 = time.process_time(), time.perf_counter()
    for _ in range(args.steps):
        t = time.perf_counter()
        O.fast_project(plan, ys)
        times.append(time.perf_counter() - t)
    wall, cpu = time.perf_counter() - t0, time.process_time() - c0
    step = sum(times) / len(times)
    value = sample.shape[0] * N / step
    line = {
        "impl": "reference", "metric": "projected samples/s", "value": value, "unit": "samples/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOADS[args.workload]["desc"],
                                         "sample_signals_per_step": int(sample.shape[0])},
        "cpu_baseline": {"value": value, "unit": "samples/s", "cores": max(1, round(cpu / wall)),
                         "kind": "oracle",
                         "sample": f"{sample.shape[0]} signals of the workload per step, FP64 oracle fast "
                                   f"projection, plan prebuilt"},
        "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_ragged_bench(args):
    """Ragged batch: fst_plan_many (timed apart), then fst_project_ragged per step,
    against the same signals projected by one fst_project call per signal."""
    import numpy as np
    import torch
    from paper_1611_04950_gb300 import fst as F
    from paper_1611_04950_gb300 import workloads as WL
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    count = args.batch or 4096
    params = WL.ragged_params(count, seed=3)
    t0 = time.perf_counter()
    ps = F.PlanSet(params)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    # every signal is a view of one contiguous device buffer (one host copy per direction)
    lens = [N for (N, W, e) in params]
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    total = int(offs[-1])
    gen = torch.Generator(device="cuda").manual_seed(3)
    yall = torch.randn(total, device="cuda", generator=gen)
    oall = torch.empty_like(yall)
    ys = [yall[offs[i]:offs[i + 1]] for i in range(count)]
    outs = [oall[offs[i]:offs[i + 1]] for i in range(count)]
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        ps.project(ys, outs)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    l0 = F.fst_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ps.project(ys, outs)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = F.fst_launch_count() - l0
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1) / args.steps
    tuning = {f"M=2^{lg}": {"slots_per_group": n, "ms": t} for lg, (n, t) in ps.tuning(ys, outs).items()}
    # per-kernel device time of one batched call (events around every launch: direct launches)
    F.fst_profile_enable(True)
    ps.project(ys, outs)
    torch.cuda.synchronize()
    per = {}
    for name, t_ms, units in F.fst_profile_records():
        d = per.setdefault(name, {"launches": 0, "ms": 0.0})
        d["launches"] += 1
        d["ms"] += t_ms
    F.fst_profile_enable(False)
    ktot = sum(d["ms"] for d in per.values()) or 1.0
    kernels = {k: {"launches": v["launches"], "ms_per_step": v["ms"], "share": v["ms"] / ktot} for k, v in per.items()}
    # one fst_project call per signal (each plan's own cached graph)
    def per_signal():
        for h, y, o in zip(ps.h, ys, outs):
            F.fst_project(h, y.data_ptr(), o.data_ptr(), 1, 0, F.FST_F32, stream.cuda_stream)
    for _ in range(2):
        per_signal()
    torch.cuda.synchronize()
    kp = max(2, args.steps // 4)
    e0.record(stream)
    for _ in range(kp):
        per_signal()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_per_signal = e0.elapsed_time(e1) / kp
    # end to end: pinned host signals -> device, the ragged projection, results -> host
    e2e = None
    if not args.no_e2e:
        yh = yall.cpu().pin_memory()
        oh = torch.empty_like(yh).pin_memory()

        def e2e_step():
            yall.copy_(yh, non_blocking=True)
            ps.project(ys, outs)
            oh.copy_(oall, non_blocking=True)
        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k2 = max(3, args.steps // 2)
        for _ in range(k2):
            e2e_step()
        torch.cuda.synchronize()
        wall = (time.perf_counter() - t0) / k2
        e2e = {"value": total / wall, "unit": "samples/s", "h2d_bytes_per_step": total * 4,
               "d2h_bytes_per_step": total * 4, "ms_per_step": wall * 1e3}
    # every signal against the FP64 oracle would take minutes on the host: a spread sample
    err, cpu = None, None
    if not (args.no_err and args.no_cpu):
        from oracle import fst_oracle as O
        idx = list(range(0, count, max(1, count // 12)))[:12]
        oplans = {i: O.make_plan(params[i][0], params[i][1], O.default_K(params[i][0], params[i][1]), params[i][2])
                  for i in idx}
        yh64 = {i: ys[i].double().cpu().numpy() for i in idx}
        if not args.no_err:
            es = {}
            for i in idx:
                ref = O.fast_project(oplans[i], yh64[i])
                es[str(i)] = float(np.linalg.norm(outs[i].double().cpu().numpy() - ref) / np.linalg.norm(yh64[i]))
            err = {"max": max(es.values()), "per_signal": es, "tolerance": 1e-5,
                   "against": "FP64 oracle fast projection with each signal's own plan"}
        if not args.no_cpu:
            n_done, c0, t0 = 0, time.process_time(), time.perf_counter()
            while time.perf_counter() - t0 < 10.0:
                for i in idx:
                    O.fast_project(oplans[i], yh64[i])
                    n_done += params[i][0]
            wall, cpu_t = time.perf_counter() - t0, time.process_time() - c0
            cpu = {"value": n_done / wall, "unit": "samples/s", "cores": max(1, round(cpu_t / wall)),
                   "kind": "oracle", "sample": f"{len(idx)} signals spread over the ragged batch (own plans, "
                                               f"prebuilt), repeated over {wall:.1f} s"}
    peaks, src = measured_peaks()
    rsum = sum(F.fst_plan_info(h)["r"] for h in ps.h)
    alg = sum(N * 8 + N * F.fst_plan_info(h)["r"] * 4 for h, (N, W, e) in zip(ps.h, params))
    line = {
        "metric": "projected samples/s", "value": total / (ms * 1e-3), "unit": "samples/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS["ragged"]["desc"], "signals": count, "samples": total,
                   "mean_r": rsum / count, "plan_many_s": plan_s, "autotune": tuning,
                   "l2": "inputs + outputs + S_T exceed the 129 MB L2; no flush"},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "achieved": alg / (ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": alg / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"], "traffic": None,
                     "kernel": "whole ragged step", "peak_source": src, "kernels": kernels},
        "plan_s": plan_s,
        "plain": {"ms_per_step": ms_per_signal, "form": "one fst_project call per signal"},
        "plain_ms_per_step": ms_per_signal, "batched_over_plain": ms_per_signal / ms,
        "max_rel_err_vs_oracle": err,
        "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks,
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c65k", choices=sorted(WORKLOADS))
    ap.add_argument("--batch", type=int, default=None)
    ap.add_argument("--n", type=int, default=None,
                    help="signal length other than the workload's (small cases for profiling only)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain one-signal-per-launch arm")
    ap.add_argument("--no-err", action="store_true", help="skip the per-signal error against the oracle")
    ap.add_argument("--err-signals", type=int, default=16, help="signals checked against the oracle")
    ap.add_argument("--coeffs", default="auto", choices=["auto", "on", "off"],
                    help="also compute the fast coefficient vector each step (auto: on for c4m)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ragged":
        return run_ragged_bench(args)

    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1611_04950_gb300 import fst as F

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    wl = make_workload(args.workload, "cuda", args.batch, args.n)
    y = wl.y.contiguous()
    out = torch.empty_like(y)
    B, N = y.shape
    torch.cuda.synchronize()
    t_plan = time.perf_counter()
    plan = F.Plan(N, wl.W, eps=wl.eps)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t_plan
    stream = torch.cuda.current_stream()
    with_coeffs = args.coeffs == "on" or (args.coeffs == "auto" and args.workload == "c4m")
    coef_buf = None
    if with_coeffs:
        Kp = F.fst_coeffs_info(plan.h)["Kprime"]
        ct = torch.complex128 if y.dtype in (torch.float64, torch.complex128) else torch.complex64
        coef_buf = torch.empty((B, Kp), dtype=ct, device=y.device)

    def step():
        plan.project(y, out)
        if with_coeffs:
            F.fst_coeffs(plan.h, y.data_ptr(), coef_buf.data_ptr(), B, N, F._dtype_code(y.dtype),
                         stream.cuda_stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    l0 = F.fst_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = F.fst_launch_count() - l0
    clocks = sampler.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, "cuda")
    samples_per_step = B * N * world
    value = job_throughput(B * N, world, ms * 1e-3)

    # per-kernel launch times (separate pass with events around every launch)
    F.fst_profile_enable(True)
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    recs = F.fst_profile_records()
    F.fst_profile_enable(False)
    per = {}
    for name, t_ms, units in recs:
        d = per.setdefault(name, {"launches": 0, "ms": 0.0, "pairs": 0})
        d["launches"] += 1
        d["ms"] += t_ms
        d["pairs"] += units
    tot = sum(d["ms"] for d in per.values()) or 1.0
    dom = max(per, key=lambda k: per[k]["ms"])
    dd = per[dom]
    peaks, peak_src = measured_peaks()
    sig_bytes = N * (8 if y.is_complex() else 4)          # bytes of one signal
    pairs_per_launch = dd["pairs"] / dd["launches"]
    signals_per_launch = pairs_per_launch * (1 if y.is_complex() else 2)
    launch_ms = dd["ms"] / dd["launches"]
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = sms * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    log2M = int(round(math.log2(plan.M)))
    log2Q = min(14, max(12, log2M - 5))
    if dom.startswith("k_fastB") or dom.startswith("k_passB"):
        # the row-FFT pass is bound by FP32 instruction issue: its share log2 Q / log2 M of the
        # FFT flops, 5 M log2 Q per real signal (twice per complex one), per launch
        flops = signals_per_launch * (2 if y.is_complex() else 1) * 5.0 * plan.M * log2Q
        achieved = flops / (launch_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": achieved / alu_peak, "flops_per_launch": flops,
                    "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 x SM max clock"}
    else:
        alg_bytes = signals_per_launch * 2 * sig_bytes + N * plan.r * 4 + plan.M * 4
        achieved = alg_bytes / (launch_ms * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"], "peak_source": peak_src}
    roofline["traffic"] = ncu_traffic(dom, pairs_per_launch, plan.M)
    roofline["kernel"] = dom
    roofline["kernels"] = {k: {"launches": v["launches"] // 3, "ms_per_step": v["ms"] / 3,
                               "share": v["ms"] / tot} for k, v in per.items()}
    # whole path against the same roofline (all kernels of one step)
    step_alg = B * 2 * sig_bytes + N * plan.r * 4 + plan.M * 4
    roofline["path_frac"] = step_alg / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"]
    # and against the FP32 ALU: forward + inverse FFT of length M (5 M log2 M flops per real
    # signal, twice that per complex one) plus the rank-r correction (4 N r per real signal,
    # 8 N r per complex one); peak = SMs x 128 FP32 lanes x 2 flops x the maximum SM clock
    cf = 2 if y.is_complex() else 1
    flops = B * cf * (5.0 * plan.M * math.log2(plan.M) + 4.0 * N * plan.r)
    alu_ach = flops / (ms * 1e-3) / 1e12
    roofline["alu"] = {"achieved": alu_ach, "peak": alu_peak, "unit": "TFLOP/s", "frac": alu_ach / alu_peak,
                       "flops_per_step": flops, "peak_source": f"{sms} SMs x 128 lanes x 2 x SM max clock"}

    # the plain FP32 form on the same GPU: one fst_project call per signal, generic four-step
    # kernels with the CUDA-core correction, no graph, no tensor cores (FST_PLAIN=1)
    plain = None
    if not args.no_plain:
        out_plain = torch.empty_like(y)
        code = F._dtype_code(y.dtype)

        def plain_step():
            for b in range(B):
                F.fst_project(plan.h, y[b].data_ptr(), out_plain[b].data_ptr(), 1, N, code, stream.cuda_stream)
        os.environ["FST_PLAIN"] = "1"
        try:
            plain_step()
            torch.cuda.synchronize()
            kp = max(2, args.steps // 5)
            e0.record(stream)
            for _ in range(kp):
                plain_step()
            e1.record(stream)
            torch.cuda.synchronize()
        finally:
            os.environ.pop("FST_PLAIN", None)
        plain_ms = max_over_ranks(e0.elapsed_time(e1) / kp, world, "cuda")
        step()
        torch.cuda.synchronize()
        diff = torch.linalg.vector_norm((out_plain - out).reshape(B, -1), dim=1)
        ynrm = torch.linalg.vector_norm(y.reshape(B, -1), dim=1)
        plain = {"ms_per_step": plain_ms, "value": job_throughput(B * N, world, plain_ms * 1e-3),
                 "batched_over_plain": plain_ms / ms,
                 "max_rel_diff_vs_batched": float((diff / ynrm).max().item()),
                 "form": "one fst_project per signal; generic FP32 four-step kernels, CUDA-core rank-r "
                         "correction, no CUDA graph, no tensor cores"}

    # error against the FP64 oracle's fast projection, per signal of a sample (outside the
    # timed regions); the oracle plan is reused by the CPU baseline below
    oplan, err = None, None
    if rank == 0 and not (args.no_err and args.no_cpu):
        from oracle import fst_oracle as O
        t0 = time.perf_counter()
        oplan = O.make_plan(N, wl.W, plan.K, wl.eps)
        oplan_s = time.perf_counter() - t0
    if rank == 0 and not args.no_err:
        nsamp = min(B, args.err_signals)
        idx = sorted(set(int(round(i * (B - 1) / max(1, nsamp - 1))) for i in range(nsamp)))
        ys = y[idx].cpu()
        ys = ys.to(torch.complex128) if ys.is_complex() else ys.double()
        ref = O.fast_project(oplan, ys.numpy().T).T
        got = out[idx].cpu().numpy()
        e = np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ys.numpy(), axis=1)
        err = {"max": float(e.max()), "per_signal": {str(i): float(v) for i, v in zip(idx, e)},
               "tolerance": 1e-5, "against": "FP64 oracle fast projection at the same eps",
               "oracle_plan_s": oplan_s}

    # end to end: pinned host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        yh = y.cpu().pin_memory()
        oh = torch.empty_like(yh).pin_memory()
        nbytes_in = nbytes_out = B * sig_bytes
        if with_coeffs:
            # projection + coefficient vector: host y -> device, both results -> host
            ch = torch.empty(coef_buf.shape, dtype=coef_buf.dtype).pin_memory()
            nbytes_out += ch.numel() * ch.element_size()

            def e2e_step():
                y.copy_(yh, non_blocking=True)
                step()
                oh.copy_(out, non_blocking=True)
                ch.copy_(coef_buf, non_blocking=True)
        else:
            # the host-buffer entry point: chunked copies overlapped with the projection
            def e2e_step():
                plan.project_host(yh, oh)
        e2e_step()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k2 = max(3, args.steps // 2)
        for _ in range(k2):
            e2e_step()
        torch.cuda.synchronize()
        wall = max_over_ranks((time.perf_counter() - t0) / k2, world, "cuda")
        e2e = {"value": job_throughput(B * N, world, wall), "unit": "samples/s", "h2d_bytes_per_step": nbytes_in,
               "d2h_bytes_per_step": nbytes_out, "ms_per_step": wall * 1e3}

    cpu = None
    if rank == 0 and not args.no_cpu:
        ys = y[: min(8, B)].cpu()
        ys = ys.to(torch.complex128) if ys.is_complex() else ys.double()
        rate, threads, sample = cpu_oracle_rate(args.workload, ys.numpy(), oplan)
        cpu = {"value": rate, "unit": "samples/s", "cores": threads, "kind": "oracle", "sample": sample}

    if rank == 0:
        line = {
            "metric": "projected samples/s", "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "c64" if y.is_complex() else "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload]["desc"] + (f"; N overridden to {N} (profiling case)"
                                                                       if args.n else ""),
                       "N": N, "W": wl.W, "eps": wl.eps,
                       "batch_per_gpu": B, "K": plan.K, "r": plan.r, "M": plan.M,
                       "step": "projection + fast coefficient vector" if with_coeffs else "projection",
                       "l2": f"inputs {B * sig_bytes / 2**20:.0f} MiB + outputs of the same size exceed "
                             f"the 129 MB L2; no flush"},
            "gpu_launches": launches,
            "roofline": roofline,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clocks,
            "plan_s": plan_s,
            "plain": plain,
            "plain_ms_per_step": plain["ms_per_step"] if plain else None,
            "batched_over_plain": plain["batched_over_plain"] if plain else None,
            "max_rel_err_vs_oracle": err,
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
