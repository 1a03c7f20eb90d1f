#!/usr/bin/env python
"""Benchmark of the mode-wise flexible st-HOSVD on B300: input GB/s.

One step = one full st-HOSVD (Alg. 2) of each tensor of the workload:
  * 640 x 640 x 640, ranks (64, 64, 64)
  * 128 x 128 x 128 x 128, ranks (16, 16, 16, 16)
Both are random Tucker tensors plus 1e-3 N(0,1) noise (synthetic).  They are
float32, column-major, and resident in HBM before the timed region.  Each
tensor (1.05 GB and 1.07 GB) is larger than the 126 MB L2, so nothing is
flushed between steps.
metric = sum of input bytes / step time.

Printed JSON line (one, rank 0): value, e2e (host buffers through the C ABI,
copies included), roofline of the dominant kernel (timed live with CUDA events
inside the library on the launching stream), the CPU oracle baseline on a
bounded sample, clocks sampled during the timed region, and kernel launches.

``--impl reference`` times the CPU oracle (float64, explicit matricization) on
a bounded sample of the same workload, per step.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "st-HOSVD input GB/s"
UNIT = "GB/s"
TENSORS = [((640, 640, 640), (64, 64, 64)), ((128, 128, 128, 128), (16, 16, 16, 16))]
WORKLOAD = "plain FP32 st-HOSVD (EIG every mode): 640^3 R64 + 128^4 R16, random Tucker + 1e-3 noise"
FP32_ALU_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12  # SMs x FP32 lanes x 2 flop x max SM clock
GRAM_TRAFFIC_RATIO = 1.19  # DRAM read + write bytes / input bytes per Gram launch (ncu, mode-1 Gram)
CPU_SAMPLE = ((640, 640, 8), (64, 64, 8))       # cpu_baseline: a 640 x 640 x 8 slab of the workload
REF_SAMPLE = ((640, 160, 8), (64, 64, 8))       # reference arm: one such slab sample per step


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def gram_flops(dims, ranks, solver, mode_order=None):
    """Algorithmic Gram flops of one st-HOSVD, I_n^2 J_n per EIG mode (Eq. 4)."""
    cur = list(dims)
    total = 0.0
    for n in (mode_order or range(len(dims))):
        J = float(np.prod(cur)) / cur[n]
        if solver[n] == 0:
            total += float(cur[n]) ** 2 * J
        cur[n] = ranks[n]
    return total


class ClockSampler:
    """nvidia-smi clocks during the timed region.

    The sampler starts first and the region begins only after its first
    sample; the samples kept run from the last one before the region to the
    first one after it (20 ms apart), so even a region of a few tens of ms
    is covered."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self.first = self.last = 0

    def _wait_lines(self, count, timeout):
        t_end = time.time() + timeout
        while len(self.lines) < count and time.time() < t_end and self.proc.poll() is None:
            time.sleep(0.002)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            self._wait_lines(1, 5.0)
            self.first = max(0, len(self.lines) - 1)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self._wait_lines(len(self.lines) + 1, 1.0)
            self.last = len(self.lines)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[self.first:self.last]:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return int(os.environ.get("RANK", "0")), ws, int(os.environ.get("LOCAL_RANK", "0"))


def cpu_oracle_sample(sample, reps=1):
    import oracle
    import synth
    dims, ranks = sample
    x, _, _ = synth.random_tucker(dims, ranks, seed=0)
    x64 = x.astype(np.float64)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.sthosvd(x64, dims, ranks, solver=[0] * len(dims))
        times.append(time.perf_counter() - t0)
    return x.nbytes, times


def run_reference(args):
    rank, ws, _ = dist_env()
    if rank != 0:
        return 0
    import oracle  # noqa: F401  (builds the C oracle once before timing)
    oracle.build()
    dims, ranks = REF_SAMPLE
    import synth
    x, _, _ = synth.random_tucker(dims, ranks, seed=0)
    x64 = x.astype(np.float64)
    for _ in range(args.warmup):
        oracle.sthosvd(x64, dims, ranks, solver=[0] * len(dims))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sthosvd(x64, dims, ranks, solver=[0] * len(dims))
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    gbs = x.nbytes / dt / 1e9
    cores = os.cpu_count()
    sample = f"oracle st-HOSVD-EIG (float64, OpenMP loops) of a {dims[0]}x{dims[1]}x{dims[2]} slab sample, ranks {ranks}"
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": gbs, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": gbs, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    rank, ws, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo", init_method="env://")
    torch.cuda.set_device(local)
    import paper_2010_10131_b300 as atk
    import synth
    atk.lib()
    main = torch.cuda.current_stream()
    # The tensors are independent: each has its own plan on its own stream, and
    # a step runs them concurrently (atucker_sthosvd_many), so one tensor's
    # eigensolver (a few CTAs) overlaps the other's Gram.  The tensor with the
    # most Gram work, the longest chain, gets the highest stream priority.
    work = [gram_flops(d, r, [0] * len(d)) for d, r in TENSORS]
    top = max(range(len(TENSORS)), key=lambda t: work[t])
    streams = [torch.cuda.Stream(priority=-5 if t == top else 0) for t in range(len(TENSORS))]
    plans, xs, hosts, xnps = [], [], [], []
    for (dims, ranks), st in zip(TENSORS, streams):
        x, _, _ = synth.random_tucker(dims, ranks, seed=rank)
        xnps.append(x)
        xt = torch.from_numpy(x).cuda()
        p = atk.Plan(dims, ranks, solver=[0] * len(dims), stream=st)
        core = torch.empty(p.core_numel, device="cuda")
        fac = torch.empty(p.factors_numel, device="cuda")
        plans.append((p, core, fac))
        xs.append(xt)
        hosts.append(torch.from_numpy(x).pin_memory())
    torch.cuda.synchronize()
    in_bytes = sum(int(np.prod(d)) * 4 for d, _ in TENSORS)

    def concurrent_step(pl):
        atk.run_many([q for q, _, _ in pl], xs, [c for _, c, _ in pl], [f for _, _, f in pl])

    def serial_step(pl):
        # The same runs one tensor after the other (each stream waits for the previous one).
        prev = None
        for (q, c, f), x, st in zip(pl, xs, streams):
            if prev is not None:
                st.wait_event(prev)
            q.run(x, c, f)
            prev = torch.cuda.Event()
            prev.record(st)
        return prev

    def timed(pl, steps, fn):
        """Device ms per step of `steps` calls of fn(pl), all streams joined at both ends."""
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(main)
        for st in streams:
            st.wait_event(e0)
        for _ in range(steps):
            fn(pl)
        for st in streams:
            done = torch.cuda.Event()
            done.record(st)
            main.wait_event(done)
        e1.record(main)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / max(steps, 1)

    # Warm-up: serial first, so that every cached CUDA graph is captured by one
    # host thread, then concurrent.
    for _ in range(max(args.warmup, 1)):
        serial_step(plans)
    for _ in range(args.warmup):
        concurrent_step(plans)
    # Serial leg: one tensor at a time, so that each Gram launch has the GPU to
    # itself; its CUDA-event durations give the kernel's roofline figure.  The
    # fused TTM + next-mode Gram is off in this leg, so every mode's Gram runs
    # in the Gram kernel whose flops the figure counts.
    for p, _, _ in plans:
        p.sync()
        p.set_option(atk.OPT_FUSE_TTM_GRAM, 0)
        p.set_timing(True)
    serial_ms = timed(plans, args.steps, serial_step)
    stims = [p.timings() for p, _, _ in plans]
    # Headline leg: the concurrent step.
    for p, _, _ in plans:
        p.set_timing(True)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    with ClockSampler(local) as clk:
        ms = timed(plans, args.steps, concurrent_step)
    if ws > 1:
        torch.distributed.barrier()
    for p, _, _ in plans:
        p.sync()
    tims = [p.timings() for p, _, _ in plans]
    if ws > 1:
        t = torch.tensor([ms], dtype=torch.float64)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    value = in_bytes * ws / (ms * 1e-3) / 1e9

    # Dominant kernel: the Gram partial-tile kernel (float32 CUDA cores).
    # DRAM traffic per Gram call, scaled from one ncu capture of a smaller view
    # of the mode-1 Gram: each launch reads its input about once (measured read
    # + write / input bytes = 1.19; the writes are the split-K partial tiles).
    # A contiguous mode-1 view (lo == 1, I_n % 4 == 0) runs all its tiles in
    # one launch; a strided view with more than 128 rows makes two (diagonal
    # and off-diagonal tiles), each reading the input.
    calls, traffic_bytes, alg_bytes = 0, 0.0, 0.0
    for d, r in TENSORS:
        cur = list(d)
        for nmode in range(len(d)):
            size = float(np.prod(cur)) * 4
            lo = int(np.prod(cur[:nmode]))
            launches = 1 if (cur[nmode] <= 128 or (lo == 1 and cur[nmode] % 4 == 0)) else 2
            traffic_bytes += GRAM_TRAFFIC_RATIO * size * launches
            alg_bytes += size
            calls += 1
            cur[nmode] = r[nmode]
    flops = sum(gram_flops(d, r, [0] * len(d)) for d, r in TENSORS) * args.steps
    gram_ms = sum(t["gram"] for t in stims)
    achieved = flops / (gram_ms * 1e-3) / 1e12 if gram_ms > 0 else None
    gram_ms_conc = sum(t["gram"] for t in tims)
    achieved_conc = flops / (gram_ms_conc * 1e-3) / 1e12 if gram_ms_conc > 0 else None
    phases = {k: sum(t[k] for t in tims) / max(args.steps, 1) for k in
              ("gram", "gram_reduce", "eig", "ttm", "als", "norms", "total")}
    launches = int(sum(t["launches"] for t in tims))

    def relerr_recon(x, core, fac, dims, ranks):
        """||X - G x_1 U1 ... x_N UN|| / ||X|| by reconstruction on the GPU:
        valid for any core (the identity ||X||^2 - ||G||^2 needs the exact
        projection, which a rounded TTM is not)."""
        facs = [f.view(r, d).t() for f, d, r in zip(torch.split(fac, [d * r for d, r in zip(dims, ranks)]), dims, ranks)]
        return reconstruct_relerr(x, core, facs, dims, ranks)

    def time_variant(precision=atk.FP32, mode_solver=atk.EIG):
        """ms per step (concurrent, like the headline) and relerr of the same
        workload under other plan settings (`mode_solver` for every mode: EIG,
        ALS or AUTO)."""
        vplans = []
        for (dims, ranks), st in zip(TENSORS, streams):
            vp = atk.Plan(dims, ranks, solver=[mode_solver] * len(dims), precision=precision, stream=st)
            vplans.append((vp, torch.empty(vp.core_numel, device="cuda"), torch.empty(vp.factors_numel, device="cuda")))
        serial_step(vplans)
        for _ in range(args.warmup):
            concurrent_step(vplans)
        vms = timed(vplans, args.steps, concurrent_step)
        rel = [relerr_recon(x, c, f, list(d), list(r)) for x, (_, c, f), (d, r) in zip(xs, vplans, TENSORS)]
        classes = [vp.classes for vp, _, _ in vplans]
        for vp, _, _ in vplans:
            vp.close()
        return vms, rel, classes

    rel_plain = [relerr_recon(x, c, f, list(d), list(r)) for x, (_, c, f), (d, r) in zip(xs, plans, TENSORS)]
    # Mixed precision on the same tensors: the tensor-core Gram forms, timed
    # like the plain step, each compared by relative error with the plain output.
    mixed = None
    if not args.no_mixed:
        mixed = {"relerr_plain": rel_plain, "forms": {}}
        for name, prec in (("BF16X3", atk.BF16X3), ("TF32", atk.TF32), ("BF16", atk.BF16)):
            mms, rel, _ = time_variant(precision=prec)
            mixed["forms"][name] = {"ms_per_step": mms, "value": in_bytes / (mms * 1e-3) / 1e9,
                                    "speedup_vs_plain": ms / mms, "relerr": rel,
                                    "max_relerr_delta_vs_plain": max(abs(a - b) for a, b in zip(rel, rel_plain))}
    # The solvers on the same workload: every mode ALS (Alg. 3, 5 sweeps), and
    # every mode chosen by the learned selector when its weights are present.
    solvers = None
    if not args.no_mixed:
        # Every solver leg on fresh plans timed the same way (EIG again too, so
        # the comparison does not mix the headline leg's longer warm-up in).
        ems, erel, _ = time_variant(mode_solver=atk.EIG)
        solvers = {"EIG": {"ms_per_step": ems, "value": in_bytes / (ems * 1e-3) / 1e9, "relerr": erel}}
        ams, arel, _ = time_variant(mode_solver=atk.ALS)
        solvers["ALS"] = {"ms_per_step": ams, "value": in_bytes / (ams * 1e-3) / 1e9, "relerr": arel,
                          "speedup_vs_EIG": ems / ams}
        from paper_2010_10131_b300 import selector as atk_selector
        if atk_selector.install():
            sms, srel, scls = time_variant(mode_solver=atk.AUTO)
            solvers["AUTO"] = {"ms_per_step": sms, "value": in_bytes / (sms * 1e-3) / 1e9, "relerr": srel,
                               "speedup_vs_EIG": ems / sms, "classes": scls}

    # The form the method's target names: learned selector and a split-product
    # precision form together, against the plain float32 step.
    mixed_selector = None
    if not args.no_mixed and solvers is not None and "AUTO" in solvers:
        best = None
        for name, prec in (("BF16X3", atk.BF16X3), ("TF32", atk.TF32)):
            mms, rel, cls = time_variant(precision=prec, mode_solver=atk.AUTO)
            row = {"form": name, "ms_per_step": mms, "value": in_bytes / (mms * 1e-3) / 1e9,
                   "speedup_vs_plain": ms / mms, "relerr": rel, "classes": cls,
                   "max_relerr_delta_vs_plain": max(abs(a - b) for a, b in zip(rel, rel_plain))}
            if row["max_relerr_delta_vs_plain"] <= 1e-4 and (best is None or mms < best["ms_per_step"]):
                best = row
        mixed_selector = best

    # End to end through the C ABI with host buffers (copies inside the timed
    # region): the concurrent host-buffer call, so one tensor's copies overlap
    # the other's kernels.
    cores_h = [torch.empty(p.core_numel).pin_memory() for p, _, _ in plans]
    facs_h = [torch.empty(p.factors_numel).pin_memory() for p, _, _ in plans]
    pl_only = [p for p, _, _ in plans]
    atk.run_many_host(pl_only, hosts, cores_h, facs_h)
    e2e_steps = max(1, min(args.steps, 5))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        atk.run_many_host(pl_only, hosts, cores_h, facs_h)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    d2h = sum((p.core_numel + p.factors_numel) * 4 for p, _, _ in plans)

    line = None
    if rank == 0:
        pk = peaks()
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            nb, ts = cpu_oracle_sample(CPU_SAMPLE)
            cpu = {"value": nb / min(ts) / 1e9, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"oracle st-HOSVD-EIG of one {CPU_SAMPLE[0]} slab of the workload, ranks "
                             f"{CPU_SAMPLE[1]} ({min(ts):.1f} s)"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "tensors": [list(d) for d, _ in TENSORS],
                       "ranks": [list(r) for _, r in TENSORS], "solver": "EIG every mode",
                       "precision": "FP32 CUDA cores", "l2": "inputs (1.05 GB, 1.07 GB) larger than L2; no flush",
                       "execution": "the tensors' plans run concurrently (atucker_sthosvd_many), one stream each, "
                                    "the 640^3 tensor's at the highest priority",
                       "serial_ms_per_step": serial_ms},
            "roofline": {"bound": "alu",
                         "kernel": "FP32 Gram (gram_async_kernel for contiguous mode-1 views, gram_ci_kernel for "
                                   "strided ones; float32 FMA)",
                         "achieved": achieved, "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": (achieved / FP32_ALU_PEAK_TFLOPS) if achieved else None,
                         "timed_in": "serial leg of this run (one tensor at a time, same steps), so each Gram "
                                     "launch has the GPU to itself",
                         "achieved_concurrent": achieved_conc,
                         "traffic": traffic_bytes / calls, "traffic_unit": "bytes per Gram call",
                         "algorithmic_bytes": alg_bytes / calls,
                         "traffic_source": "scaled from ncu dram read + write bytes of gram:1,640,80000 (ratio 1.19 x input)",
                         "peak_source": "derived: 148 SMs x 128 FP32 lanes x 2 flop x 2032 MHz",
                         "flops_per_step": flops / max(args.steps, 1),
                         "ms_per_step": gram_ms / max(args.steps, 1)},
            "phases_ms_per_step": phases,
            "mixed": mixed,
            "solvers": solvers,
            "mixed_selector": mixed_selector,
            "e2e": {"value": in_bytes / e2e_s / 1e9, "unit": UNIT, "h2d_bytes_per_step": in_bytes,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
            "hbm_peak_gbs": pk.get("hbm_gbs"),
        }
    for p, _, _ in plans:
        p.close()
    xs.clear()
    torch.cuda.empty_cache()
    if rank == 0 and not args.no_extra:
        # The other workloads of the metric, each a bounded leg (few steps):
        # precision sweep, batched form, learned selector against the paper's
        # decision tree, the Table II stand-ins, the matricization ablation and the
        # fused TTM + next-mode Gram against the separate kernels.
        xargs = argparse.Namespace(**vars(args))
        xargs.steps, xargs.warmup = min(args.steps, 3), 1
        extra = {}
        for key, fn in (("precision_sweep", run_precision), ("roofline_48x5", run_roofline_small),
                        ("batched", run_batched), ("selector", run_selector_summary),
                        ("table2", run_table2), ("explicit_ablation", run_explicit),
                        ("fused_ttm_gram", run_fused)):
            t0 = time.time()
            try:
                extra[key] = fn(xargs)
            except Exception as e:  # a leg that cannot run is reported, not fatal
                extra[key] = {"error": str(e)[:200]}
            extra[key + "_wall_s"] = time.time() - t0
            torch.cuda.empty_cache()
        line.update(extra)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_case(args):
    """Time one step-level operation: --case gram:LO,N,HI, ttm:LO,N,HI,R, als:LO,N,HI,R,
    ttmgram:LO,N,HI,R,S,I_M or eig:N,R[,METHOD].

    Used for kernel profiles: the input is synthetic N(0,1) float32 on the
    device, the call goes through the C ABI, and the line reports the
    operation's device time (CUDA events) and its algorithmic rate.
    """
    import torch
    import paper_2010_10131_b300 as atk
    prec = args.precision
    kind, _, shape = args.case.partition(":")
    if kind == "selector":
        print(json.dumps({"case": "selector", **run_selector(args)}), flush=True)
        return 0
    if kind == "precision":
        print(json.dumps({"case": "precision", "sweep": run_precision(args)}), flush=True)
        return 0
    if kind == "table2":
        print(json.dumps({"case": "table2", "stand_ins": run_table2(args)}), flush=True)
        return 0
    if kind == "explicit":
        print(json.dumps({"case": "explicit", "ablation": run_explicit(args)}), flush=True)
        return 0
    if kind == "batchrun":
        # The batched kernel alone (fixed launch variant, no tuning and no
        # one-at-a-time leg): the command profiles of the kernel use.
        import paper_2010_10131_b300 as atk
        vals = [int(v) for v in shape.split(",")] if shape else [512]
        shapes, xs_np = batched_inputs(vals[0])
        xs = [torch.from_numpy(x).cuda() for x in xs_np]
        b = atk.Batch([d for d, _ in shapes], [r for _, r in shapes])
        b.set_option(atk.BATCH_OPT_VARIANT, vals[1] if len(vals) > 1 else 0)
        cores, facs = b.outputs()
        for _ in range(max(args.warmup, 0) + max(args.steps, 1)):
            b.run(xs, cores, facs)
        b.close()
        print(json.dumps({"case": args.case, "tensors": vals[0]}), flush=True)
        return 0
    if kind == "batched":
        out = run_batched(args, count=int(shape) if shape else 4096)
        print(json.dumps({"case": args.case, **out}), flush=True)
        return 0
    vals = [int(v) for v in shape.split(",")]
    g = torch.Generator(device="cuda").manual_seed(0)
    if kind == "eig":
        # S = Q diag(lambda) Q^T: R signal eigenvalues in [1, 10] over a noise
        # floor 1e-6 (the spectrum of a rank-R Tucker tensor's Gram plus 1e-3 noise).
        n, R = vals[0], vals[1]
        method = vals[2] if len(vals) > 2 else atk.EIG_AUTO
        q, _ = torch.linalg.qr(torch.randn(n, n, device="cuda", dtype=torch.float64, generator=g))
        lam = torch.cat([1 + 9 * torch.rand(R, device="cuda", dtype=torch.float64, generator=g),
                         1e-6 * (1 + torch.rand(n - R, device="cuda", dtype=torch.float64, generator=g))])
        S = ((q * lam) @ q.t()).contiguous()
        U = torch.empty(n * R, device="cuda", dtype=torch.float32)
        lamo = torch.empty(n, device="cuda", dtype=torch.float64)
        disc = torch.empty(1, device="cuda", dtype=torch.float64)
        L = atk.lib()
        stream = torch.cuda.current_stream().cuda_stream

        def fn():
            st = L.atucker_eig(S.data_ptr(), n, R, atk.EIG_ROT_FP32, method, U.data_ptr(), lamo.data_ptr(),
                               disc.data_ptr(), stream)
            if st != 0:
                raise SystemExit(f"atucker_eig failed: {st}")
        flops, lo, hi = 2.0 * n * n * R, 1, n  # one S Q product as the unit of work
    else:
        lo, n, hi = vals[:3]
        y = torch.randn(lo * n * hi, device="cuda", generator=g)
    if kind == "eig":
        pass
    elif kind == "gram":
        fn = lambda: atk.gram(y, lo, n, hi, precision=prec)  # noqa: E731
        flops = float(n) * n * lo * hi  # I_n^2 J_n (Eq. 4)
    elif kind == "ttm":
        R = vals[3]
        U = torch.randn(n, R, device="cuda", generator=g)
        fn = lambda: atk.ttm(y, lo, n, hi, U, precision=prec)  # noqa: E731
        flops = 2.0 * n * R * lo * hi
    elif kind == "als":
        # one ALS mode update, 5 sweeps (Alg. 3): 4 I_n J_n R_n flops per sweep (Eq. 5)
        R = vals[3]
        fn = lambda: atk.als_mode(y, lo, n, hi, R, precision=prec)  # noqa: E731
        flops = 5 * 4.0 * n * R * lo * hi
    elif kind == "ttmgram":
        # fused TTM + next-mode Gram: ttmgram:LO,N,HI,R,S,I_M
        R, s_m, i_m = vals[3], vals[4], vals[5]
        U = torch.linalg.qr(torch.randn(n, R, device="cuda", generator=g))[0]
        fn = lambda: atk.ttm_gram(y, lo, n, hi, U, s_m, i_m)  # noqa: E731
        flops = 2.0 * n * R * lo * hi + float(i_m) * lo * hi * R  # TTM + I_m^2 J_m with J_m = J R / I_m
    else:
        raise SystemExit(f"unknown case {kind}")
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    print(json.dumps({"case": args.case, "precision": prec, "ms": ms, "tflops": flops / (ms * 1e-3) / 1e12,
                      "input_gbs": lo * n * hi * 4 / (ms * 1e-3) / 1e9}), flush=True)
    return 0


def batched_inputs(count: int, seed: int = 0):
    """The batched workload: `count` random-Tucker order-3 tensors (synth recipe)."""
    import synth
    shapes = synth.batched_shapes(count=count, seed=seed)
    return shapes, [synth.batched_tensor(shapes, t, seed=seed) for t in range(count)]


def run_batched(args, count: int = 4096, serial_sample: int = 256):
    """Time the batched form: one tuned, graph-replayed persistent launch over
    `count` small tensors, against the single-tensor plan path called one
    tensor at a time (plans created beforehand) on the first `serial_sample`
    tensors, scaled to the whole batch.  Returns a dict for the JSON line."""
    import torch
    import paper_2010_10131_b300 as atk
    t0 = time.time()
    shapes, xs_np = batched_inputs(count)
    gen_s = time.time() - t0
    in_bytes = sum(x.nbytes for x in xs_np)
    xs = [torch.from_numpy(x).cuda() for x in xs_np]
    b = atk.Batch([s[0] for s in shapes], [s[1] for s in shapes])
    cores, facs = b.outputs()
    tune_ms = b.tune(xs, cores, facs, reps=2)
    variant = b.variant
    for _ in range(max(args.warmup, 1)):
        b.run(xs, cores, facs, sync=False)
    b.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(args.steps, 1)
    e0.record()
    for _ in range(steps):
        b.run(xs, cores, facs, sync=False)
    e1.record()
    b.sync()
    ms = e0.elapsed_time(e1) / steps
    b.close()
    # One at a time: the regular plan per tensor, created outside the timed region.
    k = min(serial_sample, count)
    plans = [atk.Plan(shapes[t][0], shapes[t][1], solver=[0, 0, 0]) for t in range(k)]
    outs = [(torch.empty(int(np.prod(shapes[t][1])), device="cuda"),
             torch.empty(sum(d * r for d, r in zip(*shapes[t])), device="cuda")) for t in range(k)]
    for t in range(k):
        plans[t].run(xs[t], outs[t][0], outs[t][1])
    torch.cuda.synchronize()
    e0.record()
    for t in range(k):
        plans[t].run(xs[t], outs[t][0], outs[t][1])
    e1.record()
    torch.cuda.synchronize()
    serial_ms = e0.elapsed_time(e1) * count / k
    for pl in plans:
        pl.close()
    return {
        "workload": f"{count} order-3 tensors, dims uniform in [16, 96], ranks uniform in [4, 16] "
                    "(feasibility-clamped), random Tucker + 1e-3 noise, EIG every mode",
        "input_bytes": in_bytes, "ms": ms, "gbs": in_bytes / (ms * 1e-3) / 1e9,
        "tensors_per_s": count / (ms * 1e-3), "variant": variant,
        "variants": [{"threads": th, "chunk": kc, "ms": m} for (th, kc), m in zip(atk.Batch.variants(), tune_ms)],
        "one_at_a_time_ms": serial_ms, "one_at_a_time_sample": f"first {k} of {count} tensors, scaled",
        "speedup_vs_one_at_a_time": serial_ms / ms, "graph": True, "generate_s": gen_s,
    }


PRECISION_SWEEP = [((768, 768, 768), 32), ((768, 768, 768), 64), ((768, 768, 768), 128), ((48, 48, 48, 48, 48), 8)]


def decaying_tucker_gpu(dims, r_max: int, seed: int = 0, noise: float = 1e-3):
    """The decaying-spectrum recipe of synth.decaying_tucker built on the GPU
    with torch (the full-size inputs are too large to build on the host):
    core Z x_1 D ... x_N D, Z ~ N(0,1) of size (2 r_max)^N, D = diag(k^-1.5),
    orthonormal factors, signal RMS 1, plus noise N(0,1).  Column-major flat."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(seed)
    N = len(dims)
    kk = [min(2 * r_max, d) for d in dims]
    z = torch.randn(*reversed(kk), device="cuda", generator=g)
    for n in range(N):
        dvec = torch.arange(1, kk[n] + 1, device="cuda", dtype=torch.float32) ** -1.5
        shape = [1] * N
        shape[N - 1 - n] = kk[n]
        z = z * dvec.view(shape)
    for n in range(N):
        u, _ = torch.linalg.qr(torch.randn(dims[n], kk[n], device="cuda", generator=g))
        ax = N - 1 - n
        z = torch.movedim(torch.tensordot(u, z, dims=([1], [ax])), 0, ax)
    z = z * (1.0 / torch.sqrt(torch.mean(z.double() ** 2))).float()
    z = z + noise * torch.randn(z.shape, device="cuda", generator=g)
    return z.contiguous().view(-1)


def run_precision(args):
    """The precision sweep: every form (Gram and TTM) on 768^3 (R 32, 64, 128)
    and 48^5 (R 8), decaying spectrum; time per st-HOSVD (CUDA events) and
    relative error by reconstruction, beside the float32 plan's."""
    import torch
    import paper_2010_10131_b300 as atk
    forms = (("FP32", atk.FP32), ("TF32", atk.TF32), ("BF16", atk.BF16), ("BF16X3", atk.BF16X3),
             ("FP8E4M3", atk.FP8E4M3))
    out = []
    for dims, R in PRECISION_SWEEP:
        x = decaying_tucker_gpu(dims, R)
        ranks = [R] * len(dims)
        row = {"dims": list(dims), "ranks": ranks, "forms": {}}
        for name, prec in forms:
            p = atk.Plan(dims, ranks, solver=[atk.EIG] * len(dims), precision=prec)
            core = torch.empty(p.core_numel, device="cuda")
            fac = torch.empty(p.factors_numel, device="cuda")
            for _ in range(max(args.warmup, 1)):
                p.run(x, core, fac)
            p.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(max(args.steps, 1)):
                p.run(x, core, fac)
            e1.record()
            p.sync()
            ms = e0.elapsed_time(e1) / max(args.steps, 1)
            facs = [f.view(r, d).t() for f, d, r in zip(torch.split(fac, [d * r for d, r in zip(dims, ranks)]),
                                                        dims, ranks)]
            rel = reconstruct_relerr(x, core, facs, list(dims), ranks)
            row["forms"][name] = {"ms": ms, "gbs": x.numel() * 4 / (ms * 1e-3) / 1e9, "relerr": rel}
            p.close()
        base = row["forms"]["FP32"]
        for v in row["forms"].values():
            v["relerr_delta_vs_fp32"] = v["relerr"] - base["relerr"]
            v["speedup_vs_fp32"] = base["ms"] / v["ms"]
        out.append(row)
        del x
        torch.cuda.empty_cache()
    return out


def run_roofline_small(args):
    """HBM roofline of the memory-bound contractions: the mode-1 Gram and the
    R = 8 TTM of the 48^5 tensor (view 1 x 48 x 48^4), float32, through the C
    ABI, device time by CUDA events.  Algorithmic bytes: the input read once
    (Gram); input read once plus the output written (TTM)."""
    import torch
    import paper_2010_10131_b300 as atk
    lo, n, hi, R = 1, 48, 48 ** 4, 8
    g = torch.Generator(device="cuda").manual_seed(0)
    y = torch.randn(lo * n * hi, device="cuda", generator=g)
    U = torch.linalg.qr(torch.randn(n, R, device="cuda", generator=g))[0]
    hbm = peaks().get("hbm_gbs") or 6400.0
    out = {"view": [lo, n, hi], "hbm_peak_gbs": hbm}
    for name, fn, nbytes in (("gram", lambda: atk.gram(y, lo, n, hi), 4.0 * y.numel()),
                             ("ttm", lambda: atk.ttm(y, lo, n, hi, U), 4.0 * y.numel() * (1 + R / n))):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 10
        gbs = nbytes / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "algorithmic_bytes": nbytes, "gbs": gbs, "frac_of_measured_hbm": gbs / hbm}
    return out


def run_selector_summary(args, e2e_shapes: int = 24):
    """The learned selector as installed (weights trained by the library's
    kernels on the committed timing sets) against the paper's decision tree
    trained on the same timings: held-out regret and host inference time, then
    end to end on held-out shapes, every mode AUTO against every mode EIG."""
    import torch
    import paper_2010_10131_b300 as atk
    from paper_2010_10131_b300 import selector
    out = selector.compare_tree_mlp()
    shapes, _ = selector.load_timings(selector.TIMINGS)
    held = shapes[192:192 + e2e_shapes]
    tot = {"AUTO": 0.0, "EIG": 0.0}
    for i, (dims, ranks) in enumerate(held):
        x = selector.random_tucker_gpu(dims, ranks, 900001 + i)
        for name, sv in (("AUTO", atk.AUTO), ("EIG", atk.EIG)):
            ms, _, _, _, _ = time_plan(x, dims, ranks, 2, 1, solver=[sv] * len(dims))
            tot[name] += ms
        del x
        torch.cuda.empty_cache()
    out["end_to_end"] = {"shapes": len(held), "auto_ms": tot["AUTO"], "eig_ms": tot["EIG"],
                         "gain_vs_fixed_EIG": tot["EIG"] / tot["AUTO"]}
    return out


def run_selector(args, e2e_shapes: int = 64):
    """The learned selector: train on the committed timing sets with the
    library's kernels, regret on the 64 held-out shapes against exhaustive
    search, then end to end on the held-out shapes: plans with every mode AUTO
    (the selector) against every mode EIG (the method without it), timed with
    CUDA events."""
    import torch
    import paper_2010_10131_b300 as atk
    from paper_2010_10131_b300 import selector
    t0 = time.time()
    report, packed = selector.train_and_evaluate()
    train_s = time.time() - t0
    selector.install(packed)
    shapes, _ = selector.load_timings(selector.TIMINGS)
    held = shapes[192:192 + e2e_shapes]
    tot = {"AUTO": 0.0, "EIG": 0.0}
    for i, (dims, ranks) in enumerate(held):
        x = selector.random_tucker_gpu(dims, ranks, 900001 + i)
        for name, sv in (("AUTO", atk.AUTO), ("EIG", atk.EIG)):
            p = atk.Plan(dims, ranks, solver=[sv] * len(dims))
            core = torch.empty(p.core_numel, device="cuda")
            fac = torch.empty(p.factors_numel, device="cuda")
            p.run(x, core, fac)
            p.sync()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(2):
                p.run(x, core, fac)
            e1.record()
            p.sync()
            tot[name] += e0.elapsed_time(e1) / 2
            p.close()
        del x
        torch.cuda.empty_cache()
    report["end_to_end"] = {"shapes": len(held), "auto_ms": tot["AUTO"], "eig_ms": tot["EIG"],
                            "gain_vs_fixed_EIG": tot["EIG"] / tot["AUTO"],
                            "inputs": "random Tucker + 1e-3 noise built on the GPU, new seeds"}
    report["train_s"] = train_s
    return report


# Table II of the paper (its six real tensors, not available here) as
# synthetic stand-ins: the same shapes and truncations, random Tucker cores
# with those ranks plus 10 % noise (the real tensors' errors are 0.2 - 0.9).
# MNIST's R_2 = 142 is clamped to the library's rank limit of 128.
TABLE_II = (("MNIST", (784, 5000, 10), (65, 128, 10)),
            ("Cavity", (100, 100, 10000), (20, 20, 20)),
            ("Boats", (320, 240, 7000), (10, 10, 10)),
            ("Air", (30648, 376, 6), (10, 10, 5)),
            ("Video", (112, 160, 3, 32), (10, 10, 3, 32)),
            ("HSI", (1021, 1340, 33, 8), (10, 10, 10, 5)))


def random_tucker_big(dims, ranks, seed, noise):
    """Random Tucker signal scaled to RMS 1 per element plus noise * N(0,1),
    built on the GPU (the stand-ins are too large to build on the host),
    column-major flat.  With 10 % noise the relative errors land where the
    paper's real tensors do (0.1 - 0.4) and the signal stays above the noise."""
    import torch
    from paper_2010_10131_b300 import selector
    x = selector.random_tucker_gpu(dims, ranks, seed, noise=0.0)
    x *= (1.0 / torch.sqrt(torch.mean(x.double() ** 2))).float()
    g = torch.Generator(device="cuda").manual_seed(int(seed) + 1)
    x += noise * torch.randn(x.shape, device="cuda", generator=g)
    return x


def reconstruct_relerr(x, core, facs, dims, ranks):
    """||X - G x_1 U1 ... x_N UN|| / ||X|| on the GPU (float64 sums)."""
    import torch
    N = len(dims)
    g = core.view(*reversed(ranks)).double()
    for n in range(N):
        ax = N - 1 - n
        g = torch.movedim(torch.tensordot(facs[n].double(), g, dims=([1], [ax])), 0, ax)
    xx = x.view(*reversed(dims)).double()
    return float(torch.linalg.norm(xx - g) / torch.linalg.norm(xx))


def time_plan(x, dims, ranks, steps, warmup, **kw):
    """ms per st-HOSVD (CUDA events), device memory the plan took (free memory
    before creation minus after the first run) and the result."""
    import torch
    import paper_2010_10131_b300 as atk
    explicit = kw.pop("explicit", 0)
    fuse = kw.pop("fuse", 0)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    p = atk.Plan(dims, ranks, **kw)
    if explicit:
        p.set_option(atk.OPT_EXPLICIT_UNFOLD, 1)
    if fuse:
        p.set_option(atk.OPT_FUSE_TTM_GRAM, 1)
    core = torch.empty(p.core_numel, device="cuda")
    fac = torch.empty(p.factors_numel, device="cuda")
    for _ in range(max(warmup, 1)):
        p.run(x, core, fac)
    p.sync()
    mem = free0 - torch.cuda.mem_get_info()[0]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(max(steps, 1)):
        p.run(x, core, fac)
    e1.record()
    p.sync()
    ms = e0.elapsed_time(e1) / max(steps, 1)
    facs = [f.view(r, d).t() for f, d, r in zip(torch.split(fac, [d * r for d, r in zip(dims, ranks)]), dims, ranks)]
    classes = p.classes
    p.close()
    return ms, mem, core, facs, classes


def run_table2(args):
    """The Table II stand-ins with EIG in every mode, ALS in every mode and
    the learned selector (AUTO): time, device memory and relative error."""
    import torch
    import paper_2010_10131_b300 as atk
    from paper_2010_10131_b300 import selector
    selector.install()
    out = []
    for i, (name, dims, ranks) in enumerate(TABLE_II):
        x = random_tucker_big(dims, ranks, 7000 + i, noise=0.1)
        row = {"name": name, "dims": list(dims), "ranks": list(ranks), "solvers": {}}
        for sname, sv in (("EIG", atk.EIG), ("ALS", atk.ALS), ("AUTO", atk.AUTO)):
            try:
                ms, mem, core, facs, cls = time_plan(x, list(dims), list(ranks), args.steps, args.warmup,
                                                     solver=[sv] * len(dims))
                row["solvers"][sname] = {"ms": ms, "gbs": x.numel() * 4 / (ms * 1e-3) / 1e9,
                                         "plan_mem_gb": mem / 1e9,
                                         "relerr": reconstruct_relerr(x, core, facs, dims, ranks)}
                if sv == atk.AUTO:
                    row["solvers"][sname]["classes"] = [atk.CLASS_NAMES[c] for c in cls]
            except Exception as e:  # a solver that cannot run this shape
                row["solvers"][sname] = {"error": str(e)[:160]}
            torch.cuda.empty_cache()
        out.append(row)
        del x
        torch.cuda.empty_cache()
    return out


def run_explicit(args):
    """Ablation of the matricization-free design (Sec. VI-E): the same plans
    with every mode with I_<n > 1 explicitly unfolded into a buffer and the
    result folded back (ATK_OPT_EXPLICIT_UNFOLD), EIG every mode; time and the
    device memory each plan took."""
    import torch
    import paper_2010_10131_b300 as atk
    shapes = [("640^3 R64", (640, 640, 640), (64, 64, 64)), ("128^4 R16", (128, 128, 128, 128), (16, 16, 16, 16))]
    shapes += [(n, d, r) for n, d, r in TABLE_II if n in ("Cavity", "Boats", "Video", "HSI")]
    out = []
    for i, (name, dims, ranks) in enumerate(shapes):
        x = random_tucker_big(dims, ranks, 8000 + i, noise=0.1)
        row = {"name": name, "dims": list(dims), "ranks": list(ranks)}
        for label, ex in (("free", 0), ("explicit", 1)):
            ms, mem, core, facs, _ = time_plan(x, list(dims), list(ranks), args.steps, args.warmup,
                                               solver=[atk.EIG] * len(dims), explicit=ex)
            row[label] = {"ms": ms, "plan_mem_gb": mem / 1e9, "relerr": reconstruct_relerr(x, core, facs, dims, ranks)}
            torch.cuda.empty_cache()
        row["speedup_free_vs_explicit"] = row["explicit"]["ms"] / row["free"]["ms"]
        row["memory_saved"] = 1.0 - row["free"]["plan_mem_gb"] / max(row["explicit"]["plan_mem_gb"], 1e-12)
        out.append(row)
        del x
        torch.cuda.empty_cache()
    return out


def run_fused(args):
    """The fused TTM + next-mode Gram (ATK_OPT_FUSE_TTM_GRAM) against the
    separate kernels, EIG every mode, float32: whole st-HOSVD time of plans
    that differ only in that option."""
    import torch
    import paper_2010_10131_b300 as atk
    shapes = [("48^5 R8", (48,) * 5, (8,) * 5), ("128^4 R16", (128,) * 4, (16,) * 4),
              ("96^3 R8", (96,) * 3, (8,) * 3), ("384x96^3 R(32,16,16,16)", (384, 96, 96, 96), (32, 16, 16, 16))]
    out = []
    for i, (name, dims, ranks) in enumerate(shapes):
        x = random_tucker_big(dims, ranks, 9000 + i, noise=0.1)
        row = {"name": name, "dims": list(dims), "ranks": list(ranks)}
        for label, fz in (("separate", 0), ("fused", 1)):
            ms, mem, core, facs, _ = time_plan(x, list(dims), list(ranks), args.steps, args.warmup,
                                               solver=[atk.EIG] * len(dims), fuse=fz)
            row[label] = {"ms": ms, "relerr": reconstruct_relerr(x, core, facs, dims, ranks)}
        row["speedup_fused"] = row["separate"]["ms"] / row["fused"]["ms"]
        out.append(row)
        del x
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--case", default=None, help="profile one op: gram:LO,N,HI, ttm:LO,N,HI,R, als:LO,N,HI,R, "
                    "ttmgram:LO,N,HI,R,S,I_M, eig:N,R[,METHOD] or batched[:COUNT]")
    ap.add_argument("--precision", type=int, default=0,
                    help="0 FP32, 1 TF32, 2 BF16, 3 3xBF16, 4 FP8-e4m3, 5 FP32 compensated (--case)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision comparison")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other workloads (precision sweep, batched, selector, Table II, ablation)")
    args = ap.parse_args()
    if args.case:
        return run_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
