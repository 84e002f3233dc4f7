#!/usr/bin/env python
"""Benchmark of the GB300 trans_ev_tridi_to_band (back-transformation of
eigenvectors from tridiagonal to band form, Kus et al. Sec. 2 / Sec. 3.1).

One step = one call of gb_trans_ev_tridi_to_band_d on the whole workload:
n = 16384, nev = 4096 eigenvectors (25%), band width nbw = 64, FP64 real,
reflectors in the bulge-chase layout (seeded synthetic, see
paper_1811_01277_gb300/inputs.py) and a seeded Z.  Inputs (Z 0.54 GB,
reflectors 1.07 GB) are larger than the 129 MB L2, so no flush is needed.

Prints ONE JSON line (rank 0).  Under torchrun every rank runs its own
independent problem (weak scaling) and the time is the max over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

# Solves overlapping on many streams (batched and serve stages) need as many
# hardware work queues; the CUDA driver reads this before the context exists.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "n16384": dict(n=16384, nev=4096, nbw=64),
    "n6144": dict(n=6144, nev=2048, nbw=64),   # small case for ncu captures
    "n1024": dict(n=1024, nev=1024, nbw=32),
}
# FP64 DFMA: 2 lanes per clock per SM on GB300 (1.25 TFLOP/s nominal at the
# 2070 MHz maximum SM clock over 152 SMs: 152 * 2 * 2 flop * 2.07e9).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# measured constants of this part (one GB300, SM clock 2070 MHz throughout;
# profiles/fp64_peak_and_variant_sweep.md): the DFMA pipe and the legacy
# warp-level bf16 mma.sync m16n8k16 path
FP64_DFMA_MEASURED_TFLOPS = 1.256
MMA_SYNC_BF16_TFLOPS = 606.0


def measured_peaks():
    """The measured copy bandwidth and cuBLAS bf16 rates (MEASURED_PEAKS.json),
    or fallback figures from an earlier GB300 measurement when the file is absent."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained"), "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def tc_executed_flops(n, nbw, nev):
    """bf16 tensor-core flops one pipeline_tc call executes: per tile (16
    sweeps) and 64-column item, W = V^T Z (16 x LP x 64) and dZ = U W
    (LP x 16 x 64), each over the 53 digit-plane pairs (i + j <= 9 of nine
    digits per operand), LP = nbw + 15 rounded up to 16."""
    lp = (nbw + 15 + 15) // 16 * 16
    G = (n - 1 + 15) // 16
    tiles = sum((n - (1 + 16 * g) + nbw - 1) // nbw for g in range(G))
    items = tiles * ((nev + 63) // 64)
    pairs = sum(min(9, 10 - i) for i in range(9))     # 53
    return items * pairs * 2 * (2 * 16 * lp * 64)


def tc5_executed_flops_z(n, nbw, nev):
    """pipeline_tc5 on complex data (the real 2 x 2-block form): per tile of
    8 sweeps and 128-column item, W'^T (128 x LP x 16) and dZ'^T
    (128 x 16 x LP) over 43 digit pairs, LP = 2 (nbw + 7) rounded up to 16."""
    lp = (2 * (nbw + 7) + 15) // 16 * 16
    G = (n - 1 + 7) // 8
    tiles = sum((n - (1 + 8 * g) + nbw - 1) // nbw for g in range(G))
    items = tiles * ((nev + 127) // 128)
    return items * 43 * 2 * (2 * 128 * 16 * lp)


def tc5_executed_flops(n, nbw, nev):
    """FP16 tensor-core flops one pipeline_tc5 call executes: per tile (NB
    sweeps: 32 for nbw = 64, else 16) and 128-column item, W^T = Z^T V
    (128 x LP x NB) and dZ^T = W^T U^T (128 x NB x LP), each over the 43
    digit-plane pairs (s + t <= 8 of eight digits per operand),
    LP = nbw + NB - 1 rounded up to 16."""
    nb = 32 if nbw == 64 else 16
    lp = (nbw + nb - 1 + 15) // 16 * 16
    G = (n - 1 + nb - 1) // nb
    tiles = sum((n - (1 + nb * g) + nbw - 1) // nbw for g in range(G))
    items = tiles * ((nev + 127) // 128)
    pairs = sum(1 for s_ in range(8) for t_ in range(8) if s_ + t_ <= 8)     # 43
    return items * pairs * 2 * (2 * 128 * nb * lp)


def algorithmic_flops(n, nev, cplx=False):
    """4 flops per reflector element and column (16 for complex); the
    reflectors of a sweep s cover n-s rows, so sum len = n(n-1)/2."""
    return (16 if cplx else 4) * nev * n * (n - 1) // 2


KERNEL_SOURCES = {
    "pipeline_d": ["trans_ev_pipeline.cu", "tile_apply.cuh", "layout.cuh"],
    "wavefront_tile_d": ["trans_ev_wavefront.cu", "tile_apply.cuh", "layout.cuh"],
    "pipeline_tc": ["trans_ev_tc.cu", "mma_bf16.cuh", "layout.cuh"],
    "pipeline_tc5": ["trans_ev_tc5.cu", "tcgen05.cuh", "tc_fixed.cuh", "mma_bf16.cuh", "layout.cuh"],
}


def kernel_sources_sha1(kernel):
    """Hash of the source files a kernel is compiled from (traffic figures in
    profiles/ are only reported while this matches)."""
    h = hashlib.sha1()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1811_01277_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def profile_traffic(kernel, workload, variant, sha):
    """DRAM bytes per step from a committed ncu summary, if it was taken on
    the current kernel sources; None otherwise."""
    for p in glob.glob(os.path.join(ROOT, "profiles", "*.md")) + glob.glob(os.path.join(ROOT, "profiles", "*.txt")):
        with open(p) as f:
            for line in f:
                if line.startswith("traffic:") and f"kernel={kernel}" in line and \
                        f"workload={workload}" in line and f"variant={variant}" in line:
                    kv = dict(x.split("=", 1) for x in line.split()[1:] if "=" in x)
                    if kv.get("sha1") == sha:
                        return float(kv["bytes_per_step"])
    return None


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(world, steps, max_elapsed_s):
    """Whole-job throughput: every rank ran `steps` back-transforms of its own
    problem; the job took the slowest rank's time."""
    return world * steps / max_elapsed_s


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def cpu_baseline(n, nev, nbw, hv, ht, Z, target_s=12.0):
    """The oracle as it stands, on a bounded sample of the workload's columns
    (columns are independent, so time scales linearly with the count)."""
    import numpy as np
    import oracle
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    cols = cores
    t0 = time.perf_counter()
    oracle.trans_ev(n, nbw, hv, ht, np.asfortranarray(Z[:, :cols]))
    t1 = time.perf_counter() - t0
    reps = max(1, int(target_s / max(t1, 1e-3)))
    cols2 = min(nev, cols * reps)
    t0 = time.perf_counter()
    oracle.trans_ev(n, nbw, hv, ht, np.asfortranarray(Z[:, :cols2]))
    t2 = time.perf_counter() - t0
    return {"value": (cols2 / nev) / t2, "unit": "back-transforms/s", "cores": cores, "kind": "oracle",
            "sample": f"{cols2} of {nev} columns (n={n}, nbw={nbw}), {t2:.1f} s; "
                      f"value scaled to the full nev (columns are independent)"}


def run_reference(args, wl):
    """The oracle (plain C, OpenMP over columns) on this host's cores."""
    import numpy as np
    from paper_1811_01277_gb300 import inputs
    import oracle
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    n, nev, nbw = wl["n"], wl["nev"], wl["nbw"]
    hv, ht = inputs.synthetic_reflectors(n, nbw, seed=2024)
    Z = inputs.z_gaussian(n, nev, seed=2025)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    cols = min(nev, cores)
    Zs = np.asfortranarray(Z[:, :cols])
    for _ in range(args.warmup):
        oracle.trans_ev(n, nbw, hv, ht, Zs)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.trans_ev(n, nbw, hv, ht, Zs)
    el = time.perf_counter() - t0
    value = args.steps * (cols / nev) / el
    sample = f"each step {cols} of {nev} columns (n={n}, nbw={nbw}); value scaled to the full nev"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "back-transforms/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * el / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(wl), "variant": "oracle",
        "cpu_baseline": {"value": value, "unit": "back-transforms/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "back-transforms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


METRIC = ("solve s at n=16384 (25% vecs); trans_ev % of FP64 peak; batched solves/s, p99 -- value: "
          "trans_ev_tridi_to_band back-transforms/s at n=16384, nev=4096, nbw=64 (FP64 accuracy); "
          "keys solve (full two-stage solve at that size) and batched (512 problems) carry the rest")


def config_of(wl, shards=1):
    n, nev, nbw = wl["n"], wl["nev"], wl["nbw"]
    count = sum((n - s + nbw - 1) // nbw for s in range(1, n))
    c = {"workload": f"trans_ev_tridi_to_band n={n} nev={nev} nbw={nbw} real FP64",
         "n": n, "nev": nev, "nbw": nbw,
         "l2": "inputs larger than L2 (Z %.2f GB, reflectors %.2f GB); no flush" % (
             8 * n * nev / 1e9, 8 * nbw * count / 1e9)}
    c["parallelism"] = (f"one problem, columns sharded over {shards} GPUs (reflectors replicated, no exchange "
                        f"during the step)") if shards > 1 else "one independent problem per GPU"
    return c


def run_ours(args, wl):
    import numpy as np
    import torch
    import paper_1811_01277_gb300 as gb
    from paper_1811_01277_gb300 import build as gbuild
    from paper_1811_01277_gb300 import inputs

    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    gbuild.build()
    gb.load()
    n, nev, nbw = wl["n"], wl["nev"], wl["nbw"]
    opts = {"variant": args.variant, "sweeps_per_tile": args.nb, "cols_per_block": args.threads,
            "column_batch": args.column_batch, "lead_tiles": args.lead_tiles}
    if args.variant == 0 and args.nb == 0 and args.threads == 0 and args.column_batch == 0 and args.lead_tiles == 0:
        opts = None  # the library's default choice

    shard = args.shard and world > 1
    if shard:
        # one problem for the whole job: every rank builds the same reflectors
        # (the replicated set; sharded.broadcast_reflectors would send them
        # from one rank instead) and back-transforms its own column block
        from paper_1811_01277_gb300.sharded import column_shard
        hv, ht = inputs.synthetic_reflectors(n, nbw, seed=2024)
        c0, nev_loc = column_shard(nev, world, rank)
        Z = np.asfortranarray(inputs.z_gaussian(n, nev, seed=2025)[:, c0:c0 + nev_loc])
        nev_job, nev = nev, nev_loc
    else:
        hv, ht = inputs.synthetic_reflectors(n, nbw, seed=2024 + 1000 * rank)
        Z = inputs.z_gaussian(n, nev, seed=2025 + 1000 * rank)
    hv_d = torch.from_numpy(hv).to(dev)
    ht_d = torch.from_numpy(ht).to(dev)
    Z_d = torch.from_numpy(np.ascontiguousarray(Z.T)).to(dev)  # (nev, n) row-major = column-major Z
    tuned = None
    if args.autotune:
        # the paper's on-the-fly autotuning: one back-transformation per setting
        level = gb.GB_AUTOTUNE_MEDIUM if args.autotune == "medium" else gb.GB_AUTOTUNE_FAST
        t = gb.gb_autotune_create(level, n, nbw, nev)
        st0 = torch.cuda.current_stream(dev)
        trials = []
        while True:
            o = gb.gb_autotune_step(t)
            if o is None:
                break
            wsb0 = gb.gb_trans_ev_workspace_bytes(n, nbw, nev, 0, o)
            ws0 = torch.zeros(max(wsb0, 256), dtype=torch.uint8, device=dev)
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(st0)
            gb.gb_trans_ev_tridi_to_band_d(n, nbw, nev, hv_d, ht_d, Z_d, n, ws0, wsb0, st0, o)
            a1.record(st0)
            torch.cuda.synchronize(dev)
            sec = a0.elapsed_time(a1) / 1e3
            gb.gb_autotune_report(t, sec)
            trials.append({"variant": o.variant, "nb": o.sweeps_per_tile, "cols": o.cols_per_block,
                           "column_batch": o.column_batch, "s": sec})
        best, _ = gb.gb_autotune_best(t)
        gb.gb_autotune_destroy(t)
        opts = {"variant": best.variant, "sweeps_per_tile": best.sweeps_per_tile,
                "cols_per_block": best.cols_per_block, "column_batch": best.column_batch}
        tuned = {"level": args.autotune, "chosen": opts, "trials": trials}
    launches_per_call = gb.gb_trans_ev_launch_count(n, nbw, nev, 0, opts)
    # the tensor-core pipelines are six launches (scales, to fixed point, tile
    # offsets, tile prep, pipeline, back); the DFMA pipeline one
    variant_name = {gb.GB_VARIANT_PIPELINE_TC5: "pipeline_tc5", gb.GB_VARIANT_PIPELINE_TC: "pipeline_tc",
                    gb.GB_VARIANT_PIPELINE: "pipeline"}.get(gb.gb_trans_ev_variant(n, nbw, nev, 0, opts), "wavefront")
    wsb = gb.gb_trans_ev_workspace_bytes(n, nbw, nev, 0, opts)
    ws = torch.zeros(max(wsb, 256), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    # the dominant kernel's own launch time, live: the library records a pair
    # of caller events around that launch on the call's stream (the events
    # exist once recorded, so each is recorded once beforehand)
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in kev:
        a.record(stream)
        b.record(stream)
    kopts = [dict(opts or {}, kernel_begin_event=a.cuda_event, kernel_end_event=b.cuda_event) for a, b in kev]

    def step(i=None):
        gb.gb_trans_ev_tridi_to_band_d(n, nbw, nev, hv_d, ht_d, Z_d, n, ws, wsb, stream,
                                       opts if i is None else kopts[i])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    smi_index = vis.split(",")[local] if vis else str(local)
    sampler = ClockSampler(smi_index) if rank == 0 else None
    barrier(world)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        step(i)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    el_ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    kernel_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in kev) / args.steps, world, dev)
    clocks = sampler.stop() if sampler else None
    ms_per_step = el_ms / args.steps
    # replicas: every rank finished its own problem per step; shard: the
    # ranks together finished one problem per step
    value = args.steps / (el_ms / 1e3) if shard else aggregate(world, args.steps, el_ms / 1e3)
    F = algorithmic_flops(n, nev)
    achieved = F / (ms_per_step / 1e3) / 1e12
    launches = launches_per_call
    kernel = {"pipeline": "pipeline_d", "pipeline_tc": "pipeline_tc",
              "pipeline_tc5": "pipeline_tc5"}.get(variant_name, "wavefront_tile_d")
    sha = kernel_sources_sha1(kernel)
    # the committed ncu figure is for the default configuration only
    traffic = profile_traffic(kernel, args.workload, variant_name, sha) if opts is None else None

    # end to end through the host-buffer entry point: H2D of reflectors and Z,
    # the kernels, D2H of Z, per step
    e2e = None
    if not args.no_e2e:
        hv_h = torch.from_numpy(hv).pin_memory()
        ht_h = torch.from_numpy(ht).pin_memory()
        Z_h = torch.from_numpy(np.ascontiguousarray(Z.T)).pin_memory()
        bufb = gb.gb_trans_ev_host_buffer_bytes(n, nbw, nev, n, 0, opts)
        buf = torch.empty(bufb, dtype=torch.uint8, device=dev)

        def hstep():
            gb.gb_trans_ev_tridi_to_band_d_host(n, nbw, nev, hv_h, ht_h, Z_h, n, buf, bufb, stream, opts)

        for _ in range(max(1, min(args.warmup, 2))):
            hstep()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            hstep()
        el = max_over_ranks(time.perf_counter() - t0, world, dev)
        h2d = hv.nbytes + ht.nbytes + Z.nbytes
        e2e = {"value": args.steps / el if shard else aggregate(world, args.steps, el), "unit": "back-transforms/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(Z.nbytes),
               "api": "gb_trans_ev_tridi_to_band_d_host (pinned host buffers)"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(n, nev, nbw, hv, ht, Z)

    # roofline of the dominant kernel: its executed work per launch over its
    # own average launch time (CUDA events recorded by the library around the
    # launch, on the call's stream); the whole call's FP64-equivalent rate of
    # the algorithmic work beside it
    step_fp64 = {"achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                 "frac": achieved / FP64_PEAK_TFLOPS, "algorithmic_tflop_per_step": F / 1e12,
                 "per": "step (the whole call: scales, tile preparation, pipeline, conversions)"}
    if variant_name == "pipeline_tc5":
        # tcgen05 MMAs on FP16 digit planes (same dense rate as bf16): executed
        # tensor flops against the measured bf16 peak (cuBLAS, tcgen05 path).
        # The kernel is timed alone (the step is this one call, and it runs at
        # the maximum clock), so the burst figure is the denominator; the
        # sustained one (cuBLAS under the power cap) beside it
        pk = measured_peaks()
        Ft = tc5_executed_flops(n, nbw, nev)
        tc_ach = Ft / (kernel_ms / 1e3) / 1e12
        peak = pk["bf16_tflops"]
        roof = {"bound": "tensor", "achieved": tc_ach, "peak": peak, "unit": "TFLOP/s",
                "frac": tc_ach / peak, "traffic": traffic,
                "peak_source": f"MEASURED_PEAKS.json bf16_tflops, burst ({pk['source']}; cuBLAS bf16 on the "
                               f"tcgen05 path, FP16 runs at the same dense rate)",
                "frac_of_sustained_peak": tc_ach / (pk["bf16_tflops_sustained"] or pk["bf16_tflops"]),
                "kernel": kernel, "per": "launch", "kernel_ms_per_launch": kernel_ms,
                "executed_fp16_tflop_per_launch": Ft / 1e12, "fp64_equivalent": step_fp64}
    elif variant_name == "pipeline_tc":
        # legacy bf16 mma.sync: executed tensor flops against the measured
        # bf16 peak
        pk = measured_peaks()
        Ft = tc_executed_flops(n, nbw, nev)
        tc_ach = Ft / (kernel_ms / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": tc_ach, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                "frac": tc_ach / pk["bf16_tflops"], "traffic": traffic,
                "peak_source": f"MEASURED_PEAKS.json bf16_tflops ({pk['source']}, cuBLAS on the tcgen05 path); "
                               f"this kernel issues legacy bf16 mma.sync, measured at {MMA_SYNC_BF16_TFLOPS} TFLOP/s",
                "frac_of_mma_sync_peak": tc_ach / MMA_SYNC_BF16_TFLOPS,
                "kernel": kernel, "per": "launch", "kernel_ms_per_launch": kernel_ms,
                "executed_bf16_tflop_per_launch": Ft / 1e12, "fp64_equivalent": step_fp64}
    else:
        k_ach = F / (kernel_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": k_ach, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": k_ach / FP64_PEAK_TFLOPS, "traffic": traffic,
                "peak_source": "FP64 DFMA: 152 SMs x 2 lanes/clk x 2 flop x 2070 MHz "
                               f"(DFMA microbenchmark {FP64_DFMA_MEASURED_TFLOPS} TFLOP/s)",
                "kernel": kernel, "per": "launch" if variant_name == "pipeline" else "call's launches",
                "kernel_ms_per_launch": kernel_ms, "algorithmic_tflop_per_launch": F / 1e12,
                "fp64_equivalent": step_fp64}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "back-transforms/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "strong" if shard else "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config_of(wl, world if shard else 1), "variant": variant_name,
            "roofline": roof,
            "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": int(launches) * args.steps,
            "clocks": clocks, "kernel_sources_sha1": sha,
        }
        if opts is not None:
            line["opts"] = dict(opts) if isinstance(opts, dict) else {
                f: getattr(opts, f) for f, _ in gb.gb_trans_ev_opts._fields_}
        if tuned:
            line["autotune"] = tuned
        if world == 1 and not args.no_extra:
            # the rest of the metric: the full solve at the same size (one
            # warm-up, one timed solve) and the 512-problem batch (one warm-up
            # batch, one timed batch), after the back-transformation's buffers
            # are released
            del Z_d, hv_d, ht_d, ws
            if e2e is not None:
                del buf, hv_h, ht_h, Z_h
            torch.cuda.empty_cache()
            sv = measure_solve(n, nev, nbw, steps=1, warmup=1, record_stages=False)
            line["solve"] = {"seconds_per_solve": sv["seconds_per_solve"], "n": n, "nev": nev, "nbw": nbw,
                             "status": sv["status"], "accuracy": sv["accuracy"], "roofline": sv["roofline"],
                             "steps": 1, "warmup": 1, "data": sv["data"], "clocks": sv["clocks"]}
            bt = measure_batched(512, 128, 2048, 16, steps=1, warmup=1)
            line["batched"] = {k_: bt[k_] for k_ in ("solves_per_s", "p50_ms", "p99_ms", "seconds_per_batch",
                                                     "streams", "plain_solve_one_at_a_time",
                                                     "accuracy_worst_over_50nu", "data", "clocks", "metric",
                                                     "graph", "graph_tuned_nbw", "staged", "staged_tuned_nbw")}
            line["batched"].update(steps=1, warmup=1, form="streams (gb_solve_batched_d); the graph forms beside it")
        print(json.dumps(line))
    return 0


def chase_flops(n, b):
    """Algorithmic flops of the band -> tridiagonal bulge chase, summed over
    tasks (s,k): left block 4*len*(r-c-1), below block 4*len*rows_below,
    p = tau*A*v 2*len^2, symmetric rank-2 update 2*len*(len+1); the reflector
    itself (O(len)) is not counted."""
    import numpy as np
    total = 0
    for s_ in range(1, n):
        nk = (n - s_ + b - 1) // b
        k = np.arange(nk)
        r = s_ + k * b
        ln = np.minimum(b, n - r)
        c = np.where(k == 0, s_ - 1, s_ + (k - 1) * b)
        below = np.minimum(b, np.maximum(n - r - ln, 0))
        active = ln > 1
        total += int(np.sum(np.where(active, 4 * ln * (r - c - 1) + 4 * ln * below + 2 * ln * ln + 2 * ln * (ln + 1), 0)))
    return total


def run_stage_band_to_tridi(args):
    """Time gb_band_to_tridi_d (device bulge chase) on an n x n band matrix
    with U[-1,1] entries; one JSON line."""
    import numpy as np
    import torch
    import paper_1811_01277_gb300 as gb
    from paper_1811_01277_gb300 import build as gbuild
    from paper_1811_01277_gb300 import inputs
    gbuild.build()
    gb.load()
    n, b = args.chase_n, args.chase_b
    dev = torch.device("cuda", 0)
    g = np.random.default_rng(args.chase_n)
    AB = np.zeros((n, b + 1))                      # row j = column j of the lower band storage
    AB[:, :] = g.uniform(-1.0, 1.0, (n, b + 1))
    for dd in range(b + 1):
        AB[n - dd:, dd] = 0.0
    AB_d = torch.from_numpy(AB).to(dev)
    cnt = gb.gb_hh_count(n, b)
    d = torch.empty(n, dtype=torch.float64, device=dev)
    e = torch.empty(n, dtype=torch.float64, device=dev)
    hv = torch.empty(cnt * b, dtype=torch.float64, device=dev)
    ht = torch.empty(cnt, dtype=torch.float64, device=dev)
    wsb = gb.gb_band_to_tridi_workspace_bytes(n, b)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream(dev)

    def step():
        gb.gb_band_to_tridi_d(n, b, AB_d, b + 1, d, e, hv, ht, ws, wsb, st)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    status = gb.gb_trans_ev_query(ws, wsb, st)
    ms = e0.elapsed_time(e1) / args.steps
    F = chase_flops(n, b)
    ach = F / (ms / 1e3) / 1e12
    print(json.dumps({
        "stage": "band_to_tridi", "metric": f"band->tridiagonal bulge chase, n={n}, nbw={b}",
        "value": 1e3 / ms, "unit": "reductions/s", "ms_per_step": ms, "steps": args.steps,
        "warmup": args.warmup, "status": status, "dtype": "f64", "data": "synthetic U[-1,1] band",
        "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": ach / FP64_PEAK_TFLOPS, "algorithmic_gflop": F / 1e9},
        "gpu_launches": 3 * args.steps, "clocks": clocks}))
    return 0


def solve_flops(n, nev, nbw, cplx=False):
    """Algorithmic flops of the two-stage solve by stage (real flops; a
    complex multiply-add counts 8): full->band (4/3) n^3 (two-sided panel
    reduction), the bulge chase (chase_flops), the back-transformations
    trans_ev (algorithmic_flops) and band->full 2 n^2 nev, and the
    Newton-Schulz step n nev^2 (Z^T Z, one triangle) + 2 n nev^2 (Z M).
    Bisection and inverse iteration are O(n nev) per round and not counted."""
    f = 4 if cplx else 1
    st = {"full_to_band": f * 4 * n ** 3 // 3,
          "band_to_tridi": f * chase_flops(n, nbw),
          "orthogonalise": f * 3 * n * nev * nev,
          "trans_ev_tridi_to_band": algorithmic_flops(n, nev, cplx),
          "band_to_full": f * 2 * n * n * nev}
    return sum(st.values()), st


def prescribed_symmetric_gpu(lam, k, seed, dev, cplx=False):
    """A = Q diag(lam) Q^H on the device, Q = H_1 ... H_k a product of k seeded
    random Householder reflectors (tau = 2/||y||^2), built in O(n^2 k) from the
    compact form Q = I - Y T Y^H (input synthesis; eigenvalues known exactly)."""
    import torch
    n = lam.numel()
    g = torch.Generator(device=dev).manual_seed(seed)
    dt = torch.complex128 if cplx else torch.float64
    Y = torch.randn(n, k, generator=g, device=dev, dtype=torch.float64)
    if cplx:
        Y = torch.complex(Y, torch.randn(n, k, generator=g, device=dev, dtype=torch.float64))
    tau = (2.0 / (Y.abs() ** 2).sum(0)).to(dt)
    G = Y.conj().T @ Y
    T = torch.zeros(k, k, dtype=dt, device=dev)
    for j in range(k):
        if j:
            T[:j, j] = -tau[j] * (T[:j, :j] @ G[:j, j])
        T[j, j] = tau[j]
    U = Y @ T                                   # Q = I - U Y^H
    L = lam.to(dt)
    LY = L[:, None] * Y                         # Lambda Y
    A = torch.diag(L) - U @ LY.conj().T - LY @ U.conj().T + U @ ((Y.conj().T @ LY) @ U.conj().T)
    return 0.5 * (A + A.conj().T)


def measure_solve(n, nev, nbw, cplx=False, spectrum="clustered", steps=1, warmup=1, dfma_products=False,
                  emulated_gemm=False, record_stages=True):
    """Time gb_solve_d / gb_solve_z (the full two-stage solve) on A = Q L Q^T
    with a prescribed spectrum L, and check the eigenvalues against L and the
    residual and orthogonality on all nev columns.  Returns a dict."""
    import torch
    import paper_1811_01277_gb300 as gb
    from paper_1811_01277_gb300 import build as gbuild
    from paper_1811_01277_gb300 import inputs
    gbuild.build()
    gb.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    spec = inputs.gapped_uniform_spectrum if spectrum == "uniform-gapped" else inputs.clustered_spectrum
    lam = torch.from_numpy(spec(n, seed=n)).to(dev)
    A = prescribed_symmetric_gpu(lam, 256, seed=n + 1, dev=dev, cplx=cplx)
    Acm = A.T.contiguous() if cplx else A       # column-major storage (A Hermitian: A^T = conj(A))
    ev = torch.zeros(nev, dtype=torch.float64, device=dev)
    Z = torch.zeros((nev, n), dtype=torch.complex128 if cplx else torch.float64, device=dev)
    wsb = (gb.gb_solve_workspace_bytes_z if cplx else gb.gb_solve_workspace_bytes)(n, nev, nbw)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream(dev)

    base_flags = gb.GB_SOLVE_FP64_EMULATED_GEMM if emulated_gemm else 0
    if dfma_products:
        base_flags |= gb.GB_SOLVE_DFMA_PRODUCTS

    def step(flags=0):
        flags |= base_flags
        if cplx:
            gb.gb_solve_z(n, nev, nbw, Acm, n, ev, Z, n, ws, wsb, st, flags & ~gb.GB_SOLVE_RECORD_STAGES)
        else:
            gb.gb_solve_d(n, nev, nbw, Acm, n, ev, Z, n, ws, wsb, st, flags)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(steps):
        step()
    e1.record(st)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    status = (gb.gb_solve_query_z if cplx else gb.gb_solve_query)(ws, n, nev, nbw, st)
    ms = e0.elapsed_time(e1) / steps
    F, Fst = solve_flops(n, nev, nbw, cplx)
    stages = None
    if not cplx and record_stages:
        step(gb.GB_SOLVE_RECORD_STAGES)        # one more solve, outside the timed region
        stages = gb.gb_solve_stage_ms(st)
    # accuracy: eigenvalues against the prescribed ones, residual and
    # orthogonality on all nev columns (GEMMs on the device)
    Zc = Z.T                                   # n x nev view, column-major data
    anorm = lam.abs().max().item()
    dlam = (ev - lam[:nev]).abs().max().item() / anorm
    R = A @ Zc - Zc * ev[None, :].to(Zc.dtype)
    resid = (torch.linalg.norm(R) / torch.linalg.norm(A)).item()
    del R
    orth = (Zc.conj().T @ Zc - torch.eye(nev, dtype=Zc.dtype, device=dev)).abs().max().item()
    u = 2.0 ** -53
    out = {
        "emulated_gemm": bool(emulated_gemm), "products": "dfma" if dfma_products else "sliced",
        "metric": f"two-stage eigensolve s at n={n} ({100 * nev // n}% vecs), nbw={nbw}, "
                  f"{'complex128 Hermitian' if cplx else 'real FP64'}",
        "n": n, "nev": nev, "nbw": nbw,
        "value": 1e3 / ms, "unit": "solves/s", "ms_per_step": ms, "seconds_per_solve": ms / 1e3,
        "steps": steps, "warmup": warmup, "status": status, "dtype": "f64",
        "data": ("synthetic: A = Q diag(uniform [-1,1] spectrum, 10% in clusters with 1e-6 gaps) Q^T"
                 if spectrum == "uniform-gapped" else "synthetic: A = Q diag(clustered spectrum) Q^T")
                + ", Q a product of 256 seeded Householders",
        "stage_ms": stages,
        "roofline": {"bound": "alu", "achieved": F / (ms / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": F / (ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS, "algorithmic_tflop": F / 1e12,
                     "by_stage_tflop": {k_: v_ / 1e12 for k_, v_ in Fst.items()},
                     "note": "algorithmic FP64 flops of the whole solve against the FP64 DFMA peak; "
                             "large products on the bf16 tensor cores by exact digit slicing (FP64 "
                             "accuracy; the DFMA kernels with --dfma-products), the rest in DFMA kernels"},
        "accuracy": {"max_dlambda_over_norm": dlam, "residual_rel_fro": resid, "orth_max": orth,
                     "bound_50nu": 50 * n * u,
                     "within": bool(dlam <= 1e-11 and resid <= 50 * n * u and orth <= 50 * n * u)},
        "clocks": clocks}
    del A, Acm, Z, ws, ev
    torch.cuda.empty_cache()
    return out


def run_stage_solve(args):
    """Time gb_solve_d (full two-stage solve) on A = Q L Q^T with a clustered
    spectrum L; checks the eigenvalues against L and reports one JSON line."""
    import torch
    torch.cuda.set_device(0)
    r = measure_solve(args.solve_n, args.solve_nev, args.solve_nbw, cplx=args.complex, spectrum=args.spectrum,
                      steps=args.steps, warmup=args.warmup, dfma_products=args.dfma_products,
                      emulated_gemm=args.emulated_gemm, record_stages=not args.no_stages)
    r = dict(stage="solve", **r)
    print(json.dumps(r))
    return 0


def run_stage_gemm(args):
    """The solver's FP64 products at the shapes of an n = 16384, nev = 4096,
    nbw = 64 solve: this library's DFMA kernels (gb_dgemm / gb_dsymm /
    gb_dsyr2k / gb_dsyrk), its sliced bf16 tensor-core forms (gb_*_sliced)
    and torch's float64 products on the same device (cuBLAS); one JSON line
    with TFLOP/s (FP64 flops of the product) for each, the fraction of the
    FP64 DFMA peak, and the largest difference of the sliced result from the
    DFMA one relative to the largest entry."""
    import torch
    import paper_1811_01277_gb300 as gb
    from paper_1811_01277_gb300 import build as gbuild
    gbuild.build()
    gb.load()
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream(dev)
    g = torch.Generator(device=dev).manual_seed(77)
    n, nev, b = 16384, 4096, 64
    m = n - b
    A = torch.rand(n, n, generator=g, device=dev, dtype=torch.float64) - 0.5      # column-major view: A.T
    Y = torch.rand(b, m, generator=g, device=dev, dtype=torch.float64) - 0.5      # m x b column-major
    X = torch.rand(b, m, generator=g, device=dev, dtype=torch.float64) - 0.5
    Zt = torch.rand(nev, n, generator=g, device=dev, dtype=torch.float64) - 0.5   # n x nev column-major
    Cb = torch.empty(b, m, device=dev, dtype=torch.float64)
    G = torch.empty(nev, nev, device=dev, dtype=torch.float64)
    Zo = torch.empty(nev, n, device=dev, dtype=torch.float64)
    wsb = gb.gb_dgemm_workspace_bytes(n, b)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    swb = max(gb.gb_dsymm_sliced_workspace_bytes("L", m, b), gb.gb_dsyr2k_sliced_workspace_bytes(m, b),
              gb.gb_dgemm_sliced_workspace_bytes(b, nev, n), gb.gb_dgemm_sliced_workspace_bytes(n, nev, b),
              gb.gb_dsyrk_sliced_workspace_bytes(nev, n), gb.gb_dsymm_sliced_workspace_bytes("R", n, nev))
    sws = torch.empty(swb, dtype=torch.uint8, device=dev)
    G2 = torch.empty(nev, nev, device=dev, dtype=torch.float64)
    Zs = torch.empty(nev, n, device=dev, dtype=torch.float64)
    Asym = A.T                                  # only the lower triangle matters to gb_dsymm
    # (name, flops, DFMA call, sliced call, cuBLAS call, (DFMA output, sliced output) or None)
    cases = [
        ("symm_L m=16320 n=64 (full->band X = A2 YT)", 2.0 * m * m * b,
         lambda: gb.gb_dsymm("L", m, b, 1.0, A, n, Y, m, 0.0, Cb, m, ws, wsb, st),
         lambda: gb.gb_dsymm_sliced("L", m, b, 1.0, A, n, Y, m, 0.0, X, m, sws, swb, st),
         lambda: torch.mm(Asym[:m, :m], Y.T), (Cb, X)),
        ("syr2k m=16320 k=64 (full->band rank-2b update)", 2.0 * m * m * b,
         lambda: gb.gb_dsyr2k(m, b, -1.0, X, m, Y, m, 1.0, A, n, st),
         lambda: gb.gb_dsyr2k_sliced(m, b, -1.0, X, m, Y, m, 1.0, A, n, sws, swb, st),
         lambda: A[:m, :m].addmm_(X.T, Y, alpha=-1.0).addmm_(Y.T, X, alpha=-1.0), None),
        ("gemm TN 64 x 4096 k=16384 (band->full Y^T Z)", 2.0 * b * nev * n,
         lambda: gb.gb_dgemm("T", "N", b, nev, n, 1.0, A, n, Zt, n, 0.0, G, b, ws, wsb, st),
         lambda: gb.gb_dgemm_sliced("T", "N", b, nev, n, 1.0, A, n, Zt, n, 0.0, G2, b, sws, swb, st),
         lambda: torch.mm(A[:b, :], Zt.T), (G.view(-1)[:b * nev], G2.view(-1)[:b * nev])),
        ("gemm NN 16384 x 4096 k=64 (band->full Z -= Y S2)", 2.0 * n * nev * b,
         lambda: gb.gb_dgemm("N", "N", n, nev, b, -1.0, A, n, G, b, 1.0, Zo, n, ws, wsb, st),
         lambda: gb.gb_dgemm_sliced("N", "N", n, nev, b, -1.0, A, n, G, b, 1.0, Zo, n, sws, swb, st),
         lambda: Zo.T.addmm_(A[:b, :].T, G.view(-1)[:b * nev].view(nev, b).T, alpha=-1.0), None),
        ("syrk 4096 k=16384 (Newton-Schulz Z^T Z)", 1.0 * nev * nev * n,
         lambda: gb.gb_dsyrk(nev, n, 1.0, Zt, n, 0.0, G, nev, st),
         lambda: gb.gb_dsyrk_sliced(nev, n, 1.0, Zt, n, 0.0, G2, nev, sws, swb, st),
         # the lower triangle of the column-major result is the upper one of the row-major view
         lambda: torch.mm(Zt, Zt.T, out=G), (lambda: G.triu(), lambda: G2.triu())),
        ("symm_R 16384 x 4096 (Newton-Schulz Z M)", 2.0 * n * nev * nev,
         lambda: gb.gb_dsymm("R", n, nev, 1.0, G2, nev, Zt, n, 0.0, Zo, n, ws, wsb, st),
         lambda: gb.gb_dsymm_sliced("R", n, nev, 1.0, G2, nev, Zt, n, 0.0, Zs, n, sws, swb, st),
         lambda: torch.mm(G2, Zt, out=Zo), (Zo, Zs)),
    ]
    res = {}
    for name, flops, ours, sliced, ref, outs in cases:
        out = {}
        if outs is not None:               # accuracy of the sliced form against the DFMA form
            ours()
            sliced()
            torch.cuda.synchronize(dev)
            d, s_ = (o() if callable(o) else o for o in outs)
            out["sliced_vs_dfma_maxdiff_rel"] = float((s_ - d).abs().max() / d.abs().max().clamp_min(1e-300))
        for label, f in (("dfma", ours), ("sliced", sliced), ("torch_cublas", ref)):
            for _ in range(max(1, args.warmup)):
                f()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            for _ in range(args.steps):
                f()
            e1.record(st)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / args.steps
            out[label] = {"ms": ms, "tflops": flops / (ms / 1e3) / 1e12}
        out["frac_of_fp64_peak"] = out["dfma"]["tflops"] / FP64_PEAK_TFLOPS
        out["sliced_speedup_over_dfma"] = out["dfma"]["ms"] / out["sliced"]["ms"]
        out["cublas_note"] = "torch float64 matmul (cuBLAS DGEMM); syr2k as two full GEMMs, so twice the flops"
        res[name] = out
    print(json.dumps({"stage": "gemm", "metric": "FP64 products of the n=16384 solve, TFLOP/s",
                      "peak_tflops": FP64_PEAK_TFLOPS, "steps": args.steps, "warmup": args.warmup,
                      "dtype": "f64", "data": "synthetic U[-0.5,0.5]", "cases": res}))
    return 0


def measure_batched(count, lo, hi, nstreams, steps=1, warmup=1, plain_every=8):
    """Many independent problems (sizes U[lo, hi], N(0,1) entries symmetrised,
    all eigenpairs) through gb_solve_batched_d on several streams: solves/s
    over the whole batch, p50/p99 of the per-solve times, and the plain
    gb_solve_d one problem at a time on every `plain_every`-th problem for
    comparison.  Returns a dict."""
    import numpy as np
    import torch
    import paper_1811_01277_gb300 as gb
    from paper_1811_01277_gb300 import build as gbuild
    gbuild.build()
    gb.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    g = np.random.default_rng(512)
    sizes = [int(x) for x in g.integers(lo, hi + 1, count)]
    gen = torch.Generator(device=dev).manual_seed(513)
    A = []
    for n in sizes:
        R = torch.randn(n, n, generator=gen, device=dev, dtype=torch.float64)
        A.append(0.5 * (R + R.T))
    ev = [torch.zeros(n, dtype=torch.float64, device=dev) for n in sizes]
    Z = [torch.zeros((n, n), dtype=torch.float64, device=dev) for n in sizes]
    streams = [torch.cuda.Stream(device=dev) for _ in range(nstreams)]
    wsb = gb.gb_solve_batched_workspace_bytes(sizes, sizes, len(streams))
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    es = [torch.cuda.Event(enable_timing=True) for _ in sizes]
    ee = [torch.cuda.Event(enable_timing=True) for _ in sizes]

    def batch(events):
        gb.gb_solve_batched_d(sizes, sizes, A, sizes, ev, Z, sizes, ws, wsb, streams,
                              es if events else None, ee if events else None)

    for _ in range(warmup):
        batch(False)
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    t0 = time.perf_counter()
    for _ in range(steps):
        batch(True)
    issue = time.perf_counter() - t0          # host time to issue the work
    torch.cuda.synchronize(dev)
    el = time.perf_counter() - t0
    clocks = sampler.stop()
    per = np.array([a.elapsed_time(b) for a, b in zip(es, ee)])   # last batch, ms
    # the plain solve on the same problems, one after another on one stream
    # (every plain_every-th problem: the rate, not the whole batch's time, is compared)
    sample = list(range(0, len(sizes), plain_every))
    pst = torch.cuda.Stream(device=dev)
    pmax = max(gb.gb_solve_workspace_bytes(sizes[i], sizes[i], gb.gb_solve_default_nbw(sizes[i])) for i in sample)
    pws = torch.empty(pmax, dtype=torch.uint8, device=dev)

    def plain(i):
        n_, b_ = sizes[i], gb.gb_solve_default_nbw(sizes[i])
        gb.gb_solve_d(n_, n_, b_, A[i], n_, ev[i], Z[i], n_, pws, pmax, pst, 0)

    plain(sample[0])
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    for i in sample:
        plain(i)
    torch.cuda.synchronize(dev)
    plain_rate = len(sample) / (time.perf_counter() - t1)
    # accuracy on a few problems
    worst = 0.0
    for i in range(0, len(sizes), max(1, len(sizes) // 8)):
        n = sizes[i]
        Zi = Z[i].T
        r = torch.linalg.norm(A[i] @ Zi - Zi * ev[i][None, :]) / torch.linalg.norm(A[i])
        o = (Zi.T @ Zi - torch.eye(n, dtype=torch.float64, device=dev)).abs().max()
        worst = max(worst, float(r) / (50 * n * 2.0 ** -53), float(o) / (50 * n * 2.0 ** -53))
    rate = steps * len(sizes) / el

    # the same batch as one CUDA graph (captured once, replayed), first with
    # the default band widths, then with the band widths a size-class tuner
    # picked from one timed solve per (class, nbw) trial
    def graph_form(nbw):
        gwsb = gb.gb_solve_batched_workspace_bytes_nbw(sizes, sizes, nbw, len(streams))
        gws = ws if gwsb <= wsb else torch.empty(gwsb, dtype=torch.uint8, device=dev)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        graph = gb.gb_solve_batched_graph_create(sizes, sizes, nbw, A, sizes, ev, Z, sizes, gws, gwsb,
                                                 len(streams), es, ee)
        create_s = time.perf_counter() - t0
        try:
            gst = torch.cuda.Stream(device=dev)
            for _ in range(warmup):
                gb.gb_solve_batched_graph_launch(graph, gst)
            torch.cuda.synchronize(dev)
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            smp = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
            g0.record(gst)
            for _ in range(steps):
                gb.gb_solve_batched_graph_launch(graph, gst)
            g1.record(gst)
            torch.cuda.synchronize(dev)
            gclk = smp.stop()
            gel = g0.elapsed_time(g1) / 1e3
            gper = np.array([a.elapsed_time(b) for a, b in zip(es, ee)])
            nodes = gb.gb_solve_batched_graph_nodes(graph)
        finally:
            gb.gb_solve_batched_graph_destroy(graph)
        return {"value": steps * len(sizes) / gel, "unit": "solves/s", "seconds_per_batch": gel / steps,
                "p50_ms": float(np.percentile(gper, 50)), "p99_ms": float(np.percentile(gper, 99)),
                "graph_nodes": int(nodes), "branches": len(streams), "capture_and_instantiate_s": create_s,
                "clocks": gclk}

    # stage by stage: every front on the streams, all chases in one launch,
    # every back on the streams (the tuned band widths, once known, below)
    def staged_form(nbw):
        swsb = gb.gb_solve_batched_staged_workspace_bytes(sizes, sizes, nbw, len(streams))
        sws = torch.empty(swsb, dtype=torch.uint8, device=dev)
        for _ in range(warmup):
            gb.gb_solve_batched_staged_d(sizes, sizes, nbw, A, sizes, ev, Z, sizes, sws, swsb, streams)
        torch.cuda.synchronize(dev)
        smp = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
        t0 = time.perf_counter()
        for _ in range(steps):
            gb.gb_solve_batched_staged_d(sizes, sizes, nbw, A, sizes, ev, Z, sizes, sws, swsb, streams, es, ee)
        torch.cuda.synchronize(dev)
        sel = time.perf_counter() - t0
        sclk = smp.stop()
        status = gb.gb_solve_batched_staged_query(sws, sizes, sizes, nbw, streams)
        sper = np.array([a.elapsed_time(b) for a, b in zip(es, ee)])
        del sws
        torch.cuda.empty_cache()
        return {"value": steps * len(sizes) / sel, "unit": "solves/s", "seconds_per_batch": sel / steps,
                "p50_ms": float(np.percentile(sper, 50)), "p99_ms": float(np.percentile(sper, 99)),
                "workspace_gb": swsb / 1e9, "status": status, "clocks": sclk}

    def guarded(f, *a):
        # the extra forms must not take the stream form's line down with them
        try:
            return f(*a)
        except Exception as exc:          # noqa: BLE001 -- reported in the line
            return {"error": f"{type(exc).__name__}: {exc}"}

    staged_default = guarded(staged_form, None)
    graph_default = guarded(graph_form, None)
    # a trial is a mini-batch: one problem of the class's order per stream,
    # all solved at once with the trial's band width (the batch's throughput,
    # not a lone solve's latency, is what the choice has to serve)
    tuner = gb.gb_solve_tuner_create(lo, hi, 4)
    trials = []
    while True:
        tr = gb.gb_solve_tuner_step(tuner)
        if tr is None:
            break
        tn, tb = tr
        k = len(streams)
        At = []
        for _ in range(k):
            R = torch.randn(tn, tn, generator=gen, device=dev, dtype=torch.float64)
            At.append(0.5 * (R + R.T))
        evt = [torch.zeros(tn, dtype=torch.float64, device=dev) for _ in range(k)]
        Zt_ = [torch.zeros((tn, tn), dtype=torch.float64, device=dev) for _ in range(k)]
        tsz, tbw = [tn] * k, [tb] * k
        twsb = gb.gb_solve_batched_workspace_bytes_nbw(tsz, tsz, tbw, k)
        tws = torch.empty(twsb, dtype=torch.uint8, device=dev)
        gb.gb_solve_batched_nbw_d(tsz, tsz, tbw, At, tsz, evt, Zt_, tsz, tws, twsb, streams)   # warm-up
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        gb.gb_solve_batched_nbw_d(tsz, tsz, tbw, At, tsz, evt, Zt_, tsz, tws, twsb, streams)
        torch.cuda.synchronize(dev)
        sec = time.perf_counter() - t0
        gb.gb_solve_tuner_report(tuner, sec)
        trials.append({"n": tn, "nbw": tb, "problems": k, "s": sec})
        del At, evt, Zt_, tws
    tuned_nbw = [gb.gb_solve_tuner_nbw(tuner, n_) for n_ in sizes]
    gb.gb_solve_tuner_destroy(tuner)
    graph_tuned = guarded(graph_form, tuned_nbw)
    staged_tuned = guarded(staged_form, tuned_nbw)
    graph_tuned.setdefault("tuner", {})
    graph_tuned["tuner"] = {"classes": 4, "trials": trials,
                            "chosen": sorted({(n_, b_) for n_, b_ in zip(sizes, tuned_nbw)})[::max(1, count // 16)]}
    out = {
        "metric": f"batched eigensolves/s, {len(sizes)} problems n~U[{lo},{hi}], all eigenpairs",
        "value": rate, "unit": "solves/s", "solves_per_s": rate, "seconds_per_batch": el / steps,
        "host_issue_seconds_per_batch": issue / steps,
        "p50_ms": float(np.percentile(per, 50)), "p99_ms": float(np.percentile(per, 99)),
        "streams": len(streams), "steps": steps, "warmup": warmup, "dtype": "f64",
        "plain_solve_one_at_a_time": {"value": plain_rate, "unit": "solves/s",
                                      "sample": f"every {plain_every}th problem ({len(sample)})",
                                      "speedup_of_batched": rate / plain_rate},
        "data": "synthetic N(0,1) symmetrised", "accuracy_worst_over_50nu": worst, "clocks": clocks,
        "graph": graph_default, "graph_tuned_nbw": graph_tuned, "staged": staged_default,
        "staged_tuned_nbw": staged_tuned}
    del A, Z, ev, ws, pws
    torch.cuda.empty_cache()
    return out


def run_stage_batched(args):
    import torch
    torch.cuda.set_device(0)
    r = measure_batched(args.batch_count, args.batch_lo, args.batch_hi, args.batch_streams, steps=args.steps,
                        warmup=args.warmup)
    print(json.dumps(dict(stage="batched", **r)))
    return 0


def run_stage_refine(args):
    """The mixed-precision configuration's refinement step measured against
    the direct FP64 solve: all eigenpairs of A = Q L Q^T (L uniform in
    [-1, 1] with runs of eigenvalues 1e-6 apart) by gb_solve_d (divide and
    conquer), then the same eigenvectors rounded to FP32 -- the accuracy an
    FP32 solve would deliver -- refined by gb_refine_syev_d (Ogita-Aishima)
    step by step, with orthogonality and residual after each step.  An FP32
    solve plus k steps can only beat the FP64 solve if the FP32 solve takes
    less than the FP64 solve minus k steps."""
    import torch
    import paper_1811_01277_gb300 as gb
    from paper_1811_01277_gb300 import build as gbuild
    from paper_1811_01277_gb300 import inputs
    gbuild.build()
    gb.load()
    n, nbw = args.refine_n, 64
    dev = torch.device("cuda", 0)
    lam0 = torch.from_numpy(inputs.gapped_uniform_spectrum(n, seed=n)).to(dev)
    A = prescribed_symmetric_gpu(lam0, 256, seed=n + 1, dev=dev)
    st = torch.cuda.current_stream(dev)
    ev = torch.zeros(n, dtype=torch.float64, device=dev)
    Z = torch.zeros((n, n), dtype=torch.float64, device=dev)
    wsb = gb.gb_solve_workspace_bytes(n, n, nbw)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    gb.gb_solve_d(n, n, nbw, A, n, ev, Z, n, ws, wsb, st, 0)      # warm-up
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    gb.gb_solve_d(n, n, nbw, A, n, ev, Z, n, ws, wsb, st, 0)
    e1.record(st)
    torch.cuda.synchronize(dev)
    solve_s = e0.elapsed_time(e1) / 1e3
    del ws
    torch.cuda.empty_cache()
    eye = torch.eye(n, dtype=torch.float64, device=dev)
    nrmA = float(torch.linalg.norm(A))

    def accuracy(Xc, lam):       # Xc: column-major storage (rows of the tensor are columns of X)
        X = Xc.T
        return {"orth_max": float((X.T @ X - eye).abs().max()),
                "residual_rel_fro": float(torch.linalg.norm(A @ X - X * lam[None, :]) / nrmA),
                "max_dlambda_over_norm": float((torch.sort(lam).values - lam0).abs().max() / lam0.abs().max())}

    direct = accuracy(Z, ev)
    X = Z.float().double()        # FP32-accurate eigenvectors
    lam = ev.clone()
    rws_b = gb.gb_refine_syev_workspace_bytes(n)
    rws = torch.empty(rws_b, dtype=torch.uint8, device=dev)
    steps = [{"step": 0, "seconds": 0.0, **accuracy(X, lam)}]
    for k in range(1, args.steps + 1):
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(st)
        gb.gb_refine_syev_d(n, A, n, lam, X, n, rws, rws_b, st)
        r1.record(st)
        torch.cuda.synchronize(dev)
        steps.append({"step": k, "seconds": r0.elapsed_time(r1) / 1e3, **accuracy(X, lam)})
    clocks = sampler.stop()
    step_s = min(x["seconds"] for x in steps[1:]) if len(steps) > 1 else None
    flops = 6.0 * n ** 3
    print(json.dumps({
        "stage": "refine", "metric": f"Ogita-Aishima refinement step vs the direct FP64 solve, n={n}, all eigenpairs",
        "n": n, "direct_fp64_solve_s": solve_s, "direct_accuracy": direct, "refine_steps": steps,
        "refine_step_s": step_s,
        "refine_step_tflops_fp64_equivalent": flops / step_s / 1e12 if step_s else None,
        "two_steps_s": 2 * step_s if step_s else None,
        "fp32_solve_budget_for_break_even_s": solve_s - 2 * step_s if step_s else None,
        "data": "synthetic: A = Q diag(uniform in [-1,1], runs of 8 spaced 1e-6) Q^T; FP32 start = FP64 eigenvectors rounded",
        "dtype": "f64", "clocks": clocks}))
    return 0


def run_stage_gemm_fp32(args):
    """The FP32 split product (gb_dgemm_fp32split, the mixed solve's
    reduction and back-transformation products) beside the FP64-accurate
    sliced product (gb_dgemm_sliced) at the band->full shapes of an
    n = 16384 solve and at a square size: TFLOP/s on 2 m n k flops (CUDA
    events, best of --steps after --warmup) and each result's largest error
    against torch's float64 product relative to sum_k |a| |b|."""
    import torch
    import paper_1811_01277_gb300 as gb
    from paper_1811_01277_gb300 import build as gbuild
    gbuild.build()
    gb.load()
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream(dev)
    g = torch.Generator(device=dev).manual_seed(78)
    q = args.gemm_n
    shapes = [("T", "N", 64, 4096, 16384, "band->full Y^T Z"), ("N", "N", 16384, 4096, 64, "band->full Z -= Y S"),
              ("N", "N", q, q, q, "square")]
    rows = []
    for ta, tb, m, n, k, what in shapes:
        A = torch.rand(m if ta == "T" else k, k if ta == "T" else m, generator=g, device=dev,
                       dtype=torch.float64) - 0.5                                  # column-major op(A) storage
        B = torch.rand(n, k, generator=g, device=dev, dtype=torch.float64) - 0.5  # k x n column-major
        lda = k if ta == "T" else m
        wsb = gb.gb_dgemm_sliced_workspace_bytes(m, n, k)
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        opA = A if ta == "T" else A.T              # m x k op(A)
        ref = opA @ B.T
        absref = opA.abs() @ B.T.abs()
        row = {"shape": f"{ta}{tb} {m} x {n}, k = {k} ({what})"}
        for name, fn in (("fp32split", gb.gb_dgemm_fp32split), ("fp64_sliced", gb.gb_dgemm_sliced)):
            C = torch.zeros(n, m, device=dev, dtype=torch.float64)              # m x n column-major
            call = lambda: fn(ta, tb, m, n, k, 1.0, A, lda, B, k, 0.0, C, m, ws, wsb, st)
            for _ in range(max(args.warmup, 1)):
                call()
            best = None
            for _ in range(max(args.steps, 1)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                call()
                e1.record(st)
                torch.cuda.synchronize(dev)
                t = e0.elapsed_time(e1) / 1e3
                best = t if best is None else min(best, t)
            row[name] = {"ms": best * 1e3, "tflops": 2.0 * m * n * k / best / 1e12,
                         "max_err_over_abs_sum": float(((C.T - ref).abs() / absref.clamp_min(1e-300)).max())}
        rows.append(row)
        del A, B, C, ws, ref, absref
        torch.cuda.empty_cache()
    print(json.dumps({"stage": "gemm_fp32", "metric": "FP32 split vs FP64-accurate sliced products, TFLOP/s",
                      "cases": rows, "dtype": "f64 in/out", "data": "synthetic: uniform [-0.5, 0.5]"}))
    return 0


def run_stage_mixed(args):
    """The mixed-precision configuration: gb_solve_mixed_d (all eigenpairs
    with FP32 products in full -> band and band -> full, then FP64
    Ogita-Aishima steps with Rayleigh-Ritz on clusters, the lowest nev
    returned) timed beside the FP64 solve gb_solve_d on the same matrix,
    A = Q diag(uniform [-1, 1], 10% in runs of 8 spaced 1e-6) Q^T; the
    eigenvalue error against the prescribed spectrum, the residual and the
    orthogonality of both, and of the mixed solve with no refinement step
    (the low-precision half alone).  One solve per form, CUDA events."""
    import torch
    import paper_1811_01277_gb300 as gb
    from paper_1811_01277_gb300 import build as gbuild
    from paper_1811_01277_gb300 import inputs
    gbuild.build()
    gb.load()
    n, nbw, K = args.mixed_n, 64, args.mixed_steps
    nev = args.mixed_nev or n // 2
    dev = torch.device("cuda", 0)
    st = torch.cuda.current_stream(dev)
    lam0 = torch.from_numpy(inputs.gapped_uniform_spectrum(n, seed=n)).to(dev)
    A = prescribed_symmetric_gpu(lam0, 256, seed=n + 1, dev=dev)
    u = 2.0 ** -53
    nrmA = float(torch.linalg.norm(A))

    def accuracy(ev, Z):
        Zc = Z.T
        dlam = float((ev - lam0[:nev]).abs().max() / lam0.abs().max())
        R = A @ Zc - Zc * ev[None, :]
        res = float(torch.linalg.norm(R) / nrmA)
        del R
        orth = float((Zc.T @ Zc - torch.eye(nev, dtype=torch.float64, device=dev)).abs().max())
        return {"max_dlambda_over_norm": dlam, "residual_rel_fro": res, "orth_max": orth,
                "within": bool(dlam <= 1e-11 and res <= 50 * n * u and orth <= 50 * n * u)}

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / 1e3

    sampler = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    ev = torch.zeros(nev, dtype=torch.float64, device=dev)
    Z = torch.zeros((nev, n), dtype=torch.float64, device=dev)
    out = {"stage": "mixed", "n": n, "nev": nev, "nbw": nbw, "refine_steps": K}
    wsb = gb.gb_solve_workspace_bytes(n, nev, nbw)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    if args.warmup:
        gb.gb_solve_d(n, nev, nbw, A, n, ev, Z, n, ws, wsb, st, 0)
    t = timed(lambda: gb.gb_solve_d(n, nev, nbw, A, n, ev, Z, n, ws, wsb, st, 0))
    out["fp64_solve"] = {"seconds": t, "status": gb.gb_solve_query(ws, n, nev, nbw, st), **accuracy(ev, Z)}
    del ws
    torch.cuda.empty_cache()
    wsb = gb.gb_solve_mixed_workspace_bytes(n, nev, nbw)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    runs = []
    for steps in ([0, K] if K else [0]):
        ev.zero_()
        Z.zero_()
        t = timed(lambda: gb.gb_solve_mixed_d(n, nev, nbw, A, n, ev, Z, n, steps, ws, wsb, st))
        runs.append({"refine_steps": steps, "seconds": t, "status": gb.gb_solve_mixed_query(ws, n, nev, nbw, st),
                     **accuracy(ev, Z)})
    out["mixed_solve"] = runs
    if K:
        out["refine_step_s"] = (runs[1]["seconds"] - runs[0]["seconds"]) / K
        out["mixed_over_fp64_time"] = runs[1]["seconds"] / out["fp64_solve"]["seconds"]
    out.update({
        "metric": f"mixed-precision solve s vs FP64 solve s, n={n}, nev={nev}",
        "workspace_gb": {"fp64": gb.gb_solve_workspace_bytes(n, nev, nbw) / 1e9, "mixed": wsb / 1e9},
        "data": "synthetic: A = Q diag(uniform [-1,1], 10% in runs of 8 spaced 1e-6) Q^T, Q a product of 256 "
                "seeded Householders",
        "dtype": "f64 (FP32 products in the mixed solve's reduction and back-transformation)",
        "clocks": sampler.stop()})
    print(json.dumps(out))
    del ws, A, Z, ev
    torch.cuda.empty_cache()
    return 0


def run_stage_trans_ev_z(args):
    """The complex128 back-transformation alone: synthetic unitary reflectors
    (the bulge chase's layout) applied to Gaussian Z, timed with CUDA events
    on the launching stream; FP64 TFLOP/s on the algorithmic flops
    (16 nev per reflector element: one complex dot and one complex update)."""
    import numpy as np
    import torch
    import paper_1811_01277_gb300 as gb
    from paper_1811_01277_gb300 import build as gbuild
    from paper_1811_01277_gb300 import inputs
    gbuild.build()
    gb.load()
    n, nev, nbw = args.zn, args.znev, args.solve_nbw
    dev = torch.device("cuda", 0)
    hv, ht = inputs.synthetic_reflectors(n, nbw, seed=n, cplx=True)
    Z = inputs.z_gaussian(n, nev, seed=nev, cplx=True)
    hv_d = torch.from_numpy(np.ascontiguousarray(hv)).to(dev)
    ht_d = torch.from_numpy(np.ascontiguousarray(ht)).to(dev)
    Zt = torch.from_numpy(np.ascontiguousarray(Z.T)).to(dev)     # column-major n x nev data
    wsb = gb.gb_trans_ev_workspace_bytes(n, nbw, nev, 1, None)
    ws = torch.zeros(max(wsb, 256), dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream(dev)

    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in kev:          # the events exist once recorded
        a.record(st)
        b.record(st)
    zopts = {"column_batch": args.column_batch} if args.column_batch else {}
    kopts = [dict(zopts, kernel_begin_event=a.cuda_event, kernel_end_event=b.cuda_event) for a, b in kev]

    def step(i=None):
        gb.gb_trans_ev_tridi_to_band_z(n, nbw, nev, hv_d, ht_d, Zt, n, ws if wsb else None, wsb, st,
                                       (zopts or None) if i is None else kopts[i])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for i in range(args.steps):
        step(i)
    e1.record(st)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    status = gb.gb_trans_ev_query(ws if wsb else None, wsb, st)
    ms = e0.elapsed_time(e1) / args.steps
    kernel_ms = sum(a.elapsed_time(b) for a, b in kev) / args.steps
    F = algorithmic_flops(n, nev, cplx=True)
    # unitary reflectors keep every column's norm
    norms = torch.linalg.norm(Zt, dim=1).cpu().numpy()
    drift = float(np.max(np.abs(norms / np.linalg.norm(Z, axis=0) - 1.0)))
    variant = gb.gb_trans_ev_variant(n, nbw, nev, 1, None)
    fp64 = {"achieved": F / (ms / 1e3) / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": F / (ms / 1e3) / 1e12 / FP64_PEAK_TFLOPS, "algorithmic_tflop": F / 1e12}
    if variant == gb.GB_VARIANT_PIPELINE_TC5:
        pk = measured_peaks()
        Ft = tc5_executed_flops_z(n, nbw, nev)
        ach = Ft / (kernel_ms / 1e3) / 1e12
        peak = pk["bf16_tflops"]
        roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "kernel": "pipeline_tc5 (complex, real 2x2-block form)", "per": "launch",
                "kernel_ms_per_launch": kernel_ms, "executed_fp16_tflop_per_launch": Ft / 1e12,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst: the kernel is timed alone)",
                "frac_of_sustained_peak": ach / (pk["bf16_tflops_sustained"] or pk["bf16_tflops"]),
                "fp64_equivalent_per_step": fp64}
    else:
        roof = dict(bound="alu", kernel_ms_per_launch=kernel_ms, **fp64)
    print(json.dumps({
        "stage": "trans_ev_z", "metric": f"complex128 trans_ev_tridi_to_band s at n={n}, nev={nev}, nbw={nbw}",
        "value": 1e3 / ms, "unit": "back-transforms/s", "ms_per_step": ms, "steps": args.steps,
        "warmup": args.warmup, "status": status, "dtype": "complex128",
        "variant": {gb.GB_VARIANT_PIPELINE_TC5: "pipeline_tc5", gb.GB_VARIANT_WAVEFRONT: "wavefront_smem"}.get(variant, variant),
        "data": "synthetic unitary reflectors (v0 = 1, v U[-1,1]/sqrt(len), tau = (1 - e^{i theta})/|v|^2), Z iid N(0,1/n)",
        "roofline": roof, "column_norm_drift_max": drift, "clocks": clocks}))
    return 0


def run_stage_serve(args):
    """Poisson stream of complex Hermitian requests through the
    continuous-batching server: `systems` systems with sizes drawn from
    --serve-sizes, each re-submitted --serve-repeats times as
    A <- A + 1e-3 E (E Hermitian, ||E||_2 = 1, kept on the device), nev = 30%."""
    import numpy as np
    import torch
    import paper_1811_01277_gb300 as gb
    from paper_1811_01277_gb300 import build as gbuild
    from paper_1811_01277_gb300 import serve
    gbuild.build()
    gb.load()
    dev = torch.device("cuda", 0)
    g = np.random.default_rng(200)
    sizes = [int(x) for x in args.serve_sizes.split(",")]
    gen = torch.Generator(device=dev).manual_seed(201)
    reqs, t, rid = [], 0.0, 0
    systems = []
    for k in range(args.serve_systems):
        n = int(g.choice(sizes))
        R = torch.complex(torch.randn(n, n, generator=gen, device=dev, dtype=torch.float64),
                          torch.randn(n, n, generator=gen, device=dev, dtype=torch.float64))
        A = 0.5 * (R + R.conj().T)
        R = torch.complex(torch.randn(n, n, generator=gen, device=dev, dtype=torch.float64),
                          torch.randn(n, n, generator=gen, device=dev, dtype=torch.float64))
        E = 0.5 * (R + R.conj().T)
        E = E / torch.linalg.matrix_norm(E, ord=2)
        systems.append((n, A, E))
    arrivals = np.cumsum(g.exponential(1.0 / args.serve_rate, args.serve_systems * args.serve_repeats))
    for j in range(args.serve_repeats):
        for k, (n, A, E) in enumerate(systems):
            M = A + (1e-3 * j) * E
            reqs.append(serve.Request(rid=rid, A=M.T.contiguous(), nev=int(0.3 * n), arrival=float(arrivals[rid])))
            rid += 1
    torch.cuda.synchronize(dev)
    warm = serve.EigenServer(slots=args.serve_slots)
    warm.run([serve.Request(rid=-1, A=reqs[0].A, nev=reqs[0].nev, arrival=0.0)])
    srv = serve.EigenServer(slots=args.serve_slots, hbm_budget_bytes=args.serve_budget_gb << 30)
    sampler = ClockSampler(os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0])
    done = srv.run(reqs)
    clocks = sampler.stop()
    summ = serve.latency_summary(done)
    # the same requests with the bulge chases batched across requests (one
    # chase launch in flight at a time, or up to four)
    stage_batched = {}
    for lanes in (1, 4):
        for r in reqs:
            r.start = r.done = r.status = r.ev = r.Z = None
        srv_b = serve.EigenServer(slots=args.serve_slots, hbm_budget_bytes=args.serve_budget_gb << 30,
                                  stage_batching=True, chase_lanes=lanes)
        done_b = srv_b.run(reqs)
        summ_b = serve.latency_summary(done_b)
        stage_batched[f"lanes_{lanes}"] = {
            "value": summ_b["solves_per_s"], "unit": "solves/s", "p50_ms": summ_b["p50_ms"],
            "p99_ms": summ_b["p99_ms"], "failed": sum(1 for r in done_b if r.status != 0),
            "chases_per_launch_mean": float(np.mean(srv_b.chase_sizes)), "chase_launches": len(srv_b.chase_sizes)}
    # the plain solve on the same requests, one after another on one stream
    pst = torch.cuda.Stream(device=dev)
    pmax = max(gb.gb_solve_workspace_bytes_z(r.n, r.nev, gb.gb_solve_default_nbw(r.n)) for r in reqs)
    pws = torch.empty(pmax, dtype=torch.uint8, device=dev)
    pev = torch.empty(max(r.nev for r in reqs), dtype=torch.float64, device=dev)
    pZ = torch.empty(max(r.n * r.nev for r in reqs), dtype=torch.complex128, device=dev)
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    for r in reqs:
        b_ = gb.gb_solve_default_nbw(r.n)
        gb.gb_solve_z(r.n, r.nev, b_, r.A, r.n, pev, pZ, r.n, pws, pmax, pst, 0)
    torch.cuda.synchronize(dev)
    plain_rate = len(reqs) / (time.perf_counter() - t1)
    print(json.dumps({
        "stage": "serve", "metric": "served complex Hermitian eigensolves: solves/s and latency",
        "value": summ["solves_per_s"], "unit": "solves/s", "p50_ms": summ["p50_ms"], "p99_ms": summ["p99_ms"],
        "max_ms": summ["max_ms"], "requests": summ["requests"], "arrival_rate_per_s": args.serve_rate,
        "sizes": sizes, "systems": args.serve_systems, "repeats": args.serve_repeats, "slots": args.serve_slots,
        "hbm_budget_gb": args.serve_budget_gb, "failed": sum(1 for r in done if r.status != 0),
        "plain_solve_one_at_a_time": {"value": plain_rate, "unit": "solves/s", "sample": "the same requests",
                                      "speedup_of_served": summ["solves_per_s"] / plain_rate},
        "stage_batched_chases": stage_batched,
        "dtype": "complex128", "data": "synthetic Hermitian, A <- A + 1e-3 E per re-submission",
        "clocks": clocks}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="n16384")
    ap.add_argument("--variant", type=int, default=0, help="0 library default, 1 wavefront, 2 pipeline")
    ap.add_argument("--nb", type=int, default=0, help="sweeps per tile (0 = default)")
    ap.add_argument("--threads", type=int, default=0, help="columns per block (0 = default)")
    ap.add_argument("--column-batch", type=int, default=0, help="pipeline: column blocks per ticket batch (0 = default)")
    ap.add_argument("--lead-tiles", type=int, default=0, help="pipeline: tiles a sweep group may lead the next (0 = default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--autotune", choices=["fast", "medium"], default=None,
                    help="walk the autotuner first and time its fastest setting")
    ap.add_argument("--shard", action="store_true",
                    help="with N > 1 ranks: split one problem's columns over the ranks (strong scaling) "
                         "instead of one independent problem per rank")
    ap.add_argument("--no-extra", action="store_true",
                    help="default stage: skip the solve and batched measurements that complete the metric")
    ap.add_argument("--stage", choices=["trans_ev", "trans_ev_z", "band_to_tridi", "solve", "batched", "serve", "gemm",
                                        "refine", "mixed", "gemm_fp32"],
                    default="trans_ev")
    ap.add_argument("--refine-n", type=int, default=8192, help="refine stage: n (all eigenpairs)")
    ap.add_argument("--mixed-n", type=int, default=8192, help="mixed stage: n")
    ap.add_argument("--gemm-n", type=int, default=8192, help="gemm_fp32 stage: the square size")
    ap.add_argument("--mixed-nev", type=int, default=0, help="mixed stage: nev (0: n/2)")
    ap.add_argument("--mixed-steps", type=int, default=3, help="mixed stage: refinement steps")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--batch-lo", type=int, default=128)
    ap.add_argument("--batch-hi", type=int, default=2048)
    ap.add_argument("--batch-streams", type=int, default=16)
    ap.add_argument("--solve-n", type=int, default=16384)
    ap.add_argument("--solve-nev", type=int, default=4096)
    ap.add_argument("--solve-nbw", type=int, default=64)
    ap.add_argument("--complex", action="store_true", help="solve stage: complex128 Hermitian")
    ap.add_argument("--zn", type=int, default=8192, help="trans_ev_z stage: n")
    ap.add_argument("--znev", type=int, default=2048, help="trans_ev_z stage: nev")
    ap.add_argument("--spectrum", choices=["clustered", "uniform-gapped"], default="clustered",
                    help="solve stage: clustered in [-50, 50] (1e-8 clusters), or uniform in [-1, 1] with 1e-6 gaps")
    ap.add_argument("--no-stages", action="store_true", help="solve stage: skip the extra stage-timing solve")
    ap.add_argument("--dfma-products", action="store_true",
                    help="solve stage: run the real solve's products on the FP64 FMA pipe (not sliced)")
    ap.add_argument("--emulated-gemm", action="store_true",
                    help="solve stage: let cuBLAS use its fixed-point FP64 emulation for the GEMMs")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-sizes", default="512,1024,2048")
    ap.add_argument("--serve-systems", type=int, default=6)
    ap.add_argument("--serve-repeats", type=int, default=10)
    ap.add_argument("--serve-slots", type=int, default=12)
    ap.add_argument("--serve-budget-gb", type=int, default=64)
    ap.add_argument("--chase-n", type=int, default=16384)
    ap.add_argument("--chase-b", type=int, default=64)
    args = ap.parse_args()
    if args.stage == "band_to_tridi":
        return run_stage_band_to_tridi(args)
    if args.stage == "solve":
        return run_stage_solve(args)
    if args.stage == "gemm":
        return run_stage_gemm(args)
    if args.stage == "batched":
        return run_stage_batched(args)
    if args.stage == "refine":
        return run_stage_refine(args)
    if args.stage == "mixed":
        return run_stage_mixed(args)
    if args.stage == "gemm_fp32":
        return run_stage_gemm_fp32(args)
    if args.stage == "trans_ev_z":
        return run_stage_trans_ev_z(args)
    if args.stage == "serve":
        return run_stage_serve(args)
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)
    return run_ours(args, wl)


if __name__ == "__main__":
    sys.exit(main())
