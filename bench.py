"""Benchmark of the hot path on synthetic images shaped like the paper's workloads.

One step = one pass of the whole path over one batch: critical-table extraction of
64 grayscale 2048 x 2048 images (Gaussian random field, correlation length 16,
quantised to 0..255), ECT at 1024 directions x 512 thresholds, and the Laplace,
Fourier and Bessel hybrid transforms at 4096 directions (|xi| log-uniform in
[0.01, 1]) in FP32 with compensated sums.  The plain FP64 hybrid path is timed on a
direction sample beside it.  Inputs (268 MB) and tables (~1.4 GB) exceed the 129 MB
L2, so no flush is needed between steps.

Prints one JSON line: the metric, the timed step, the roofline of the dominant kernel,
the CPU-oracle baseline, the end-to-end rate through host buffers, the clocks seen and
the other rows of the path.  ``--impl reference`` times the CPU oracle instead (a
bounded sample of the same workload, same metric).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "hybrid dir×crit-pt evals/s (FP32c vs FP64), ECT dirs/s, extraction GB/s"
UNIT = "dir×crit-pt evals/s"
WORKLOAD = "2D grayscale GRF, 64 x 2048x2048 uint8 (ell=16); ECT 1024 dirs x 512 thresholds; " \
           "Laplace/Fourier/Bessel HT at 4096 dirs, |xi| log-uniform [0.01, 1]"
B_IMAGES, SIDE, ELL = 64, 2048, 16.0
D_ECT, T_ECT, D_HT = 1024, 512, 4096
KERNELS = ("laplace", "fourier", "bessel")
FP64_SAMPLE_DIRS = 128
# DRAM bytes (read + write) per image of one FP32C hybrid launch: dram__bytes_read.sum +
# dram__bytes_write.sum of the packed launches in an ncu capture of the 8-image case (the
# tables are read once per work item, so the traffic grows with the number of images)
HT_DRAM_BYTES_PER_IMAGE = {"ht_laplace": (84.03e6 + 3.71e6) / 8, "ht_fourier": (86.93e6 + 4.30e6) / 8,
                           "ht_bessel": (96.63e6 + 0.95e6) / 8}


def bench_config(n_img: int, side: int, world: int) -> dict:
    """The workload both arms report (the reference arm times the CPU oracle on samples of it)."""
    return {"workload": WORKLOAD, "images": n_img, "side": side, "ect_dirs": D_ECT, "thresholds": T_ECT,
            "ht_dirs": D_HT, "l2": "inputs larger than L2 (no flush)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def make_images(count: int, side: int):
    from paper_2405_02256_gb300 import synth
    return [synth.grf((side, side), ELL, seed=1000 + b) for b in range(count)]


def make_dirs():
    from paper_2405_02256_gb300 import synth
    return synth.circle_dirs(D_ECT), synth.random_2d_dirs(D_HT, 2, 0.01, 1.0)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(ms: float, device) -> float:
    """Job time: the maximum over ranks (a no-op without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job throughput: units processed by all ranks over the job time."""
    return units_per_rank * world / (ms / 1e3)


def _dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2405_02256_gb300 import binding as tb
    from paper_2405_02256_gb300 import synth

    rank, world, local = _dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    n_img = args.images

    # ---- inputs (host, seeded), resident in HBM before the timed region ----------------
    t0 = time.time()
    imgs = make_images(n_img, args.side)
    batch = tb.pack_images(imgs, device=dev)
    host_pixels = batch.pixels.cpu().pin_memory()
    dirs_ect_h, dirs_ht_h = make_dirs()
    dirs_ect = torch.from_numpy(dirs_ect_h).to(dev)
    dirs_ht = torch.from_numpy(dirs_ht_h).to(dev)
    R = synth.image_radius(2)
    setup_s = time.time() - t0

    tabs = tb.tables_create(batch.shapes, batch.offsets)
    tabs.build(batch.pixels)
    tabs.sync()
    # table sizes: nl[b, o] = |Delta^-_o|, nd[b, o] = |Delta_rep(o)| (the table direction o uses)
    nl = np.array([[tabs.info(b, o)[0] for o in range(4)] for b in range(n_img)], dtype=np.int64)
    nd = np.array([[tabs.info(b, o)[1] for o in range(4)] for b in range(n_img)], dtype=np.int64)
    orth = np.array([sum(1 << k for k in range(2) if x[k] < 0) for x in dirs_ht_h])
    orth_e = np.array([sum(1 << k for k in range(2) if x[k] < 0) for x in dirs_ect_h])
    cnt_ht = np.bincount(orth, minlength=4)
    cnt_ect = np.bincount(orth_e, minlength=4)
    terms = int((nd * cnt_ht[None, :]).sum())            # evaluations per kernel per step
    ect_updates = int((nl * cnt_ect[None, :]).sum())
    n_lower = int(nl.sum())
    seg_entries = n_lower + int(nd[:, :2].sum())         # 4 lower tables + 2 Delta tables per image
    ext_bytes = batch.pixels.numel() * 1 + seg_entries * 6      # u8 in, int32 idx + int16 value out

    ect_out = torch.empty((n_img, D_ECT, T_ECT), dtype=torch.int32, device=dev)
    ht_out = {k: torch.empty((n_img, D_HT, 2) if k == "fourier" else (n_img, D_HT), dtype=torch.float64, device=dev)
              for k in KERNELS}
    stream = torch.cuda.current_stream(dev)

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        tabs.build(batch.pixels)
        if ev is not None:
            ev[1].record(stream)
        tb.ect(tabs, dirs_ect, -R, R, T_ECT, out=ect_out)
        if ev is not None:
            ev[2].record(stream)
        for i, k in enumerate(KERNELS):
            tb.hybrid_transform(tabs, k, dirs_ht, "fp32c", out=ht_out[k])
            if ev is not None:
                ev[3 + i].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    tabs.sync()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        start.record(stream)
        for s in range(args.steps):
            step(evs[s])
        stop.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    total_ms = max_over_ranks(start.elapsed_time(stop), dev)
    ms_step = total_ms / args.steps
    ph = np.array([[evs[s][i].elapsed_time(evs[s][i + 1]) for i in range(5)] for s in range(args.steps)])
    ph_ms = ph.mean(axis=0)
    value = whole_job_rate(terms * 3, world, ms_step)

    # ---- plain FP64 hybrid path on a direction sample ---------------------------------------
    sample = dirs_ht[:FP64_SAMPLE_DIRS].contiguous()
    sample_terms = int((nd * np.bincount(orth[:FP64_SAMPLE_DIRS], minlength=4)[None, :]).sum())
    fp64 = {}
    fp32_s = {}
    for k in KERNELS:
        for prec, store in (("fp64", fp64), ("fp32c", fp32_s)):
            tb.hybrid_transform(tabs, k, sample, prec)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            o64 = tb.hybrid_transform(tabs, k, sample, prec)
            e1.record(stream)
            torch.cuda.synchronize()
            store[k] = {"ms": e0.elapsed_time(e1), "evals_per_s": sample_terms / (e0.elapsed_time(e1) / 1e3),
                        "out": o64}
    # accuracy of FP32C against the FP64 GPU path on the sample (relative to sum |Delta kbar| ~ |HT| bound)
    acc = {}
    for k in KERNELS:
        a, b_ = fp32_s[k]["out"], fp64[k]["out"]
        acc[k] = float(((a - b_).abs().max() / b_.abs().max().clamp_min(1e-300)).item())

    # ---- end to end through the public API: host pixels in, results out -----------------------
    ect_host = torch.empty(ect_out.shape, dtype=torch.int32).pin_memory()
    ht_host = {k: torch.empty(v.shape, dtype=torch.float64).pin_memory() for k, v in ht_out.items()}
    e2e_start, e2e_stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    e2e_start.record(stream)
    for _ in range(e2e_steps):
        batch.pixels.copy_(host_pixels, non_blocking=True)
        step()
        ect_host.copy_(ect_out, non_blocking=True)
        for k in KERNELS:
            ht_host[k].copy_(ht_out[k], non_blocking=True)
    e2e_stop.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e2e_start.elapsed_time(e2e_stop) / e2e_steps
    h2d = host_pixels.numel() * host_pixels.element_size()
    d2h = ect_host.numel() * 4 + sum(v.numel() * 8 for v in ht_host.values())

    clocks = clk.summary()
    # dominant kernel of the step -> roofline
    names = ["extract", "ect", "ht_laplace", "ht_fourier", "ht_bessel"]
    dom = int(np.argmax(ph_ms))
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0))
    # FP32 pipe: 128 lanes per SM per clock; issue: 4 schedulers x 32 lanes per SM per clock
    lane_ops = sm_count * 128 * mhz * 1e6
    # FP32-pipe lane operations per term of each hybrid kernel as written (a packed f32x2
    # operation counts 2, MUFU operations are not counted; the average over the MUFU and
    # polynomial halves for Fourier), and issued instructions per (point, direction)
    # update of the ECT kernel; both counted from the kernel source
    # (packed f32x2: argument 2, accumulation 1 per component, block-compensated sums about
    # 0.6 per component; Fourier: the mean of a polynomial pair, 12.25, and a MUFU pair with
    # the FMUL range reduction of sin and cos, 8.5; Bessel: 7.6 on the |z| <= 0.5 path that
    # almost every tile of this direction law takes)
    fp32_ops = {"ht_laplace": 3.6, "ht_fourier": 10.4, "ht_bessel": 7.6}
    # warp instructions per 32 (point, direction) updates of k_hist, from its ncu
    # capture (instructions executed / updates x 32)
    ect_instr = 23.0
    if names[dom] == "extract":
        achieved = ext_bytes / (ph_ms[dom] / 1e3) / 1e9
        roof = {"kernel": "k_extract", "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": None, "peak_source": "MEASURED_PEAKS hbm_gbs (of measured)"}
    elif names[dom] == "ect":
        achieved = ect_updates * ect_instr / 32 / (ph_ms[dom] / 1e3) / 1e12
        peak = lane_ops / 32 / 1e12
        roof = {"kernel": "k_hist", "bound": "alu", "achieved": achieved, "peak": peak, "unit": "Twarp-instr/s",
                "frac": achieved / peak, "traffic": None,
                "peak_source": "152 SMs x 4 issue slots x max SM clock (recipe unit counts)"}
    else:
        nm = names[dom]
        term_rate = terms / (ph_ms[dom] / 1e3)
        achieved = term_rate * fp32_ops[nm] / 1e12
        peak = lane_ops / 1e12
        roof = {"kernel": "k_ht_f32<" + nm[3:] + ">", "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "Tlane-ops/s (FP32 pipe)", "frac": achieved / peak,
                "traffic": HT_DRAM_BYTES_PER_IMAGE[nm] * n_img,
                "terms_per_s": term_rate, "fp32_lane_ops_per_term": fp32_ops[nm],
                "peak_source": "152 SMs x 128 FP32 lanes x max SM clock (recipe unit counts)"}

    # extraction 1; ECT: direction prep, plan, histogram, finish; each hybrid transform:
    # direction prep, plan, packed and wide-range launches, combine
    launches_per_step = 1 + 4 + 5 * len(KERNELS)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8 tables / fp32c hybrid", "data": "synthetic",
        "config": bench_config(n_img, args.side, world),
        "phases_ms": dict(zip(names, [float(x) for x in ph_ms])),
        "ect_dirs_per_s": n_img * D_ECT * world / (ph_ms[1] / 1e3),
        "ect_updates_per_s": ect_updates / (ph_ms[1] / 1e3),
        "extraction_gbs": ext_bytes / (ph_ms[0] / 1e3) / 1e9,
        "extraction_hbm_frac": ext_bytes / (ph_ms[0] / 1e3) / 1e9 / hbm,
        "hybrid_fp32c_evals_per_s": {k: terms / (ph_ms[2 + i] / 1e3) for i, k in enumerate(KERNELS)},
        "hybrid_fp64_evals_per_s": {k: fp64[k]["evals_per_s"] for k in KERNELS},
        "fp32c_over_fp64_speedup": {k: fp32_s[k]["evals_per_s"] / fp64[k]["evals_per_s"] for k in KERNELS},
        "fp32c_rel_err_vs_fp64": acc,
        "fp32c_rel_err_norm": "max |FP32C - FP64| / max |FP64| over all sampled outputs; the tests bound the "
                              "per-direction error normalised by sum |Delta kappa-bar| at 1e-6",
        "fp64_sample": f"{FP64_SAMPLE_DIRS} of {D_HT} directions, all images",
        "work": {"hybrid_terms_per_kernel": terms, "ect_updates": ect_updates, "lower_entries": n_lower,
                 "algorithmic_extraction_bytes": ext_bytes},
        "roofline": roof,
        "e2e": {"value": terms * 3 / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "setup_s": setup_s,
    }
    if not args.no_extra:
        out["rows"] = extra_rows(tabs, batch, dirs_ect, dirs_ect_h, dirs_ht, dirs_ht_h, nl, nd, n_img, dev)
        tabs.free()
        del batch
        torch.cuda.empty_cache()
        out["rows"].update(extra_workloads(dev))
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        out["cpu_baseline"] = cpu_baseline(imgs[0], dirs_ect_h, dirs_ht_h, budget_s=args.cpu_budget)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def _time_cuda(fn, reps: int = 3) -> float:
    """Mean ms of fn over reps launches, after one warm-up (CUDA events, current stream)."""
    import torch
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _orthants(dirs: np.ndarray) -> np.ndarray:
    n = dirs.shape[1]
    return sum(((dirs[:, k] < 0).astype(np.int64) << k) for k in range(n))


def _sizes(tabs, n_img, NO):
    nl = np.array([[tabs.info(b, o)[0] for o in range(NO)] for b in range(n_img)], dtype=np.int64)
    nd = np.array([[tabs.info(b, o)[1] for o in range(NO)] for b in range(n_img)], dtype=np.int64)
    return nl, nd


_ROWS = None   # names of the extra rows to run (None: all)


def _hbm_gbs() -> float:
    """Measured HBM copy bandwidth (GB/s) of this machine's GPUs, else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f).get("hbm_gbs", 6800.0))
    except OSError:
        return 6800.0


def _want(name: str) -> bool:
    return _ROWS is None or name in _ROWS


def extra_rows(tabs, batch, dirs_ect, dirs_ect_h, dirs_ht, dirs_ht_h, nl, nd, n_img, dev):
    """Every other row of the hot path, measured on its own workload."""
    import torch

    from paper_2405_02256_gb300 import binding as tb
    from paper_2405_02256_gb300 import synth
    rows = {}
    R2 = synth.image_radius(2)
    # (point, direction) terms of one hybrid transform over the 4096 directions
    terms = int((nd * np.bincount(_orthants(dirs_ht_h), minlength=4)[None, :]).sum())

    if _want("radon_2d"):
        # Radon on the same 2048^2 tables, 1024 directions x 512 thresholds (two tables per direction)
        out = torch.empty((n_img, D_ECT, T_ECT), dtype=torch.int32, device=dev)
        ms = _time_cuda(lambda: tb.radon(tabs, dirs_ect, -R2, R2, T_ECT, out=out))
        cnt = np.bincount(_orthants(dirs_ect_h), minlength=4)
        upd = int(sum(cnt[o] * (nl[:, o] + nl[:, o ^ 3]).sum() for o in range(4)))
        rows["radon_2d"] = {"workload": "same 64 x 2048^2 tables; 1024 dirs x 512 thresholds", "ms": ms,
                            "dirs_per_s": n_img * D_ECT / (ms / 1e3), "updates_per_s": upd / (ms / 1e3)}

    if _want("adjoint_2d"):
        # adjoint of Laplace and Fourier at the 4096 hybrid directions
        g = torch.empty_like(dirs_ht)
        adj = {}
        for k in ("laplace", "fourier"):
            gout = torch.ones((n_img, D_HT, 2) if k == "fourier" else (n_img, D_HT), dtype=torch.float64, device=dev)
            ms = _time_cuda(lambda: tb.hybrid_transform_grad(tabs, k, dirs_ht, gout, "fp32c", out=g), reps=1)
            adj[k] = {"ms": ms, "terms_per_s": terms / (ms / 1e3)}
        rows["adjoint_2d"] = {"workload": "same tables; 4096 dirs, d/dxi of sum_b,d HT", **adj}

    if _want("sine_2d"):
        # kappa = sin (the kernel of the paper's experiments)
        o_sine = torch.empty((n_img, D_HT), dtype=torch.float64, device=dev)
        ms = _time_cuda(lambda: tb.hybrid_transform(tabs, "sine", dirs_ht, "fp32c", out=o_sine), reps=1)
        rows["sine_2d"] = {"workload": "same tables; 4096 dirs, kappa = sin (kbar = -cos), FP32C",
                           "ms": ms, "terms_per_s": terms / (ms / 1e3)}
        del o_sine

    if _want("table_2d"):
        # a tabulated kernel, kbar given by K samples (piecewise linear, constant ends);
        # here K = 1024 samples of sin(2 s) + 0.3 s^2 on [-R, R]
        tab_rows = {}
        for K in (64, 1024):
            sk = -R2 + 2 * R2 / (K - 1) * np.arange(K)
            kt = tb.KernelTable(np.sin(2.0 * sk) + 0.3 * sk * sk, -R2, R2)
            o_tab = torch.empty((n_img, D_HT), dtype=torch.float64, device=dev)
            ms = _time_cuda(lambda: tb.hybrid_transform(tabs, kt, dirs_ht, "fp32c", out=o_tab), reps=1)
            tab_rows[f"K{K}_ms"] = ms
            tab_rows[f"K{K}_terms_per_s"] = terms / (ms / 1e3)
            del o_tab
            kt.free()
        rows["table_2d"] = {"workload": "same tables; 4096 dirs, kbar tabulated by K samples on [-R, R], FP32C",
                            **tab_rows}

    if _want("exact_2d"):
        # exact representations (T, E) and (T', E') at 4 directions per image, and their
        # evaluation at 4096 arbitrary thresholds
        tabs.sync()                                   # sizes on the host (the step rebuilt the tables)
        d4 = dirs_ht[:4].contiguous()
        o4 = _orthants(dirs_ht_h[:4])
        ent0 = int(sum(nl[:, o].sum() for o in o4))
        ent1 = int(sum(nd[:, o if o < 2 else o ^ 3].sum() for o in o4))
        cap0 = int(nl.max())
        cap1 = int(nd.max())
        reps = {}
        ms0 = _time_cuda(lambda: reps.__setitem__(0, tb.exact_representation(tabs, 0, d4, cap=cap0)), reps=2)
        ms1 = _time_cuda(lambda: reps.__setitem__(1, tb.exact_representation(tabs, 1, d4, cap=cap1)), reps=2)
        q = torch.linspace(-R2, R2, 4096, dtype=torch.float64, device=dev)
        ms_e = _time_cuda(lambda: tb.ect_exact_eval(reps[0], q))
        ms_r = _time_cuda(lambda: tb.radon_exact_eval(reps[0], reps[1], q))
        rows["exact_2d"] = {
            "workload": f"same {n_img} x 2048^2 tables; exact representations at 4 hybrid directions per image "
                        "(sort of the FP64 dot products, ties merged), evaluated at 4096 thresholds",
            "ect_rep_ms": ms0, "ect_rep_entries_per_s": ent0 / (ms0 / 1e3),
            "radon_rep_ms": ms1, "radon_rep_entries_per_s": ent1 / (ms1 / 1e3),
            "ect_eval_ms": ms_e, "radon_eval_ms": ms_r,
            "evals_per_s": n_img * 4 * 4096 / (ms_e / 1e3),
        }
        del reps

    if _want("top_2d"):
        # top-dimensional construction of the same images (tables on the 2049^2 pixel
        # corners): corner-image pre-pass + extraction, then the ECT at the 1024 x 512 grid
        ttop = tb.tables_create(batch.shapes, batch.offsets, construction="top")
        ms_top = _time_cuda(lambda: ttop.build(batch.pixels))
        ttop.sync()
        ntop = _sizes(ttop, n_img, 4)
        ent_top = int(ntop[0].sum() + ntop[1][:, :2].sum())
        out_top = torch.empty((n_img, D_ECT, T_ECT), dtype=torch.int32, device=dev)
        ms_top_ect = _time_cuda(lambda: tb.ect(ttop, dirs_ect, -R2, R2, T_ECT, out=out_top))
        rows["top_2d"] = {
            "workload": f"same {n_img} x 2048^2 images, top-dimensional construction (tables on 2049^2 corners); "
                        "extraction, then ECT at 1024 dirs x 512 thresholds",
            "extract_ms": ms_top, "extract_gbs": (batch.pixels.numel() + 6 * ent_top) / (ms_top / 1e3) / 1e9,
            "extract_hbm_frac": (batch.pixels.numel() + 6 * ent_top) / (ms_top / 1e3) / 1e9 / _hbm_gbs(),
            "ect_ms": ms_top_ect, "ect_dirs_per_s": n_img * D_ECT / (ms_top_ect / 1e3),
        }
        ttop.free()
        del out_top
    return rows


def ragged_workload():
    """The ragged batch: 10,000 grey images, sides log-uniform in [28, 512] (non-square),
    uniform noise blurred by sigma = 2 px; ECT directions (64 on the circle) and Laplace
    directions (256 unit vectors, uniform angle) shared by every image."""
    from paper_2405_02256_gb300 import synth
    shapes = synth.ragged_shapes(10000, 28, 512, seed=4)
    imgs = [synth.blurred_noise(s, 2.0, seed=400000 + i) for i, s in enumerate(shapes)]
    return imgs, synth.circle_dirs(64), synth.random_2d_dirs(256, 44, 1.0, 1.0)


def ragged_pipeline(tb, batch, ect_h, ht_h, dev):
    """The graph the bench times: extraction, ECT 64 x 64 and Laplace FP32C, tuned tiles."""
    import torch

    from paper_2405_02256_gb300 import synth
    R2 = synth.image_radius(2)
    pipe = tb.Pipeline(batch.shapes, batch.offsets, batch.pixels.numel(),
                       ect=(torch.from_numpy(ect_h).to(dev), -R2, R2, 64),
                       hybrid=[("laplace", torch.from_numpy(ht_h).to(dev), "fp32c")], tune=True)
    pipe.pixels.copy_(batch.pixels)
    return pipe.capture()


def extra_workloads(dev):
    """The ragged batch under a CUDA graph, 256^3 binary volumes, gradients on a 128^3 volume."""
    import torch

    from paper_2405_02256_gb300 import binding as tb
    from paper_2405_02256_gb300 import synth
    rows = {}

    if _want("ragged_graph_2d"):
        # 10,000 ragged grey images, one CUDA graph per step (tuned tiles)
        t0 = time.time()
        imgs, ect_h, ht_h = ragged_workload()
        gen_s = time.time() - t0
        batch = tb.pack_images(imgs, device=dev)
        R2 = synth.image_radius(2)
        pipe = ragged_pipeline(tb, batch, ect_h, ht_h, dev)
        ms = _time_cuda(lambda: pipe.run(), reps=5)
        # the three parts of the step, each launched on its own (outside the graph)
        ect_d = torch.from_numpy(ect_h).to(dev)
        ht_d = torch.from_numpy(ht_h).to(dev)
        ect_o = torch.empty((len(imgs), 64, 64), dtype=torch.int32, device=dev)
        ht_o = torch.empty((len(imgs), 256), dtype=torch.float64, device=dev)
        ms_parts = {"extract_ms": _time_cuda(lambda: pipe.tables.build(pipe.pixels)),
                    "ect_ms": _time_cuda(lambda: tb.ect(pipe.tables, ect_d, -R2, R2, 64, out=ect_o)),
                    "laplace_ms": _time_cuda(lambda: tb.hybrid_transform(pipe.tables, "laplace", ht_d, "fp32c",
                                                                         out=ht_o))}
        pipe.tables.sync()
        nl, nd = _sizes(pipe.tables, len(imgs), 4)
        terms = int((nd * np.bincount(_orthants(ht_h), minlength=4)[None, :]).sum())
        px = int(batch.pixels.numel())
        rows["ragged_graph_2d"] = {
            "workload": "10,000 grey images, sides log-uniform in [28, 512], blurred noise sigma 2; ECT 64 x 64 and "
                        "Laplace at 256 unit dirs per image; extraction + ECT + Laplace replayed as one CUDA graph",
            "ms_per_step": ms, "images_per_s": len(imgs) / (ms / 1e3), "pixels": px,
            "ect_dirs_per_s": len(imgs) * 64 / (ms / 1e3), "laplace_terms_per_s_whole_step": terms / (ms / 1e3),
            "laplace_terms_per_s": terms / (ms_parts["laplace_ms"] / 1e3),
            "ect_updates_per_s": int((nl * np.bincount(_orthants(ect_h), minlength=4)[None, :]).sum())
                                 / (ms_parts["ect_ms"] / 1e3),
            "tuned_tiles": pipe.tuned, "parts": ms_parts, "input_gen_s": gen_s}
        pipe.tables.free()
        del pipe, batch, imgs

    if _want("volumes_3d"):
        # 4 binary volumes 256^3, ECT / Radon at 2048 Fibonacci dirs x 256, Fourier at 8192
        vols = [synth.grf((256, 256, 256), 8.0, seed=300 + b, binary=True) for b in range(4)]
        batch = tb.pack_images(vols, device=dev)
        R3 = synth.image_radius(3)
        fib = synth.fibonacci_dirs(2048)
        four = synth.scale_norms(synth.fibonacci_dirs(8192), 3, 0.05, 2.0)
        tabs = tb.tables_create(batch.shapes, batch.offsets)
        ms_ext = _time_cuda(lambda: tabs.build(batch.pixels))
        tabs.sync()
        nl, nd = _sizes(tabs, 4, 8)
        ent = int(nl.sum() + nd[:, :4].sum())
        d_f = torch.from_numpy(fib).to(dev)
        d_4 = torch.from_numpy(four).to(dev)
        out = torch.empty((4, 2048, 256), dtype=torch.int32, device=dev)
        ms_ect = _time_cuda(lambda: tb.ect(tabs, d_f, -R3, R3, 256, out=out))
        ms_rad = _time_cuda(lambda: tb.radon(tabs, d_f, -R3, R3, 256, out=out))
        o4 = torch.empty((4, 8192, 2), dtype=torch.float64, device=dev)
        ms_f = _time_cuda(lambda: tb.hybrid_transform(tabs, "fourier", d_4, "fp32c", out=o4))
        terms = int((nd * np.bincount(_orthants(four), minlength=8)[None, :]).sum())
        rows["volumes_3d"] = {
            "workload": "4 binary GRF volumes 256^3 (ell=8); ECT and Radon at 2048 Fibonacci dirs x 256; "
                        "Fourier at 8192 dirs, |xi| uniform [0.05, 2]",
            "extract_ms": ms_ext, "extract_gbs": (batch.pixels.numel() + 6 * ent) / (ms_ext / 1e3) / 1e9,
            "extract_hbm_frac": (batch.pixels.numel() + 6 * ent) / (ms_ext / 1e3) / 1e9 / _hbm_gbs(),
            "extract_path": "binary volumes: bit-sliced pack, count, scan and write kernels",
            "ect_ms": ms_ect, "ect_dirs_per_s": 4 * 2048 / (ms_ect / 1e3),
            "radon_ms": ms_rad, "radon_dirs_per_s": 4 * 2048 / (ms_rad / 1e3),
            "fourier_ms": ms_f, "fourier_terms_per_s": terms / (ms_f / 1e3)}
        tabs.free()
        del batch, vols

    if _want("gradients_3d"):
        # one 128^3 grey volume, Laplace and Fourier forward + adjoint at 8192 dirs
        vol = synth.grf((128, 128, 128), 6.0, seed=5)
        batch = tb.pack_images([vol], device=dev)
        tabs = tb.build_critical_tables(batch)
        xi = synth.sphere_dirs(8192, 6, 0.1, 1.0)
        d = torch.from_numpy(xi).to(dev)
        nl, nd = _sizes(tabs, 1, 8)
        terms = int((nd * np.bincount(_orthants(xi), minlength=8)[None, :]).sum())
        res = {}
        for k in ("laplace", "fourier"):
            o = torch.empty((1, 8192, 2) if k == "fourier" else (1, 8192), dtype=torch.float64, device=dev)
            ms_fw = _time_cuda(lambda: tb.hybrid_transform(tabs, k, d, "fp32c", out=o))
            g = torch.empty_like(d)
            gout = torch.ones_like(o)
            ms_bw = _time_cuda(lambda: tb.hybrid_transform_grad(tabs, k, d, gout, "fp32c", out=g))
            res[k] = {"forward_ms": ms_fw, "adjoint_ms": ms_bw, "forward_terms_per_s": terms / (ms_fw / 1e3),
                      "adjoint_terms_per_s": terms / (ms_bw / 1e3)}
        rows["gradients_3d"] = {"workload": "128^3 grey GRF (ell=6); 8192 dirs, |xi| in [0.1, 1]", **res}
        tabs.free()
    return rows


# ---- CPU baseline: the oracle on the host's cores ------------------------------------------
# The oracle (plain numpy, FP64 / int64) as it stands, run the way the paper parallelises
# (Section 5.3): the tables split over vertices (row blocks), the transforms over
# directions (oracle/parallel.py).  Worker processes are spawned, never forked from a
# process that holds a CUDA context.

def cpu_baseline(img, dirs_ect, dirs_ht, budget_s: float = 20.0, procs: int = None):
    """The oracle on a bounded sample of the bench workload, on every host core and on one.

    Sample: one 2048^2 image; its tables (split over row blocks); ECT and Radon at some of
    the 1024 directions x 512 thresholds; the three hybrid transforms at some of the 4096
    directions (counts sized to the budget from a one-direction probe).  value = hybrid
    terms per second on all cores (the bench's unit); the one-process figures come from
    one task run alone."""
    import multiprocessing as mp
    import tempfile

    from oracle import parallel as OP
    nproc = os.cpu_count() or 1
    P = procs or nproc
    ctx = mp.get_context("spawn")
    R = math.sqrt(2.0) / 2.0
    tmp = tempfile.mkdtemp(prefix="topot_oracle_")
    paths = []
    try:
        with ctx.Pool(P) as pool:
            pool.map(abs, range(P))                        # start the workers (imports excluded)
            t0 = time.time()
            parts = pool.map(OP.block_tables, OP.row_blocks(img, P))
            t_tables = time.time() - t0
        t0 = time.time()
        OP.block_tables(OP.row_blocks(img, 1)[0])
        t_tables_1 = time.time() - t0
        tab = OP.merge_blocks(img.shape, parts)
        for s_, (idx, val) in enumerate(zip(tab.lower_idx + tab.delta_idx, tab.lower_val + tab.delta_val)):
            for j, arr in enumerate((idx, val)):
                path = os.path.join(tmp, f"t{s_}_{j}.npy")
                np.save(path, arr)
                paths.append(path)
        rates = {}
        with ctx.Pool(P, initializer=OP.worker_init, initargs=(paths, img.shape, tab.chi)) as pool:
            pool.map(abs, range(P))
            for what, dirs in (("ect", dirs_ect), ("radon", dirs_ect), ("ht", dirs_ht)):
                extra = (-R, R, T_ECT) if what != "ht" else (KERNELS,)
                dt, _ = pool.apply(OP.transform_task, ((what, dirs[:1]) + extra,))
                per = max(1, int((budget_s / 3.0) / max(dt, 1e-3)))
                chunks = []
                for i in range(P):
                    s0 = (i * per) % len(dirs)
                    chunks.append((what, dirs[s0:s0 + per]) + extra)
                t0 = time.time()
                out = pool.map(OP.transform_task, chunks)
                wall = time.time() - t0
                n_dirs = sum(len(c[1]) for c in chunks)
                terms = sum(o[1] for o in out)
                rates[what] = {"dirs": n_dirs, "terms": terms,
                               "all_cores": (terms if what == "ht" else n_dirs) / wall,
                               "one_process": (out[0][1] if what == "ht" else len(chunks[0][1])) / out[0][0]}
    finally:
        for pth in paths:
            os.remove(pth)
        os.rmdir(tmp)
    ht = rates["ht"]
    return {"value": ht["all_cores"], "unit": UNIT, "cores": P, "nproc": nproc, "kind": "oracle",
            "one_thread": {"value": ht["one_process"], "unit": UNIT,
                           "ect_dirs_per_s": rates["ect"]["one_process"],
                           "radon_dirs_per_s": rates["radon"]["one_process"],
                           "tables_s_per_image": t_tables_1},
            "ect_dirs_per_s": rates["ect"]["all_cores"], "radon_dirs_per_s": rates["radon"]["all_cores"],
            "tables_s_per_image": t_tables,
            "sample": (f"1 image {'x'.join(map(str, img.shape))}: tables over {P} row blocks "
                       f"({t_tables:.2f} s; one process {t_tables_1:.2f} s); ECT {rates['ect']['dirs']} and "
                       f"Radon {rates['radon']['dirs']} directions x {T_ECT} thresholds; hybrid transforms "
                       f"{ht['dirs']} directions x 3 kernels ({ht['terms']} terms), split over {P} processes; "
                       f"one-process figures from one task alone")}


def run_reference(args):
    """The reference arm: the oracle (this repository's CPU statement of the method) on the
    host's cores, one bounded sample of the bench workload per step."""
    rank, world, _ = _dist_info()
    if rank != 0:
        return
    imgs = make_images(1, SIDE)
    dirs_ect, dirs_ht = make_dirs()
    per = max(3.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):   # untimed
        cpu_baseline(imgs[0], dirs_ect, dirs_ht, budget_s=min(per, 3.0))
    vals, samples, walls, last = [], [], [], None
    for _ in range(max(1, args.steps)):
        t0 = time.time()
        last = cpu_baseline(imgs[0], dirs_ect, dirs_ht, budget_s=per)
        walls.append(time.time() - t0)
        vals.append(last["value"])
        samples.append(last["sample"])
    v = float(np.mean(vals))
    cb = dict(last)
    cb["value"] = v
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": float(np.mean(walls)) * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": bench_config(args.images, args.side, world),
           "cpu_baseline": cb,
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--images", type=int, default=B_IMAGES)
    p.add_argument("--side", type=int, default=SIDE)
    p.add_argument("--cpu-budget", type=float, default=20.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extra", action="store_true", help="skip the other rows and configurations")
    p.add_argument("--rows", default=None,
                   help="comma-separated extra rows to run (radon_2d, adjoint_2d, sine_2d, table_2d, exact_2d, "
                        "top_2d, ragged_graph_2d, volumes_3d, gradients_3d); default all")
    args = p.parse_args()
    if args.rows:
        global _ROWS
        _ROWS = set(args.rows.split(","))
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
