#!/usr/bin/env python3
"""Benchmark of the bank filter (Eqs. 1, 3, 4 of arXiv:0906.4175) on one GB300.

A step is one pass of the hot path over the 1024-template, N = 2^20 workload
(32x32 mass lattice over [1, 3] Msun, fs = 4096 Hz, 256 s of seeded coloured
Gaussian noise with 8 injections, threshold rho = 6): segment conditioning
(mf_segment_refresh of the resident samples) plus the bank filter
(mf_filter_bank), captured once as a CUDA graph and replayed per step
(--eager times the plain calls).  Inputs are resident in HBM when timing
starts; L2 is flushed (256 MiB write) before every timed step; each step is
timed with CUDA events on the launching stream.  The per-stage shares and the
roofline come from the same number of eager steps with per-stage events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mfgb|reference]

--impl reference times the FP64 CPU oracle (the reference arm of this build)
on a bounded sample of the same workload.  Under torchrun (N > 1) every rank
filters its own replica of the workload (weak scaling, no data-path
collective); rank 0 prints the JSON line with the max time over ranks.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "templates/s filtered at N=2^20 (FP32), % HBM roofline, max ρ rel err vs FP64"
UNIT = "templates/s"
WORKLOAD = "1024 templates (32x32 lattice, m1,m2 in [1,3] Msun), 1 segment N=2^20 at 4096 Hz, 8 injections, thr 6"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
KERNEL_SOURCES = ["mf_fft.cuh", "mf_passes.cuh", "mf_filter.cuh", "mf_persist.cu", "mf_rows.cu", "mf_pass1.cu",
                  "mf_internal.h", "mf_async.cuh"]
# the sources each profiled stage's kernel is built from (its ncu figures stay valid while they do not change)
STAGE_SOURCES = {"pass1": ["mf_fft.cuh", "mf_passes.cuh", "mf_filter.cuh", "mf_pass1.cuh", "mf_pass1.cu",
                           "mf_async.cuh"],
                 "pass2": ["mf_fft.cuh", "mf_filter.cuh", "mf_rows.cuh", "mf_rows.cu", "mf_async.cuh"]}


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mfgb", choices=["mfgb", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU work of the oracle baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--templates", type=int, default=0,
                    help="use only the first T templates of the workload (small profiling cases; not a bench line)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default schedule (MFGB_SCHED may force one)")
    ap.add_argument("--eager", action="store_true", help="time eager calls instead of CUDA-graph replays")
    ap.add_argument("--conditioning", default="fp64", choices=["fp64", "fp32"],
                    help="precision of the forward FFT of the per-step segment refresh (mf_segment_set_conditioning)")
    ap.add_argument("--fft-mode", default="fp32", choices=["fp32", "tc_fp16", "tc_bf16"],
                    help="FFT form of the scale workload: FP32 butterflies (the benchmark line) or the tensor-core "
                         "DFT stage of pass 2 with FP16 / BF16 splits (precision-sweep forms)")
    ap.add_argument("--seed", type=int, default=0, help="seed of the synthetic workload (bank order, noise, injections)")
    ap.add_argument("--config", type=int, default=0, choices=[0, 2, 3, 4, 5],
                    help="the workload by its configuration number: 2 = scale (the benchmark line), 3 = uneven, "
                         "4 = precision, 5 = refine (config 1, the 16-template case, is a parity test)")
    ap.add_argument("--workload", default="scale",
                    choices=["scale", "uneven", "precision", "refine", "chisq", "fft", "events"],
                    help="scale: the benchmark line; the others print their own measurement line "
                         "(uneven bank over mixed segment lengths, phase precision forms, trigger refinement)")
    a = ap.parse_args()
    if a.config:
        a.workload = {2: "scale", 3: "uneven", 4: "precision", 5: "refine"}[a.config]
    return a


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks (every rank gets it): the job's time is
    its slowest rank's."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: int, ms: float) -> float:
    """Units all ranks processed (each rank filters its own replica) per
    second of the slowest rank's time."""
    return world * units_per_rank / (ms / 1e3)


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _hbm_peak():
    try:
        with open(PEAKS_PATH) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash(files=None) -> str:
    h = hashlib.sha256()
    for f in (files or KERNEL_SOURCES):
        with open(os.path.join(ROOT, "paper_0906_4175_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic(kernel_stage: str):
    """DRAM bytes per launch of the dominant kernel from the committed ncu
    summary, if it was taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        e = d.get(kernel_stage)
        if e and e.get("source_hash") == kernel_source_hash(STAGE_SOURCES.get(kernel_stage)):
            return float(e["dram_bytes_per_launch"]), float(e.get("templates_per_launch", 0)) or None
    except Exception:
        pass
    return None, None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms; start()
    waits for the first sample, and only samples taken between mark_begin()
    and mark_end() (host wall clock) are kept."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(prefix="mfgb_clocks_", suffix=".csv")
        self.proc = None
        self.gpu = gpu_index
        self.t0 = self.t1 = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
            deadline = time.time() + 10.0
            while time.time() < deadline and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None

    def mark_begin(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    @staticmethod
    def _stamp(text):
        import datetime
        for fmt in ("%Y/%m/%d %H:%M:%S.%f", "%Y/%m/%d %H:%M:%S"):
            try:
                return datetime.datetime.strptime(text, fmt).timestamp()
            except ValueError:
                pass
        return None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                ts = self._stamp(p[0])
                if ts is not None and self.t0 is not None and not (self.t0 - 0.1 <= ts <= self.t1 + 0.1):
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for n, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def cpu_baseline(wl, cpu_seconds: float, gpu_check=None):
    """Time the FP64 oracle as it stands on a bounded template sample of the
    workload (its own FP64 synthesis of the same seeded segment), on all host
    cores.  If gpu_check is given, also measure the GPU's rho error on the
    same input and sample."""
    import numpy as np
    import oracle
    oracle.build()
    spec = wl.segments[0]
    s = oracle.synth(spec.normals(), spec.N, spec.fs, wl.f_low, spec.injections).astype(np.float32)
    s64 = s.astype(np.float64)
    rng = np.random.default_rng(12345)
    order = rng.permutation(wl.n_templates)
    # calibrate with one template on all cores (OpenMP across templates -> one thread busy)
    t0 = time.perf_counter()
    oracle.filter_bank(wl.m1[order[:1]], wl.m2[order[:1]], s64, spec.fs, wl.f_low, wl.threshold, n_threads=1)
    t1 = time.perf_counter() - t0
    ncores = os.cpu_count() or 1
    n_s = int(max(1, min(wl.n_templates, round(cpu_seconds / max(t1, 1e-3)))))
    n_s = max(ncores, (n_s // ncores) * ncores) if n_s >= ncores else n_s
    n_s = min(n_s, wl.n_templates)
    sel = np.sort(order[:n_s])
    t0 = time.perf_counter()
    peaks, trig, ntr, used = oracle.filter_bank(wl.m1[sel], wl.m2[sel], s64, spec.fs, wl.f_low, wl.threshold)
    dt = time.perf_counter() - t0
    res = {"value": n_s / dt, "unit": UNIT, "cores": int(used), "kind": "oracle",
           "sample": "%d of %d templates (seeded), full N=2^20 segment, FP64 radix-2 FFT, %.1f s wall on %d threads"
                     % (n_s, wl.n_templates, dt, used),
           "single_thread_value": 1.0 / max(t1, 1e-9)}
    acc = None
    if gpu_check is not None:
        acc = gpu_check(s, sel, peaks)
    return res, acc


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    import workloads
    wl = workloads.scale(args.seed)
    import numpy as np
    import oracle
    oracle.build()
    spec = wl.segments[0]
    s64 = oracle.synth(spec.normals(), spec.N, spec.fs, wl.f_low, spec.injections).astype(np.float32).astype(np.float64)
    ncores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.filter_bank(wl.m1[:1], wl.m2[:1], s64, spec.fs, wl.f_low, wl.threshold, n_threads=1)
    t1 = time.perf_counter() - t0
    # each step: a bounded sample sized so that warmup + steps end within a few minutes
    budget = 150.0 / max(1, args.steps + args.warmup)
    per_step = int(max(1, min(wl.n_templates, ncores * max(1, int(budget / max(t1, 1e-3))))))
    per_step = min(per_step, wl.n_templates)
    rng = np.random.default_rng(0)
    times, used = [], 1
    for k in range(args.warmup + args.steps):
        sel = np.sort(rng.choice(wl.n_templates, per_step, replace=False))
        t0 = time.perf_counter()
        _, _, _, used = oracle.filter_bank(wl.m1[sel], wl.m2[sel], s64, spec.fs, wl.f_low, wl.threshold)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = per_step * len(times) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded coloured Gaussian noise, Eq. 2 PSD, 8 injections)",
            "config": {"workload": WORKLOAD, "seed": args.seed, "step_sample_templates": per_step},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": int(used), "kind": "oracle",
                             "sample": "%d random templates of 1024 per step, full N=2^20 segment" % per_step},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _timed_steps(torch, run, steps, warmup, flush, stream):
    """ms per step of run() over `steps` CUDA-event-timed steps after `warmup`
    untimed ones, L2 flushed before each timed step."""
    for _ in range(warmup):
        run()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        run()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev) / steps


def _capture(torch, run):
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        run()
    return g


def run_uneven(args, mf, torch, dev):
    """4096 templates (m1, m2 in [1, 34], M <= 35, each cut at its own ISCO
    frequency) over 8 segments of 2^18, 2^18, 2^19, 2^19, 2^20, 2^20, 2^21,
    2^21 samples in one mf_filter_bank call: the per-segment persistent
    launches as one CUDA graph, the per-batch launches, the fused scheduler
    (2^19 and 2^20 segments; the others per batch), per-template launches,
    and the autotuner's choice."""
    import workloads
    wl = workloads.uneven(args.seed)
    segs = [mf.Segment(mf.synth_segment(sp.normals(), sp.N, sp.fs, wl.f_low, sp.injections), sp.fs)
            for sp in wl.segments]
    bank = mf.Bank(wl.m1, wl.m2, f_low=wl.f_low)
    cap = 1 << 22
    n_seg = len(segs)
    out = (torch.empty((wl.n_templates * n_seg, 4), dtype=torch.float32, device=dev),
           torch.empty((cap, 6), dtype=torch.float32, device=dev), torch.zeros(1, dtype=torch.int64, device=dev))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def call():
        mf.filter_bank(bank, segs, wl.threshold, trig_cap=cap, out=out)

    res = {}
    # units run widest band first by default; the *_bank_order runs keep bank order for comparison
    for name, env in (("persistent_graph", {"MFGB_SCHED": "persistent"}), ("batch_graph", {"MFGB_SCHED": "batch"}),
                      ("fused_graph", {"MFGB_SCHED": "fused"}),
                      ("persistent_graph_bank_order", {"MFGB_SCHED": "persistent", "MFGB_UNIT_ORDER": "bank"}),
                      ("batch_graph_bank_order", {"MFGB_SCHED": "batch", "MFGB_UNIT_ORDER": "bank"}),
                      ("per_template_eager", {"MFGB_SCHED": "batch", "MFGB_BATCH": "1"})):
        old = {k: os.environ.get(k) for k in ("MFGB_SCHED", "MFGB_BATCH", "MFGB_UNIT_ORDER")}
        for k in old:
            os.environ.pop(k, None)
        os.environ.update(env)
        call()
        torch.cuda.synchronize()
        assert bank.check() == 0
        l0 = mf.launch_count()
        call()
        launches = mf.launch_count() - l0
        if name.endswith("graph"):
            g = _capture(torch, call)
            ms = _timed_steps(torch, g.replay, args.steps, args.warmup, flush, stream)
        else:
            ms = _timed_steps(torch, call, max(3, args.steps // 10), 1, flush, stream)
        assert bank.check() == 0
        bank.profile(True)
        call()
        torch.cuda.synchronize()
        stages = {k: round(v[0], 3) for k, v in bank.profile_read().items() if v[2] > 0}
        bank.profile(False)
        res[name] = {"ms_per_call": ms, "launches_per_call": launches, "n_trig": int(out[2].item()),
                     "stage_ms_eager": stages}
        for k, v in old.items():
            os.environ.pop(k, None)
            if v is not None:
                os.environ[k] = v
    # the autotuner's choice (scheduler, exchange budget, kernel forms of the two passes) on this call
    if not args.no_autotune and not any(os.environ.get(k) for k in ("MFGB_SCHED", "MFGB_BATCH", "MFGB_UNIT_ORDER")):
        cache = os.path.join(tempfile.gettempdir(), "mfgb_autotune_uneven.json")
        mf.autotune(bank, segs, wl.threshold, repeats=1, cache_path=cache)
        with open(cache) as fh:
            choice = json.loads(fh.readline())
        call()
        torch.cuda.synchronize()
        g = _capture(torch, call)
        ms = _timed_steps(torch, g.replay, args.steps, args.warmup, flush, stream)
        assert bank.check() == 0
        res["autotuned_graph"] = {"ms_per_call": ms, "n_trig": int(out[2].item()), "choice": choice}
    units = wl.n_templates * n_seg
    eq = wl.n_templates * sum(sp.N for sp in wl.segments) / float(1 << 20)
    best = min(res.values(), key=lambda r: r["ms_per_call"])["ms_per_call"]
    line = {"workload": "uneven", "metric": "template-segment units/s (uneven bank, mixed segment lengths)",
            "value": units / (best / 1e3), "unit": "units/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": best, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic (seeded coloured Gaussian noise, Eq. 2 PSD, 2 injections per segment)",
            "config": {"workload": "4096 templates m1,m2 in [1,34] Msun with M <= 35, 8 segments "
                                   "N = 2^18,2^18,2^19,2^19,2^20,2^20,2^21,2^21 at 4096 Hz, thr 6",
                       "l2": "flushed before every timed step (256 MiB write)",
                       "unit_order": "descending band width (f_isco) per segment; *_bank_order: bank order"},
            "equivalent_2p20_templates_per_s": eq / (best / 1e3), "schedules": res}
    print(json.dumps(line))
    return 0


def run_precision(args, mf, torch, dev):
    """The phase forms and the FFT forms (FP32 butterflies, or the first
    radix-32 stage of pass 2's rows as split FP16 / BF16 tensor-core products)
    on the 1024-template, N = 2^20 workload: speed of each (one CUDA-graph
    replay per step) and, in the CPU-baseline leg, its rho error against the
    FP64 oracle on a seeded sample of templates (full series,
    oracle-synthesised input)."""
    import numpy as np
    import workloads
    wl = workloads.scale(args.seed)
    spec = wl.segments[0]
    seg = mf.Segment(mf.synth_segment(spec.normals(), spec.N, spec.fs, wl.f_low, spec.injections), spec.fs)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    forms = {}
    cap = 1 << 22
    modes = (("fp64_anchors_fp32_taylor", mf.MF_PHASE_ANCHOR, mf.MF_FFT_FP32),
             ("fp64_per_bin", mf.MF_PHASE_FP64, mf.MF_FFT_FP32),
             ("fp32_only", mf.MF_PHASE_FP32, mf.MF_FFT_FP32),
             ("tc_fp16_split_stage", mf.MF_PHASE_ANCHOR, mf.MF_FFT_TC_FP16),
             ("tc_bf16_split_stage", mf.MF_PHASE_ANCHOR, mf.MF_FFT_TC_BF16))
    for name, mode, fmode in modes:
        bank = mf.Bank(wl.m1, wl.m2, f_low=wl.f_low, phase_mode=mode, fft_mode=fmode)
        out = (torch.empty((wl.n_templates, 4), dtype=torch.float32, device=dev),
               torch.empty((cap, 6), dtype=torch.float32, device=dev),
               torch.zeros(1, dtype=torch.int64, device=dev))

        def call():
            mf.filter_bank(bank, [seg], wl.threshold, trig_cap=cap, out=out)

        call()
        torch.cuda.synchronize()
        g = _capture(torch, call)
        ms = _timed_steps(torch, g.replay, args.steps, args.warmup, flush, stream)
        forms[name] = {"templates_per_s": wl.n_templates / (ms / 1e3), "ms_per_call": ms}
    acc = None
    if not args.no_cpu_baseline:
        acc = _precision_cpu_baseline(mf, torch, dev, wl, modes)
        for name in forms:
            forms[name].update(acc["forms"][name])
    line = {"workload": "precision", "metric": "templates/s and max rho rel err vs FP64 per phase and FFT form",
            "value": forms["fp64_anchors_fp32_taylor"]["templates_per_s"], "unit": "templates/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic (seeded coloured Gaussian noise, Eq. 2 PSD, 8 injections)",
            "config": {"workload": WORKLOAD, "error_sample": acc["sample"] if acc else None,
                       "l2": "flushed before every timed step (256 MiB write)",
                       "phase_forms": "FFT in FP32; phase from FP64 anchors + FP32 Taylor, FP64 per bin, FP32 only",
                       "fft_forms": "tc_*: FP64-anchor phase; first radix-32 stage of pass 2's 1024-point rows as "
                                    "tcgen05 products of hi + lo FP16 / BF16 splits (hi*hi + hi*lo + lo*hi), FP32 "
                                    "accumulate; all other stages FP32"},
            "forms": forms, "cpu_baseline": acc["cpu_baseline"] if acc else None}
    print(json.dumps(line))
    return 0


def _precision_cpu_baseline(mf, torch, dev, wl, modes):
    """The oracle's full rho series for 8 seeded templates (timed, host cores)
    and each phase form's error against it on the same input."""
    import numpy as np
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    oracle.build()
    spec = wl.segments[0]
    s32 = oracle.synth(spec.normals(), spec.N, spec.fs, wl.f_low, spec.injections).astype(np.float32)
    s64 = s32.astype(np.float64)
    seg = mf.Segment(torch.from_numpy(s32).to(dev), spec.fs)
    rng = np.random.default_rng(77)
    sample = np.sort(rng.choice(wl.n_templates, 8, replace=False))
    ncores = os.cpu_count() or 1
    t0 = time.perf_counter()
    st, S = oracle.data_spectrum(s64, spec.fs), oracle.psd_bins(spec.N, spec.fs)
    with ThreadPoolExecutor(max_workers=min(8, ncores)) as ex:
        ref = list(ex.map(lambda t: oracle.filter_template(float(wl.m1[t]), float(wl.m2[t]), st, S, spec.N,
                                                           spec.fs, wl.f_low)["rho"], sample))
    cpu_s = time.perf_counter() - t0
    forms = {}
    for name, mode, fmode in modes:
        b2 = mf.Bank(wl.m1[sample], wl.m2[sample], f_low=wl.f_low, phase_mode=mode, fft_mode=fmode)
        p, t, n = mf.filter_bank(b2, [seg], 0.0, trig_cap=len(sample) * spec.N)
        tr = mf.triggers_to_numpy(t, n)
        rho = tr["rho"].reshape(len(sample), spec.N).astype(np.float64)
        pk = mf.peaks_to_numpy(p)
        err = np.concatenate([np.abs(rho[i] - ref[i]) / np.maximum(ref[i], 1.0) for i in range(len(sample))])
        idx = sum(int(pk["j"][i]) == int(np.argmax(ref[i])) for i in range(len(sample)))
        mism = sum(int(np.sum((rho[i] > wl.threshold) != (ref[i] > wl.threshold))) for i in range(len(sample)))
        forms[name] = {"rho_err_max": float(err.max()), "rho_err_median": float(np.median(err)),
                       "peak_index_agree": "%d/%d" % (idx, len(sample)), "trigger_mismatches": mism}
    return {"forms": forms, "sample": "%d seeded templates, all 2^20 samples" % len(sample),
            "cpu_baseline": {"value": len(sample) / cpu_s, "unit": "templates/s", "cores": min(8, ncores),
                             "kind": "oracle", "sample": "%d templates, full N=2^20 rho series" % len(sample)}}


def run_fft(args, mf, torch, dev):
    """The batched complex FFT alone (the paper's Figs. 1-2 experiment): for
    N = 2^10 .. 2^22, batches of 2^26 points (512 MiB in, 512 MiB out) through
    mf_fft_c2c, CUDA events; the CPU-baseline leg times the oracle's FP64
    radix-2 FFT on the host cores for a bounded number of transforms."""
    import ctypes
    import numpy as np
    from paper_0906_4175_gb300 import _native
    total = 1 << 26
    x = torch.randn(total, dtype=torch.complex64, device=dev)
    y = torch.empty_like(x)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    peak, peak_kind = _hbm_peak()
    rows = {}
    for lg in range(10, 23):
        N = 1 << lg
        batch = total // N

        def call():
            _native.check(_native.lib().mf_fft_c2c(x.data_ptr(), y.data_ptr(), N, batch, -1,
                                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))

        l0 = mf.launch_count()
        call()
        launches = mf.launch_count() - l0
        ms = _timed_steps(torch, call, max(3, args.steps // 10), args.warmup, flush, torch.cuda.current_stream())
        gbs = 16.0 * total / (ms / 1e3) / 1e9
        rows["2^%d" % lg] = {"batch": batch, "ms": ms, "transforms_per_s": batch / (ms / 1e3),
                             "gflops": 5.0 * N * lg * batch / (ms / 1e3) / 1e9, "algorithmic_gbs": gbs,
                             "hbm_frac": gbs / peak, "launches": launches}
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        from concurrent.futures import ThreadPoolExecutor
        oracle.build()
        ncores = os.cpu_count() or 1
        cpu = {}
        for lg in (10, 14, 18, 20, 22):
            N = 1 << lg
            n_t = max(ncores, int(min(256, (1 << 22) // N)) // ncores * ncores)
            xs = [np.random.default_rng(i).standard_normal(N) + 0j for i in range(n_t)]
            t0 = time.perf_counter()
            with ThreadPoolExecutor(max_workers=ncores) as ex:
                list(ex.map(lambda v: oracle.fft(v, -1), xs))
            dt = time.perf_counter() - t0
            cpu["2^%d" % lg] = {"transforms_per_s": n_t / dt, "gflops": 5.0 * N * lg * n_t / dt / 1e9,
                                "transforms": n_t}
        cpu = {"kind": "oracle", "cores": ncores, "unit": "transforms/s", "per_N": cpu,
               "sample": "FP64 radix-2 oracle FFT, forward, one transform per thread at a time"}
    r20 = rows["2^20"]
    line = {"workload": "fft", "metric": "batched complex FFT transforms/s (FP32, forward), 2^26 points per call",
            "value": r20["transforms_per_s"], "unit": "transforms/s at N=2^20", "n_gpus": 1, "higher_is_better": True,
            "dtype": "c64", "data": "synthetic (normal complex samples)",
            "config": {"workload": "batches of 2^26 complex points, N = 2^10..2^22 (batch = 2^26 / N)",
                       "l2": "input and output 512 MiB each (larger than L2), L2 flushed before every timed call"},
            "roofline": {"bound": "hbm", "kernel": "fft_c2c (both passes)", "achieved": r20["algorithmic_gbs"],
                         "peak": peak, "unit": "GB/s", "frac": r20["hbm_frac"], "peak_kind": peak_kind,
                         "traffic": None, "algorithmic_bytes": "16 per point (read x, write y)"},
            "per_N": rows, "cpu_baseline": cpu}
    print(json.dumps(line))
    return 0


def run_events(args, mf, torch, dev):
    """The search tail on the bench workload: filter (1024 templates, 2^20
    samples, threshold 6) -> events (mf_cluster_triggers, 1 s window) -> chi^2
    of Eq. (5) at every event (mf_chisq_points, p = 16); CUDA events per
    stage over the timed steps."""
    import numpy as np
    import workloads
    wl = workloads.scale(args.seed)
    spec = wl.segments[0]
    seg = mf.Segment(mf.synth_segment(spec.normals(), spec.N, spec.fs, wl.f_low, spec.injections), spec.fs)
    bank = mf.Bank(wl.m1, wl.m2, f_low=wl.f_low)
    cap = 1 << 22
    out = (torch.empty((wl.n_templates, 4), dtype=torch.float32, device=dev),
           torch.empty((cap, 6), dtype=torch.float32, device=dev), torch.zeros(1, dtype=torch.int64, device=dev))
    W = int(spec.fs)                      # 1 s
    ev_cap = 1 << 16
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream()
    steps = max(3, args.steps // 10)
    times = {"filter": 0.0, "cluster": 0.0, "chisq": 0.0}
    n_ev = 0
    chi = None
    for k in range(args.warmup + steps):
        flush.fill_(k & 0xFF)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(st)
        mf.filter_bank(bank, [seg], wl.threshold, trig_cap=cap, out=out)
        e[1].record(st)
        ev, n_e = mf.cluster_triggers(out[1], out[2], wl.n_templates, 1, spec.N, W, ev_cap=ev_cap)
        e[2].record(st)
        n_ev = min(int(n_e.item()), ev_cap)    # host read between stages (the event count sizes the chi^2 call)
        e2 = torch.cuda.Event(enable_timing=True)
        e2.record(st)
        chi = mf.chisq_points(bank, [seg], ev[:n_ev], p=16)
        e[3].record(st)
        torch.cuda.synchronize()
        if k >= args.warmup:
            times["filter"] += e[0].elapsed_time(e[1])
            times["cluster"] += e[1].elapsed_time(e[2])
            times["chisq"] += e2.elapsed_time(e[3])
    evs = mf.events_to_numpy(ev, n_e)
    chi = chi.cpu().numpy()
    order = np.argsort(-evs["rho"])[:8]
    line = {"workload": "events", "metric": "events/s through filter -> clustering -> per-event chi^2",
            "value": n_ev / ((times["filter"] + times["cluster"] + times["chisq"]) / steps / 1e3), "unit": "events/s",
            "n_gpus": 1, "steps": steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic (seeded coloured Gaussian noise, Eq. 2 PSD, 8 injections)",
            "config": {"workload": WORKLOAD, "window_samples": W, "p": 16, "n_trig": int(out[2].item()),
                       "n_events": n_ev, "l2": "flushed before every step"},
            "ms_per_step": {k: v / steps for k, v in times.items()},
            "loudest_events": [{"tmpl": int(evs["tmpl"][i]), "j": int(evs["j"][i]), "rho": float(evs["rho"][i]),
                                "chisq": float(chi[i]), "n_trig": int(evs["n_trig"][i]),
                                "n_tmpl": int(evs["n_tmpl"][i])} for i in order],
            "injections_j": [int((spec.N - int(x["j0"])) % spec.N) for x in spec.injections]}
    print(json.dumps(line))
    return 0


MSUN_S = 4.925490947e-6


def _band_bins(m1, m2, N, fs, f_low):
    """In-band bin counts K_t (Sec. 1.1 band rule: f_cut = min(f_isco, fs/2),
    k_lo = ceil(f_low/df), k_hi = min(floor(f_cut/df) + 1, N/2)), for the
    algorithmic-byte models."""
    import numpy as np
    fisco = 1.0 / (6.0 * np.sqrt(6.0) * np.pi * (np.asarray(m1) + np.asarray(m2)) * MSUN_S)
    fc = np.minimum(fisco, 0.5 * fs)
    lo = np.maximum(1, np.ceil(f_low * N / fs)).astype(np.int64)
    hi = np.minimum(np.floor(fc * N / fs).astype(np.int64) + 1, N // 2)
    return np.maximum(hi - lo, 0)


def run_chisq(args, mf, torch, dev):
    """Eq. (5) chi^2 series (p = 16 sub-bands, every one of the 2^20 samples)
    for the 64 loudest templates of the 1024-template bench workload: one
    mf_chisq_series call per step, CUDA events, L2 flushed.  The CPU-baseline
    leg times the FP64 oracle on a bounded template sample and measures the
    GPU's chi^2 error on the same (oracle-synthesised) input."""
    import numpy as np
    import workloads
    wl = workloads.scale(args.seed)
    spec = wl.segments[0]
    N = spec.N
    s_dev = mf.synth_segment(spec.normals(), N, spec.fs, wl.f_low, spec.injections)
    seg = mf.Segment(s_dev, spec.fs)
    bank = mf.Bank(wl.m1, wl.m2, f_low=wl.f_low)
    pk = mf.peaks_to_numpy(mf.filter_bank(bank, [seg], wl.threshold, trig_cap=1 << 20)[0])
    n, p = 64, 16
    sel = np.sort(np.argsort(-pk["rho"])[:n]).astype(np.int32)
    tmpl = torch.tensor(sel, device=dev)
    chi = torch.empty((n, N), dtype=torch.float32, device=dev)
    edges = torch.empty((n, p + 1), dtype=torch.int64, device=dev)
    import ctypes
    from paper_0906_4175_gb300 import _native

    def call(segment=seg):
        _native.check(_native.lib().mf_chisq_series(bank.handle, segment.handle, tmpl.data_ptr(), n, p,
                                                    chi.data_ptr(), edges.data_ptr(),
                                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    l0 = mf.launch_count()
    call()
    launches = mf.launch_count() - l0
    steps = max(3, args.steps // 10)
    ms = _timed_steps(torch, call, steps, args.warmup, flush, torch.cuda.current_stream())
    # algorithmic bytes per template (model): the W band once; anchors and the
    # exchange write + read for each sub-band and the full band; one write of
    # chi^2 (at N = 2^20 the rows kernel sums every sub-band of a row in
    # registers: no accumulator in memory)
    K = _band_bins(wl.m1[sel], wl.m2[sel], N, spec.fs, wl.f_low).astype(np.float64)
    n_anc = K / 128.0
    per_t = 8.0 * K + (p + 1) * (20.0 * n_anc + 16.0 * N) + 4.0 * N
    achieved = float(per_t.sum()) / (ms / 1e3) / 1e9
    peak, peak_kind = _hbm_peak()
    cpu = None
    err = None
    if not args.no_cpu_baseline:
        cpu, err = _chisq_cpu_baseline(mf, torch, dev, wl, bank, sel, p, call, chi)
    line = {"workload": "chisq", "metric": "templates/s of the Eq. (5) chi^2 series at N=2^20, p=16",
            "value": n / (ms / 1e3), "unit": "templates/s", "n_gpus": 1, "steps": steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "dtype": "f32 (FP64 anchors, FP64 band edges)",
            "data": "synthetic (seeded coloured Gaussian noise of the bench workload, 8 injections)",
            "config": {"workload": "64 loudest of the 1024-template bench bank, 1 segment N=2^20 at 4096 Hz, "
                                   "p = 16 sub-bands, every sample", "l2": "flushed before every timed step"},
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "traffic": None,
                         "model_bytes_per_template": float(per_t.mean())},
            "chisq_err": err, "cpu_baseline": cpu}
    print(json.dumps(line))
    return 0


def _chisq_cpu_baseline(mf, torch, dev, wl, bank, sel, p, call, chi):
    """The oracle's chi^2 series on a bounded sample of the templates (all
    host cores), and the GPU's error on the same oracle-synthesised input."""
    import numpy as np
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    oracle.build()
    spec = wl.segments[0]
    N = spec.N
    s32 = oracle.synth(spec.normals(), N, spec.fs, wl.f_low, spec.injections).astype(np.float32)
    st, S = oracle.data_spectrum(s32.astype(np.float64), spec.fs), oracle.psd_bins(N, spec.fs)
    ncores = os.cpu_count() or 1
    m_cpu = min(len(sel), max(ncores, 16))
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=ncores) as ex:
        refs = list(ex.map(lambda t: oracle.chisq_series(float(wl.m1[t]), float(wl.m2[t]), st, S, N, spec.fs,
                                                         wl.f_low, p), sel[:m_cpu]))
    cpu_s = time.perf_counter() - t0
    seg2 = mf.Segment(torch.from_numpy(s32).to(dev), spec.fs)
    call(seg2)
    got = chi[:m_cpu].cpu().numpy().astype(np.float64)
    rel = max(float(np.max(np.abs(got[i] - r["chisq"]) / (r["chisq"] + 2 * r["rho"] ** 2 + 1.0)))
              for i, r in enumerate(refs))
    cpu = {"value": m_cpu / cpu_s, "unit": "templates/s", "cores": ncores, "kind": "oracle",
           "sample": "%d of the 64 templates, full N=2^20 series, p=16, %.1f s wall" % (m_cpu, cpu_s)}
    err = {"max": rel, "measure": "|chi2_gpu - chi2_fp64| / (chi2 + 2 rho^2 + 1), all samples of the sample"}
    return cpu, err


def _ascend(mf, torch, seg, theta0, steps, rel_m=5e-3, step_t=2e-4, row_seg=None):
    """Adam ascent of rho^2 on (m1, m2, t) through RefineFn (x = theta / scale,
    unit learning rate); best point per row over steps + 1 evaluations."""
    th0 = theta0
    sc = torch.stack([rel_m * th0[:, 0], rel_m * th0[:, 1], torch.full_like(th0[:, 2], step_t)], dim=1)
    x = (th0 / sc).clone().requires_grad_(True)
    opt = torch.optim.Adam([x], lr=1.0)
    best_th = th0.clone()
    best_J = torch.full((th0.shape[0],), -1.0, dtype=torch.float64, device=th0.device)
    for k in range(steps + 1):
        th = x * sc
        J = mf.RefineFn.apply(th, seg, None, 40.0, row_seg)
        with torch.no_grad():
            better = J > best_J
            best_J = torch.where(better, J.detach(), best_J)
            best_th = torch.where(better[:, None], th.detach(), best_th)
        if k == steps:
            break
        opt.zero_grad()
        (-J.sum()).backward()
        opt.step()
    return best_th, best_J


def _ascend_graph(mf, torch, segs, theta0, steps, row_seg, rel_m=5e-3, step_t=2e-4):
    """The ascent of _ascend (every trigger of every segment, one
    objective+gradient launch per evaluation) captured once as a CUDA graph:
    autograd backward and a capturable Adam step included.  Returns
    (run, best_th, best_J); run() restarts from theta0 and replays."""
    th0 = theta0
    sc = torch.stack([rel_m * th0[:, 0], rel_m * th0[:, 1], torch.full_like(th0[:, 2], step_t)], dim=1)
    x0 = th0 / sc
    x = x0.clone().requires_grad_(True)
    opt = torch.optim.Adam([x], lr=1.0, capturable=True)
    best_th = th0.clone()
    best_J = torch.full((th0.shape[0],), -1.0, dtype=torch.float64, device=th0.device)

    def body():
        for k in range(steps + 1):
            th = x * sc
            J = mf.RefineFn.apply(th, segs, None, 40.0, row_seg)
            with torch.no_grad():
                better = J > best_J
                best_J.copy_(torch.where(better, J.detach(), best_J))
                best_th.copy_(torch.where(better[:, None], th.detach(), best_th))
            if k == steps:
                break
            opt.zero_grad(set_to_none=False)
            (-J.sum()).backward()
            opt.step()

    def reset():
        with torch.no_grad():
            x.copy_(x0)
            best_J.fill_(-1.0)
            best_th.copy_(th0)
            for st in opt.state.values():
                for v in st.values():
                    if torch.is_tensor(v):
                        v.zero_()

    side = torch.cuda.Stream()   # warm-up (optimiser state, gradient buffer) off the capture
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        body()
    torch.cuda.current_stream().wait_stream(side)
    reset()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        body()

    def run():
        reset()
        g.replay()

    return run, best_th, best_J


def run_refine(args, mf, torch, dev):
    """Coarse triggers of the 210-template 1-Msun bank on 32 segments of 2^20
    samples with 8 injections each (256), then 20 Adam steps of rho^2 on
    (m1, m2, t) per trigger through RefineFn; reports the refinement
    throughput, the SNR gain and the recovered-mass error."""
    import numpy as np
    import workloads
    wl = workloads.refine_bank(args.seed)
    fs = wl.segments[0].fs
    N = wl.segments[0].N
    segs = [mf.Segment(mf.synth_segment(sp.normals(), sp.N, sp.fs, wl.f_low, sp.injections), sp.fs)
            for sp in wl.segments]
    bank = mf.Bank(wl.m1, wl.m2, f_low=wl.f_low)
    cap = 1 << 24
    t0 = time.perf_counter()
    p, t, n = mf.filter_bank(bank, segs, 4.0, trig_cap=cap)
    torch.cuda.synchronize()
    coarse_s = time.perf_counter() - t0
    assert bank.check() == 0
    tr = mf.triggers_to_numpy(t, n)
    starts, truth, rho0 = [], [], []
    for si, sp in enumerate(wl.segments):
        ts = tr[tr["seg"] == si]
        th, tru, r0 = [], [], []
        for inj in sp.injections:
            jc = (N - int(inj["j0"])) % N
            d = np.abs(((ts["j"].astype(np.int64) - jc + N // 2) % N) - N // 2)
            near = ts[d < int(2.0 * fs)]
            if near.size == 0:
                continue
            b = near[np.argmax(near["rho"])]
            th.append([wl.m1[int(b["tmpl"])], wl.m2[int(b["tmpl"])], int(b["j"]) / fs])
            tru.append([inj["m1"], inj["m2"], jc / fs])
            r0.append(float(b["rho"]))
        starts.append(torch.tensor(th, dtype=torch.float64, device=dev))
        truth.append(np.array(tru))
        rho0.append(np.array(r0))
    n_trig = sum(int(x.shape[0]) for x in starts)
    row_seg = torch.tensor(np.concatenate([np.full(int(x.shape[0]), si, dtype=np.int32)
                                           for si, x in enumerate(starts)]), device=dev)
    steps = 20
    # warm-up of both forms (module loading, allocator pools, optimiser state)
    _ascend(mf, torch, segs, torch.cat(starts), 2, row_seg=row_seg)
    _ascend(mf, torch, segs[0], starts[0], 2)
    # timed: the ascent of every segment's triggers (steps + 1 objective+gradient evaluations each),
    # captured once as a CUDA graph and replayed
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    run, th_all, J_all = _ascend_graph(mf, torch, segs, torch.cat(starts), steps, row_seg)
    run()
    torch.cuda.synchronize()
    ms_g = []
    for _ in range(5):
        ev0.record()
        run()
        ev1.record()
        torch.cuda.synchronize()
        ms_g.append(ev0.elapsed_time(ev1))
    ms = statistics.median(ms_g)
    # the same ascent eager (one refine launch pair per step, optimiser kernels launched from Python)
    ev0.record()
    th_e, J_e = _ascend(mf, torch, segs, torch.cat(starts), steps, row_seg=row_seg)
    ev1.record()
    torch.cuda.synchronize()
    ms_eager = ev0.elapsed_time(ev1)
    agree = float(torch.max(torch.abs(J_e - J_all) / torch.clamp(J_e, min=1.0)).item())
    # the objective+gradient launches alone over the same rows (no optimiser), per evaluation
    ev0.record()
    for _ in range(steps + 1):
        mf.refine(segs, th_all, row_seg=row_seg)
    ev1.record()
    torch.cuda.synchronize()
    ms_kernels = ev0.elapsed_time(ev1)
    # per-segment call loop (one refine launch pair per segment and step), for comparison
    ev0.record()
    for si in range(len(segs)):
        _ascend(mf, torch, segs[si], starts[si], steps)
    ev1.record()
    torch.cuda.synchronize()
    ms_per_seg = ev0.elapsed_time(ev1)
    results, o = [], 0
    for si in range(len(segs)):
        k = int(starts[si].shape[0])
        results.append((th_all[o:o + k], J_all[o:o + k]))
        o += k
    gain, dmc, dm = [], [], []
    for si, (th, J) in enumerate(results):
        thn = th.cpu().numpy()
        rho = np.sqrt(J.cpu().numpy())
        gain.extend(list(rho / rho0[si]))
        tru = truth[si]
        mc = lambda a, b: (a * b) ** 0.6 / (a + b) ** 0.2
        for k in range(thn.shape[0]):
            a, b = sorted(thn[k, :2], reverse=True)
            ta, tb = sorted(tru[k, :2], reverse=True)
            dmc.append(abs(mc(a, b) - mc(ta, tb)) / mc(ta, tb))
            dm.append(max(abs(a - ta), abs(b - tb)))
        # starting-point errors for comparison
    dmc0, dm0 = [], []
    for si in range(len(segs)):
        s0 = starts[si].cpu().numpy()
        for k in range(s0.shape[0]):
            a, b = sorted(s0[k, :2], reverse=True)
            ta, tb = sorted(truth[si][k, :2], reverse=True)
            mcf = lambda x, y: (x * y) ** 0.6 / (x + y) ** 0.2
            dmc0.append(abs(mcf(a, b) - mcf(ta, tb)) / mcf(ta, tb))
            dm0.append(max(abs(a - ta), abs(b - tb)))
    # against the injection truth: rho^2 of the exact template at the exact coalescence time
    # (the best any refinement of that trigger can reach, noise aside), per trigger
    th_true = torch.tensor(np.concatenate(truth), dtype=torch.float64, device=dev)
    J_true, _ = mf.refine(segs, th_true, row_seg=row_seg)
    rho_true = np.sqrt(np.maximum(J_true.cpu().numpy(), 0.0))
    rho_ref = np.sqrt(np.maximum(J_all.cpu().numpy(), 0.0))
    rho_start = np.concatenate(rho0)
    frac_ref, frac_start = rho_ref / rho_true, rho_start / rho_true
    q = lambda a: {"median": float(np.median(a)), "p10": float(np.percentile(a, 10)),
                   "min": float(np.min(a)), "max": float(np.max(a))}
    evals = n_trig * (steps + 1)
    line = {"workload": "refine", "metric": "trigger objective+gradient evaluations/s (Adam ascent of rho^2)",
            "value": evals / (ms / 1e3), "unit": "evaluations/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "f64 anchor phase + f32 Taylor, f32 sums", "ms_total": ms,
            "gpu_launches": 3 * (steps + 1),
            "ascent": "CUDA graph of the whole ascent (refine launches, autograd backward, capturable Adam), "
                      "median of 5 replays",
            "ms_total_eager": ms_eager, "graph_vs_eager_max_rel_diff_rho2": agree,
            "ms_total_per_segment_calls": ms_per_seg, "ms_refine_launches_only": ms_kernels,
            "data": "synthetic (seeded coloured Gaussian noise, 8 injections per segment, m in [1, 20], SNR 8-15)",
            "config": {"workload": "210-template 1-Msun bank (m1 >= m2 in 1..20), 32 segments N=2^20 at 4096 Hz, "
                                   "256 injections; coarse threshold 4; %d Adam steps, steps rel 5e-3 m and 2e-4 s"
                                   % steps,
                       "coarse_filter_s": coarse_s},
            "triggers": n_trig,
            "snr_gain": {"median": float(np.median(gain)), "min": float(np.min(gain)),
                         "max": float(np.max(gain))},
            "chirp_mass_rel_err": {"coarse_median": float(np.median(dmc0)), "refined_median": float(np.median(dmc))},
            "component_mass_err_msun": {"coarse_median": float(np.median(dm0)), "refined_median": float(np.median(dm))},
            "vs_truth": {"note": "rho at the injected (m1, m2, t_c) with the exact template (direct Eq. 1 sum); "
                                 "fractions of it reached by the coarse trigger and by the refined point",
                         "rho_true": q(rho_true), "coarse_fraction": q(frac_start), "refined_fraction": q(frac_ref),
                         "refined_within_1pct_of_truth": float(np.mean(frac_ref >= 0.99)),
                         "coarse_within_1pct_of_truth": float(np.mean(frac_start >= 0.99))}}
    print(json.dumps(line))
    return 0


def main():
    args = _args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "scale":
        if args.warmup < 3:
            args.warmup = 3
        import torch
        torch.cuda.set_device(0)
        from paper_0906_4175_gb300 import build as _b
        _b.build()
        import paper_0906_4175_gb300 as mf
        fn = {"uneven": run_uneven, "precision": run_precision, "refine": run_refine,
              "chisq": run_chisq, "fft": run_fft, "events": run_events}[args.workload]
        return fn(args, mf, torch, torch.device("cuda", 0))
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local = _dist()
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = dist_mod
    from paper_0906_4175_gb300 import build as _b
    _b.build()
    import paper_0906_4175_gb300 as mf
    import workloads

    wl = workloads.scale(seed=args.seed + rank)
    if args.templates > 0:
        wl.m1, wl.m2 = wl.m1[:args.templates], wl.m2[:args.templates]
    spec = wl.segments[0]
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    # inputs: seeded coloured noise + injections synthesised on the device by the library
    s_dev = mf.synth_segment(spec.normals(), spec.N, spec.fs, wl.f_low, spec.injections)
    fft_mode = {"fp32": mf.MF_FFT_FP32, "tc_fp16": mf.MF_FFT_TC_FP16, "tc_bf16": mf.MF_FFT_TC_BF16}[args.fft_mode]
    bank = mf.Bank(wl.m1, wl.m2, f_low=wl.f_low, fft_mode=fft_mode)
    cap = 1 << 22
    outb = (torch.empty((wl.n_templates, 4), dtype=torch.float32, device=dev),
            torch.empty((cap, 6), dtype=torch.float32, device=dev),
            torch.zeros(1, dtype=torch.int64, device=dev))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    # one segment handle: every step re-conditions the resident samples into it
    seg = mf.Segment(s_dev, spec.fs)
    seg.set_conditioning(args.conditioning)
    seg.refresh(s_dev)

    def step():
        seg.refresh(s_dev)
        mf.filter_bank(bank, [seg], wl.threshold, trig_cap=cap, out=outb)

    schedule = {"scheduler": "default"}
    if not args.no_autotune:
        cache = os.path.join(tempfile.gettempdir(), "mfgb_autotune_%d.json" % rank)
        mf.autotune(bank, [seg], wl.threshold, repeats=2, cache_path=cache)
        with open(cache) as fh:
            schedule = json.load(fh)
        os.unlink(cache)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert bank.check() == 0
    n_trig = int(outb[2].item())

    graph = None
    launches_per_step = None
    if not args.eager:
        # one CUDA graph per step: refresh + filter, replayed on the current stream
        l0 = mf.launch_count()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        launches_per_step = mf.launch_count() - l0
        for _ in range(args.warmup):
            graph.replay()
        torch.cuda.synchronize()
        assert bank.check() == 0
        assert int(outb[2].item()) == n_trig

    step_medians = []

    def timed(run, profile):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        if profile:
            bank.profile(True)
        l0 = mf.launch_count()
        w0 = time.perf_counter()
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            run()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        w = time.perf_counter() - w0
        n_l = mf.launch_count() - l0
        pr = None
        if profile:
            pr = bank.profile_read()
            bank.profile(False)
        per = [a.elapsed_time(b) for a, b in ev]
        step_medians.append(statistics.median(per))
        return sum(per), w, n_l, pr

    sampler = ClockSampler(local)
    sampler.mark_begin()
    # eager steps with per-stage CUDA events: the stage shares and the roofline
    eager_ms, eager_wall, eager_launches, prof = timed(step, True)
    if graph is not None:
        tot_ms, wall, _, _ = timed(graph.replay, False)
        launches = launches_per_step * args.steps
    else:
        tot_ms, wall, launches = eager_ms, eager_wall, eager_launches
    sampler.mark_end()
    clocks = sampler.stop()
    assert bank.check() == 0
    if dist:
        tot_ms = max_over_ranks(tot_ms, dist, dev)
        dist.barrier()
    value = whole_job_rate(world, wl.n_templates * args.steps, tot_ms)

    # roofline of the dominant kernel (largest share of the filter's device time)
    stages = {k: v for k, v in prof.items() if v[2] > 0}
    dom = max(stages, key=lambda k: stages[k][0])
    d_ms, d_bytes, d_n = stages[dom]
    peak, peak_kind = _hbm_peak()
    achieved = d_bytes / (d_ms / 1e3) / 1e9
    traffic, traffic_tmpl = _ncu_traffic(dom)
    tmpl_per_launch = wl.n_templates * args.steps / max(1, d_n) if dom in ("pass1", "pass2", "anchors", "fused") else None
    if traffic is not None and traffic_tmpl and tmpl_per_launch:
        traffic *= tmpl_per_launch / traffic_tmpl   # the exchange traffic grows with the templates per launch
    roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
            "timed_on": "the eager steps (same workload, per-stage CUDA events on the launching stream)",
            "effective": bool(traffic is not None and traffic < d_bytes / max(1, d_n)),
            "algorithmic_bytes_per_launch": d_bytes / max(1, d_n), "launches": d_n,
            "avg_launch_ms": d_ms / max(1, d_n), "templates_per_launch": tmpl_per_launch,
            "stage_share": {k: v[0] / sum(x[0] for x in stages.values()) for k, v in stages.items()}}
    # whole-path roofline with the per-template model B = 8 K + 16 N + 24 n_trig
    b_total = sum(v[1] for k, v in prof.items() if k in ("pass1", "pass2", "fused")) + 24.0 * n_trig * args.steps
    path = {"model_bytes_per_template": b_total / (wl.n_templates * args.steps),
            "achieved_gbs": b_total / (tot_ms / 1e3) / 1e9, "frac": b_total / (tot_ms / 1e3) / 1e9 / peak}

    # segment conditioning timed on its own, and the filter without it (the
    # step above includes mf_segment_refresh, so `value` is the inclusive rate)
    conditioning = None
    if graph is not None and rank == 0:
        g_ref = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_ref):
            seg.refresh(s_dev)
        g_fil = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_fil):
            mf.filter_bank(bank, [seg], wl.threshold, trig_cap=cap, out=outb)
        ms_ref = _timed_steps(torch, g_ref.replay, args.steps, args.warmup, flush, stream)
        ms_fil = _timed_steps(torch, g_fil.replay, args.steps, args.warmup, flush, stream)
        ups = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            s_new = mf.Segment(s_dev, spec.fs)   # mf_segment_upload: allocation + conditioning
            e1.record(stream)
            torch.cuda.synchronize()
            ups.append(e0.elapsed_time(e1))
            del s_new
        assert bank.check() == 0
        conditioning = {"segment_upload_ms": statistics.median(ups), "segment_refresh_ms": ms_ref,
                        "filter_only_ms": ms_fil, "filter_only_templates_per_s": wl.n_templates / (ms_fil / 1e3),
                        "note": "value includes mf_segment_refresh in every step; filter_only excludes it "
                                "(each timed on its own CUDA graph, L2 flushed per step)"}

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    s_host = torch.empty(spec.N, dtype=torch.float32, pin_memory=True)
    s_host.copy_(s_dev.cpu())
    peaks_h = torch.empty((wl.n_templates, 4), dtype=torch.float32, pin_memory=True)
    ntr_h = torch.empty(1, dtype=torch.int64, pin_memory=True)
    trig_h = torch.empty((cap, 6), dtype=torch.float32, pin_memory=True)
    # Two forms of the same user loop.  eager: mf_segment_refresh from the
    # pinned host samples (its H2D copy inside) and an eager mf_filter_bank.
    # graph: the H2D copy of the samples into a device staging buffer, then one
    # CUDA-graph replay of mf_segment_refresh (device samples) + mf_filter_bank,
    # the pattern the boundary documents for a fixed-shape search.  Both read
    # back peaks, n_trig and the triggers every step.
    s_stage = torch.empty(spec.N, dtype=torch.float32, device=dev)
    g_e2e = None
    if graph is not None:
        s_stage.copy_(s_dev)
        g_e2e = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_e2e):
            seg.refresh(s_stage)
            mf.filter_bank(bank, [seg], wl.threshold, trig_cap=cap, out=outb)

    def e2e_run(form):
        d2h, ms = [], []
        for k in range(args.e2e_steps + 2 if args.e2e_steps > 0 else 0):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if form == "graph":
                s_stage.copy_(s_host, non_blocking=True)   # H2D of the step's samples (pinned)
                g_e2e.replay()
            else:
                seg.refresh(s_host.numpy())     # H2D of the step's samples (pinned) + conditioning
                mf.filter_bank(bank, [seg], wl.threshold, trig_cap=cap, out=outb)
            peaks_h.copy_(outb[0], non_blocking=True)
            ntr_h.copy_(outb[2], non_blocking=True)
            torch.cuda.synchronize()
            n = min(int(ntr_h.item()), cap)
            trig_h[:n].copy_(outb[1][:n], non_blocking=True)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            if k >= 2:
                ms.append(dt * 1e3)
                d2h.append(peaks_h.numel() * 4 + 8 + n * 24)
        tot = sum(ms) if ms else float("nan")
        if dist:
            tot = max_over_ranks(tot, dist, dev)
        rate = whole_job_rate(world, wl.n_templates * len(ms), tot) if ms else None
        return rate, (int(statistics.mean(d2h)) if d2h else 0)

    # Pipelined form of the graph loop, as a streaming search runs it: two
    # staging buffers, two output sets and two graphs, so that the H2D copy of
    # step k + 1's samples and the D2H reads of step k - 1's results (on a copy
    # stream) overlap the replay of step k.  Every step still copies its own
    # samples in and its own peaks, n_trig and triggers out inside the timed
    # region; the rate is steps x templates over the wall time of the loop.
    def e2e_pipelined():
        if g_e2e is None or args.e2e_steps <= 0:
            return None, 0
        stage = [s_stage, torch.empty_like(s_stage)]
        outs = [outb, tuple(torch.empty_like(x) for x in outb)]
        ph = [peaks_h, torch.empty_like(peaks_h).pin_memory()]
        nh = [ntr_h, torch.empty_like(ntr_h).pin_memory()]
        th = [trig_h, torch.empty_like(trig_h).pin_memory()]
        graphs = []
        for i in range(2):
            stage[i].copy_(s_dev)
            gi = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gi):
                seg.refresh(stage[i])
                mf.filter_bank(bank, [seg], wl.threshold, trig_cap=cap, out=outs[i])
            graphs.append(gi)
        comp = torch.cuda.current_stream()
        cp = torch.cuda.Stream()
        ev_h2d = [torch.cuda.Event() for _ in range(2)]
        ev_done = [torch.cuda.Event() for _ in range(2)]
        ev_d2h = [torch.cuda.Event() for _ in range(2)]
        ev_peaks = torch.cuda.Event()

        def run(K):
            d2h = []
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(cp):
                stage[0].copy_(s_host, non_blocking=True)
                ev_h2d[0].record(cp)
            for k in range(K + 1):
                if k < K:
                    i = k % 2
                    comp.wait_event(ev_h2d[i])
                    if k >= 2:
                        comp.wait_event(ev_d2h[i])   # step k - 2's outputs are read back
                    graphs[i].replay()
                    ev_done[i].record(comp)
                    if k + 1 < K:
                        j = (k + 1) % 2
                        with torch.cuda.stream(cp):
                            if k >= 1:
                                cp.wait_event(ev_done[j])   # step k - 1 has read its staging buffer
                            stage[j].copy_(s_host, non_blocking=True)
                            ev_h2d[j].record(cp)
                if k >= 1:   # the results of step k - 1, while step k runs
                    i = (k - 1) % 2
                    with torch.cuda.stream(cp):
                        cp.wait_event(ev_done[i])
                        ph[i].copy_(outs[i][0], non_blocking=True)
                        nh[i].copy_(outs[i][2], non_blocking=True)
                        ev_peaks.record(cp)
                    ev_peaks.synchronize()
                    n = min(int(nh[i].item()), cap)
                    with torch.cuda.stream(cp):
                        th[i][:n].copy_(outs[i][1][:n], non_blocking=True)
                        ev_d2h[i].record(cp)
                    ev_d2h[i].synchronize()
                    d2h.append(ph[i].numel() * 4 + 8 + n * 24)
            torch.cuda.synchronize()
            return time.perf_counter() - t0, d2h

        run(2)   # warm-up
        tot, d2h = run(args.e2e_steps)
        assert int(nh[0].item()) == int(nh[1].item())   # the same samples every step
        tot_ms = tot * 1e3
        if dist:
            tot_ms = max_over_ranks(tot_ms, dist, dev)
        return whole_job_rate(world, wl.n_templates * args.e2e_steps, tot_ms), int(statistics.mean(d2h))

    e2e_eager, d2h_bytes = e2e_run("eager")
    e2e_graph = None
    if g_e2e is not None:
        e2e_graph, d2h_bytes = e2e_run("graph")
        assert bank.check() == 0
    e2e_pipe, d2h_pipe = e2e_pipelined()
    if e2e_pipe is not None:
        assert bank.check() == 0
    best = e2e_pipe if e2e_pipe is not None else (e2e_graph if e2e_graph is not None else e2e_eager)
    e2e = {"value": best, "unit": UNIT,
           "h2d_bytes_per_step": spec.N * 4, "d2h_bytes_per_step": d2h_pipe if e2e_pipe is not None else d2h_bytes,
           "form": "graph, pipelined" if e2e_pipe is not None else ("graph" if e2e_graph is not None else "eager"),
           "includes": ("H2D of the pinned host samples, mf_segment_refresh + mf_filter_bank (one CUDA-graph replay "
                        "in the graph forms, eager calls in the eager form), D2H of peaks + n_trig + triggers; "
                        "pipelined: step k + 1's H2D and step k - 1's D2H overlap step k's replay"),
           "graph_value": e2e_graph, "eager_value": e2e_eager}

    cpu = None
    acc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        def gpu_check(s32, sel, opeaks):
            b2 = mf.Bank(wl.m1[sel], wl.m2[sel], f_low=wl.f_low, fft_mode=fft_mode)
            sg = mf.Segment(torch.from_numpy(s32).to(dev), spec.fs)
            p, _, _ = mf.filter_bank(b2, [sg], wl.threshold, trig_cap=1 << 16)
            pk = mf.peaks_to_numpy(p)
            err = np.abs(pk["rho"].astype(np.float64) - opeaks["rho"]) / np.maximum(opeaks["rho"], 1.0)
            # full rho series of two templates (threshold 0 returns every sample)
            b3 = mf.Bank(wl.m1[sel[:2]], wl.m2[sel[:2]], f_low=wl.f_low, fft_mode=fft_mode)
            p3, t3, n3 = mf.filter_bank(b3, [sg], 0.0, trig_cap=2 * spec.N)
            tr = mf.triggers_to_numpy(t3, n3)
            import oracle
            S = oracle.psd_bins(spec.N, spec.fs)
            st = oracle.data_spectrum(s32.astype(np.float64), spec.fs)
            series = 0.0
            for i in range(2):
                ref = oracle.filter_template(float(wl.m1[sel[i]]), float(wl.m2[sel[i]]), st, S, spec.N, spec.fs,
                                             wl.f_low)["rho"]
                got = tr["rho"][tr["tmpl"] == i].astype(np.float64)
                series = max(series, float(np.max(np.abs(got - ref) / np.maximum(ref, 1.0))))
            return {"peak_max": float(err.max()), "peak_median": float(np.median(err)),
                    "series_max": series, "templates": int(len(sel)),
                    "measure": "|rho_gpu - rho_fp64| / max(rho_fp64, 1)"}
        cpu, acc = cpu_baseline(wl, args.cpu_seconds, gpu_check)

    launch_mode = {"mode": "eager" if graph is None else "cuda_graph",
                   "median_ms_per_step": step_medians[-1],
                   "eager_ms_per_step": eager_ms / args.steps,
                   "graph_ms_per_step": tot_ms / args.steps if graph is not None else None,
                   "launches_per_step": launches / args.steps}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded coloured Gaussian noise, Eq. 2 PSD, 8 injections; no LIGO data)",
            "config": {"workload": WORKLOAD, "seed": args.seed, "templates": wl.n_templates, "N": spec.N, "fs": spec.fs,
                       "segments": 1, "threshold": wl.threshold, "n_trig_per_step": n_trig,
                       "l2": "flushed before every timed step (256 MiB write)",
                       "step": "mf_segment_refresh (device s) + mf_filter_bank, one CUDA-graph replay"
                               if graph is not None else "mf_segment_refresh (device s) + mf_filter_bank",
                       "launch": launch_mode,
                       "conditioning": conditioning,
                       "schedule": schedule,
                       "segment_fft": args.conditioning.upper() + " forward FFT in mf_segment_refresh",
                       "phase": "FP64 anchors + FP32 Taylor; FFT " + {
                           "fp32": "FP32", "tc_fp16": "FP32 but pass 2's first radix-32 stage on the tensor cores "
                           "(FP16 hi + lo splits)", "tc_bf16": "FP32 but pass 2's first radix-32 stage on the tensor "
                           "cores (BF16 hi + lo splits)"}[args.fft_mode]},
            "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roof, "path_roofline": path,
            "rho_err": acc, "cpu_baseline": cpu, "wall_s_timed": wall}
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
