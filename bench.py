#!/usr/bin/env python
"""Benchmark of the editable-Gaussian rasterizer path on GB300.

One step = one pass of the whole path over one batch: edit table (compose/edit), projection +
shading of every (view, Gaussian), tile binning + radix sort, compositing of every view, and
the backward of all of it for a fixed dL/dRGBA. Default workload: 1,000,000 Gaussians over 4
basic models, 8 views of uneven sizes (512^2, 800^2, 1024x768, 1280^2, twice), 6.65 Mpix.
Metric: Mpix/s of forward+backward (also reported: forward only).

`--impl reference` times the FP64 CPU oracle instead (a bounded sample of the same workload).
Multi-GPU (torchrun): every rank renders its own replica of the workload (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd / fwd+bwd Mpix/s at 1M Gaussians, batched-mixed vs plain, max|Δ|≤2e-4"
UNIT = "Mpix/s"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ivrgs", choices=["ivrgs", "reference"])
    ap.add_argument("--workload", default="cfg4", choices=["cfg1", "cfg2", "cfg3", "cfg4", "cfg4-2v"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-only", action="store_true", help="run warmup + 2 steps, print nothing else")
    ap.add_argument("--opt", action="append", default=[], help="library option name=value (launch shapes)")
    ap.add_argument("--eager", action="store_true", help="time eager launches instead of CUDA-graph replays")
    ap.add_argument("--no-mixed", action="store_true", help="skip the 16-bit storage and single-view forms")
    ap.add_argument("--autotune", action="store_true", help="pick launch shapes by timing (cached per GPU)")
    ap.add_argument("--no-inverse", action="store_true", help="skip the inverse-exploration iteration timing")
    ap.add_argument("--layout", default="morton", choices=["morton", "composed"],
                    help="Gaussian order in memory: per model by Morton code (one-time reorder) or as composed")
    return ap.parse_args()


def workload(name):
    import scenegen as sg
    return {"cfg1": sg.config1, "cfg2": sg.config2, "cfg3": sg.config3, "cfg4": sg.config4,
            "cfg4-2v": sg.config4_two_views}[name]()


# ------------------------------------------------------------------------------------ clocks
CLOCK_LOAD_S = 0.8


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout: float = 3.0):
        """Wait (bounded) until the sampler has printed its first line."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.01)

    def mark(self):
        """Samples before this point (an idle GPU) are left out of the report."""
        self.first = len(self.lines)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines[getattr(self, "first", 0):] or self.lines
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------ roofline
def peaks():
    p = {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            m = json.load(f)
        p.update({"hbm_gbs": float(m["hbm_gbs"]), "sm_max_mhz": float(m.get("sm_max_mhz", 2070.0)),
                  "source": "measured"})
    return p


N_SM = 152
FP32_LANES = 128
OPS_FWD = 20.0  # FP32 lane operations per evaluated (pixel, Gaussian) entry in the forward blend
OPS_BWD = 40.0  # backward blend: recompute alpha + transmittance recovery + nine gradient terms


def kernel_work(name, w, stats):
    """Algorithmic work of one launch of `name`: (bound, amount, unit). Bytes count each array
    once (what the kernel must read and write), operations the FP32 lane ops per evaluated entry."""
    n, V, pairs, evals = stats["n"], stats["V"], stats["pairs"], stats["evals"]
    if name == "k_render":
        return "alu", OPS_FWD * evals, "op"
    if name == "k_render_bwd":
        return "alu", OPS_BWD * evals, "op"
    if name == "k_onesweep":  # one tile-id pass: key + u32 value, read and written (u16 keys but the
        # last pass's output below 2^16 tiles: 12 B and 14 B, averaged over the two passes)
        return "hbm", (13.0 if stats.get("tiles", 1 << 16) < (1 << 16) else 16.0) * pairs, "B"
    if name == "k_project":  # 86 B of attributes per Gaussian in, a 44 B record per (view, Gaussian) out
        return "hbm", 86.0 * n + 44.0 * n * V, "B"
    if name == "k_project_bwd":  # attributes in, 36 B of record gradients per (view, Gaussian) in, 84 B out
        return "hbm", 86.0 * n + 36.0 * n * V + 84.0 * n, "B"
    if name == "k_emit":  # the pairs written: u16 or u32 tile id + u32 value (record reads not counted)
        return "hbm", (6.0 if stats.get("tiles", 1 << 16) < (1 << 16) else 8.0) * pairs, "B"
    if name == "k_count":  # position, conic + opacity and radius in, the pair count out, per record
        return "hbm", 32.0 * n * V, "B"
    return None


# ------------------------------------------------------------------------------------ GPU arm
class Harness:
    """Buffers, CUDA graphs and timing of the fwd+bwd step for one workload and one storage."""

    def __init__(self, args, w, comp, table, dev, world, graphs=True):
        import torch

        from paper_2504_17954_gb300 import Gaussians, Rasterizer
        self.args, self.w, self.comp, self.table, self.dev, self.world = args, w, comp, table, dev, world
        self.ed = w.edits
        self.rast = Rasterizer(w.cameras, comp.n, len(w.models), device=dev, lowpass=w.lowpass, bg=w.bg)
        self.rast.forward(comp, table, mode="exact")  # sizes the pair buffer
        torch.cuda.synchronize()
        self.n_pairs = self.rast.n_pairs
        self.rast._ensure_capacity(int(self.n_pairs * 1.1) + 4096)
        gen = torch.Generator(device=dev).manual_seed(4)
        self.dL = torch.randn((self.rast.n_pix, 4), generator=gen, device=dev, dtype=torch.float32) * 1e-3
        self.grad = Gaussians.empty(comp.n, len(w.models), dev)
        self.grad.model_id = None
        self.flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
        self.stream = torch.cuda.current_stream()
        for _ in range(max(3, args.warmup)):
            self.step()
        torch.cuda.synchronize()
        self.graphs = {}
        if graphs and not args.eager:
            self.graphs[True] = self.rast.capture(comp, table, self.dL, grad=self.grad)
            self.graphs[False] = self.rast.capture(comp, table)

    def edit(self):
        from paper_2504_17954_gb300 import compose_edit
        ed = self.ed
        compose_edit(None, ed.palette, ed.opacity_scale, ed.visible, ed.lam, ed.bias, device=self.dev,
                     edit_table=self.table)

    def step(self, backward=True):
        """Eager: edit table, projection, binning (CAPACITY mode), compositing, backward."""
        self.edit()
        self.rast.forward(self.comp, self.table, mode="capacity")
        if backward:
            self.rast.backward(self.comp, self.table, self.dL, grad=self.grad)

    def run_step(self, backward):
        if self.graphs:
            self.edit()
            self.graphs[backward].replay()
        else:
            self.step(backward)

    def timed(self, k, backward, prof=False):
        """Device ms of k steps (L2 flushed between steps, outside the timed events), max over ranks."""
        import torch

        from paper_2504_17954_gb300 import _native as N
        world = self.world
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        evs = []
        if prof:
            N.prof_report()
            N.prof_enable(True)
        for _ in range(k):
            self.flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(self.stream)
            if prof:
                self.step(backward)  # eager launches, each bracketed by the library's events
            else:
                self.run_step(backward)
            b.record(self.stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        rep = {}
        if prof:
            N.prof_enable(False)
            rep = N.prof_report()
        if world > 1:
            torch.distributed.barrier()
        ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), self.dev, world)
        if int(self.rast.d_n_pairs.item()) > self.rast.capacity:
            raise RuntimeError("pair buffer overflow during the timed steps")
        return ms, rep

    def mpix(self, ms, k):
        return whole_job_mpix(self.rast.n_pix, self.world, k, ms)


def max_over_ranks(ms: float, device, world: int) -> float:
    """The slowest rank's time (replicas are timed between barriers; the job is as slow as its
    slowest replica)."""
    import torch
    if world <= 1:
        return float(ms)
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_mpix(pixels_per_replica: int, world: int, steps: int, ms: float) -> float:
    """Whole-job throughput: every replica renders its own copy of the workload."""
    return pixels_per_replica * world * steps / (ms / 1e3) / 1e6


def source_hash():
    """Hash of the CUDA sources: ncu traffic figures are used only for the build they came from."""
    import glob
    import hashlib
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_2504_17954_gb300", "csrc", "*"))):
        with open(p, "rb") as f:
            h.update(os.path.basename(p).encode() + f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel, workload):
    """dram bytes per launch of `kernel` from the committed ncu summary, if it matches these CUDA sources."""
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}.md")
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.startswith("traffic-json: "):
            d = json.loads(line[len("traffic-json: "):])
            if d.get("source_hash") == source_hash():
                return d["kernels"].get(kernel)
    return None


def run_gpu(args, rank, world):
    import torch

    from paper_2504_17954_gb300 import _native as N
    from paper_2504_17954_gb300 import build as B
    from paper_2504_17954_gb300 import Gaussians, compose_edit, pack_mixed, reorder_spatial

    B.build()
    opts = {}
    for kv in args.opt:
        k, v = kv.split("=")
        N.ivrgs_set_option(k, int(v))
    for k in ("render_pixels_per_thread", "render_bwd_pixels_per_thread", "sort_match", "sort_scan", "sort_early"):
        opts[k] = N.ivrgs_get_option(k)
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w = workload(args.workload)
    ed = w.edits
    attrs = ("mean", "log_scale", "quat", "opacity_logit", "dcolor", "normal", "kads")
    models = [Gaussians.from_arrays({k: getattr(m, k) for k in attrs}, device=dev) for m in w.models]
    comp, table = compose_edit(models, ed.palette, ed.opacity_scale, ed.visible, ed.lam, ed.bias, device=dev)
    del models
    if args.layout == "morton":  # one-time layout step of the model set, outside the timed region
        comp, _ = reorder_spatial(comp)
    if args.profile_only:  # a short run for profilers: warm-up plus one step, no report
        h = Harness(args, w, comp, table, dev, world, graphs=False)
        h.step()
        torch.cuda.synchronize()
        return None
    h = Harness(args, w, comp, table, dev, world)
    rast, n_pairs = h.rast, h.n_pairs
    evals = float(rast.last.double().sum().item())
    if args.autotune:
        from paper_2504_17954_gb300 import autotune
        autotune.tune(lambda: h.step(True), f"{args.workload}|n={comp.n}|pairs~{n_pairs // 1000000}M")
        for k in opts:
            opts[k] = N.ivrgs_get_option(k)
        h = Harness(args, w, comp, table, dev, world)
        rast = h.rast
    for _ in range(2):
        h.run_step(True)
    K = args.steps
    # nvidia-smi samples every 200 ms, longer than the timed steps take: the sampler starts
    # before CLOCK_LOAD_S of the same step replayed back to back (untimed), and runs on through
    # the timed regions, so its samples see the clocks of this load
    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    sampler.start()
    sampler.wait_first()
    sampler.mark()
    n_load, t_load = 0, time.perf_counter()
    while time.perf_counter() - t_load < CLOCK_LOAD_S:
        h.run_step(True)
        torch.cuda.synchronize()
        n_load += 1
    ms_total, _ = h.timed(K, True)
    ms_fwd_total, _ = h.timed(K, False)
    ms_eager, kernels = h.timed(K, True, prof=True)
    clocks = sampler.stop()
    clocks["window"] = f"{n_load} untimed steps ({CLOCK_LOAD_S} s) back to back, then the timed steps"
    value, fwd_value = h.mpix(ms_total, K), h.mpix(ms_fwd_total, K)

    # the batched form with 16-bit attribute storage, same workload
    mixed = None
    if not args.no_mixed:
        packed, _ = pack_mixed(comp)
        hm = Harness(args, w, packed, table, dev, world)
        mm, _ = hm.timed(K, True)
        mf, _ = hm.timed(K, False)
        mixed = {"mpix_s": hm.mpix(mm, K), "fwd_mpix_s": hm.mpix(mf, K), "ms_per_step": mm / K,
                 "storage": "FP16 mean offsets from per-256 FP32 anchors, BF16 log-scale/dc/normal, FP16 q/o/k",
                 "bytes_per_gaussian": 44}
        del hm, packed
    # the vector-quantised storage (Sec. 4.4): k = 256 codebooks per model and attribute
    vqd = None
    if not args.no_mixed:
        from paper_2504_17954_gb300 import vq_compress
        ta, tb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ta.record()
        q = vq_compress(comp, k=256, iters=16)
        tb.record()
        torch.cuda.synchronize()
        hq = Harness(args, w, q, table, dev, world)
        qm, _ = hq.timed(K, True)
        qf, _ = hq.timed(K, False)
        vqd = {"mpix_s": hq.mpix(qm, K), "fwd_mpix_s": hq.mpix(qf, K), "ms_per_step": qm / K,
               "storage": "FP32 mean and normal, uint8 indices into per-model k=256 scalar codebooks",
               "bytes_per_gaussian": 41, "codebook_build_ms": ta.elapsed_time(tb)}
        del hq, q
    # the plain single-view form (500k Gaussians, one 800x800 view, float32)
    single = None
    if not args.no_mixed and args.workload == "cfg4":
        ws = workload("cfg2")
        ms_ = [Gaussians.from_arrays({k: getattr(m, k) for k in attrs}, device=dev) for m in ws.models]
        c2, t2 = compose_edit(ms_, ws.edits.palette, ws.edits.opacity_scale, ws.edits.visible, ws.edits.lam,
                              ws.edits.bias, device=dev)
        h2 = Harness(args, ws, c2, t2, dev, world)
        sm, _ = h2.timed(K, True)
        sf, _ = h2.timed(K, False)
        single = {"workload": ws.name, "mpix_s": h2.mpix(sm, K), "fwd_mpix_s": h2.mpix(sf, K), "ms_per_step": sm / K}
        del h2

    inverse = None
    if not args.no_inverse and args.workload == "cfg4":
        inverse = inverse_bench(args, dev)

    # roofline of the dominant kernel (largest share of device time in the eager timed steps)
    pk = peaks()
    stats = {"n": comp.n, "V": len(w.cameras), "pairs": n_pairs, "evals": evals, "tiles": rast.n_tiles}
    kern_table = {}
    for name, (cnt, tot) in kernels.items():
        kern_table[name] = {"launches": cnt, "ms_per_launch": tot / cnt, "share": tot / sum(x[1] for x in kernels.values())}
    dom = max(kernels.items(), key=lambda kv: kv[1][1])[0]
    cnt, tot = kernels[dom]
    per_launch_s = tot / cnt / 1e3
    wk = kernel_work(dom, w, stats)
    launches_per_step = sum(c for c, _ in kernels.values()) / K
    traffic = recorded_traffic(dom, args.workload)
    if wk is None:
        roof = {"bound": None, "kernel": dom}
    elif wk[0] == "hbm":
        ach = wk[1] / per_launch_s / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"], "peak_source": pk["source"], "traffic": traffic}
    else:
        peak = N_SM * FP32_LANES * pk["sm_max_mhz"] * 1e6 / 1e12
        ach = wk[1] / per_launch_s / 1e12
        roof = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": peak, "unit": "Top/s (FP32 lane ops)",
                "frac": ach / peak, "peak_source": f"{N_SM} SMs x {FP32_LANES} FP32 lanes x {pk['sm_max_mhz']:.0f} MHz",
                "traffic": traffic}
    roof["work_per_launch"] = wk[1] if wk else None
    # every kernel with an algorithmic work figure, against the same peaks
    stages = {}
    for name, (c_, t_) in kernels.items():
        kw = kernel_work(name, w, stats)
        if kw is None:
            continue
        sec = t_ / c_ / 1e3
        if kw[0] == "hbm":
            a_ = kw[1] / sec / 1e9
            stages[name] = {"bound": "hbm", "achieved": a_, "unit": "GB/s", "frac": a_ / pk["hbm_gbs"]}
        else:
            pk_alu = N_SM * FP32_LANES * pk["sm_max_mhz"] * 1e6 / 1e12
            a_ = kw[1] / sec / 1e12
            stages[name] = {"bound": "alu", "achieved": a_, "unit": "Top/s", "frac": a_ / pk_alu}
    roof["timing"] = "per-kernel CUDA events (library, launching stream) over K eager steps"
    roof["evaluated_entries_per_launch"] = evals

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
           "ms_per_step": ms_total / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32", "data": "synthetic (seeded volume-band Gaussians; no paper datasets)",
           "config": {"workload": w.name, "gaussians": comp.n, "models": len(w.models), "views": len(w.cameras),
                      "pixels_per_replica": rast.n_pix, "pairs": n_pairs, "l2": "flushed between timed steps",
                      "layout": "per model in Morton order (one-time reorder)" if args.layout == "morton"
                      else "as composed",
                      "options": opts,
                      "parallelism": f"replicas x{world}"},
           "fwd_mpix_s": fwd_value, "fwd_ms_per_step": ms_fwd_total / K,
           "launch": "eager" if args.eager else "cuda-graph replay",
           "eager_mpix_s": h.mpix(ms_eager, K),
           "roofline": roof, "stage_roofline": stages, "kernels": kern_table, "clocks": clocks,
           "batched_mixed": mixed, "batched_vq": vqd, "plain_single_view": single, "inverse_exploration": inverse,
           "source_hash": source_hash(),
           "gpu_launches": int(round(launches_per_step * K))}

    if not args.no_e2e:
        out["e2e"] = e2e(rast, comp, table, w, ed, h.dL, h.grad, K, dev, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w)
    return out


def inverse_bench(args, dev, iters: int = 50):
    """Inverse volume exploration (Sec. 4.6) at the size of the paper's five-jet case (1.48M
    primitives): the 1.5M-Gaussian, 6-model scene fitted to one 1024x1024 reference view with an
    orbital light; all edit parameters and the light direction learnable. One iteration =
    projection, binning, compositing, loss, backward and Adam step, replayed as a CUDA graph."""
    import numpy as np
    import torch

    import scenegen as sg
    from paper_2504_17954_gb300 import Gaussians, Rasterizer, compose_edit
    from paper_2504_17954_gb300.inverse import LEARN_ALL, InverseExplorer
    w = workload("cfg3")
    cam = w.cameras[0]
    attrs = ("mean", "log_scale", "quat", "opacity_logit", "dcolor", "normal", "kads")
    models = [Gaussians.from_arrays({k: getattr(m, k) for k in attrs}, device=dev) for m in w.models]
    M = len(w.models)
    ref = sg.random_edits(w.models, seed=5)
    ref_dir = np.array([0.5, -0.3, 0.81])
    comp, tref = compose_edit(models, ref.palette, ref.opacity_scale, ref.visible, [1.2, 0.9, 1.1, 1.0],
                              [0.02, 0.0, 0.0, 1.0], device=dev, light_dir=ref_dir)
    del models
    rast = Rasterizer([cam], comp.n, M, device=dev, bg=(0.0, 0.0, 0.0))
    rast.forward(comp, tref)
    target = rast.rgba.clone()
    start = sg.identity_edits(w.models)
    _, table = compose_edit(None, start.palette, start.opacity_scale, start.visible, start.lam, start.bias,
                            device=dev, light_dir=[0.2, 0.4, 0.9])
    ex = InverseExplorer(rast, comp, table, target, learn=LEARN_ALL, lr=0.01)
    ex.capture()
    for _ in range(max(args.warmup, 3)):
        ex.graph.replay()
    loss0 = float(ex.loss[0].item())
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(iters):
        ex.graph.replay()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / iters
    if ex.overflowed():
        raise RuntimeError("inverse exploration: pair buffer overflowed during replay")
    return {"workload": f"1.5M Gaussians / {M} models, one {cam.W}x{cam.H} reference view, orbital light; "
                        "learnable c_p, opacity scale, lambda, b, light polar/azimuth",
            "gaussians": comp.n, "ms_per_iter": ms, "iters_timed": iters,
            "loss_after_warmup": loss0, "loss_last": float(ex.loss[0].item()),
            "paper_ms_per_iter": {"five-jet (1,484,642)": 48.0, "combustion (5,432,519)": 88.0,
                                  "vortex (7,104,441)": 122.0, "hardware": "RTX 4090 (context, not a target)"},
            "l2": "not flushed (one iteration's working set; the loop reuses it every iteration)"}


def e2e(rast, comp, table, w, ed, dL, grad, K, dev, world):
    """Same metric through the public API with the inputs in pinned host memory
    (paper_2504_17954_gb300.hostio.HostPipeline): every step copies the Gaussian attributes in,
    runs forward + backward, and reads the image and the gradients back; the transfers of
    neighbouring steps overlap the compute on their own streams."""
    import torch

    from paper_2504_17954_gb300.hostio import HostPipeline, pack_host
    pipe = HostPipeline(rast, comp.model_id, comp.n_models, table, dL)
    blk = pack_host(comp)
    out_img = torch.empty(rast.rgba.shape, dtype=torch.float32).pin_memory()
    out_grad = torch.empty_like(blk).pin_memory()
    stream = torch.cuda.current_stream()
    pipe.run([blk] * 2, [out_img] * 2, [out_grad] * 2)  # warm-up
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    pipe.run([blk] * K, [out_img] * K, [out_grad] * K)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.barrier()
    ms = float(t.item())
    return {"value": rast.n_pix * world * K / (ms / 1e3) / 1e6, "unit": UNIT, "h2d_bytes_per_step": pipe.h2d_bytes,
            "d2h_bytes_per_step": pipe.d2h_bytes, "ms_per_step": ms / K,
            "transfers": "pinned host blocks; copies of neighbouring steps overlap the compute (3 streams); "
                         "compute replayed from CUDA graphs"}


# ------------------------------------------------------------------------------------ oracle
def oracle_sample_step(w, comp, table):
    """One bounded sample of the workload on the FP64 oracle: view 0, forward + backward."""
    import numpy as np

    import oracle
    cam = w.cameras[0]
    r = oracle.render(w.models, w.edits, [cam], bg=w.bg, comp=comp, table=table)
    dl = np.full((cam.H, cam.W, 4), 1e-3)
    oracle.render_backward(r, [cam], [dl], bg=w.bg)
    return cam.W * cam.H


def cpu_baseline(w, steps=1):
    import oracle
    oracle.build()
    comp = oracle.compose(w.models)
    table = oracle.edit_table(w.edits)
    t0 = time.perf_counter()
    px = 0
    for _ in range(steps):
        px += oracle_sample_step(w, comp, table)
    dt = time.perf_counter() - t0
    c = w.cameras[0]
    return {"value": px / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"view 0 ({c.W}x{c.H}) of the workload, forward + backward, all {comp.n} Gaussians, "
                      f"{steps} step(s), {dt:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle
    oracle.build()
    w = workload(args.workload)
    comp = oracle.compose(w.models)
    table = oracle.edit_table(w.edits)
    for _ in range(min(args.warmup, 1)):
        oracle_sample_step(w, comp, table)
    t0 = time.perf_counter()
    px = 0
    for _ in range(args.steps):
        px += oracle_sample_step(w, comp, table)
    dt = time.perf_counter() - t0
    v = px / dt / 1e6
    c = w.cameras[0]
    sample = (f"view 0 ({c.W}x{c.H}) of {w.name}, forward + backward over all {comp.n} Gaussians per step, "
              f"single-threaded FP64 C oracle")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "gaussians": comp.n, "models": len(w.models), "views": len(w.cameras),
                       "pixels_per_replica": sum(q.W * q.H for q in w.cameras), "sample": sample,
                       "parallelism": "rank 0 only, host cores"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl != "reference":
        import torch
        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_gpu(args, rank, world)
    if rank == 0 and out is not None and not args.profile_only:
        print(json.dumps(out))
    if world > 1 and args.impl != "reference":
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
