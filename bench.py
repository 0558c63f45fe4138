"""Benchmark of the GB300 render path (arXiv 2410.08129 hot path).

Headline workload: 1,000,000 clustered Gaussians (SH degree 3) rendered at
1920x1080 with hybrid transparency, K = 8 (the paper's benchmark resolution,
between its Francis 0.44M and Bicycle 4.35M scenes). A step is one full
render: preprocess, binning, radix sort, blend. value = frames/s over all
ranks. Also reported: the training step (500k Gaussians at 1200x800: render,
L1 loss gradient, render backward) in steps/s, the end-to-end frame rate
through the C ABI with host buffers, the blend kernel's roofline fraction
and the FP64 oracle timed on this host.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank renders its own replica (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1080p frames/s @1M Gaussians and fwd+bwd steps/s, batched vs plain, at oracle tol"
UNIT = "frames/s"
WORKLOAD = "1M clustered Gaussians, SH deg 3, 1920x1080, 60deg vFOV, K=8, tau_alpha=1/255, tau_K=0.05"
FP32_LANES = 128  # FP32 lanes per SM (sm_100 family)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region
    runs, every 50 ms. Entering waits for the first sample (taken right after
    the warm-up) so that the sampler is live when the region starts; leaving
    waits for one more, so that a region shorter than the interval is still
    bracketed by samples."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
            return self
        deadline = time.time() + 5.0
        while not self.rows and time.time() < deadline and self.proc.poll() is None:
            time.sleep(0.01)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *exc):
        if self.proc is not None:
            n, deadline = len(self.rows), time.time() + 0.5
            while len(self.rows) == n and time.time() < deadline and self.proc.poll() is None:
                time.sleep(0.01)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def source_digest(names) -> str:
    """sha256 of the kernel sources with comments and blank lines removed, so
    that a comment edit does not retire counters taken on unchanged code."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2410_08129_gb300", "csrc", name)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        code = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
        h.update(code.encode())
    return h.hexdigest()


def recorded_traffic():
    """DRAM bytes per launch of the forward blend on the headline workload,
    as measured by ncu (profiles/blend_fwd_traffic.json); None when the
    kernel's code changed since the counters were taken."""
    prof = os.path.join(ROOT, "profiles", "blend_fwd_traffic.json")
    try:
        with open(prof) as f:
            rec = json.load(f)
        digest = source_digest(rec["sources"])
    except (OSError, ValueError, KeyError):
        return None
    return rec.get("bytes_per_launch_1080p_1M") if digest == rec.get("sources_code_sha256") else None


def dist_summary(ms) -> dict:
    """Median, mean and extremes of per-step times (ms)."""
    a = np.asarray(ms, dtype=np.float64)
    return {"n": int(a.size), "median": float(np.median(a)), "mean": float(a.mean()),
            "min": float(a.min()), "max": float(a.max())}


def per_step_ms(step, stream, warmup: int, n: int) -> dict:
    """`warmup` untimed calls of `step`, then `n` timed ones with a CUDA event
    recorded on `stream` between consecutive calls (the events sit between
    steps, never inside one)."""
    import torch
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(n + 1)]
    ev[0].record(stream)
    for i in range(n):
        step()
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    out = dist_summary([ev[i].elapsed_time(ev[i + 1]) for i in range(n)])
    out["note"] = f"{warmup} warm-ups, {n} steps, an event between consecutive steps"
    return out


def reduce_max(x: float, world: int, device) -> float:
    """Largest value of x over the ranks of the default process group (the
    job's time is that of its slowest rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job throughput of replicas: every rank processes units_per_rank
    units; the job ends with its slowest rank (max_ms)."""
    return world * units_per_rank / (max_ms / 1e3)


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _lscpu():
    """Host CPU description from lscpu (model, logical CPUs)."""
    out = {"os_cpu_count": os.cpu_count()}
    try:
        txt = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
    except (OSError, subprocess.SubprocessError):
        return out
    for ln in txt.splitlines():
        k, _, v = ln.partition(":")
        if k.strip() in ("CPU(s)", "Model name", "Architecture", "Thread(s) per core", "Core(s) per socket"):
            out[k.strip()] = v.strip()
    return out


def _oracle_window(scene64, cam, prm, window):
    import oracle
    t0 = time.perf_counter()
    oracle.render(scene64, cam, prm, window=window)
    return time.perf_counter() - t0


def cpu_baseline(scene, cam, prm, stress_scene, stress_cam):
    """The FP64 oracle as it stands (brute force: every Gaussian against every
    pixel) on the host cores, on the samples the measurement plan names: the
    64x64 frame of 256 Gaussians in full, a 128x128 crop of the headline 1080p
    frame and a 128x128 crop of the 6M-Gaussian stress frame (16 of its 128
    rows, the rest extrapolated). value = headline frames/s extrapolated from
    the crop's time per pixel."""
    import oracle
    from paper_2410_08129_gb300 import scenes
    runs = []
    s1, c1, p1, _ = scenes.config1()
    dt = _oracle_window(s1.astype(np.float64), c1.rounded(), p1, None)
    runs.append({"sample": "256 Gaussians, 64x64, full frame", "s": dt, "pairs": s1.n * 64 * 64,
                 "pairs_per_s": s1.n * 64 * 64 / dt})
    cx, cy = cam.width // 2 - 64, cam.height // 2 - 64
    dt2 = _oracle_window(scene.astype(np.float64), cam, prm, (cx, cy, 128, 128))
    runs.append({"sample": f"{scene.n} Gaussians, 128x128 crop at ({cx},{cy}) of 1920x1080", "s": dt2,
                 "pairs": scene.n * 128 * 128, "pairs_per_s": scene.n * 128 * 128 / dt2})
    sx, sy = stress_cam.width // 2 - 64, stress_cam.height // 2 - 64
    dt5 = _oracle_window(stress_scene.astype(np.float64), stress_cam, prm, (sx, sy, 128, 16))
    runs.append({"sample": f"{stress_scene.n} Gaussians, rows 0-15 of the 128x128 crop at ({sx},{sy}) of "
                           f"the stress frame; crop time extrapolated", "s": dt5, "crop_s_extrapolated": 8 * dt5,
                 "pairs": stress_scene.n * 128 * 16, "pairs_per_s": stress_scene.n * 128 * 16 / dt5})
    fps = 1.0 / (dt2 * cam.width * cam.height / (128 * 128))
    return {"value": fps, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
            "sample": "headline frames/s extrapolated from a 128x128 crop of the 1080p frame "
                      f"({dt2:.1f} s, all Gaussians brute-forced per pixel)",
            "runs": runs, "lscpu": _lscpu()}


def fp32_peak(local):
    """FP32 FMA rate of this device: SM count from the device properties and
    the rate measured by the FMA-chain probe (best of 5 launches of about
    5 ms, CUDA events), with the SM clock sampled during the probe."""
    import torch
    from paper_2410_08129_gb300 import binding as B
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    blocks, iters = sms * 8, 5000
    out = torch.empty(blocks * 256, dtype=torch.float32, device="cuda")
    B.htgs_fma_probe(blocks, iters, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    with ClockSampler(local) as ck:
        for _ in range(5):
            e0.record()
            n = B.htgs_fma_probe(blocks, iters, out)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
    rate = n / (best / 1e3)
    clk = ck.summary()
    mhz = clk["sm_mhz"] or clk["sm_max_mhz"]
    nominal = sms * FP32_LANES * mhz * 1e6 if mhz else None
    return {"sms": sms, "fma_per_s": rate, "probe_ms": best, "sm_mhz": mhz, "clocks": clk,
            "nominal_at_clock": nominal, "frac_of_nominal": rate / nominal if nominal else None}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    from paper_2410_08129_gb300 import scenes
    import oracle
    scene, cam, prm = scenes.config2()
    cam = cam.rounded()
    s64 = scene.astype(np.float64)
    win = (952, 532, 16, 16)
    for _ in range(args.warmup):
        oracle.render(s64, cam, prm, window=win)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.render(s64, cam, prm, window=win)
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    fps = 1.0 / (dt * cam.width * cam.height / (win[2] * win[3]))
    line = {"impl": "reference", "metric": METRIC, "value": fps, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "16x16 window per step, extrapolated"},
            "cpu_baseline": {"value": fps, "unit": UNIT, "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": f"16x16 window of the 1080p frame per step ({dt:.3f} s)"},
            "e2e": {"value": fps, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _chunks(instances, limit):
    """Consecutive groups of views whose instance sums stay under `limit`."""
    out, cur, tot = [], [], 0
    for i, n in enumerate(instances):
        if cur and tot + n > limit:
            out.append(cur)
            cur, tot = [], 0
        cur.append(i)
        tot += n
    if cur:
        out.append(cur)
    return out


def plain_vs_batched(gs, tgs, cams, prm, steps, warmup, tune_views=None, graph=True):
    """One training-style step over a set of views, (a) as the plain per-view
    loop (htgs_render, htgs_l1_loss_grad, htgs_render_backward per view,
    gradients of a shared scene summed) and (b) as the batched form
    (htgs_render_batch + per-view loss + htgs_render_batch_backward, captured
    in a CUDA graph), both with the launch configuration the autotuner picks.
    Returns frames/s of the forward alone and steps/s of the whole step."""
    import torch
    from paper_2410_08129_gb300 import binding as B
    from paper_2410_08129_gb300.autotune import autotune
    from paper_2410_08129_gb300.renderer import FIELDS, BatchRenderer, Renderer

    n_views = len(cams)
    dev = torch.device("cuda")
    gen = torch.Generator(device=dev).manual_seed(7)

    # -- autotune (tile shape, forward pixels per thread) on fwd+bwd of a subset
    sub = tune_views if tune_views is not None else list(range(n_views))

    def step_for_launch(launch):
        br = BatchRenderer([gs[i] for i in sub], [cams[i] for i in sub], prm, launch=launch)
        br.forward(check=True)
        dls = [torch.randn(im.shape, device=dev, generator=gen) * 1e-3 for im in br.images]
        grads = br.gradient_buffers()

        def step():
            br.forward(check=False)
            br.backward(dls, grads=grads)
        return step

    t0 = time.perf_counter()
    launch, tune_ms = autotune(step_for_launch, warmup=1, repeats=2)
    tune_s = time.perf_counter() - t0
    torch.cuda.empty_cache()
    tile, ppt, sbatch = (launch.tile_w, launch.tile_h), launch.px_per_thread, launch.smem_batch

    # -- plain: one Renderer per view ------------------------------------------
    rs = [Renderer(c, prm, g.n, launch=launch) for g, c in zip(gs, cams)]
    imgs = [r.image_buffer() for r in rs]
    targets = [r.forward(t, save=False, check=True).clone() for r, t in zip(rs, tgs)]
    for r, g, im in zip(rs, gs, imgs):
        r.forward(g, image=im, save=True, check=True)
    inst = [int(r.last_instances) for r in rs]
    dls = [torch.empty_like(im) for im in imgs]
    losses = torch.zeros(n_views, dtype=torch.float32, device=dev)
    distinct = {}
    for g in gs:
        distinct.setdefault(id(g), g)
    acc = {k: {f: torch.zeros_like(getattr(g, f)) for f in FIELDS} for k, g in distinct.items()}
    tmp = {k: {f: torch.empty_like(getattr(g, f)) for f in FIELDS} for k, g in distinct.items()}

    def plain_fwd():
        for r, g, im in zip(rs, gs, imgs):
            r.forward(g, image=im, save=False, check=False)

    def plain_step():
        seen = set()
        for i, (r, g, im) in enumerate(zip(rs, gs, imgs)):
            r.forward(g, image=im, save=True, check=False)
            B._check(B.htgs_l1_loss_grad(im, targets[i], dls[i], losses[i:i + 1]), "l1")
            if id(g) not in seen:
                r.backward(g, dls[i], grads=acc[id(g)])
                seen.add(id(g))
            else:
                r.backward(g, dls[i], grads=tmp[id(g)])
                for f in FIELDS:
                    acc[id(g)][f].add_(tmp[id(g)][f])

    # -- batched: as few batches as the instance limit allows -------------------
    groups = _chunks(inst, int(0.97 * B.HTGS_MAX_CAPACITY))
    brs, bviews_f, bviews_b, bgrads, bdls, blosses = [], [], [], [], [], []
    for grp in groups:
        br = BatchRenderer([gs[i] for i in grp], [cams[i] for i in grp], prm, launch=launch,
                           capacity=min(int(sum(inst[i] for i in grp) * 1.02) + 4096, B.HTGS_MAX_CAPACITY))
        br.forward(check=True)
        gr = br.gradient_buffers()
        dl = [torch.empty_like(im) for im in br.images]
        brs.append(br)
        bdls.append(dl)
        bgrads.append(gr)
        blosses.append(torch.zeros(len(grp), dtype=torch.float32, device=dev))
        bviews_f.append(br.views())
        bviews_b.append(br.views(dl_dimages=dl, grads=gr))
    bacc = {k: {f: torch.zeros_like(getattr(g, f)) for f in FIELDS} for k, g in distinct.items()} \
        if len(groups) > 1 else bgrads[0]

    def batched_fwd():
        for br, v in zip(brs, bviews_f):
            B._check(B.htgs_render_batch(v, prm, launch, br.workspace, br.capacity), "htgs_render_batch")

    def batched_step():
        for j, (br, grp) in enumerate(zip(brs, groups)):
            B._check(B.htgs_render_batch(bviews_f[j], prm, launch, br.workspace, br.capacity), "htgs_render_batch")
            for k, i in enumerate(grp):
                B._check(B.htgs_l1_loss_grad(br.images[k], targets[i], bdls[j][k], blosses[j][k:k + 1]), "l1")
            B._check(B.htgs_render_batch_backward(bviews_b[j], prm, launch, br.workspace, br.capacity),
                     "htgs_render_batch_backward")
            if len(groups) > 1:
                for key, gd in bgrads[j].items():
                    for f in FIELDS:
                        bacc[key][f].add_(gd[f]) if j else bacc[key][f].copy_(gd[f])

    graphs = {}
    if graph:
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            batched_fwd()
            batched_step()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        for name, fn in (("fwd", batched_fwd), ("step", batched_step)):
            gph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gph, stream=side):
                fn()
            graphs[name] = gph
    run_bfwd = graphs["fwd"].replay if graph else batched_fwd
    run_bstep = graphs["step"].replay if graph else batched_step

    def timed(fn, k):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    ms = {"plain_fwd": timed(plain_fwd, steps), "batched_fwd": timed(run_bfwd, steps),
          "plain_step": timed(plain_step, steps), "batched_step": timed(run_bstep, steps)}
    for r in rs:
        st, _ = r.status()
        assert st == B.HTGS_OK, B.htgs_status_string(st)
    for br in brs:
        st, _ = B.htgs_get_error(br.workspace)
        assert st == B.HTGS_OK, B.htgs_status_string(st)

    # Same images and (up to atomic summation order) the same gradients.
    plain_step()
    run_bstep()
    torch.cuda.synchronize()
    img_diff = 0.0
    for j, grp in enumerate(groups):
        for k, i in enumerate(grp):
            img_diff = max(img_diff, float((brs[j].images[k] - imgs[i]).abs().max()))
    grad_rel = 0.0
    for key in distinct:
        for f in FIELDS:
            a, b = acc[key][f], bacc[key][f]
            grad_rel = max(grad_rel, float((a - b).abs().max() / a.abs().max().clamp_min(1e-30)))
    return {
        "views": n_views, "gaussians": [int(g.n) for g in distinct.values()],
        "pixels": int(sum(c.width * c.height for c in cams)), "instances": int(sum(inst)),
        "launch": {"tile": f"{tile[0]}x{tile[1]}", "px_per_thread": int(ppt), "smem_batch": int(sbatch),
                   "autotune_ms_per_step": {f"{t[0]}x{t[1]}/ppt{p}/b{b}": round(v, 3)
                                            for (t, p, b), v in tune_ms.items()},
                   "autotune_views": len(sub), "autotune_s": round(tune_s, 1)},
        "batches": len(groups), "cuda_graph": bool(graph),
        "fwd": {"plain_frames_per_s": n_views * 1e3 / ms["plain_fwd"],
                "batched_frames_per_s": n_views * 1e3 / ms["batched_fwd"],
                "speedup": ms["plain_fwd"] / ms["batched_fwd"]},
        "fwd_bwd": {"plain_steps_per_s": 1e3 / ms["plain_step"], "batched_steps_per_s": 1e3 / ms["batched_step"],
                    "speedup": ms["plain_step"] / ms["batched_step"]},
        "ms": {k: round(v, 3) for k, v in ms.items()},
        "max_abs_image_diff": img_diff, "max_rel_grad_diff": grad_rel,
    }


def batched_leg(steps, warmup):
    """Config-4 workloads: 32 views (320x240 .. 1600x1064) of a 3M-Gaussian
    scene, and 8 scenes of 50k .. 2M Gaussians at 1280x720; K = 8."""
    import torch
    from paper_2410_08129_gb300 import scenes
    from paper_2410_08129_gb300.renderer import GaussianTensors
    prm = scenes.Params(K=8)
    rng = np.random.Generator(np.random.PCG64(44))
    scene = scenes.config4_scene()
    g = GaussianTensors.from_scene(scene)
    tg = GaussianTensors.from_scene(scenes.perturbed(scene, rng))
    del scene
    cams = [c.rounded() for c in scenes.config4_views()]
    out = {"views32": plain_vs_batched([g] * len(cams), [tg] * len(cams), cams, prm, steps, warmup,
                                       tune_views=list(range(0, len(cams), 8)))}
    out["views32"]["workload"] = ("32 views of one 3M-Gaussian scene (config-1 distribution), "
                                  "320x240..1600x1064, cameras on a 6 m sphere, K=8")
    del g, tg
    torch.cuda.empty_cache()
    multi = scenes.config4_multi()
    gs = [GaussianTensors.from_scene(s) for s, _ in multi]
    tgs = [GaussianTensors.from_scene(scenes.perturbed(s, rng)) for s, _ in multi]
    cams = [c.rounded() for _, c in multi]
    del multi
    out["scenes8"] = plain_vs_batched(gs, tgs, cams, prm, steps, warmup)
    out["scenes8"]["workload"] = "8 scenes of 50k..2M Gaussians (config-1 distribution), 1280x720 each, K=8"
    torch.cuda.empty_cache()
    return out


def profile_case(which: str, warmup: int, tile=None, ppt: int = 1, binning: int = 0, batch: int = 128):
    """A few untimed steps of the headline render (fwd) or of the training
    step (train): `warmup` steps, then 2 more, nothing else on the GPU. The
    launch shape defaults to the one the autotuner picks for the workload on
    a GB300 (16x16 for the render, 32x16 for the training step, 1 pixel per
    thread); `batch` is the forward's staging batch."""
    import torch
    from paper_2410_08129_gb300 import binding as B
    from paper_2410_08129_gb300 import scenes
    from paper_2410_08129_gb300.renderer import GaussianTensors, Renderer
    if which == "fwd":
        scene, cam, prm = scenes.config2()
        g = GaussianTensors.from_scene(scene)
        r = Renderer(cam.rounded(), prm, scene.n, launch=B.c_launch(tile or (16, 16), ppt, binning=binning, smem_batch=batch))
        img = r.image_buffer()
        r.forward(g, image=img, save=False, check=True)
        for _ in range(warmup + 2):
            r.forward(g, image=img, save=False, check=False)
    else:
        scene, target, cam, prm = scenes.config3()
        g = GaussianTensors.from_scene(scene)
        r = Renderer(cam.rounded(), prm, scene.n, launch=B.c_launch(tile or (32, 16), ppt, binning=binning, smem_batch=batch))
        img = r.image_buffer()
        tgt = r.forward(GaussianTensors.from_scene(target), save=False, check=True).clone()
        dl = torch.empty_like(img)
        loss = torch.zeros(1, device="cuda")
        r.forward(g, image=img, save=True, check=True)
        for _ in range(warmup + 2):
            r.forward(g, image=img, save=True, check=False)
            B._check(B.htgs_l1_loss_grad(img, tgt, dl, loss), "l1")
            r.backward(g, dl)
    torch.cuda.synchronize()
    st, inst = r.status()
    assert st == B.HTGS_OK, st
    print(f"profile case {which}: ok, {inst} instances")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the plain-vs-batched comparison")
    ap.add_argument("--batched-steps", type=int, default=3)
    ap.add_argument("--batched-warmup", type=int, default=3)
    ap.add_argument("--profile", choices=["fwd", "train"], default=None,
                    help="run a few untimed steps of one workload (for an external profiler) and exit")
    ap.add_argument("--profile-tile", default=None, help="tile shape WxH of --profile (default: the autotuner's pick)")
    ap.add_argument("--profile-ppt", type=int, default=1, help="forward pixels per thread of --profile")
    ap.add_argument("--profile-binning", choices=["radix", "counting"], default="radix",
                    help="tile binning of --profile (the lists are the same)")
    ap.add_argument("--profile-batch", type=int, default=128, choices=[32, 64, 128, 192],
                    help="forward staging batch of --profile")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile:
        tile = tuple(int(v) for v in args.profile_tile.split("x")) if args.profile_tile else None
        profile_case(args.profile, args.warmup, tile, args.profile_ppt,
                     binning=2 if args.profile_binning == "counting" else 1, batch=args.profile_batch)
        return

    import torch
    import torch.distributed as dist

    from paper_2410_08129_gb300 import binding as B
    from paper_2410_08129_gb300 import scenes
    from paper_2410_08129_gb300.renderer import GaussianTensors, Renderer

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x):
        return reduce_max(x, world, "cuda")

    stream = torch.cuda.current_stream()
    peaks, peak_src = _peaks()

    # ---- headline: 1080p frames/s at 1M Gaussians --------------------------
    scene, cam, prm = scenes.config2(seed=1 + rank)
    cam = cam.rounded()
    g = GaussianTensors.from_scene(scene)
    # Launch shape (tile, pixels per thread, staging batch) from the autotuner.
    from paper_2410_08129_gb300.autotune import autotune
    sorted_candidates = [((16, 16), 1), ((32, 16), 1), ((16, 8), 1)]

    def fwd_step_for(launch_):
        rr = Renderer(cam, prm, scene.n, launch=launch_)
        im = rr.image_buffer()
        rr.forward(g, image=im, save=False, check=True)
        return lambda: rr.forward(g, image=im, save=False, check=False)

    best_fwd, tune_fwd = autotune(fwd_step_for, warmup=2, repeats=5)
    torch.cuda.empty_cache()
    fwd_shape = ((best_fwd.tile_w, best_fwd.tile_h), best_fwd.px_per_thread, best_fwd.smem_batch)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    for e in ev:
        e.record(stream)
    # The timed renders carry no phase events (with events between its
    # phases a render launches its kernels without programmatic dependencies);
    # the per-phase times come from a separate pass with them.
    launch_ev = B.c_launch(fwd_shape[0], fwd_shape[1], 0, ev, smem_batch=fwd_shape[2])
    launch = B.c_launch(fwd_shape[0], fwd_shape[1], 0, None, smem_batch=fwd_shape[2])
    r = Renderer(cam, prm, scene.n, launch=launch)
    image = r.image_buffer()
    r.forward(g, image=image, save=False, check=True)       # sizes the instance capacity
    for _ in range(max(args.warmup, 3)):
        r.forward(g, image=image, save=False, check=False)
    torch.cuda.synchronize()
    blend_ms, pre_ms, bin_ms = [], [], []
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        barrier()
        torch.cuda.synchronize()
        t_start.record(stream)
        for _ in range(args.steps):
            r.forward(g, image=image, save=False, check=False)
        t_end.record(stream)
        torch.cuda.synchronize()
        barrier()
    # per-phase times: a separate, identical pass (events between steps)
    r.launch = launch_ev
    for _ in range(min(args.steps, 20)):
        r.forward(g, image=image, save=False, check=False)
        torch.cuda.synchronize()
        pre_ms.append(ev[0].elapsed_time(ev[1]))
        bin_ms.append(ev[2].elapsed_time(ev[3]))
        blend_ms.append(ev[4].elapsed_time(ev[5]))
    r.launch = launch
    # Per-frame distribution (10 warm-ups, then 100 frames, an event between
    # consecutive frames): median and mean of the frame time.
    frame_dist = per_step_ms(lambda: r.forward(g, image=image, save=False, check=False), stream, 10, 100)
    st, inst = r.status()
    assert st == B.HTGS_OK, B.htgs_status_string(st)
    counters = B.htgs_get_counters(r.workspace)
    total_ms = max_over_ranks(t_start.elapsed_time(t_end))
    ms_per_step = total_ms / args.steps
    fps = job_throughput(args.steps, world, total_ms)

    # ---- the same frame with the 3D smoothing filter (Sec. 4.2) -----------
    fscene = scene.with_filter(scenes.filter_variance_from_cameras(scene.means, [cam]))
    fg = GaussianTensors.from_scene(fscene)
    fr = Renderer(cam, prm, scene.n, launch=B.c_launch(*fwd_shape[:2], smem_batch=fwd_shape[2]))
    fimg = fr.image_buffer()
    fr.forward(fg, image=fimg, save=False, check=True)
    for _ in range(max(args.warmup, 3)):
        fr.forward(fg, image=fimg, save=False, check=False)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        fr.forward(fg, image=fimg, save=False, check=False)
    f1.record(stream)
    torch.cuda.synchronize()
    st3, finst = fr.status()
    assert st3 == B.HTGS_OK
    filter_ms = max_over_ranks(f0.elapsed_time(f1))
    filtered = {"value": job_throughput(args.steps, world, filter_ms), "unit": UNIT,
                "ms_per_step": filter_ms / args.steps, "instances": finst,
                "workload": "the headline frame with the 3D filter, variance (0.2 depth / focal)^2 per Gaussian"}
    del fr, fg, fimg

    # ---- the same frame from baked records (App. A) --------------------------
    kev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    for e in kev:
        e.record(stream)
    kg = g.bake()
    klaunch_ev = B.c_launch(*fwd_shape[:2], 0, kev, smem_batch=fwd_shape[2])
    kr = Renderer(cam, prm, scene.n, launch=B.c_launch(*fwd_shape[:2], smem_batch=fwd_shape[2]))
    kimg = kr.image_buffer()
    kr.forward(kg, image=kimg, save=False, check=True)
    assert torch.equal(kimg, image), "a baked render must equal the raw one"
    for _ in range(max(args.warmup, 3)):
        kr.forward(kg, image=kimg, save=False, check=False)
    torch.cuda.synchronize()
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(args.steps):
        kr.forward(kg, image=kimg, save=False, check=False)
    k1.record(stream)
    torch.cuda.synchronize()
    assert kr.status()[0] == B.HTGS_OK
    baked_ms = max_over_ranks(k0.elapsed_time(k1))
    kpre = []
    kr.launch = klaunch_ev
    for _ in range(min(args.steps, 20)):
        kr.forward(kg, image=kimg, save=False, check=False)
        torch.cuda.synchronize()
        kpre.append(kev[0].elapsed_time(kev[1]))
    baked = {"value": job_throughput(args.steps, world, baked_ms), "unit": UNIT,
             "ms_per_step": baked_ms / args.steps, "preprocess_ms": float(np.mean(kpre)),
             "bytes_per_gaussian": B.baked_floats(scene.sh_degree) * 4,
             "workload": "the headline frame from baked records (activations folded in, one buffer per "
                         "Gaussian); image identical to the raw render"}
    del kr, kg, kimg

    # ---- the headline frame at K = 4 and K = 16 (the K sweep) ----------------
    k_sweep = {}
    for kk in (4, 16):
        kprm = scenes.Params(K=kk, tau_alpha=prm.tau_alpha, tau_K=prm.tau_K, alpha_max=prm.alpha_max, bg=prm.bg)
        ksr = Renderer(cam, kprm, scene.n, launch=B.c_launch(*fwd_shape[:2], smem_batch=fwd_shape[2]))
        ksimg = ksr.image_buffer()
        ksr.forward(g, image=ksimg, save=False, check=True)
        for _ in range(max(args.warmup, 3)):
            ksr.forward(g, image=ksimg, save=False, check=False)
        torch.cuda.synchronize()
        w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0.record(stream)
        for _ in range(args.steps):
            ksr.forward(g, image=ksimg, save=False, check=False)
        w1.record(stream)
        torch.cuda.synchronize()
        assert ksr.status()[0] == B.HTGS_OK
        kms = max_over_ranks(w0.elapsed_time(w1))
        k_sweep[str(kk)] = {"value": job_throughput(args.steps, world, kms), "unit": UNIT,
                            "ms_per_step": kms / args.steps, "counters": B.htgs_get_counters(ksr.workspace)}
        del ksr, ksimg

    # ---- the same frame rendered without the tail (inference variant) ------
    nprm = scenes.Params(K=prm.K, tau_alpha=prm.tau_alpha, tau_K=prm.tau_K, alpha_max=prm.alpha_max,
                         bg=prm.bg, no_tail=True)
    nr = Renderer(cam, nprm, scene.n, launch=B.c_launch(*fwd_shape[:2], smem_batch=fwd_shape[2]))
    nimg = nr.image_buffer()
    nr.forward(g, image=nimg, save=False, check=True)
    for _ in range(max(args.warmup, 3)):
        nr.forward(g, image=nimg, save=False, check=False)
    torch.cuda.synchronize()
    n0, n1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0.record(stream)
    for _ in range(args.steps):
        nr.forward(g, image=nimg, save=False, check=False)
    n1.record(stream)
    torch.cuda.synchronize()
    assert nr.status()[0] == B.HTGS_OK
    notail_ms = max_over_ranks(n0.elapsed_time(n1))
    no_tail = {"value": job_throughput(args.steps, world, notail_ms), "unit": UNIT,
               "ms_per_step": notail_ms / args.steps, "workload": "the headline frame without the tail"}
    del nr, nimg

    # ---- the variant without per-pixel hybrid transparency (Tab. 3) -------
    sprm = scenes.Params(K=prm.K, tau_alpha=prm.tau_alpha, tau_K=prm.tau_K, alpha_max=prm.alpha_max,
                         bg=prm.bg, sorted_blend=True)
    # The sorted kernels differ from the hybrid ones, so they get their own
    # tile shape (one pixel per thread; the forward's staging batch stays 128).
    def sorted_frame_for(launch_):
        rr = Renderer(cam, sprm, scene.n, launch=launch_)
        im = rr.image_buffer()
        rr.forward(g, image=im, save=False, check=True)
        return lambda: rr.forward(g, image=im, save=False, check=False)

    best_sorted, tune_sorted = autotune(sorted_frame_for, candidates=sorted_candidates, batches=(128,),
                                        warmup=2, repeats=5)
    sorted_tile = (best_sorted.tile_w, best_sorted.tile_h)
    sr = Renderer(cam, sprm, scene.n, launch=B.c_launch(sorted_tile, 1))
    simg = sr.image_buffer()
    sr.forward(g, image=simg, save=False, check=True)
    for _ in range(max(args.warmup, 3)):
        sr.forward(g, image=simg, save=False, check=False)
    torch.cuda.synchronize()
    q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    q0.record(stream)
    for _ in range(args.steps):
        sr.forward(g, image=simg, save=False, check=False)
    q1.record(stream)
    torch.cuda.synchronize()
    assert sr.status()[0] == B.HTGS_OK
    sorted_ms = max_over_ranks(q0.elapsed_time(q1))
    sorted_blend = {"value": job_throughput(args.steps, world, sorted_ms), "unit": UNIT,
                    "ms_per_step": sorted_ms / args.steps,
                    "workload": "the headline frame, mean-depth-sorted alpha blending with early termination"}
    del sr, simg

    # ---- end to end through the C ABI with host buffers --------------------
    # Every step uploads its inputs from pinned host memory and reads its image
    # back. The copies run on streams of their own with two device buffers of
    # each, so the upload of step i + 1 and the read-back of step i - 1 overlap
    # the render of step i: the render waits for its inputs and for the
    # read-back of the image buffer it overwrites, an upload waits for the
    # render that last read its buffer.
    # The five parameter arrays sit in one pinned host buffer and, per slot,
    # in one device buffer (each array starting on a 16-byte boundary), so a
    # step's upload is a single copy; the renders take views of the device
    # buffer.
    keys = ("means", "log_scales", "quats", "opacity_logits", "sh")
    arrs = [np.ascontiguousarray(getattr(scene, k), dtype=np.float32) for k in keys]
    offs, o = [], 0
    for arr in arrs:
        offs.append(o)
        o += -(-arr.size // 4) * 4
    host_all = torch.zeros(o, dtype=torch.float32).pin_memory()
    for arr, off in zip(arrs, offs):
        host_all[off:off + arr.size] = torch.from_numpy(arr.ravel())
    host_img = [torch.empty(image.shape, dtype=torch.float32).pin_memory() for _ in range(2)]
    h2d = host_all.numel() * 4
    d2h = host_img[0].numel() * 4
    dev_all = [torch.empty(o, dtype=torch.float32, device="cuda") for _ in range(2)]
    dev = [GaussianTensors(*[buf[off:off + arr.size].view(arr.shape) for arr, off in zip(arrs, offs)],
                           g.sh_degree) for buf in dev_all]
    imgs = [image, torch.empty_like(image)]
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    inputs_ready = [torch.cuda.Event() for _ in range(2)]
    inputs_free = [torch.cuda.Event() for _ in range(2)]
    image_done = [torch.cuda.Event() for _ in range(2)]
    image_free = [torch.cuda.Event() for _ in range(2)]

    def e2e_step(i):
        b = i % 2
        up.wait_event(inputs_free[b])
        with torch.cuda.stream(up):
            dev_all[b].copy_(host_all, non_blocking=True)
        inputs_ready[b].record(up)
        stream.wait_event(inputs_ready[b])
        stream.wait_event(image_free[b])
        r.forward(dev[b], image=imgs[b], save=False, check=False)
        inputs_free[b].record(stream)
        image_done[b].record(stream)
        down.wait_event(image_done[b])
        with torch.cuda.stream(down):
            host_img[b].copy_(imgs[b], non_blocking=True)
        image_free[b].record(down)

    for i in range(4):
        e2e_step(i)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    up.wait_event(e0)
    for i in range(args.steps):
        e2e_step(i)
    stream.wait_stream(down)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1))
    e2e_fps = job_throughput(args.steps, world, e2e_ms)
    last = (args.steps - 1) % 2
    assert torch.equal(host_img[last], imgs[last].cpu()), "the read-back image must be the render's"
    # The host link's own rate: one step's uploads alone, back to back (the
    # best of three rounds of five, as the host's memory is shared with other
    # work). It bounds the end-to-end rate at h2d bytes / rate, whatever the
    # render does.
    link_gbs = 0.0
    for _ in range(3):
        torch.cuda.synchronize()
        l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0.record(up)
        with torch.cuda.stream(up):
            for _ in range(5):
                dev_all[1].copy_(host_all, non_blocking=True)
        l1.record(up)
        torch.cuda.synchronize()
        link_gbs = max(link_gbs, 5 * h2d / (l0.elapsed_time(l1) * 1e-3) / 1e9)
    del dev, dev_all, imgs[1]

    # ---- training step: render + L1 + backward (500k Gaussians, 1200x800) --
    tscene, ttarget, tcam, tprm = scenes.config3(seed=2 + rank)
    tcam = tcam.rounded()
    tg = GaussianTensors.from_scene(tscene)
    tt = GaussianTensors.from_scene(ttarget)
    def train_step_for(launch_):
        rr = Renderer(tcam, tprm, tscene.n, launch=launch_)
        tgt = rr.forward(tt, save=False, check=True).clone()
        im = rr.image_buffer()
        dl_ = torch.empty_like(im)
        loss_ = torch.zeros(1, dtype=torch.float32, device="cuda")
        grads_ = {k: torch.empty_like(getattr(tg, k)) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
        rr.forward(tg, image=im, save=True, check=True)

        def step():
            rr.forward(tg, image=im, save=True, check=False)
            B._check(B.htgs_l1_loss_grad(im, tgt, dl_, loss_), "htgs_l1_loss_grad")
            rr.backward(tg, dl_, grads=grads_)
        return step

    best_train, tune_train = autotune(train_step_for, warmup=1, repeats=3)
    torch.cuda.empty_cache()
    train_shape = ((best_train.tile_w, best_train.tile_h), best_train.px_per_thread, best_train.smem_batch)
    bev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    for e in bev:
        e.record(stream)
    tlaunch_ev = B.c_launch(train_shape[0], train_shape[1], 0, bev, smem_batch=train_shape[2])
    tr = Renderer(tcam, tprm, tscene.n, launch=B.c_launch(train_shape[0], train_shape[1], smem_batch=train_shape[2]))
    target = tr.forward(tt, save=False, check=True).clone()
    timg = tr.image_buffer()
    dl = torch.empty_like(timg)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    grads = {k: torch.empty_like(getattr(tg, k)) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    tr.forward(tg, image=timg, save=True, check=True)

    def train_step():
        tr.forward(tg, image=timg, save=True, check=False)
        B._check(B.htgs_l1_loss_grad(timg, target, dl, loss), "htgs_l1_loss_grad")
        tr.backward(tg, dl, grads=grads)

    for _ in range(max(args.warmup, 3)):
        train_step()
    torch.cuda.synchronize()
    n_train = max(5, args.steps // 5)
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # An event between consecutive steps as well, for the per-step
    # distribution (one record per 80 ms step).
    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(n_train - 1)]
    with ClockSampler(local) as train_clocks:
        barrier()
        torch.cuda.synchronize()
        s0.record(stream)
        for i in range(n_train):
            train_step()
            if i + 1 < n_train:
                step_ev[i].record(stream)
        s1.record(stream)
        torch.cuda.synchronize()
        barrier()
    train_ms = max_over_ranks(s0.elapsed_time(s1)) / n_train
    marks = [s0] + step_ev + [s1]
    train_dist = dist_summary([marks[i].elapsed_time(marks[i + 1]) for i in range(n_train)])
    bwd_blend_ms, fwd_blend_train_ms = [], []
    tr.launch = tlaunch_ev
    for _ in range(3):
        tr.forward(tg, image=timg, save=True, check=False)
        torch.cuda.synchronize()
        fwd_blend_train_ms.append(bev[4].elapsed_time(bev[5]))
        tcounters = B.htgs_get_counters(tr.workspace)
        B._check(B.htgs_l1_loss_grad(timg, target, dl, loss), "htgs_l1_loss_grad")
        tr.backward(tg, dl, grads=grads)
        torch.cuda.synchronize()
        bwd_blend_ms.append(bev[0].elapsed_time(bev[1]))
    st2, tinst = tr.status()
    assert st2 == B.HTGS_OK
    gfinite = all(bool(torch.isfinite(v).all()) for v in grads.values())

    # the same training step with the variant without per-pixel HT (Tab. 3)
    stprm = scenes.Params(K=tprm.K, tau_alpha=tprm.tau_alpha, tau_K=tprm.tau_K, alpha_max=tprm.alpha_max,
                          bg=tprm.bg, sorted_blend=True)
    def sorted_train_step_for(launch_):
        rr = Renderer(tcam, stprm, tscene.n, launch=launch_)
        tgt = rr.forward(tt, save=False, check=True).clone()
        im = rr.image_buffer()
        dl_ = torch.empty_like(im)
        loss_ = torch.zeros(1, dtype=torch.float32, device="cuda")
        grads_ = {k: torch.empty_like(getattr(tg, k)) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
        rr.forward(tg, image=im, save=True, check=True)

        def step():
            rr.forward(tg, image=im, save=True, check=False)
            B._check(B.htgs_l1_loss_grad(im, tgt, dl_, loss_), "htgs_l1_loss_grad")
            rr.backward(tg, dl_, grads=grads_)
        return step

    best_sorted_train, tune_sorted_train = autotune(sorted_train_step_for, candidates=sorted_candidates,
                                                    batches=(128,), warmup=1, repeats=2)
    torch.cuda.empty_cache()
    sorted_train_tile = (best_sorted_train.tile_w, best_sorted_train.tile_h)
    str_ = Renderer(tcam, stprm, tscene.n, launch=B.c_launch(sorted_train_tile, 1))
    starget = str_.forward(tt, save=False, check=True).clone()
    str_.forward(tg, image=timg, save=True, check=True)

    def sorted_train_step():
        str_.forward(tg, image=timg, save=True, check=False)
        B._check(B.htgs_l1_loss_grad(timg, starget, dl, loss), "htgs_l1_loss_grad")
        str_.backward(tg, dl, grads=grads)

    for _ in range(2):
        sorted_train_step()
    torch.cuda.synchronize()
    u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    u0.record(stream)
    for _ in range(max(3, n_train // 2)):
        sorted_train_step()
    u1.record(stream)
    torch.cuda.synchronize()
    assert str_.status()[0] == B.HTGS_OK
    sorted_train_ms = max_over_ranks(u0.elapsed_time(u1)) / max(3, n_train // 2)
    del str_, starget

    # ---- roofline of every kernel group, in the work units of the plan -----
    # FP32-bound blends: algorithmic FP32 lane-instructions of the direct
    # (Pluecker) evaluation per the measurement plan: 27 per (pixel, Gaussian)
    # pair tested (8 FMA for the planes a, b; 6 for d; 6 for m; 6 for the two
    # norms; 1 compare), +20 per kept fragment (alpha, depth, blending); the
    # adjoint re-tests every pair (27) and spends 2.5x the forward's 20 per
    # kept fragment (50; the plan gives 2-3x). P = pixels inside the
    # Gaussians' tight boxes, A = kept fragments (htgs_get_counters). Peak =
    # the FMA probe's measured rate, scaled by the ratio of the SM clock
    # sampled during the timed region to the one during the probe.
    # The implementation's own instruction counts (its quadratic-form
    # evaluation needs fewer per pair) are kept as `impl_work`.
    # HBM-bound phases: algorithmic bytes per the plan (preprocess: the
    # parameters in, an 84-byte record, an 8-byte tile rectangle and a 4-byte
    # count out per Gaussian; binning and sort: 32 B per instance) over the
    # phase's CUDA-event time, against the measured copy bandwidth.
    K = prm.K
    fp32 = fp32_peak(local)
    probe_mhz = fp32["sm_mhz"]

    def fp32_peak_at(clk):
        mhz = clk.get("sm_mhz") or probe_mhz
        return fp32["fma_per_s"] * (mhz / probe_mhz if probe_mhz else 1.0)

    def plan_fwd(c):
        return 27 * c["box_pairs"] + 20 * c["kept"]

    def impl_fwd(c, k):
        return 8 * c["box_pairs"] + 14 * c["kept"] + 10 * c["admitted"] + 8 * k * c["inserted"]

    head_clocks = clocks.summary()
    peak = fp32_peak_at(head_clocks)
    alg = plan_fwd(counters)
    blend_s = float(np.mean(blend_ms)) / 1e3
    achieved = alg / blend_s
    traffic = recorded_traffic()
    hbm_peak = float(peaks["hbm_gbs"]) * 1e9
    nc = (scene.sh_degree + 1) ** 2
    pre_unit = (3 + 3 + 4 + 1 + 3 * nc) * 4 + 84 + 8 + 4
    pre_bytes = scene.n * pre_unit
    n_tiles = -(-cam.width // fwd_shape[0][0]) * -(-cam.height // fwd_shape[0][1])
    passes = -(-max(1, int(n_tiles - 1).bit_length()) // 9)
    bin_bytes = 32 * inst
    pre_s, bin_s = float(np.mean(pre_ms)) / 1e3, float(np.mean(bin_ms)) / 1e3
    tfwd_s, tbwd_s = float(np.mean(fwd_blend_train_ms)) / 1e3, float(np.mean(bwd_blend_ms)) / 1e3
    train_peak = fp32_peak_at(train_clocks.summary())

    def line(bound, work, secs, pk, unit, scale, per_unit, **extra):
        return dict({"bound": bound, "achieved": work / secs / scale, "peak": pk / scale, "unit": unit,
                     "frac": work / secs / pk, "ms": secs * 1e3, "work": work, "work_per_unit": per_unit},
                    **extra)

    fwd_units = "27 FP32 instr per box pair + 20 per kept fragment"
    kernels = {
        "preprocess_1080p": line("hbm", pre_bytes, pre_s, hbm_peak, "GB/s", 1e9,
                                 f"{pre_unit} B per Gaussian ({pre_unit - 96} in, 96 out)"),
        "binning_sort_1080p": line("hbm", bin_bytes, bin_s, hbm_peak, "GB/s", 1e9, "32 B per instance",
                                   instances=inst),
        "blend_fwd_1080p": line("alu", alg, blend_s, peak, "T FP32 instr/s", 1e12, fwd_units,
                                impl_work=impl_fwd(counters, K),
                                impl_frac=impl_fwd(counters, K) / blend_s / peak),
        "blend_fwd_train": line("alu", plan_fwd(tcounters), tfwd_s, train_peak, "T FP32 instr/s", 1e12,
                                fwd_units, impl_work=impl_fwd(tcounters, tprm.K),
                                impl_frac=impl_fwd(tcounters, tprm.K) / tfwd_s / train_peak),
        "blend_bwd_train": line("alu", 27 * tcounters["box_pairs"] + 50 * tcounters["kept"], tbwd_s, train_peak,
                                "T FP32 instr/s", 1e12, "27 FP32 instr per box pair + 50 per kept fragment",
                                impl_work=8 * tcounters["box_pairs"] + 28 * tcounters["kept"],
                                impl_frac=(8 * tcounters["box_pairs"] + 28 * tcounters["kept"]) / tbwd_s
                                / train_peak),
        "hbm_peak_source": f"hbm_gbs, {peak_src}",
        "fp32_peak": fp32,
    }

    # ---- stress: 6M Gaussians with flat, near-plane and opaque splats --------
    # (5% with one scale 1e-7, 1% near the camera or the near plane, 1% at
    # o = 0.999), 1920x1080, forward + backward at K = 4, 8, 16, 32.
    del tr, tg, tt, grads, timg, dl, target
    torch.cuda.empty_cache()
    sscene, scam, _ = scenes.config5()
    scam = scam.rounded()
    sgs = GaussianTensors.from_scene(sscene)
    stress = {}
    for kk in (4, 8, 16, 32):
        srr = Renderer(scam, scenes.Params(K=kk), sscene.n,
                       launch=B.c_launch(*fwd_shape[:2], smem_batch=fwd_shape[2]))
        simg = srr.forward(sgs, save=True, check=True)
        sdl = torch.randn(simg.shape, device=simg.device, generator=torch.Generator(device=simg.device).manual_seed(5))
        sgrads = srr.backward(sgs, sdl)
        torch.cuda.synchronize()
        x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        x0.record(stream)
        for _ in range(3):
            srr.forward(sgs, image=simg, save=True, check=False)
            srr.backward(sgs, sdl, grads=sgrads)
        x1.record(stream)
        torch.cuda.synchronize()
        st_s, sinst = srr.status()
        assert st_s == B.HTGS_OK
        finite = bool(torch.isfinite(simg).all()) and all(bool(torch.isfinite(v).all()) for v in sgrads.values())
        sms = max_over_ranks(x0.elapsed_time(x1)) / 3
        stress[str(kk)] = {"value": job_throughput(1, world, sms), "unit": "steps/s", "ms_per_step": sms,
                           "instances": sinst, "finite": finite}
        del srr, simg, sdl, sgrads
    del sgs
    torch.cuda.empty_cache()

    batched = None
    if not args.no_batched:
        del r, g, image
        torch.cuda.empty_cache()
        barrier()
        batched = batched_leg(args.batched_steps, args.batched_warmup)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(scene, cam, prm, sscene, scam)
    del sscene

    line = {
        "metric": METRIC, "value": fps, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "gaussians": scene.n, "width": cam.width, "height": cam.height,
                   "K": K, "tile": f"{fwd_shape[0][0]}x{fwd_shape[0][1]}", "px_per_thread": fwd_shape[1],
                   "smem_batch": fwd_shape[2], "parallelism": f"replicas{world}",
                   "autotune_ms": {f"{t[0]}x{t[1]}/ppt{pp}/b{bb}": round(v, 4) for (t, pp, bb), v in tune_fwd.items()},
                   "l2": "inputs larger than L2 (236 MB of Gaussian parameters per frame)"},
        "frame_ms": frame_dist,
        "phases_ms": {"preprocess": float(np.mean(pre_ms)), "binning_sort": float(np.mean(bin_ms)),
                      "blend": float(np.mean(blend_ms))},
        "instances": inst, "counters": counters,
        "fwd_bwd": {"value": job_throughput(1, world, train_ms), "unit": "steps/s", "ms_per_step": train_ms,
                    "step_ms": train_dist,
                    "workload": "500k Gaussians (box distribution), 1200x800, K=8: render + L1 + backward",
                    "launch": {"tile": f"{train_shape[0][0]}x{train_shape[0][1]}", "px_per_thread": train_shape[1],
                               "smem_batch": train_shape[2],
                               "autotune_ms": {f"{t[0]}x{t[1]}/ppt{pp}/b{bb}": round(v, 2)
                                               for (t, pp, bb), v in tune_train.items()}},
                    "instances": tinst, "blend_backward_ms": float(np.mean(bwd_blend_ms)),
                    "blend_forward_ms": float(np.mean(fwd_blend_train_ms)), "clocks": train_clocks.summary(),
                    "grads_finite": gfinite},
        "k_sweep": k_sweep,
        "stress": dict(stress, workload="6M clustered Gaussians at 1920x1080: 5% flat (one scale 1e-7), 1% at "
                                        "the camera or the near plane, 1% at o = 0.999; render + backward"),
        "filter3d": filtered,
        "baked": baked,
        "no_tail": no_tail,
        "sorted_blend": dict(sorted_blend, tile=f"{sorted_tile[0]}x{sorted_tile[1]}",
                             autotune_ms={f"{t[0]}x{t[1]}": round(v, 4) for (t, _, _), v in tune_sorted.items()},
                             fwd_bwd={"value": job_throughput(1, world, sorted_train_ms),
                                      "unit": "steps/s", "ms_per_step": sorted_train_ms,
                                      "tile": f"{sorted_train_tile[0]}x{sorted_train_tile[1]}",
                                      "autotune_ms": {f"{t[0]}x{t[1]}": round(v, 2)
                                                      for (t, _, _), v in tune_sorted_train.items()}}),
        "batched_vs_plain": batched,
        "e2e": {"value": e2e_fps, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "overlap": "uploads and read-backs on two copy streams, double-buffered, overlapping the renders",
                "h2d_link_gbs": round(link_gbs, 1),
                "link_bound": {"value": link_gbs * 1e9 / h2d * world, "unit": UNIT,
                               "note": "h2d bytes per step / the link rate measured with the same uploads alone"}},
        "roofline": {"kernel": "blend_fwd", "bound": "alu", "achieved": achieved / 1e12, "peak": peak / 1e12,
                     "unit": "T FP32 instr/s", "frac": achieved / peak, "traffic": traffic,
                     "work": f"{fwd_units}: {alg:.4g} per launch",
                     "peak_source": f"FMA-chain probe, measured {fp32['fma_per_s'] / 1e12:.2f} T/s at "
                                    f"{probe_mhz} MHz on {fp32['sms']} SMs (device properties), scaled to the "
                                    f"{head_clocks.get('sm_mhz')} MHz sampled during the timed region"},
        "kernels": kernels,
        # per frame: preprocess, scan, emit, histogram, the digit passes,
        # ranges, schedule and the blend
        "gpu_launches": args.steps * (7 + passes),
        "clocks": head_clocks,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
