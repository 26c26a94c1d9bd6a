#!/usr/bin/env python
"""Benchmark of the B300 BMND denoiser: denoised voxels/s, both stages.

Default workload: the 2-D batch (16 images of 512x512 with Poisson counts at
peaks 1, 2, 5, 10, 30 and the same 16 with Gaussian noise sigma 25/255;
patch 8x8, step 3, search 39x39, groups 16/32), all 32 images denoised in one
batched call.  One step = one such call with the inputs resident in HBM.
The line carries the plain path (one call per image) beside it, and the
serving mix (512 requests, Poisson arrivals at 200/s) served by the request
server and by the plain path, with p50/p99 latency.  Other workloads:
--workload c1 (2-D 64x64), c2 (1-D 262144 samples), c4 (3-D 128^3 with mass
conservation), c5 (the serving mix alone), schedules (Sec. 9.3 analysis).

Timing: W untimed warm-up steps, then K steps, each timed with CUDA events on
the launching stream; L2 is flushed (256 MiB write) before every timed step,
outside the events.  N > 1 (torchrun): independent replicas, one per GPU,
each on its own seeded instance of the workload; value = all ranks' voxels /
max-over-ranks time.  --impl reference times the FP64 CPU oracle on the host.
"""
from __future__ import annotations

import argparse
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

from paper_2609_34622_b300 import synth  # noqa: E402

METRIC = "denoised voxels/s (both stages)"
UNIT = "voxels/s"
SMS = 148
FP32_LANES = 128


def workload(name: str, item: int, edge: int = 128, images: int = 32):
    if name == "c1":
        j = synth.config1(item)
        return [j], "2-D 64x64 discs/rectangles, Poisson peak 10, patch 8x8, step 3, search 19x19, groups 16/32"
    if name == "c2":
        j = synth.config2(item)
        return [j], ("1-D ECG-like signal, 262144 samples, Poisson peak 50, patch 32, step 4, search 129, "
                     "groups 16/32, both stages")
    if name == "c3":
        n = max(1, images // 2)
        jobs = synth.config3(n_images=n)
        return jobs, ("2-D batch: %d images 512x512 Poisson (peaks 1,2,5,10,30) + the same %d with Gaussian "
                      "sigma 25/255, patch 8x8, step 3, search 39x39, groups 16/32, one batched call" % (n, n))
    if name == "c4":
        j = synth.config4(item, n=edge)
        return [j], ("3-D %d^3 ellipsoid phantom, Poisson 0.5-5 counts, patch 4x4x4, step 2, search 11^3, "
                     "groups 16/32, mass conservation in both stages" % edge)
    raise SystemExit("unknown workload %s" % name)


def replica_totals(dev_ms: float, e2e_ms: float, vox_step: int, steps: int, world: int, dist=None, device=None):
    """Whole-job figures of N independent replicas (one seeded instance per
    rank, no collective on the data path): the slowest rank's times (MAX over
    ranks) and the voxels all ranks processed.  Returns (dev_ms, e2e_ms,
    value, e2e value) with values in voxels/s."""
    if dist is not None:
        import torch
        t = torch.tensor([dev_ms, e2e_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dev_ms, e2e_ms = float(t[0]), float(t[1])
    total = vox_step * steps * world
    return dev_ms, e2e_ms, total / (dev_ms / 1e3), total / (e2e_ms / 1e3)


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        res = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return res
        time.sleep(0.12)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return res
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[4:8]) if v.lower() == "active"})
        busy = [s for s in sm if s > 0.5 * (max(mx) if mx else 2032)] or sm
        res.update(sm_mhz=statistics.median(busy) if busy else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=reasons, samples=len(rows))
        return res


# ---------------------------------------------------------------------------
# algorithmic work of the stage kernel
# ---------------------------------------------------------------------------

def window_counts(origins: np.ndarray, shape, patch, search) -> np.ndarray:
    """Candidates per reference (clipped window, reference included)."""
    coords = np.stack(np.unravel_index(origins, shape), axis=1)
    n = np.ones(len(origins), np.int64)
    for d, (L, j, w) in enumerate(zip(shape, patch, search)):
        rad = (w - 1) // 2
        lo = np.maximum(coords[:, d] - rad, 0)
        hi = np.minimum(coords[:, d] + rad, L - j)
        n *= hi - lo + 1
    return n


def stage_flops(ncand: np.ndarray, counts: np.ndarray, patch, stage: int, poisson: bool) -> float:
    """Algorithmic FP32 operations of one stage-kernel launch.

    matching: per candidate and patch entry, sub + fma (3), plus add + max +
    add (3) for the Poisson noise bias of stage 1;
    per group of n members and P entries: each dense DCT line of length j costs
    2 j^2 (2 n P j per axis); the Haar along the group costs 4 n P; the
    transforms run: variance (Poisson only, squared matrices), guide forward,
    observation forward (stage 2), inverse; gather/shrink/weights ~10 n P;
    weighted accumulation 4 n P."""
    P = int(np.prod(patch))
    per_entry = 6.0 if (stage == 1 and poisson) else 3.0
    match = float(np.sum(ncand - 1)) * P * per_entry
    n = counts.astype(np.float64)
    one_xform = 2.0 * n * P * float(np.sum(patch)) + 4.0 * n * P
    nx = 2 + (1 if poisson else 0) + (1 if stage == 2 else 0)
    filt = float(np.sum(nx * one_xform + 14.0 * n * P))
    return match + filt


# ---------------------------------------------------------------------------
# oracle timing (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_sample(name: str, jobs):
    """A bounded sample of the workload for the CPU oracle."""
    if name in ("c1", "c2"):
        return jobs[:1], "the full workload (%d voxels)" % jobs[0].y.size
    if name == "c3":
        j = jobs[0]
        y = np.ascontiguousarray(j.y[:96, :96])
        return [synth.Job(y, j.x[:96, :96], j.noise, j.patch, j.step, j.search)], \
            "a 96x96 crop of image 0 of the batch"
    j = jobs[0]
    y = np.ascontiguousarray(j.y[:32, :32, :32])
    return [synth.Job(y, j.x[:32, :32, :32], j.noise, j.patch, j.step, j.search, j.group_size, 2, 3)], \
        "a 32^3 crop of the volume"


def time_oracle(jobs, min_seconds: float, max_reps: int = 1000, matching=("ssd", "fixed"), ht_rule="hard",
                weight_domain="coefficient", cov_planes=0, spatial="dct"):
    import oracle
    oracle.build()
    vox, t0, reps = 0, time.perf_counter(), 0
    while True:
        for j in jobs:
            p = oracle.params(j.y.shape, j.patch, j.step, j.search, j.noise, j.group_size, j.stages,
                              j.mass_conserve, match_metric=matching[0], match_policy=matching[1], ht_rule=ht_rule,
                              weight_domain=weight_domain, cov_planes=cov_planes, spatial_transform=spatial)
            oracle.denoise(p, j.y)
            vox += j.y.size
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds or reps >= max_reps:
            return vox / el, el, reps, oracle.num_threads()


# ---------------------------------------------------------------------------

def captured_traffic(workload: str, n_arrays: int, cores=None):
    """DRAM bytes of the stage kernel per step from the committed ncu summary
    of the workload, if the kernel source is unchanged since the capture
    (else None).  The 1-D signal: one stage launch as captured.  The 2-D
    batch: stage 1 + stage 2 bytes per image of a smaller batch of the same
    images and tiles, times the images of the step (every image is its own
    set of tiles, so the traffic grows in proportion), when the step runs
    the captured tile cores."""
    import hashlib
    import re
    summ = {"c2": "k_stage_1d_262144.md", "c3": "k_stage_2d_512_batch.md"}.get(workload)
    if summ is None:
        return None
    src = os.path.join(ROOT, "paper_2609_34622_b300", "csrc", "bmnd_kernels.cu")
    try:
        text = open(os.path.join(ROOT, "profiles", summ)).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    m1 = re.search(r"kernel_source_sha: ([0-9a-f]{16})", text)
    if not m1 or m1.group(1) != sha:
        return None
    if workload == "c2":
        m2 = re.search(r"traffic_bytes_per_launch: (\d+)", text)
        return int(m2.group(1)) if m2 else None
    m2 = re.search(r"traffic_bytes_per_image: stage1 (\d+), stage2 (\d+)", text)
    m3 = re.search(r"capture_cores: (\d+)x(\d+)", text)
    if cores is not None and m3 and tuple(cores) != (int(m3.group(1)), int(m3.group(2))):
        return None  # other tiles write other partials
    return (int(m2.group(1)) + int(m2.group(2))) * n_arrays if m2 else None


SCHEDULE_SHAPES = [(481, 321), (768, 512), (256, 256), (512, 512)]
SCHEDULE_CONFIGS = [("off", 2.0, 1), ("generated", 0.0, 2), ("generated", 1.0, 2), ("generated", 2.0, 1),
                    ("generated", 2.0, 2), ("generated", 4.0, 2), ("balanced", 2.0, 1), ("balanced", 2.0, 2),
                    ("balanced", 4.0, 2), ("sparse", 2.0, 2)]


def run_schedules(args, local: int, impl: str):
    """Reference-count and coverage-uniformity analysis of the schedules
    (Sec. 9.3) on image shapes of the paper's 2-D test sets (481x321,
    768x512, 256x256, 512x512), 8x8 patches, step 3: per schedule (shift
    density, passes), the mean count relative to the off schedule and the
    median CV of the coverage map.  The official BM3D schedule the paper
    normalizes by is not available, so counts are relative to the off
    lattice.  One step = every configuration on every shape."""
    def analyse_gpu(ctx, torch, dev):
        import paper_2609_34622_b300.bmnd as bm
        res = {}
        for cfg in SCHEDULE_CONFIGS:
            out = []
            for sh in SCHEDULE_SHAPES:
                prm = bm.params(schedule=cfg[0], shift_density=cfg[1], passes=cfg[2])
                cov = torch.empty(sh, dtype=torch.int32, device=dev)
                out.append(ctx.bmnd_coverage(sh, (8, 8), (3, 3), prm, coverage=cov))
            res[cfg] = out
        return res

    def analyse_oracle():
        import oracle
        res = {}
        for cfg in SCHEDULE_CONFIGS:
            out = []
            for sh in SCHEDULE_SHAPES:
                p = oracle.params(sh, (8, 8), (3, 3), (1, 1), schedule=cfg[0], shift_density=cfg[1], passes=cfg[2])
                _, n, cv = oracle.coverage(p)
                out.append((n, cv))
            res[cfg] = out
        return res

    def table(res):
        off = res[SCHEDULE_CONFIGS[0]]
        return [{"schedule": c[0], "shift_density": c[1], "passes": c[2],
                 "count_vs_off": float(np.mean([a[0] / b[0] for a, b in zip(res[c], off)])),
                 "median_cv": float(np.median([a[1] for a in res[c]]))} for c in SCHEDULE_CONFIGS]

    pix = sum(a * b for a, b in SCHEDULE_SHAPES) * len(SCHEDULE_CONFIGS)
    desc = ("schedule analysis: %d schedules x %d shapes (%s), patch 8x8, step 3"
            % (len(SCHEDULE_CONFIGS), len(SCHEDULE_SHAPES), ", ".join("%dx%d" % s for s in SCHEDULE_SHAPES)))
    if impl == "reference":
        for _ in range(args.warmup):
            res = analyse_oracle()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            res = analyse_oracle()
        el = time.perf_counter() - t0
        import oracle
        val = pix * args.steps / el
        print(json.dumps({"metric": "coverage-analysed pixels/s", "value": val, "unit": "pixels/s", "n_gpus": args.gpus,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
                          "data": "synthetic", "impl": "reference", "config": {"workload": desc},
                          "cpu_baseline": {"value": val, "unit": "pixels/s", "cores": oracle.num_threads(),
                                           "kind": "oracle", "sample": "the full analysis"},
                          "e2e": {"value": val, "unit": "pixels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                          "table": table(res)}))
        return
    import torch
    import paper_2609_34622_b300.bmnd as bm
    from paper_2609_34622_b300 import build as B
    B.build()
    dev = torch.device("cuda", local)
    ctx = bm.Context(local)
    for _ in range(args.warmup):
        res = analyse_gpu(ctx, torch, dev)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        res = analyse_gpu(ctx, torch, dev)
    b.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = a.elapsed_time(b)
    line = {"metric": "coverage-analysed pixels/s", "value": pix * args.steps / (ms / 1e3), "unit": "pixels/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": desc, "note": "each call synchronizes to return |R| and CV (analysis path, "
                                                 "not the denoiser's hot path)"},
            "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"]},
            "gpu_launches": 2 * len(SCHEDULE_CONFIGS) * len(SCHEDULE_SHAPES) * args.steps,
            "table": table(res)}
    print(json.dumps(line))
    ctx.close()


def serving_mix(args, local: int) -> dict:
    """Serving mix: 512 requests with Poisson-process arrivals at 200/s, served
    by the library's request server (memory-budgeted admission, continuous
    batching) and, for comparison, by the plain path (one array per call, in
    arrival order).  Latency = result on the host - arrival."""
    import torch
    import paper_2609_34622_b300.bmnd as bm
    reqs = synth.config5(n_requests=args.requests)
    total_vox = sum(r.job.y.size for r in reqs)
    dev = torch.device("cuda", local)

    # warm-up of every kernel class on small inputs
    srv = bm.Server(local, mem_budget=args.budget_gb << 30, max_slots=256)
    for r in reqs[:24]:
        t = srv.bmnd_server_submit(r.job.y, r.job.cfg)
        srv.bmnd_server_wait(t)

    # served
    t0 = time.perf_counter()
    tickets = []
    for r in reqs:
        dt = t0 + r.arrival_s - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        tickets.append((srv.bmnd_server_submit(r.job.y, r.job.cfg), r))
    lat = []
    for t, r in tickets:
        _, l = srv.bmnd_server_wait(t)
        lat.append(l)
    served_span = time.perf_counter() - t0
    st = srv.bmnd_server_get_stats()
    # saturated: every request submitted at once
    t0 = time.perf_counter()
    tickets = [srv.bmnd_server_submit(r.job.y, r.job.cfg) for r in reqs]
    for t in tickets:
        srv.bmnd_server_wait(t)
    served_burst = time.perf_counter() - t0
    srv.close()

    # plain: one request at a time, host input -> device -> both stages -> host
    ctx = bm.Context(local)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    plat = []
    for r in reqs:
        dt = t0 + r.arrival_s - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        c = r.job.cfg
        y = torch.from_numpy(r.job.y).to(dev, non_blocking=False)
        o = torch.empty_like(y)
        ctx.bmnd_denoise(y, o, c["noise"], c["patch"], c["step"], c["search"], c["group_size"], c["stages"],
                         c["mass_conserve"], stream=stream)
        o.cpu()
        plat.append(1e3 * (time.perf_counter() - (t0 + r.arrival_s)))
    plain_span = time.perf_counter() - t0
    t0 = time.perf_counter()
    for r in reqs:
        c = r.job.cfg
        y = torch.from_numpy(r.job.y).to(dev, non_blocking=False)
        o = torch.empty_like(y)
        ctx.bmnd_denoise(y, o, c["noise"], c["patch"], c["step"], c["search"], c["group_size"], c["stages"],
                         c["mass_conserve"], stream=stream)
        o.cpu()
    plain_burst = time.perf_counter() - t0
    ctx.close()

    def q(v, f):
        v = sorted(v)
        return v[min(len(v) - 1, int(round(f * (len(v) - 1))))]
    return {"workload": "serving mix: %d requests, Poisson arrivals at 200/s, 40%% 1-D (8k-262k), "
                        "45%% 2-D (64^2-1024^2), 15%% 3-D (32^3-128^3), Poisson peaks 1-50" % len(reqs),
            "voxels": total_vox, "budget_gb": args.budget_gb,
            "served": {"voxels_per_s": total_vox / served_span, "p50_ms": q(lat, 0.5), "p99_ms": q(lat, 0.99),
                       "span_s": served_span, "steps": st["steps"], "mean_jobs_per_step": st["mean_jobs_per_step"]},
            "plain": {"voxels_per_s": total_vox / plain_span, "p50_ms": q(plat, 0.5), "p99_ms": q(plat, 0.99),
                      "span_s": plain_span},
            "saturated": {"note": "all requests submitted at once, host arrays in and out",
                          "served_voxels_per_s": total_vox / served_burst,
                          "plain_voxels_per_s": total_vox / plain_burst}}


def run_c5(args, local: int):
    """The serving mix alone as the line's workload (value: served voxels/s)."""
    sv = serving_mix(args, local)
    line = {"metric": METRIC, "value": sv["served"]["voxels_per_s"], "unit": UNIT, "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": 1e3 * sv["served"]["span_s"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": sv["workload"], "voxels": sv["voxels"], "budget_gb": sv["budget_gb"]},
            "served": sv["served"], "plain": sv["plain"], "saturated": sv["saturated"]}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default: 20 for the batch, 300 else)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3", choices=["c1", "c2", "c3", "c4", "c5", "schedules"])
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-mix run of the default line")
    ap.add_argument("--requests", type=int, default=512, help="serving mix size (c5)")
    ap.add_argument("--budget-gb", type=int, default=40, help="server memory budget (c5)")
    ap.add_argument("--edge", type=int, default=128, help="volume edge of the 3-D workload (c4)")
    ap.add_argument("--images", type=int, default=32,
                    help="images of the 2-D batch (c3; half Poisson, half Gaussian); smaller only for profiling")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the planner's tiles")
    ap.add_argument("--match-metric", default="ssd", choices=["ssd", "poisson_deviance", "pearson", "anscombe_ssd"],
                    help="stage-1 matching distance (Sec. 4.2)")
    ap.add_argument("--match-policy", default="fixed",
                    choices=["fixed", "reference_finite_count", "candidate_standardized"],
                    help="stage-1 acceptance policy (Sec. 4.3)")
    ap.add_argument("--ht-rule", default="hard", choices=["hard", "soft"],
                    help="stage-1 thresholding rule (Def. \"Coefficient thresholding\")")
    ap.add_argument("--weight-domain", default="coefficient", choices=["coefficient", "windowed_synthesis"],
                    help="aggregation-weight domain of both stages (Sec. 7.3)")
    ap.add_argument("--spatial-transform", default="dct", choices=["dct", "bior1.5"],
                    help="spatial transform of the hard-threshold stage (App. A lists bior1.5)")
    ap.add_argument("--cov-planes", type=int, default=0,
                    help="group-axis planes with the partial shared-source Poisson variance (Sec. 5)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.steps is None:
        args.steps = 20 if args.workload == "c3" else 300

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.workload == "schedules":
        if rank == 0:
            run_schedules(args, local, args.impl)
        return
    if args.impl == "reference":
        if rank != 0:
            return
        jobs, desc = workload(args.workload, 0, args.edge, args.images)
        sample, sdesc = oracle_sample(args.workload, jobs)
        vox = sum(j.y.size for j in sample)
        matching = (args.match_metric, args.match_policy)
        for _ in range(args.warmup):
            time_oracle(sample, 0.0, 1, matching, args.ht_rule, args.weight_domain, args.cov_planes,
                        args.spatial_transform)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            time_oracle(sample, 0.0, 1, matching, args.ht_rule, args.weight_domain, args.cov_planes,
                        args.spatial_transform)
        el = time.perf_counter() - t0
        import oracle
        val = vox * args.steps / el
        line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": {"workload": desc, "sample": sdesc},
                "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                                 "sample": sdesc},
                "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    import paper_2609_34622_b300.bmnd as bm
    from paper_2609_34622_b300 import build as B

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        B.build()
    if dist:
        dist.barrier()

    if args.workload == "c5":
        if rank == 0:
            run_c5(args, local)
        return

    jobs, desc = workload(args.workload, rank, args.edge, args.images)
    ctx = bm.Context(local)
    stream = torch.cuda.current_stream()
    ys = [torch.from_numpy(j.y).to(dev) for j in jobs]
    outs = [torch.empty_like(y) for y in ys]
    cfgs = [j.cfg for j in jobs]
    vox_step = sum(j.y.size for j in jobs)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2
    pmetric = args.match_metric != "ssd"
    variant = (pmetric or args.ht_rule != "hard" or args.weight_domain != "coefficient" or args.cov_planes > 0
               or args.spatial_transform != "dct")
    prm = (bm.params(match_metric=args.match_metric, match_policy=args.match_policy, ht_rule=args.ht_rule,
                     weight_domain=args.weight_domain, cov_planes=args.cov_planes,
                     spatial_transform=args.spatial_transform) if variant else None)

    def step(yy, oo):
        if len(jobs) == 1:
            c = cfgs[0]
            ctx.bmnd_denoise(yy[0], oo[0], c["noise"], c["patch"], c["step"], c["search"], c["group_size"],
                             c["stages"], c["mass_conserve"], prm, stream=stream)
        else:
            ctx.bmnd_denoise_batch(yy, oo, cfgs, prm, stream=stream)

    # algorithmic work per stage launch (outside any timing)
    flops = {1: 0.0, 2: 0.0}
    mflops = {1: 0.0, 2: 0.0}
    pilots = []
    refs_step = 0  # reference patches per step, both stages
    for j, y in zip(jobs, ys):
        c = j.cfg
        o, _, cnt1 = ctx.bmnd_match(y, c["noise"], c["patch"], c["step"], c["search"], c["group_size"][0], 1, prm)
        refs_step += int(o.numel()) * c["stages"]
        pilot = torch.empty_like(y)
        ctx.bmnd_stage(y, None, pilot, c["noise"], c["patch"], c["step"], c["search"], c["group_size"][0], 1,
                       c["mass_conserve"] & 1, prm)
        _, _, cnt2 = ctx.bmnd_match(pilot, c["noise"], c["patch"], c["step"], c["search"], c["group_size"][1], 2)
        ncand = window_counts(o.cpu().numpy(), j.y.shape, c["patch"], c["search"])
        pois = c["noise"][0] == "poisson"
        flops[1] += stage_flops(ncand, cnt1.cpu().numpy(), c["patch"], 1, pois)
        flops[2] += stage_flops(ncand, cnt2.cpu().numpy(), c["patch"], 2, pois)
        P = int(np.prod(c["patch"]))
        mflops[1] += float(np.sum(ncand - 1)) * P * (6.0 if pois else 3.0)
        mflops[2] += float(np.sum(ncand - 1)) * P * 3.0
        pilots.append(pilot)
        if c["mass_conserve"]:
            # the second sweep repeats the filtering (not the matching)
            pass

    # tile autotuning (outside any timing): a single array is timed alone, a
    # batch as one batched call (the arrays share the SMs)
    tuned = {}
    if not args.no_autotune and len(jobs) > 1:
        tuned["batch"] = ctx.bmnd_autotune_batch(ys, outs, cfgs, prm, stream=stream)
    if not args.no_autotune and len(jobs) == 1:
        for j, y, o in zip(jobs, ys, outs):
            c = j.cfg
            key = (tuple(j.y.shape), tuple(c["patch"]), tuple(c["step"]), tuple(c["search"]),
                   tuple(c["group_size"]), c["stages"], c["mass_conserve"])
            if key not in tuned:
                tuned[key] = ctx.bmnd_autotune(y, o, c["noise"], c["patch"], c["step"], c["search"],
                                               c["group_size"], c["stages"], c["mass_conserve"], prm,
                                               stream=stream)
    torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(ys, outs)
    torch.cuda.synchronize()
    fp32_peak = bm.bmnd_fp32_fma_peak(local)
    hbm_peak, hbm_peak_measured = 6400.0, False
    try:
        hbm_peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
        hbm_peak_measured = True
    except (OSError, KeyError, ValueError):
        pass

    # ---- matching alone: the match-only stage launches of bmnd_match ----
    match_frac = {}
    ctx.bmnd_set_profiling(True)
    reps = max(1, min(20, 2048 // len(jobs)))
    for s_ in (1, 2):
        ctx.bmnd_kernel_stats(reset=True)
        for _ in range(reps):
            for j, y, pl in zip(jobs, ys, pilots):
                c = j.cfg
                ctx.bmnd_match(y if s_ == 1 else pl, c["noise"], c["patch"], c["step"], c["search"],
                               c["group_size"][s_ - 1], s_, prm)
        n_m, ms_m = ctx.bmnd_kernel_stats(reset=True)["match"]
        match_frac[s_] = (mflops[s_] * reps / (ms_m / 1e3) / 1e12) if ms_m > 0 else None
    ctx.bmnd_set_profiling(False)
    torch.cuda.synchronize()

    # ---- device-resident timing ----
    ctx.bmnd_set_profiling(True)
    ctx.bmnd_kernel_stats(reset=True)
    clocks = ClockSampler(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.2)
    # the timed steps are the profiler range (a launch list or a capture
    # under ncu --profile-from-start off covers exactly these launches)
    torch.cuda.profiler.start()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        step(ys, outs)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    dev_ms = sum(a.elapsed_time(b) for a, b in ev)
    kstats = ctx.bmnd_kernel_stats(reset=True)
    ctx.bmnd_set_profiling(False)

    # ---- several arrays: the plain path, one call per array, same timing,
    # on a context of its own (the planner's tiles for a single array: the
    # batch's tuned cores are chosen for arrays that share the GPU) ----
    plain_ms = None
    if len(jobs) > 1:
        pctx = bm.Context(local)
        for y, o, c in zip(ys, outs, cfgs):  # untimed: scratch and tables of the new context
            pctx.bmnd_denoise(y, o, c["noise"], c["patch"], c["step"], c["search"], c["group_size"],
                              c["stages"], c["mass_conserve"], prm, stream=stream)
        torch.cuda.synchronize()
        evp = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for k in range(args.steps):
            flush.fill_(float(k))
            evp[k][0].record(stream)
            for y, o, c in zip(ys, outs, cfgs):
                pctx.bmnd_denoise(y, o, c["noise"], c["patch"], c["step"], c["search"], c["group_size"],
                                  c["stages"], c["mass_conserve"], prm, stream=stream)
            evp[k][1].record(stream)
        torch.cuda.synchronize()
        plain_ms = sum(a.elapsed_time(b) for a, b in evp)
        pctx.close()

    # ---- end to end through the C ABI with host buffers: the host-array
    # batch call copies pinned host inputs in, runs both stages, copies the
    # results back and returns when they are in host memory ----
    hy = [torch.from_numpy(j.y).pin_memory() for j in jobs]
    ho = [torch.empty(j.y.shape, dtype=torch.float32).pin_memory() for j in jobs]
    hyn = [h.numpy() for h in hy]
    hon = [h.numpy() for h in ho]
    ctx.bmnd_denoise_batch_host(hyn, hon, cfgs, prm, stream=stream)
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.bmnd_denoise_batch_host(hyn, hon, cfgs, prm, stream=stream)
        e2e_ms += 1e3 * (time.perf_counter() - t0)

    # double-precision decisions of one step (outside any timing)
    ctx.bmnd_decision_stats(reset=True)
    step(ys, outs)
    torch.cuda.synchronize()
    decisions = ctx.bmnd_decision_stats(reset=True)

    dev_ms, e2e_ms, value, e2e_val = replica_totals(dev_ms, e2e_ms, vox_step, args.steps, world,
                                                    dist if dist else None, dev)

    # tile cores of the first array as the step ran it
    c0 = cfgs[0]
    inf0 = ctx.bmnd_plan_info(jobs[0].y.shape, c0["patch"], c0["step"], c0["search"], c0["group_size"],
                              c0["stages"], c0["mass_conserve"], prm)
    plan_cores = tuple(inf0["core"]) if "core" in inf0 else None
    # roofline of the dominant kernel (the stage kernel, both stages)
    n1, ms1 = kstats["stage1"]
    n2, ms2 = kstats["stage2"]
    stage_ms = ms1 + ms2
    stage_flop = flops[1] * n1 + flops[2] * n2
    achieved = stage_flop / (stage_ms / 1e3) / 1e12 if stage_ms > 0 else None
    mhz = clk["sm_mhz"] or 2032.0
    peak_nominal = SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12
    peak = fp32_peak if fp32_peak else peak_nominal
    # reduce kernel: reads every tile's partial (float2 per region cell) and
    # writes the estimate (and eta when mass conservation runs a second sweep)
    red_bytes = 0.0
    for j, c in zip(jobs, cfgs):
        for s_ in range(1, c["stages"] + 1):
            gm = c["group_size"][s_ - 1]
            inf = ctx.bmnd_plan_info(j.y.shape, c["patch"], c["step"], c["search"], (gm, gm), 1, 0, prm)
            mc = (c["mass_conserve"] >> (s_ - 1)) & 1
            red_bytes += (1 + mc) * (8.0 * inf["tiles"] * inf["region"] + 4.0 * j.y.size) + mc * 4.0 * j.y.size
    nred, ms_red = kstats["reduce"]
    red_gbs = red_bytes * args.steps / (ms_red / 1e3) / 1e9 if ms_red > 0 else None
    launches = sum(v[0] for v in kstats.values()) + kstats["schedule"][0]  # schedule = mark + compact
    step_ms_total = sum(v[1] for v in kstats.values())

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "voxels_per_step_per_gpu": vox_step, "l2": "flushed (256 MiB) before each step",
                   "parallelism": "replicas" if world > 1 else "single",
                   "tiles": ("autotuned cores %s (%s, before the warm-up)"
                             % (sorted(set(tuned.values())),
                                "bmnd_autotune_batch on the whole batch" if len(jobs) > 1 else "bmnd_autotune")
                             if tuned else "planner")},
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"],
                   "samples": clk["samples"]},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 4 * vox_step, "d2h_bytes_per_step": 4 * vox_step,
                "path": "bmnd_denoise_batch_host: pinned host arrays in and out, copies inside the call, "
                        "host wall clock per call"},
        "gpu_launches": int(launches),
        "reference_patches_per_s": refs_step * args.steps * world / (dev_ms / 1e3),
        "decisions_per_step": dict(decisions, note="taken in double precision (or exact integer arithmetic) "
                                                   "where the FP32 error bounds could not decide"),
        "roofline": {"kernel": "k_stage (stage 1 + stage 2 launches)", "bound": "alu", "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
                     "traffic": captured_traffic(args.workload, len(jobs), plan_cores),
                     "traffic_basis": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of the stage launches "
                                       "of one step (profiles/), null once the kernel source changed"),
                     "peak_basis": ("measured FP32 FMA throughput (bmnd_fp32_fma_peak, this run); nominal "
                                    "148 SMs x 128 lanes x 2 flop x %.0f MHz = %.1f TFLOP/s" % (mhz, peak_nominal)),
                     "stage_kernel_ms_per_step": stage_ms / args.steps,
                     "kernel_ms_per_step": {k: v[1] / args.steps for k, v in kstats.items()},
                     "share_of_step": stage_ms / step_ms_total if step_ms_total else None,
                     "matching_alone": {
                         "note": "match-only launches (bmnd_match): SSD (+ Poisson bias in stage 1) and top-k "
                                 "selection; algorithmic FLOPs of the scores only",
                         "stage1_tflops": match_frac[1], "stage2_tflops": match_frac[2],
                         "stage1_frac": match_frac[1] / peak if match_frac[1] else None,
                         "stage2_frac": match_frac[2] / peak if match_frac[2] else None},
                     "reduce": {"kernel": "k_reduce", "bound": "hbm", "bytes_per_step": red_bytes,
                                "achieved_gbs": red_gbs, "peak_gbs": hbm_peak,
                                "frac": red_gbs / hbm_peak if red_gbs and hbm_peak else None,
                                "peak_basis": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth)" if hbm_peak_measured
                                else "fallback 6400 GB/s"}},
    }
    if args.ht_rule != "hard":
        line["config"]["ht_rule"] = args.ht_rule
    if args.weight_domain != "coefficient":
        line["config"]["weight_domain"] = args.weight_domain
    if args.cov_planes > 0:
        line["config"]["cov_planes"] = args.cov_planes
    if args.spatial_transform != "dct":
        line["config"]["spatial_transform"] = args.spatial_transform
    if pmetric:
        # the FLOP model above is the SSD path's; the Poisson distances spend
        # divisions, logarithms and square roots per entry pair that it does
        # not count, so no fraction is claimed for them
        line["config"]["matching"] = {"metric": args.match_metric, "policy": args.match_policy}
        line["roofline"] = {"kernel": "k_stage (generic, Poisson distances)", "bound": "alu", "achieved": None,
                            "peak": peak, "unit": "TFLOP/s", "frac": None, "traffic": None,
                            "stage_kernel_ms_per_step": stage_ms / args.steps,
                            "kernel_ms_per_step": {k: v[1] / args.steps for k, v in kstats.items()},
                            "share_of_step": stage_ms / step_ms_total if step_ms_total else None}
    line["roofline"]["fp32_peak_measured_tflops"] = fp32_peak
    if plain_ms is not None:
        line["plain"] = {"value": vox_step * args.steps / (plain_ms / 1e3), "unit": UNIT,
                         "ms_per_step": plain_ms / args.steps,
                         "path": "one bmnd_denoise call per array, same stream, same timing, planner tiles"}
        line["config"]["batched"] = "one bmnd_denoise_batch call over all %d arrays per step" % len(jobs)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample, sdesc = oracle_sample(args.workload, jobs)
        v, el, reps, cores = time_oracle(sample, 10.0, matching=(args.match_metric, args.match_policy),
                                         ht_rule=args.ht_rule, weight_domain=args.weight_domain,
                                         cov_planes=args.cov_planes, spatial=args.spatial_transform)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "%s, both stages, %d repetition(s), %.1f s" % (sdesc, reps, el)}
    ctx.close()
    if rank == 0 and world == 1 and args.workload == "c3" and not args.no_serving:
        line["serving"] = serving_mix(args, local)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
