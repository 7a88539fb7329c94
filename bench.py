"""Benchmark of the BAD / HashSIFT descriptor path on GB300.

One step = the whole extraction + matching path over one image pair:
integral image + BAD gather for both images, fused patch-warp + histogram and
tcgen05 projection (BF16 + FP32 rescue) for both images, then brute-force
Hamming top-2 + ratio matching of image A against image B for both
descriptor types.  Inputs are synthetic (seeded), shaped like the paper's
workloads; see the design doc for the recipe.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload plain|large]
    python bench.py --impl reference ...   # the CPU oracle on a bounded sample

Prints one JSON line (rank 0).
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

METRIC = ("descriptors/sec (BAD-256, HashSIFT-256) and Hamming matches/sec on 1 GB300, "
          "% of roofline")
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")


def load_peaks():
    try:
        with open(PEAKS_PATH) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

class Workload:
    """Host-side inputs of one step and their device copies."""

    def __init__(self, name: str):
        import synth
        self.name = name
        if name == "plain":
            wl = synth.plain_workload(1000)  # 640x480, 1000 keypoints, BAD-256, HashSIFT-256
            self.config = {"workload": "plain image pair 640x480, 1000 keypoints, BAD-256 + "
                                       "HashSIFT-256 (BF16+rescue), 1000x1000 top-2/ratio 0.8 "
                                       "match per descriptor",
                           "images": "2 x 640x480 uint8", "keypoints_per_image": 1000,
                           "bad_bits": 256, "hashsift_bits": 256, "angle_bins": 32}
        elif name == "large":
            wl = synth.large_pair_workload(1004)  # 2 x 3840x2160, 20000 kps, BAD-256, HashSIFT-512
            self.config = {"workload": "large image pair 3840x2160 (B = homography + noise), "
                                       "20000 keypoints each, BAD-256 + HashSIFT-512 (BF16+rescue), "
                                       "20000x20000 top-2/ratio 0.8 match per descriptor",
                           "images": "2 x 3840x2160 uint8", "keypoints_per_image": 20000,
                           "bad_bits": 256, "hashsift_bits": 512, "angle_bins": 32}
        else:
            raise SystemExit(f"unknown workload {name}")
        self.wl = wl
        self.n = int(wl.kps_a.shape[0])
        self.bad_bits = wl.bad.nbits
        self.hs_bits = wl.hs.nbits
        self.descriptors_per_step = 4 * self.n
        self.pairs_per_step = 2 * self.n * self.n

    # ---- GPU -----------------------------------------------------------
    def to_device(self, ctx):
        import torch
        import paper_2108_08380_gb300 as bd
        wl = self.wl
        dev = "cuda"
        self.img = [torch.from_numpy(wl.img_a).to(dev), torch.from_numpy(wl.img_b).to(dev)]
        self.kps = [torch.from_numpy(wl.kps_a).to(dev), torch.from_numpy(wl.kps_b).to(dev)]
        self.bp = ctx.bad_params(wl.bad)
        self.hp = ctx.hs_params(wl.hs, precision=bd.BD_HS_BF16_RESCUE)
        n = self.n
        i32 = torch.int32
        self.bad = [torch.empty((n, self.bad_bits // 32), dtype=i32, device=dev) for _ in range(2)]
        self.hs = [torch.empty((n, self.hs_bits // 32), dtype=i32, device=dev) for _ in range(2)]
        self.m_bad = torch.empty((n, 3), dtype=i32, device=dev)
        self.m_hs = torch.empty((n, 3), dtype=i32, device=dev)

    def stages(self, ctx):
        """(label, callable) of the ABI calls of one step, in order."""
        return [
            ("bad_describe_A", lambda: ctx.bad_describe(self.bp, self.img[0], self.kps[0], out=self.bad[0])),
            ("bad_describe_B", lambda: ctx.bad_describe(self.bp, self.img[1], self.kps[1], out=self.bad[1])),
            ("hashsift_describe_A", lambda: ctx.hashsift_describe(self.hp, self.img[0], self.kps[0], out=self.hs[0])),
            ("hashsift_describe_B", lambda: ctx.hashsift_describe(self.hp, self.img[1], self.kps[1], out=self.hs[1])),
            ("match_bad", lambda: ctx.match(self.bad[0], self.bad[1], self.bad_bits, 4, 5, out=self.m_bad)),
            ("match_hashsift", lambda: ctx.match(self.hs[0], self.hs[1], self.hs_bits, 4, 5, out=self.m_hs)),
        ]

    # ---- CPU oracle ----------------------------------------------------
    def oracle_step(self, sample_kp: int):
        """The oracle on the first `sample_kp` keypoints of both images (all
        stages); returns the descriptors and pairs it covered."""
        import oracle
        wl = self.wl
        s = min(sample_kp, self.n)
        ka, kb = wl.kps_a[:s], wl.kps_b[:s]
        da, _ = oracle.bad_describe(wl.img_a, ka, wl.bad)
        db, _ = oracle.bad_describe(wl.img_b, kb, wl.bad)
        ha = oracle.hs_describe(wl.img_a, ka, wl.hs)["bits"]
        hb = oracle.hs_describe(wl.img_b, kb, wl.hs)["bits"]
        oracle.match(da, db, self.bad_bits)
        oracle.match(ha, hb, self.hs_bits)
        return 4 * s, 2 * s * s


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append((time.time(), parts))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self, t0, t1):
        rows = [r for (ts, r) in self.rows if t0 <= ts <= t1] or [r for (_, r) in self.rows]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in rows if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    wl = Workload(args.workload)
    sample = args.ref_sample_kp
    # warm the oracle (build + page-in) outside the timed steps
    wl.oracle_step(8)
    t_desc = t_pairs = 0
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps)):
        d, p = wl.oracle_step(sample)
        t_desc += d
        t_pairs += p
    dt = time.perf_counter() - t0
    value = t_desc / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "descriptors/s",
        "n_gpus": 0, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8/int64/f64",
        "data": "synthetic", "config": dict(wl.config, sample_keypoints_per_image=sample),
        "matches_per_s": t_pairs / dt,
        "cpu_baseline": {"value": value, "unit": "descriptors/s", "cores": 1, "kind": "oracle",
                         "sample": f"first {sample} keypoints of each image per step, all stages "
                                   "(BAD, HashSIFT, both matchings), single-threaded C"},
        "e2e": {"value": value, "unit": "descriptors/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(wl, budget_s: float):
    """The oracle, as it stands, on host cores: steps of a bounded keypoint sample."""
    sample = min(wl.n, 250 if wl.name == "plain" else 120)
    wl.oracle_step(4)
    t0 = time.perf_counter()
    nd = npairs = steps = 0
    while True:
        d, p = wl.oracle_step(sample)
        nd += d
        npairs += p
        steps += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": nd / dt, "unit": "descriptors/s", "cores": 1, "kind": "oracle",
            "sample": f"{steps} oracle step(s) over the first {sample} keypoints of each image "
                      f"(BAD, HashSIFT, both matchings), single-threaded C, {dt:.1f} s",
            "matches_per_s": npairs / dt}


def run_ours(args):
    import torch
    import paper_2108_08380_gb300 as bd

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        pg = dist

    ctx = bd.Context(local)
    wl = Workload(args.workload)
    wl.to_device(ctx)
    stages = wl.stages(ctx)
    n_launch0 = bd.kernel_launches()

    # warm-up (also sizes the scratch area)
    for _ in range(max(3, args.warmup)):
        for _, fn in stages:
            fn()
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0, "device flags raised during warm-up"

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 2 x L2
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(stages) + 1)] for _ in range(K)]
    props = torch.cuda.get_device_properties(local)
    sampler = ClockSampler(getattr(props, "uuid", None) and f"GPU-{props.uuid}" or str(local))
    sampler.start()
    time.sleep(0.3)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    launches_before = bd.kernel_launches()
    t_wall0 = time.time()
    for s in range(K):
        flush.fill_(float(s))               # evict the previous step's data from L2
        torch.cuda._sleep(200_000)          # let the host enqueue the whole step first
        ev[s][0].record()
        for j, (_, fn) in enumerate(stages):
            fn()
            ev[s][j + 1].record()
    torch.cuda.synchronize()
    t_wall1 = time.time()
    launches = bd.kernel_launches() - launches_before
    if pg:
        pg.barrier()
    time.sleep(0.15)
    sampler.stop()
    clocks = sampler.summary(t_wall0 - 0.05, t_wall1 + 0.05)

    stage_ms = np.array([[ev[s][j].elapsed_time(ev[s][j + 1]) for j in range(len(stages))]
                         for s in range(K)])
    step_ms = stage_ms.sum(axis=1)
    ms = float(step_ms.mean())
    if pg:
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    assert ctx.sync_status() == 0, "device flags raised during the timed steps"

    # ---- end to end through the public API with pinned host buffers ----
    e2e = measure_e2e(ctx, wl, stages, max(3, min(K, 50)))

    if rank != 0:
        return
    per_stage = {lab: float(stage_ms[:, j].mean()) for j, (lab, _) in enumerate(stages)}
    roof = roofline(wl, per_stage, stage_ms, args)
    value = world * wl.descriptors_per_step / (ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "descriptors/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8/int32 (BAD, matching), f32 + bf16 tensor (HashSIFT)",
        "data": "synthetic",
        "config": dict(wl.config, l2="flushed between steps (512 MB write)",
                       parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
        "matches_per_s": world * wl.pairs_per_step / (ms * 1e-3),
        "stage_ms": per_stage,
        "roofline": roof,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": int(launches),
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_budget)
    print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def measure_e2e(ctx, wl, stages, steps):
    """Same step through the API with host buffers: H2D of both images and
    keypoint sets from pinned memory, the step, D2H of all descriptors and
    match records, inside the timed region."""
    import torch
    host_in = [torch.from_numpy(wl.wl.img_a).pin_memory(), torch.from_numpy(wl.wl.img_b).pin_memory(),
               torch.from_numpy(wl.wl.kps_a).pin_memory(), torch.from_numpy(wl.wl.kps_b).pin_memory()]
    dev_in = [wl.img[0], wl.img[1], wl.kps[0], wl.kps[1]]
    dev_out = [wl.bad[0], wl.bad[1], wl.hs[0], wl.hs[1], wl.m_bad, wl.m_hs]
    host_out = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in dev_out]
    bi = sum(t.numel() * t.element_size() for t in host_in)
    bo = sum(t.numel() * t.element_size() for t in host_out)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        for d, h in zip(dev_in, host_in):
            d.copy_(h, non_blocking=True)
        for _, fn in stages:
            fn()
        for h, d in zip(host_out, dev_out):
            h.copy_(d, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"value": wl.descriptors_per_step / (ms * 1e-3), "unit": "descriptors/s",
            "ms_per_step": ms, "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo)}


def roofline(wl, per_stage, stage_ms, args):
    """Roofline of the dominant call of the step (roofline table)."""
    peaks, kind = load_peaks()
    lab = max(per_stage, key=per_stage.get)
    t = per_stage[lab] * 1e-3
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    n = wl.n
    if lab.startswith("match"):
        K = wl.bad_bits if lab == "match_bad" else wl.hs_bits
        popc = n * n * (K // 32)
        peak = 152 * 16 * sm_mhz * 1e6 / 1e12  # Tpopc/s: 152 SMs x 16 POPC/clk
        achieved = popc / t / 1e12
        return {"bound": "alu", "kernel": lab, "achieved": achieved, "peak": peak,
                "unit": "Tpopc/s", "frac": achieved / peak, "traffic": None,
                "peak_source": f"derived: 152 SMs x 16 POPC/clk x {sm_mhz:.0f} MHz"}
    if lab.startswith("hashsift"):
        flops = 2.0 * 128 * wl.hs_bits * n
        peak = float(peaks["bf16_tflops"])
        achieved = flops / t / 1e12
        return {"bound": "tensor", "kernel": lab, "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": f"{kind} bf16 burst"}
    # BAD: integral (5 B/px) + descriptor output, HBM
    px = wl.wl.img_a.size
    byts = 5.0 * px + n * (wl.bad_bits // 8) + 16 * n
    peak = float(peaks["hbm_gbs"])
    achieved = byts / t / 1e9
    return {"bound": "hbm", "kernel": lab, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None, "peak_source": f"{kind} HBM copy"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["plain", "large"], default="plain")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--ref-sample-kp", type=int, default=250)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
