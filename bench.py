"""Benchmark of the BAD / HashSIFT descriptor path on GB300.

One step = the whole extraction + matching path over one image pair:
integral image + BAD gather for both images, fused patch-warp + histogram and
tcgen05 projection (BF16 + FP32 rescue) for both images, then brute-force
Hamming top-2 + ratio matching of image A against image B for both
descriptor types.  Inputs are synthetic (seeded), shaped like the paper's
workloads (generators in synth/).

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
    """Host-side inputs of one step, their device copies and the step's ABI calls."""

    def __init__(self, name: str, match_kind: str = "tensor", rank: int = 0):
        """rank > 0 draws its own inputs of the same shape (seed + 100 x rank):
        ranks describe independent images (weak scaling)."""
        import synth
        self.name = name
        self.rank = rank
        off = 100 * rank
        self.match = True
        self.match_kind = match_kind
        if name == "plain":
            wl = synth.plain_workload(1000 + off)  # 640x480, 1000 keypoints, BAD-256, HashSIFT-256
            self.images = [wl.img_a, wl.img_b]
            self.kps = np.concatenate([wl.kps_a, wl.kps_b])
            self.offsets = np.array([0, len(wl.kps_a), 2 * len(wl.kps_a)], np.int32)
            self.band = -1.0
            self.config = {"workload": "plain image pair 640x480 (B = A + N(0,5)), 1000 keypoints "
                                       "each, BAD-256 + HashSIFT-256 (BF16+rescue), 1000x1000 "
                                       "top-2/ratio 0.8 match per descriptor",
                           "images": "2 x 640x480 uint8", "keypoints_per_image": 1000,
                           "bad_bits": 256, "hashsift_bits": 256, "angle_bins": 32}
        elif name == "large":
            wl = synth.large_pair_workload(1004 + off)  # 2 x 3840x2160, 20000 kps, BAD-256, HashSIFT-512
            self.images = [wl.img_a, wl.img_b]
            self.kps = np.concatenate([wl.kps_a, wl.kps_b])
            self.offsets = np.array([0, len(wl.kps_a), 2 * len(wl.kps_a)], np.int32)
            self.band = -1.0
            self.config = {"workload": "large image pair 3840x2160 (B = homography + noise), "
                                       "20000 keypoints each, BAD-256 + HashSIFT-512 (BF16+rescue), "
                                       "20000x20000 top-2/ratio 0.8 match per descriptor",
                           "images": "2 x 3840x2160 uint8", "keypoints_per_image": 20000,
                           "bad_bits": 256, "hashsift_bits": 512, "angle_bins": 32}
        elif name == "batch":
            wl = synth.batch_workload(1002 + off)  # 64 images, 200k kps, BAD-512, HashSIFT-512 (BF16 W)
            self.images = wl.images
            self.kps = wl.kps
            self.offsets = wl.kp_offsets
            self.band = 1e-3
            self.match = False
            self.config = {"workload": "64 images 480x360..1920x1080, 200000 keypoints (log-uniform "
                                       "500-8000 per image), 5-level 1.2 pyramid, BAD-512 + "
                                       "HashSIFT-512 (BF16 W, rescue band 1e-3), one persistent "
                                       "launch in a CUDA graph, autotuned",
                           "images": "64 uint8", "keypoints": 200000, "bad_bits": 512,
                           "hashsift_bits": 512, "angle_bins": 32}
        else:
            raise SystemExit(f"unknown workload {name}")
        self.wl = wl
        self.n = int(self.kps.shape[0])
        self.bad_bits = wl.bad.nbits
        self.hs_bits = wl.hs.nbits
        self.descriptors_per_step = 2 * self.n
        if self.match:
            na = int(self.offsets[1])
            self.pairs_per_step = 2 * na * (self.n - na)
            if self.match_kind == "auto":
                # small pairs: matched by the describing launch itself
                self.match_kind = "tensor" if na * (self.n - na) >= (1 << 24) else "fused"
        else:
            self.pairs_per_step = 0
        self._sectors = None

    def l1_sectors(self) -> float:
        """Distinct L1 sectors of every keypoint's BAD corner reads in one step
        (bad_l1_sectors per image; the 64-image batch counts a seeded sample
        of 250 keypoints per image and scales it)."""
        if self._sectors is None:
            tot = 0.0
            for i, im in enumerate(self.images):
                lo, hi = int(self.offsets[i]), int(self.offsets[i + 1])
                if hi > lo:
                    h, w = im.shape
                    sct, _ = bad_l1_sectors(self.bp, self.wl.bad.level_scales, self.kps[lo:hi], w, h,
                                            sample=250 if self.name == "batch" else None, seed=i)
                    tot += sct
            self._sectors = tot
        return self._sectors

    def matching_in_kernel(self) -> bool:
        """The plan's matchings run as work items of the persistent kernel:
        it then holds every descriptor they read (the FP32 projection is fused;
        with the tcgen05 projection after it they run as one matching launch)."""
        return bool(self.match_kind == "fused" and self.tuned and self.tuned.get("proj_fused"))

    def projection_path(self) -> str:
        """The HashSIFT projection the launch configuration runs."""
        if self.tuned and self.tuned.get("proj_fused"):
            bits = 16 if self.tuned.get("proj_half") else 32
            return (f"FP32 CUDA-core projection tiles ({bits} bits x 32 keypoints) inside the "
                    "persistent kernel (proj_fused = 1), the FP32 path's summation order")
        return "tcgen05 BF16 head/tail split with FP32 re-check of the band (hs_proj_tc)"

    # ---- GPU -----------------------------------------------------------
    def to_device(self, ctx, autotune=True, config=None):
        import paper_2108_08380_gb300 as bd
        self.bp = ctx.bad_params(self.wl.bad)
        self.hp = ctx.hs_params(self.wl.hs, precision=bd.BD_HS_BF16_RESCUE, band=self.band)
        self.set0 = DeviceSet(self, ctx)
        for k in ("host_in", "in_arena", "dimg", "dkps", "out_arena", "bad", "hs", "plan",
                  "m_bad", "m_hs"):
            setattr(self, k, getattr(self.set0, k, None))
        self.tuned = None
        if config is not None:
            self.plan.set_config(*config)
            self.tuned = self.plan.config()
        elif autotune:
            self.tuned, _ = self.plan.autotune(self.dimg, self.dkps, self.bad, self.hs, reps=5)

    def second_set(self, ctx):
        """Another copy of the step's device buffers and plan, in the same
        launch configuration (double-buffered end-to-end steps)."""
        ds = DeviceSet(self, ctx)
        if self.tuned is not None:
            ds.plan.set_config(*[self.tuned[k] for k in BATCH_CONFIG_FIELDS])
        return ds

    def stages(self, ctx):
        return self.set0.stages(ctx)

    def outputs(self):
        return self.set0.outputs()

    # ---- CPU oracle ----------------------------------------------------
    def oracle_step(self, sample_kp: int):
        """The oracle on the first `sample_kp` keypoints of each image (all
        stages); returns the descriptors and pairs it covered."""
        import oracle
        wl = self.wl
        nd = npairs = 0
        descs = []
        for i, im in enumerate(self.images):
            lo, hi = int(self.offsets[i]), int(self.offsets[i + 1])
            k = self.kps[lo:min(hi, lo + sample_kp)]
            if len(k) == 0:
                continue
            d, _ = oracle.bad_describe(im, k, wl.bad)
            h = oracle.hs_describe(im, k, wl.hs)["bits"]
            descs.append((d, h))
            nd += 2 * len(k)
            if not self.match and nd >= 4 * sample_kp:
                break
        if self.match and len(descs) == 2:
            (da, ha), (db, hb) = descs
            oracle.match(da, db, self.bad_bits)
            oracle.match(ha, hb, self.hs_bits)
            npairs = 2 * len(da) * len(db)
        return nd, npairs


BATCH_CONFIG_FIELDS = ("bad_kp_per_item", "ctas_per_sm", "hs_first", "hs_kp_per_item",
                       "proj_fused", "bad_shared", "proj_half")


class DeviceSet:
    """One copy of a step's device buffers: an input arena (images and
    keypoints, so the end-to-end step moves them with one copy), an output
    arena (descriptors and match records, one copy back), views into both, and
    the batch plan on them (with its matchings when they are fused)."""

    def __init__(self, wl, ctx):
        import torch
        import paper_2108_08380_gb300 as bd
        self.wl = wl
        dev = "cuda"
        in_parts = [im.nbytes for im in wl.images] + [wl.kps.nbytes]
        in_off, tot = [], 0
        for nb in in_parts:
            in_off.append(tot)
            tot += (nb + 255) // 256 * 256
        self.host_in = np.zeros(tot, np.uint8)
        for im, o in zip(wl.images, in_off):
            self.host_in[o:o + im.nbytes] = im.reshape(-1)
        self.host_in[in_off[-1]:in_off[-1] + wl.kps.nbytes] = wl.kps.view(np.uint8).reshape(-1)
        self.in_arena = torch.from_numpy(self.host_in).to(dev)
        self.dimg = [self.in_arena[o:o + im.nbytes].view(im.shape) for im, o in zip(wl.images, in_off)]
        self.dkps = self.in_arena[in_off[-1]:in_off[-1] + wl.kps.nbytes].view(torch.float32) \
            .view(wl.kps.shape)
        n = wl.n
        na = int(wl.offsets[1]) if wl.match else 0
        shapes = [(n, wl.bad_bits // 32), (n, wl.hs_bits // 32)] + \
            ([(na, 3), (na, 3)] if wl.match else [])
        out_off, tot = [], 0
        for sh in shapes:
            out_off.append(tot)
            tot += (sh[0] * sh[1] + 63) // 64 * 64
        self.out_arena = torch.empty(tot, dtype=torch.int32, device=dev)
        views = [self.out_arena[o:o + sh[0] * sh[1]].view(sh) for sh, o in zip(shapes, out_off)]
        self.bad, self.hs = views[0], views[1]
        self.m_bad = self.m_hs = None
        self.plan = ctx.batch(wl.bp, wl.hp, self.dimg, wl.offsets)
        if wl.match:
            self.m_bad, self.m_hs = views[2], views[3]
            if wl.match_kind == "fused":
                # image A's descriptors against image B's, by the describing launch
                self.plan.set_matches([(bd.BD_DESC_BAD, 0, 1, self.m_bad, 4, 5),
                                       (bd.BD_DESC_HASHSIFT, 0, 1, self.m_hs, 4, 5)])

    def stages(self, ctx):
        """(label, callable) of the ABI calls of one step, in order."""
        wl = self.wl
        st = [("describe_batch", lambda: self.plan.describe(self.dimg, self.dkps, self.bad, self.hs,
                                                            graph=True))]
        if wl.match:
            na = int(wl.offsets[1])
            if wl.match_kind == "fused":
                pass  # done by describe_batch (bd_batch_set_matches)
            elif wl.match_kind == "tensor":
                st += [
                    ("match_bad", lambda: ctx.match(self.bad[:na], self.bad[na:], wl.bad_bits,
                                                    4, 5, out=self.m_bad, tensor_cores=True)),
                    ("match_hashsift", lambda: ctx.match(self.hs[:na], self.hs[na:], wl.hs_bits,
                                                         4, 5, out=self.m_hs, tensor_cores=True)),
                ]
            else:
                # both descriptor types in one launch (bd_match_batch)
                jobs = [(self.bad[:na], self.bad[na:], wl.bad_bits),
                        (self.hs[:na], self.hs[na:], wl.hs_bits)]
                st += [("match", lambda: ctx.match_batch(jobs, 4, 5, outs=[self.m_bad, self.m_hs]))]
        return st

    def outputs(self):
        return [self.bad, self.hs] + ([self.m_bad, self.m_hs] if self.wl.match else [])


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


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over all ranks (the step time the job is charged)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference_select(args):
    """The oracle on the feature-selection workload: steps of a bounded number
    of candidates over all triplets."""
    import oracle
    import synth
    sw = synth.select_workload(1005)
    n = sw.patches.shape[1]
    sample = 2
    cands = np.concatenate([sw.centres[:sample], sw.sides[:sample, None]], axis=1)
    oracle.select_feature(sw.patches[:, :64], cands[:1], sw.sim_ap[:64], sw.sim_an[:64], sw.tau)
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps)):
        oracle.select_feature(sw.patches, cands, sw.sim_ap, sw.sim_an, sw.tau)
    dt = time.perf_counter() - t0
    value = max(1, args.steps) * sample / dt
    print(json.dumps({
        "impl": "reference", "metric": "BAD feature-selection rounds: candidates evaluated per second "
        "(Algorithm 1 with Algorithm 2, 0.1 threshold grid)", "value": value, "unit": "candidates/s",
        "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / max(1, args.steps), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64 (exact integer)", "data": "synthetic",
        "config": {"workload": f"{n} triplets, {sample} of the 1000 candidates per step"},
        "cpu_baseline": {"value": value, "unit": "candidates/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
                         "sample": f"{sample} candidates over all {n} triplets per step, single-threaded C"},
        "e2e": {"value": value, "unit": "candidates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_reference_train(args):
    """The FP64 oracle's training step (forward, mining, loss, backward) on a
    bounded sample of the triplets, scaled to steps of the full batch."""
    import oracle
    import synth
    n, sample = 65536, 64
    rng = np.random.default_rng(1003)
    tw = synth.triplet_workload(1003, n=n)
    bad = synth.make_bad_params(256, rng)
    theta = rng.uniform(-20, 20, size=256).astype(np.float32)
    hs = synth.make_hashsift_params(256, rng)
    P = np.ascontiguousarray(tw.patches[:, :sample])
    oracle.train_step(P[:, :8], bad, theta, hs)  # build and page-in outside the timing
    t0 = time.perf_counter()
    for _ in range(max(1, args.steps)):
        oracle.train_step(P, bad, theta, hs)
    dt = (time.perf_counter() - t0) / max(1, args.steps)
    value = sample / n / dt
    print(json.dumps({
        "impl": "reference", "metric": "training steps (forward + backward) per second",
        "value": value, "unit": "steps/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "65536 triplets of 32x32 FP32 patches, BAD-256 + HashSIFT-256 "
                               "relaxed at T = 0.1, mining with anchor swap, full backward"},
        "cpu_baseline": {"value": value, "unit": "steps/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
                         "sample": f"forward + backward over {sample} of the {n} triplets per step "
                                   f"(FP64, single-threaded C), scaled linearly to a step (mining "
                                   f"within the sample, so the quadratic part is understated)"},
        "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    if args.workload == "select":
        return run_reference_select(args)
    if args.workload == "train":
        return run_reference_train(args)
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
        "cpu_baseline": {"value": value, "unit": "descriptors/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
                         "sample": f"first {sample} keypoints of each image per step, all stages "
                                   "(BAD, HashSIFT, both matchings), single-threaded C"},
        "e2e": {"value": value, "unit": "descriptors/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def host_cpu() -> dict:
    """The host cores this process may use and the CPU model (for the oracle
    baselines, which run single-threaded on one of them)."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    try:
        avail = len(os.sched_getaffinity(0))
    except AttributeError:
        avail = os.cpu_count() or 0
    return {"available_cores": avail, "model": model}


def cpu_baseline(wl, budget_s: float):
    """The oracle, as it stands, on host cores: steps of a bounded keypoint sample."""
    sample = {"plain": 250, "large": 120, "batch": 60}[wl.name]
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
    return {"value": nd / dt, "unit": "descriptors/s", "cores": 1, "kind": "oracle", "host": host_cpu(),
            "sample": f"{steps} oracle step(s) over the first {sample} keypoints of each image "
                      f"(BAD, HashSIFT, both matchings), single-threaded C, {dt:.1f} s",
            "matches_per_s": npairs / dt}


def oracle_parity(ctx, wl, sample: int):
    """Part of the CPU-baseline leg: the step's own outputs on the first
    `sample` keypoints of each image against the oracle (BAD words equal;
    HashSIFT bits equal wherever the oracle's margin clears the error the
    histograms can cause), and the end-to-end histogram error from the image
    (the per-image describe call, same warp and histogram routines as the
    batched kernel) against the oracle's FP64 histograms."""
    import torch
    import oracle
    bad = wl.bad.cpu().numpy().view(np.uint32)
    hsb = wl.hs.cpu().numpy().view(np.uint32)
    Wn = np.linalg.norm(np.asarray(wl.wl.hs.W, np.float64), axis=0)
    bad_bad = hs_bad = hs_checked = hs_band = 0
    herr = 0.0
    nkp = 0
    for i, im in enumerate(wl.images):
        lo, hi = int(wl.offsets[i]), int(wl.offsets[i + 1])
        hi = min(hi, lo + sample)
        if hi <= lo:
            continue
        k = wl.kps[lo:hi]
        d, _ = oracle.bad_describe(im, k, wl.wl.bad)
        bad_bad += int((d != bad[lo:hi]).sum())
        ref = oracle.hs_describe(im, k, wl.wl.hs)
        hist = torch.empty((hi - lo, 128), dtype=torch.float32, device="cuda")
        ctx.hashsift_describe(wl.hp, wl.dimg[i], wl.dkps[lo:hi], hist_out=hist)
        h = hist.cpu().numpy().astype(np.float64)
        e = np.abs(h - ref["hist"]).max(axis=1)
        herr = max(herr, float(e.max()))
        tol = (math.sqrt(128) * e[:, None] + 2.0 ** -20) * Wn[None, :] + 1e-6
        if wl.band > 0:
            tol = np.maximum(tol, wl.band)
        sure = np.abs(ref["margins"]) >= tol
        got = np.unpackbits(hsb[lo:hi].view(np.uint8), axis=1, bitorder="little")[:, :wl.hs_bits]
        hs_bad += int((got.astype(bool)[sure] != (ref["margins"] > 0)[sure]).sum())
        hs_checked += int(sure.sum())
        hs_band += int((~sure).sum())
        nkp += hi - lo
        if wl.name == "batch" and i >= 3:
            break
    return {"keypoints": nkp, "bad_word_mismatches": bad_bad,
            "hashsift_bits_checked": hs_checked, "hashsift_bit_mismatches": hs_bad,
            "hashsift_bits_in_error_band": hs_band,
            "hashsift_hist_e2e_max_abs_err": herr,
            "note": "end-to-end histogram error from the image (FP32 warp positions included); "
                    "the histogram of the same FP32 patch is held to 1e-5 in the GPU tests"}


def run_other_workloads(args):
    """The other configurations as compact records, each from a child
    `bench.py --workload X` run (a fresh process and context, a few steps):
    the 4K pair with its component rates, the 64-image batch, the training
    step and the feature-selection round."""
    steps = max(3, min(args.steps, 20))
    warm = 3
    out = {}
    for name, extra in (("large", []), ("batch", ["--no-components"]), ("train", []),
                        ("select", [])):
        cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--workload", name, "--steps",
               str(steps), "--warmup", str(warm), "--cpu-budget", "3", "--no-workloads", *extra]
        t0 = time.time()
        try:
            r = subprocess.run(cmd, capture_output=True, text=True, timeout=600,
                               env=dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0"))
            rec = None
            for ln in reversed(r.stdout.splitlines()):
                try:
                    rec = json.loads(ln)
                    break
                except ValueError:
                    continue
            if r.returncode != 0 or rec is None:
                out[name] = {"error": f"rc={r.returncode}", "stderr_tail": r.stderr[-800:]}
                continue
        except subprocess.TimeoutExpired:
            out[name] = {"error": "timed out after 600 s"}
            continue
        for k in ("probes", "item_timeline", "kernel_ms_source", "stage_ms"):
            rec.pop(k, None)
        comp = rec.get("components")
        if comp:
            comp.pop("hs_variants", None)
        rec["command"] = " ".join(["python", "bench.py"] + cmd[2:])
        rec["wall_s"] = round(time.time() - t0, 1)
        out[name] = rec
    return out


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
    wl = Workload(args.workload, args.match, rank=rank)
    cfg = tuple(int(x) for x in args.batch_config.split(",")) if args.batch_config else None
    wl.to_device(ctx, autotune=not args.no_autotune, config=cfg)
    stages = wl.stages(ctx)

    # warm-up (also sizes the scratch area)
    for _ in range(max(3, args.warmup)):
        for _, fn in stages:
            fn()
    torch.cuda.synchronize()
    assert ctx.sync_status() == 0, "device flags raised during warm-up"

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # 2 x L2
    K = args.steps
    names = [lab for lab, _ in stages]

    def run_steps(traced: bool):
        """K steps, each: L2 flush, a device sleep while the host enqueues the
        step, then the step's calls between CUDA events.  traced = kernel-level
        events inside every call as well (graph replays included)."""
        ctx.trace(traced)
        # untraced steps get events at their ends only: an event between two
        # kernels would stop the second one's programmatic early launch
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(len(stages) + 1)]
              for _ in range(K)]
        kernel_ms = []  # per step: {stage/kernel: ms}
        for s in range(K):
            flush.fill_(float(s))               # evict the previous step's data from L2
            torch.cuda._sleep(1_000_000)        # let the host enqueue the whole step first
            if traced:
                ctx.trace_reset()
            ev[s][0].record()
            for j, (_, fn) in enumerate(stages):
                fn()
                if traced or j == len(stages) - 1:
                    ev[s][j + 1].record()
            if traced:
                step_k = {}
                call = 0  # marks arrive in call order; each call opens with a 'begin' mark
                for kname, kms in ctx.trace_read_raw():
                    if kname == "begin":
                        call += 1
                        continue
                    key = f"{names[min(call, len(names) - 1)]}/{kname}"
                    step_k[key] = step_k.get(key, 0.0) + kms
                kernel_ms.append(step_k)
        torch.cuda.synchronize()
        ctx.trace(False)
        if traced:
            stage = np.array([[ev[s][j].elapsed_time(ev[s][j + 1]) for j in range(len(stages))]
                              for s in range(K)])
        else:
            stage = np.array([[ev[s][0].elapsed_time(ev[s][-1])] for s in range(K)])
        return stage, kernel_ms

    # ---- timed steps (no kernel-level events: each one drains the stream) ----
    props = torch.cuda.get_device_properties(local)
    sampler = ClockSampler(getattr(props, "uuid", None) and f"GPU-{props.uuid}" or str(local))
    sampler.start()
    time.sleep(0.3)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    ctx.rescued_count(reset=True)
    launches_before = bd.kernel_launches()
    t_wall0 = time.time()
    stage_ms, _ = run_steps(traced=False)
    t_wall1 = time.time()
    launches = bd.kernel_launches() - launches_before
    rescued = ctx.rescued_count(reset=True)
    if pg:
        pg.barrier()
    time.sleep(0.15)
    sampler.stop()
    clocks = sampler.summary(t_wall0 - 0.05, t_wall1 + 0.05)
    ms = float(stage_ms.sum(axis=1).mean())
    if pg:
        ms = max_over_ranks(ms, pg, "cuda")
    assert ctx.sync_status() == 0, "device flags raised during the timed steps"

    # ---- the same K steps again with kernel-level events: per-kernel times ----
    traced_stage_ms, kernel_ms = run_steps(traced=True)
    assert ctx.sync_status() == 0, "device flags raised during the traced steps"

    # ---- measured path rates, per-stage components ----
    probes = measure_probes(ctx)
    components = None
    if not args.no_components:
        components = measure_components(ctx, wl, probes)
    ctx.trace(False)
    ctx.trace_reset()
    ctx.rescued_count(reset=True)
    timeline = item_timeline(wl, flush)
    # ---- end to end through the public API with pinned host buffers ----
    e2e = measure_e2e(ctx, wl, stages, max(3, min(K, 50)))

    if rank != 0:
        return
    per_stage = {lab: float(traced_stage_ms[:, j].mean()) for j, (lab, _) in enumerate(stages)}
    keys = sorted({k for d in kernel_ms for k in d})
    per_kernel = {k: float(np.mean([d.get(k, 0.0) for d in kernel_ms])) for k in keys}
    roof = roofline(wl, per_kernel, clocks, probes)
    value = world * wl.descriptors_per_step / (ms * 1e-3)
    fused_proj = bool(wl.tuned and wl.tuned.get("proj_fused"))
    label = "FP32 projection fused into the persistent kernel" if fused_proj else \
        "tcgen05 BF16 + FP32 rescue projection"
    config = dict(wl.config, workload=wl.config["workload"].replace("(BF16+rescue)", f"({label})"),
                  hashsift_projection=wl.projection_path())
    line = {
        "metric": METRIC, "value": value, "unit": "descriptors/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("u8/int32 (BAD, matching), f32 (HashSIFT histogram and projection)" if fused_proj
                  else "u8/int32 (BAD, matching), f32 histogram + bf16 tensor projection with f32 "
                       "re-check (HashSIFT)"),
        "data": "synthetic",
        "config": dict(config, l2="flushed between steps (512 MB write)",
                       matching=({"tensor": "tensor cores (FP8 +-1, tcgen05), one call per "
                                            "descriptor type",
                                  "popc": "POPC, both descriptor types in one bd_match_batch launch",
                                  "fused": ("POPC, both descriptor types matched by the describing "
                                            "launch itself (bd_batch_set_matches)"
                                            if wl.matching_in_kernel() else
                                            "POPC, both descriptor types in one matching launch of "
                                            "the describing call after the tcgen05 projection "
                                            "(bd_batch_set_matches)")}[wl.match_kind]
                                 if wl.match else None),
                       parallelism=(f"{world} ranks, independent inputs per rank (weak scaling)"
                                    if world > 1 else "single GPU")),
        "matches_per_s": world * wl.pairs_per_step / (ms * 1e-3),
        "stage_ms": per_stage,  # from the traced steps
        "kernel_ms": per_kernel,
        "kernel_ms_source": "kernel-level CUDA events on the launching stream over K further steps "
                            "identical to the timed ones (traced step: "
                            f"{float(traced_stage_ms.sum(axis=1).mean()):.4f} ms)",
        "hashsift_rescued_bits_per_step": rescued / K,
        "batch_config": wl.tuned,
        "roofline": roof,
        "probes": probes,
        "components": components,
        "item_timeline": timeline,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": int(launches),
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, args.cpu_budget)
        line["parity_sample"] = oracle_parity(ctx, wl, 200)
    if world == 1 and not args.no_workloads:
        line["workloads"] = run_other_workloads(args)
    print(json.dumps(line), flush=True)
    torch.cuda.synchronize()
    ctx.close()  # plans and parameter sets first, then the context: not left to exit order
    if pg:
        pg.destroy_process_group()


# ---------------------------------------------------------------------------
# measured path rates (bd_probe) and per-stage kernels against them
# ---------------------------------------------------------------------------

def _kernel_ms(ctx, fn, reps):
    """Mean device time per call of each kernel that fn launches (trace events).
    A device sleep is queued first, so the call is enqueued before the GPU
    reaches it and the marks time the kernels, not the host's launch latency."""
    import torch
    fn()
    torch.cuda.synchronize()
    acc = {}
    for _ in range(reps):
        torch.cuda._sleep(1_000_000)
        ctx.trace_reset()
        fn()
        torch.cuda.synchronize()
        for name, ms in ctx.trace_read():
            acc[name] = acc.get(name, 0.0) + ms / reps
    return acc


def bad_l1_sectors(bp, level_scales, kps, w, h, sample=None, seed=0):
    """Distinct 32-byte sectors of an image's integral table (uint32, row
    stride w + 1, 256-byte aligned) that the 8 K corner reads of each
    keypoint touch: the least data L1 has to hand to the warps describing
    it, whatever the order of its reads.  The keypoint's pixel, pyramid level
    and angle bin follow the kernels' rules (IEEE single precision); boxes
    come from the library's own offset table.  sample: count that many
    seeded keypoints and scale to all of them.  Returns (sectors, 128-byte
    lines) summed over the keypoints."""
    off, sides = bp.table()                       # [L][NB][K][2][2], [L][K]
    L, NB, K = off.shape[0], off.shape[1], off.shape[2]
    kps = np.asarray(kps, np.float32)
    n = kps.shape[0]
    idx = np.arange(n)
    if sample is not None and sample < n:
        idx = np.sort(np.random.default_rng(seed).choice(n, size=sample, replace=False))
    k = kps[idx]
    ix = np.floor(k[:, 0] + np.float32(0.5)).astype(np.int64)
    iy = np.floor(k[:, 1] + np.float32(0.5)).astype(np.int64)
    ls = np.asarray(level_scales, np.float64)
    mids = np.float32(np.sqrt(ls[:-1] * ls[1:]))
    lev = (mids[None, :] < k[:, 2:3]).sum(axis=1) if L > 1 else np.zeros(len(k), np.int64)
    ascale = np.float32(NB / (2.0 * np.pi))
    b = np.floor((k[:, 3] * ascale) + np.float32(0.5)).astype(np.int64) % NB
    stride = w + 1
    tot_s = tot_l = 0
    for c0 in range(0, len(k), 2048):
        sl = slice(c0, c0 + 2048)
        o = off[lev[sl], b[sl]]                    # [m][K][2][2] centre offsets
        s_ = sides[lev[sl]][:, :, None]            # [m][K][1]
        x0 = ix[sl, None, None] + o[..., 0] - s_ // 2
        y0 = iy[sl, None, None] + o[..., 1] - s_ // 2
        xa, xb = np.clip(x0, 0, w), np.clip(x0 + s_, 0, w)
        ya, yb = np.clip(y0, 0, h), np.clip(y0 + s_, 0, h)
        words = np.concatenate([(ya * stride + xa).reshape(len(o), -1), (ya * stride + xb).reshape(len(o), -1),
                                (yb * stride + xa).reshape(len(o), -1), (yb * stride + xb).reshape(len(o), -1)],
                               axis=1)
        for shift in (3, 5):                       # 32-byte sectors, 128-byte lines
            q = np.sort(words >> shift, axis=1)
            d = 1 + (np.diff(q, axis=1) != 0).sum(axis=1)
            if shift == 3:
                tot_s += int(d.sum())
            else:
                tot_l += int(d.sum())
    scale = n / len(k)
    return tot_s * scale, tot_l * scale


def measure_probes(ctx):
    """Measured rates of the paths the descriptor kernels lean on (units/s):
    random 4-byte gathers from L2 (32 MB table) and within BAD-sized 8 KB
    windows (L1 hits), 32-byte sectors handed out by L1 (coalesced 16-byte
    lanes, the bound of the BAD gathers), POPC, FFMA and MUFU instructions."""
    import torch
    import paper_2108_08380_gb300 as bd
    ctx.trace(True)
    table = torch.randint(0, 1 << 20, (1 << 23,), dtype=torch.int32, device="cuda")
    cases = {
        "gather_l2": (bd.BD_PROBE_GATHER, 16, table, 1 << 23),
        "gather_l1_window_8kb": (bd.BD_PROBE_GATHER, 64, table, 1 << 11),
        "l1_sectors": (bd.BD_PROBE_L1_SECTORS, 512, table, 0),
        "popc": (bd.BD_PROBE_POPC, 256, None, 0),
        "ffma": (bd.BD_PROBE_FFMA, 1024, None, 0),
        "mufu_ex2": (bd.BD_PROBE_MUFU, 256, None, 0),
    }
    out = {}
    for name, (kind, reps, tab, win) in cases.items():
        best = None
        for _ in range(4):
            ctx.trace_reset()
            units = ctx.probe(kind, reps, tab, win)
            torch.cuda.synchronize()
            ms = sum(m for _, m in ctx.trace_read())
            best = ms if best is None else min(best, ms)
        out[name] = {"per_s": units / (best * 1e-3), "ms": best, "units": units}
    del table
    return out


def measure_components(ctx, wl, probes):
    """Each stage's kernel run on its own over image A of the workload (warm
    L2, mean of 10 calls), its rate against the measured rate of the path that
    bounds it; the BF16+rescue projection against the FP32 projection on the
    same histograms (time and bit disagreements); POPC against tensor-core
    matching (time and record equality)."""
    import torch
    import paper_2108_08380_gb300 as bd
    ctx.trace(True)
    reps = 10
    img = wl.dimg[0]
    na = int(wl.offsets[1])
    kps = wl.dkps[:na]
    h, w = img.shape
    res = {"scope": f"image A ({w}x{h}, {na} keypoints), warm L2, mean of {reps} calls"}

    # BAD: integral image + gather (Sec. III-A); 8 integral lookups per bit
    out = torch.empty((na, wl.bad_bits // 32), dtype=torch.int32, device="cuda")
    k = _kernel_ms(ctx, lambda: ctx.bad_describe(wl.bp, img, kps, out=out), reps)
    t = k.get("bad_gather", float("nan")) * 1e-3
    loads = na * wl.bad_bits * 8
    sectors, lines = bad_l1_sectors(wl.bp, wl.wl.bad.level_scales, wl.kps[:na], w, h)
    res["bad_gather"] = {
        "ms": t * 1e3, "gathers_per_s": loads / t,
        "l1_sectors_per_kp": sectors / na, "l1_lines_per_kp": lines / na,
        "l1_sectors_per_s": sectors / t,
        "frac_of_l1_sectors": sectors / t / probes["l1_sectors"]["per_s"],
        "frac_of_l2_gather": loads / t / probes["gather_l2"]["per_s"],
        "frac_of_l1_window_gather": loads / t / probes["gather_l1_window_8kb"]["per_s"],
        "work": f"{na} kps x {wl.bad_bits} bits x 8 lookups; bound: the distinct 32-byte "
                "sectors of the keypoints' corner reads at the L1 sector rate"}
    ii_ms = sum(v for kk, v in k.items() if kk.startswith("ii_"))
    res["integral"] = {"ms": ii_ms, "bytes": 6 * w * h,
                       "gbs": 6 * w * h / (ii_ms * 1e-3) / 1e9,
                       "work": "1 B read twice + 4 B written per pixel"}

    # HashSIFT: fused warp + histogram, then projection (Sec. III-B)
    hist = torch.empty((na, 128), dtype=torch.float32, device="cuda")
    bits_bf = torch.empty((na, wl.hs_bits // 32), dtype=torch.int32, device="cuda")
    k = _kernel_ms(ctx, lambda: ctx.hashsift_describe(wl.hp, img, kps, out=bits_bf,
                                                        hist_out=hist), reps)
    th = sum(v for kk, v in k.items() if kk.startswith("hs_hist")) * 1e-3
    ops = HS_OPS_PER_PIXEL * 1024.0 * na
    res["hs_histogram"] = {"ms": th * 1e3, "patches_per_s": na / th,
                           "frac_of_ffma": ops / th / probes["ffma"]["per_s"],
                           "work": f"{na} patches x 1024 px x {HS_OPS_PER_PIXEL} FP32 ops"}
    hp32 = ctx.hs_params(wl.wl.hs, precision=bd.BD_HS_FP32)
    bits32 = torch.empty_like(bits_bf)
    ctx.rescued_count(reset=True)
    k_bf = _kernel_ms(ctx, lambda: ctx.hashsift_project(wl.hp, hist, out=bits_bf), reps)
    rescued = ctx.rescued_count(reset=True) / (reps + 1)
    k_32 = _kernel_ms(ctx, lambda: ctx.hashsift_project(hp32, hist, out=bits32), reps)
    torch.cuda.synchronize()
    dis = int(np.unpackbits((bits_bf ^ bits32).cpu().numpy().view(np.uint8)).sum())
    t_bf = sum(k_bf.values())
    t_32 = sum(k_32.values())
    flops = 2.0 * 128 * wl.hs_bits * na
    res["hs_projection"] = {
        "bf16_rescue_ms": t_bf, "fp32_ms": t_32, "speedup_vs_fp32": t_32 / t_bf,
        "bit_disagreements": dis, "rescued_bits": rescued,
        "bf16_kernels": k_bf, "fp32_kernels": k_32,
        "bf16_tflops": flops / (k_bf.get("hs_proj_tc", t_bf) * 1e-3) / 1e12}
    hp32.close()

    # SIFT variants before hashing (Sec. II: RootSIFT; trilinear cell binning,
    # 0.2 clip): the same describe call with each variant on its own
    # parameter set, histogram time against the plain histogram's
    var = {}
    hpv = ctx.hs_params(wl.wl.hs, precision=bd.BD_HS_BF16_RESCUE)
    for name, flags in (("trilinear", bd.BD_HS_VARIANT_TRILINEAR), ("clip", bd.BD_HS_VARIANT_CLIP),
                        ("root", bd.BD_HS_VARIANT_ROOT),
                        ("all", bd.BD_HS_VARIANT_TRILINEAR | bd.BD_HS_VARIANT_CLIP
                         | bd.BD_HS_VARIANT_ROOT)):
        hpv.set_variant(flags)
        kv = _kernel_ms(ctx, lambda: ctx.hashsift_describe(hpv, img, kps, out=bits_bf,
                                                             hist_out=hist), reps)
        tv = sum(v for kk, v in kv.items() if kk.startswith("hs_hist")) * 1e-3
        var[name] = {"hist_ms": tv * 1e3, "patches_per_s": na / tv,
                     "vs_plain_histogram": tv / th, "kernels": kv}
    hpv.close()
    res["hs_variants"] = var

    # matching (Sec. IV-C): POPC kernel and tensor-core kernel, same records
    if wl.match:
        q, tr = wl.bad[:na], wl.bad[na:]
        nb = tr.shape[0]
        m1 = torch.empty((na, 3), dtype=torch.int32, device="cuda")
        m2 = torch.empty_like(m1)
        for lab, K, qq, tt in (("bad", wl.bad_bits, wl.bad[:na], wl.bad[na:]),
                               ("hashsift", wl.hs_bits, wl.hs[:na], wl.hs[na:])):
            kp = _kernel_ms(ctx, lambda: ctx.match(qq, tt, K, 4, 5, out=m1), reps)
            kt = _kernel_ms(ctx, lambda: ctx.match(qq, tt, K, 4, 5, out=m2, tensor_cores=True), reps)
            torch.cuda.synchronize()
            tp = sum(kp.values()) * 1e-3
            tt_ = sum(kt.values()) * 1e-3
            popc = na * nb * (K // 32)
            res[f"match_{lab}"] = {
                "popc_ms": tp * 1e3, "tensor_ms": tt_ * 1e3,
                "popc_frac_of_popc_probe": popc / tp / probes["popc"]["per_s"],
                "tensor_fp8_tflops": 2.0 * na * nb * K / tt_ / 1e12,
                "records_equal": bool(torch.equal(m1, m2)),
                "pairs_per_s_popc": na * nb / tp, "pairs_per_s_tensor": na * nb / tt_,
                "work": f"{na} x {nb} pairs x {K // 32} POPC"}
            # mutual nearest neighbours (Sec. V): both directions + cross-check
            tc = wl.match_kind == "tensor"
            mnn = torch.empty(na, dtype=torch.int32, device="cuda")
            km = _kernel_ms(ctx, lambda: ctx.match_mnn(qq, tt, K, 4, 5, tensor_cores=tc,
                                                       out=m1, mnn=mnn), reps)
            torch.cuda.synchronize()
            res[f"mnn_{lab}"] = {"ms": sum(km.values()), "kernels": km,
                                 "kernel": "tensor cores" if tc else "POPC",
                                 "mutual_pairs": int((mnn >= 0).sum().item())}
    return res


ITEM_KINDS = {0: "integral_tile", 1: "hashsift", 3: "bad", 4: "projection",
              5: "matching"}


def item_timeline(wl, flush):
    """One more step of the persistent kernel with its item timeline on (after
    the timed steps; L2 flushed first): per work-item kind, the count, when the
    first was claimed and the last ended (us from the first claim), the mean
    wait for dependencies and the mean and largest work time."""
    import torch
    plan = wl.plan
    plan.set_timeline(True)
    flush.fill_(0.5)
    torch.cuda._sleep(1_000_000)
    for _, fn in wl.stages(plan.ctx)[:1]:
        fn()
    ev = plan.timeline()
    plan.set_timeline(False)
    if len(ev) == 0:
        return None
    t0 = int(ev["t_claim"].min())
    out = {"span_us": (int(ev["t_end"].max()) - t0) / 1e3, "kinds": {}}
    for k, name in ITEM_KINDS.items():
        e = ev[ev["kind"] == k]
        if len(e) == 0:
            continue
        out["kinds"][name] = {
            "items": int(len(e)),
            "first_claim_us": (int(e["t_claim"].min()) - t0) / 1e3,
            "last_end_us": (int(e["t_end"].max()) - t0) / 1e3,
            "wait_mean_us": float(np.mean(e["t_ready"] - e["t_claim"])) / 1e3,
            "work_mean_us": float(np.mean(e["t_end"] - e["t_ready"])) / 1e3,
            "work_max_us": float(np.max(e["t_end"] - e["t_ready"])) / 1e3}
    return out


def double_buffered(steps, copy_in, compute, copy_out):
    """Times `steps` end-to-end steps over two device buffer sets: step i runs
    copy_in(i % 2) on an input stream, compute(i % 2) on the current stream
    and copy_out(i % 2) on an output stream, with events so that a set's input
    copy waits for the compute two steps back and its compute for the
    read-back two steps back.  Returns ms per step (CUDA events)."""
    import torch
    s_c = torch.cuda.current_stream()
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event(), torch.cuda.Event()]
    ev_comp = [torch.cuda.Event(), torch.cuda.Event()]
    ev_out = [torch.cuda.Event(), torch.cuda.Event()]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s_c)
    s_in.wait_stream(s_c)
    for i in range(steps):
        k = i % 2
        with torch.cuda.stream(s_in):
            if i >= 2:
                s_in.wait_event(ev_comp[k])
            copy_in(k)
            ev_in[k].record(s_in)
        s_c.wait_event(ev_in[k])
        if i >= 2:
            s_c.wait_event(ev_out[k])
        compute(k)
        ev_comp[k].record(s_c)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_comp[k])
            copy_out(k)
            ev_out[k].record(s_out)
    s_c.wait_stream(s_out)
    e1.record(s_c)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def measure_e2e(ctx, wl, stages, steps):
    """Same step through the API with host buffers, double-buffered: every
    step copies its inputs (images and keypoints, staged in one pinned
    buffer) host to device as one copy and reads all its descriptors and
    match records back as one copy, inside the timed region; two device sets
    (buffers and plans) let step i + 1's input copy and step i - 1's read-back
    run while step i computes, on their own streams, as a serving loop would."""
    import torch
    sets = [wl.set0, wl.second_set(ctx)]
    host_in = torch.from_numpy(wl.host_in).pin_memory()
    host_out = [torch.empty(wl.out_arena.shape, dtype=wl.out_arena.dtype).pin_memory()
                for _ in range(2)]
    bi = host_in.numel() * host_in.element_size()
    bo = host_out[0].numel() * host_out[0].element_size()
    s_c = torch.cuda.current_stream()
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev = lambda: torch.cuda.Event()
    ev_in, ev_comp, ev_out = [ev(), ev()], [ev(), ev()], [ev(), ev()]
    st = [ds.stages(ctx) for ds in sets]
    for k in range(2):  # warm the second set's graph outside the timed region
        for _, fn in st[k]:
            fn()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s_c)
    s_in.wait_stream(s_c)
    for i in range(steps):
        k = i % 2
        with torch.cuda.stream(s_in):
            if i >= 2:
                s_in.wait_event(ev_comp[k])  # step i - 2 has read this input arena
            sets[k].in_arena.copy_(host_in, non_blocking=True)
            ev_in[k].record(s_in)
        s_c.wait_event(ev_in[k])
        if i >= 2:
            s_c.wait_event(ev_out[k])  # step i - 2's results were read back
        for _, fn in st[k]:
            fn()
        ev_comp[k].record(s_c)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_comp[k])
            host_out[k].copy_(sets[k].out_arena, non_blocking=True)
            ev_out[k].record(s_out)
    s_c.wait_stream(s_out)
    e1.record(s_c)
    torch.cuda.synchronize()
    sets[1].plan.close()  # release the second plan here, not at interpreter exit
    ms = e0.elapsed_time(e1) / steps
    return {"value": wl.descriptors_per_step / (ms * 1e-3), "unit": "descriptors/s",
            "ms_per_step": ms, "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo),
            "pipelining": "double-buffered: the input copy of the next step and the read-back "
                          "of the previous one overlap each step's compute"}


def roofline(wl, per_kernel, clocks, probes=None, sm_count=None):
    """Roofline of the dominant kernel of the step (largest mean time per step).
    Denominators are measured: MEASURED_PEAKS.json for HBM and BF16 tensor
    throughput, the bd_probe kernels for POPC, FFMA and gather rates (derived
    from unit counts and the sampled clock only when the probes were skipped).
    Algorithmic work per unit: 6 B per pixel (integral image), the distinct
    32-byte L1 sectors of a BAD keypoint's 8 x K corner reads (bad_l1_sectors),
    HS_OPS_PER_PIXEL x 1024 per HashSIFT patch, 2 x 128 x K flop per projected
    keypoint, K/32 POPC or 2 x K flop per matched pair."""
    peaks, kind = load_peaks()
    if sm_count is None:
        import torch
        sm_count = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    key = max(per_kernel, key=per_kernel.get)
    t = per_kernel[key] * 1e-3
    stage, kname = key.split("/")
    sm_mhz = float(clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0))
    na = int(wl.offsets[1]) if wl.match else 0
    nb = wl.n - na
    out = {"kernel": key, "ms": per_kernel[key], "sm_mhz_used": sm_mhz}

    def probe(name, derived, what):
        if probes and name in probes:
            return probes[name]["per_s"], f"measured: bd_probe {name}"
        return derived, f"derived: {what} x {sm_mhz:.0f} MHz"

    if kname in ("match_top2", "match_multi"):
        if stage == "match":  # both descriptor types in one launch
            words = wl.bad_bits // 32 + wl.hs_bits // 32
        else:
            words = (wl.bad_bits if stage == "match_bad" else wl.hs_bits) // 32
        popc = na * nb * words
        peak, src = probe("popc", sm_count * 16 * sm_mhz * 1e6, f"{sm_count} SMs x 16 POPC/clk")
        out.update(bound="alu", achieved=popc / t / 1e12, peak=peak / 1e12, unit="Tpopc/s",
                   frac=popc / t / peak, peak_source=src)
    elif kname == "match_tc":
        K = wl.bad_bits if stage == "match_bad" else wl.hs_bits
        flops = 2.0 * na * nb * K
        peak = 2.0 * float(peaks["bf16_tflops"])
        ach = flops / t / 1e12
        out.update(bound="tensor", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                   peak_source=f"{kind} bf16 burst x 2 (nominal FP8/BF16 dense ratio)")
    elif kname == "hs_proj_tc":
        flops = 2.0 * 128 * wl.hs_bits * wl.n
        peak = float(peaks["bf16_tflops"])
        ach = flops / t / 1e12
        out.update(bound="tensor", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                   peak_source=f"{kind} bf16 burst (MEASURED_PEAKS.json)")
    else:
        # batch_persistent: integral images (HBM), BAD gathers and histogram
        # arithmetic fused in one launch.  Each part's minimum time at its
        # measured rate; the bound is the largest part, and the sum is the
        # time the three would take if they could not overlap.
        px = float(sum(int(im.shape[0]) * int(im.shape[1]) for im in wl.images))
        g_rate, g_src = probe("l1_sectors", sm_count * 4 * sm_mhz * 1e6,
                              f"{sm_count} SMs x 4 sectors/clk")
        f_rate, f_src = probe("ffma", sm_count * 128 * sm_mhz * 1e6, f"{sm_count} SMs x 128 FP32 lanes")
        parts = {
            "l1": (wl.l1_sectors(), g_rate, "Gsector/s", g_src),
            "alu": (HS_OPS_PER_PIXEL * 1024.0 * wl.n, f_rate, "Tops/s", f_src),
            "hbm": (6.0 * px, float(peaks["hbm_gbs"]) * 1e9, "GB/s", f"{kind} HBM copy"),
        }
        if wl.match and wl.match_kind == "fused" and wl.matching_in_kernel():  # its last items
            p_rate, p_src = probe("popc", sm_count * 16 * sm_mhz * 1e6, f"{sm_count} SMs x 16 POPC/clk")
            words = wl.bad_bits // 32 + wl.hs_bits // 32
            parts["popc"] = (float(na) * nb * words, p_rate, "Tpopc/s", p_src)
        tmin = {k: v[0] / v[1] for k, v in parts.items()}
        bound = max(tmin, key=tmin.get)
        work, rate, unit, src = parts[bound]
        scale = 1e9 if unit in ("Gsector/s", "GB/s") else 1e12  # Tops/s, Tpopc/s
        out.update(bound=bound, achieved=work / t / scale, peak=rate / scale, unit=unit,
                   frac=work / t / rate, peak_source=src,
                   parts_min_ms={k: v * 1e3 for k, v in tmin.items()},
                   frac_of_parts_sum=sum(tmin.values()) / t)
    out["traffic"] = ncu_traffic(wl.name, key)
    out["traffic_unit"] = "bytes per launch (ncu dram read + write, cold caches)"
    return out


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# step's kernels from one ncu capture per workload and kernel, with the hash
# of the kernel's own sources at capture time; a kernel whose sources changed
# since has traffic null.
KERNEL_SOURCES = {
    "batch_persistent": ["batch.cu", "bad_dev.cuh", "hashsift_dev.cuh", "integral_dev.cuh",
                         "match_dev.cuh", "bd_internal.h"],
    "hs_proj_tc": ["proj_tc.cu", "bd_internal.h"],
    "match_tc": ["match_tc.cu", "bd_internal.h"],
    "match_multi": ["match.cu", "match_dev.cuh", "bd_internal.h"],
    "select_keys": ["select.cu", "bd_internal.h"],
    "select_threshold": ["select.cu", "bd_internal.h"],
}
NCU_TRAFFIC = {
    "plain": {"describe_batch/batch_persistent": (879104 + 0, "076afb1061f29035")},
    "large": {"describe_batch/batch_persistent": (37529088 + 60882176, "076afb1061f29035"),
              "describe_batch/hs_proj_tc": (31311616 + 4352, "be87799083a5e228"),
              "match_bad/match_tc": (10279168 + 0, "59f3d684ac6a76a3"),
              "match_hashsift/match_tc": (20523520 + 0, "59f3d684ac6a76a3")},
    "select": {"select/select_keys": (201393664 + 342133504, "8d33f0ff71a1e5ba"),
               "select/select_threshold": (394337024 + 3256320, "8d33f0ff71a1e5ba")},
    "train": {"match_tc": (33593344 + 0, "59f3d684ac6a76a3")},
    "batch": {"describe_batch/batch_persistent": (286708224 + 406824704, "076afb1061f29035"),
              "describe_batch/hs_proj_tc": (162755072 + 9899776, "be87799083a5e228")},
}


def kernel_sources_hash(kernel: str) -> str:
    """sha256 (first 16 hex digits) of a kernel's CUDA sources and the C header."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2108_08380_gb300", "csrc")
    files = [os.path.join(csrc, f) for f in KERNEL_SOURCES[kernel]]
    files.append(os.path.join(ROOT, "include", "bindesc.h"))
    h = hashlib.sha256()
    for f in files:
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(wl_name: str, key: str):
    ent = NCU_TRAFFIC.get(wl_name, {}).get(key)
    kname = key.split("/")[-1]
    if ent is None or kname not in KERNEL_SOURCES:
        return None
    return ent[0] if kernel_sources_hash(kname) == ent[1] else None


# FP32/SFU operations one patch pixel of the HashSIFT histogram needs:
# sample position 4, tap split 4, bilinear 6, gradient 4, magnitude 3, orientation
# (atan2 as 1), bin split 3, Gaussian weight 1, two votes 4.
HS_OPS_PER_PIXEL = 30


def run_train(args):
    """Training-step workload: 65536 triplets of 32x32 FP32 patches, relaxed
    BAD-256 + HashSIFT-256 (T = 0.1), mining with anchor swap, loss, backward.
    The 805 MB of patches exceed L2, so no flush is needed between steps."""
    import torch
    import paper_2108_08380_gb300 as bd
    import synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    n = 65536
    rng = np.random.default_rng(1003 + 100 * rank)
    tw = synth.triplet_workload(1003 + 100 * rank, n=n)
    P = torch.from_numpy(tw.patches).cuda()
    bad = synth.make_bad_params(256, rng)
    theta = torch.from_numpy(rng.uniform(-20, 20, size=256).astype(np.float32)).cuda()
    hs = synth.make_hashsift_params(256, rng)
    W, b = torch.from_numpy(hs.W).cuda(), torch.from_numpy(hs.b).cuda()
    ctx = bd.Context(local)
    step = bd.TrainStep(ctx, ctx.bad_params(bad), 256, n, temperature=0.1)
    g = torch.ones(2, device="cuda")

    def one():
        loss, _ = step.forward(P, theta, W, b)
        grads = step.backward(P, W, g)
        return loss, grads

    for _ in range(max(3, args.warmup)):
        one()
    torch.cuda.synchronize()
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    props = torch.cuda.get_device_properties(local)
    sampler = ClockSampler(getattr(props, "uuid", None) and f"GPU-{props.uuid}" or str(local))
    sampler.start()
    time.sleep(0.3)
    launches0 = bd.kernel_launches()
    t0 = time.time()
    for s_ in range(K):
        ev[s_][0].record()
        one()
        ev[s_][1].record()
    torch.cuda.synchronize()
    t1 = time.time()
    launches = bd.kernel_launches() - launches0
    time.sleep(0.15)
    sampler.stop()
    clocks = sampler.summary(t0 - 0.05, t1 + 0.05)
    ms = float(np.mean([x.elapsed_time(y) for x, y in ev]))
    if pg is not None:
        ms = max_over_ranks(ms, pg, "cuda")
    # kernel times from a traced pass (events between kernels)
    ctx.trace(True)
    kern = {}
    for _ in range(K):
        ctx.trace_reset()
        one()
        torch.cuda.synchronize()
        for name, kms in ctx.trace_read():
            kern[name] = kern.get(name, 0.0) + kms / K
    ctx.trace(False)
    # roofline of the dominant kernel: the mining matchings (four n x n
    # matchings of K = 256 +-1 codes on the tensor cores, FP8) when they lead
    peaks, kind = load_peaks()
    dom = max(kern, key=kern.get)
    t_dom = kern[dom] * 1e-3
    if dom == "match_tc":
        flops = 4 * 2.0 * n * n * 256
        peak = 2.0 * float(peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]))
        roof = {"kernel": dom, "ms": kern[dom], "bound": "tensor", "achieved": flops / t_dom / 1e12,
                "peak": peak, "unit": "TFLOP/s", "frac": flops / t_dom / 1e12 / peak,
                "traffic": ncu_traffic("train", dom), "traffic_unit": "bytes per launch (one of "
                "the four mining matchings; ncu dram read + write)", "algorithmic_flops": flops,
                "peak_source": f"{kind} bf16 sustained x 2 (nominal FP8/BF16 dense ratio)"}
    else:
        # the patch-bound kernels: one read of the 3n patches (4 KB each)
        byts = 3.0 * n * 4096
        roof = {"kernel": dom, "ms": kern[dom], "bound": "hbm", "achieved": byts / t_dom / 1e9,
                "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                "frac": byts / t_dom / 1e9 / float(peaks["hbm_gbs"]),
                "traffic": ncu_traffic("train", dom), "algorithmic_bytes": byts,
                "peak_source": f"{kind} HBM copy"}
    # end to end, double-buffered: the patches from pinned host memory, the
    # loss back, every step (the gradients stay on the device, as in training)
    hP = torch.from_numpy(tw.patches).pin_memory()
    Ps = [P, torch.empty_like(P)]
    losses = [None, None]
    loss_h = [torch.empty(2, dtype=torch.float32).pin_memory() for _ in range(2)]

    def copy_in(k):
        Ps[k].copy_(hP, non_blocking=True)

    def compute(k):
        loss, _ = step.forward(Ps[k], theta, W, b)
        step.backward(Ps[k], W, g)
        losses[k] = loss

    def copy_out(k):
        loss_h[k].copy_(losses[k], non_blocking=True)

    e2e_ms = double_buffered(max(4, min(K, 10)), copy_in, compute, copy_out)
    line = {"metric": "training steps (forward + backward) per second", "value": world * 1e3 / ms,
            "unit": "steps/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (patches, responses, gradients), fp8 tensor (mining)", "data": "synthetic",
            "triplets_per_s": world * n * 1e3 / ms,
            "config": {"workload": "65536 triplets of 32x32 FP32 patches, BAD-256 + HashSIFT-256 "
                                   "relaxed at T = 0.1, mining with anchor swap, full backward",
                       "l2": "inputs (805 MB of patches) exceed L2"},
            "kernel_ms": kern,
            "kernel_ms_source": "kernel-level CUDA events over K further traced steps",
            "roofline": roof, "clocks": clocks,
            "e2e": {"value": world * 1e3 / e2e_ms, "unit": "steps/s", "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": int(tw.patches.nbytes), "d2h_bytes_per_step": 8},
            "gpu_launches": int(launches)}
    if not args.no_cpu_baseline and rank == 0:
        import oracle
        sample = 64
        Ps = np.ascontiguousarray(tw.patches[:, :sample])
        t0 = time.perf_counter()
        ref = oracle.train_step(Ps, bad, theta.cpu().numpy(), hs)
        dt = time.perf_counter() - t0
        # the GPU step on the same sample with the oracle's mining: gradient
        # error norm-relative to the FP64 oracle (the bound the tests hold)
        small = bd.TrainStep(ctx, step.bad, 256, sample, temperature=0.1)
        dPs = torch.from_numpy(Ps).cuda()
        fm = torch.from_numpy(np.ascontiguousarray(ref["mining"])).cuda()
        ls_, _ = small.forward(dPs, theta, W, b, fixed_mining=fm)
        gP, gth, gW, gb = small.backward(dPs, W, g)
        rel = lambda a, r: float(np.linalg.norm(a.cpu().numpy().astype(np.float64) - r)
                                 / max(np.linalg.norm(r), 1e-30))
        line["grad_rel_err_vs_oracle"] = {
            "triplets": sample, "loss": rel(ls_, ref["loss"]), "dtheta": rel(gth, ref["dtheta"]),
            "dW": rel(gW, ref["dW"]), "db": rel(gb, ref["db"]), "dpatches": rel(gP, ref["dpatches"]),
            "note": "the 65536-triplet step is held to 1e-4 against the oracle in the GPU tests; "
                    "the oracle's gradient is pinned to central finite differences in the CPU tests"}
        small.close()
        line["cpu_baseline"] = {"value": sample / n / dt, "unit": "steps/s", "cores": 1,
                                "kind": "oracle", "host": host_cpu(),
                                "sample": f"forward + backward over {sample} of the {n} triplets "
                                          f"(FP64, single-threaded C), {dt:.3f} s, scaled linearly "
                                          f"to a step (mining within the sample, so the quadratic "
                                          f"part is understated)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    torch.cuda.synchronize()
    ctx.close()
    if pg is not None:
        pg.destroy_process_group()


def run_select(args):
    """Feature-selection workload (Algorithm 1 round with Algorithm 2): 65536
    triplets of uint8 32x32 patches, 1000 candidate box pairs; one step = one
    bd_select_feature call (keys of every candidate on every patch, threshold
    search per candidate, best candidate)."""
    import torch
    import paper_2108_08380_gb300 as bd
    import synth
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    sw = synth.select_workload(1005 + 100 * rank)
    n, J = sw.patches.shape[1], sw.centres.shape[0]
    ctx = bd.Context(local)
    dP = torch.from_numpy(sw.patches).cuda()
    dap = torch.from_numpy(sw.sim_ap).cuda()
    dan = torch.from_numpy(sw.sim_an).cuda()
    step = lambda: ctx.select_feature(dP, dap, dan, sw.tau, sw.centres, sw.sides)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    props = torch.cuda.get_device_properties(local)
    sampler = ClockSampler(getattr(props, "uuid", None) and f"GPU-{props.uuid}" or str(local))
    sampler.start()
    time.sleep(0.3)
    launches0 = bd.kernel_launches()
    t0 = time.time()
    for s in range(K):
        torch.cuda._sleep(1_000_000)
        ev[s][0].record()
        step()
        ev[s][1].record()
    torch.cuda.synchronize()
    t1 = time.time()
    launches = bd.kernel_launches() - launches0
    time.sleep(0.15)
    sampler.stop()
    clocks = sampler.summary(t0 - 0.05, t1 + 0.05)
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    # kernel times from a traced pass
    ctx.trace(True)
    kern = {}
    for _ in range(K):
        torch.cuda._sleep(1_000_000)
        ctx.trace_reset()
        step()
        torch.cuda.synchronize()
        for name, kms in ctx.trace_read():
            kern[name] = kern.get(name, 0.0) + kms / K
    ctx.trace(False)
    peaks, kind = load_peaks()
    key_bytes = J * 3 * n * 2
    traffic = {"select_keys": 3 * n * 1024 + key_bytes, "select_threshold": key_bytes + 8 * n}
    dom = max((k for k in kern if k in traffic), key=kern.get)  # select_geom is set-up
    ach = traffic[dom] / (kern[dom] * 1e-3) / 1e9
    roof = {"kernel": dom, "ms": kern[dom], "bound": "hbm", "achieved": ach,
            "peak": float(peaks["hbm_gbs"]), "unit": "GB/s", "frac": ach / float(peaks["hbm_gbs"]),
            "traffic": ncu_traffic("select", "select/" + dom), "peak_source": f"{kind} HBM copy",
            "algorithmic_bytes": traffic[dom]}
    # end to end, double-buffered: patches and similarities from pinned host
    # memory, results back, every step
    hP = torch.from_numpy(sw.patches).pin_memory()
    hap = torch.from_numpy(sw.sim_ap).pin_memory()
    han = torch.from_numpy(sw.sim_an).pin_memory()
    dev_in = [(dP, dap, dan), (torch.empty_like(dP), torch.empty_like(dap), torch.empty_like(dan))]
    res = [None, None]
    out_h = [[torch.empty(J, dtype=torch.int32).pin_memory(), torch.empty(J, dtype=torch.int64).pin_memory(),
              torch.empty(1, dtype=torch.int32).pin_memory()] for _ in range(2)]

    def copy_in(k):
        for d, h in zip(dev_in[k], (hP, hap, han)):
            d.copy_(h, non_blocking=True)

    def compute(k):
        res[k] = ctx.select_feature(*dev_in[k], sw.tau, sw.centres, sw.sides)

    def copy_out(k):
        for h, d in zip(out_h[k], res[k]):
            h.copy_(d, non_blocking=True)

    e2e_ms = double_buffered(max(4, min(K, 20)), copy_in, compute, copy_out)
    line = {
        "metric": "BAD feature-selection rounds: candidates evaluated per second (Algorithm 1 with "
                  "Algorithm 2, 0.1 threshold grid)",
        "value": world * J / (ms * 1e-3), "unit": "candidates/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8/int16/int32 (exact integer)", "data": "synthetic",
        "config": {"workload": f"{n} triplets of uint8 32x32 patches, {J} candidate box pairs "
                               "(sides 1-15), 128 earlier bits, tau 64",
                   "l2": "inputs and the 393 MB key matrix exceed L2"},
        "triplet_candidate_evals_per_s": world * J * n / (ms * 1e-3),
        "kernel_ms": kern, "roofline": roof, "clocks": clocks,
        "e2e": {"value": world * J / (e2e_ms * 1e-3), "unit": "candidates/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(sw.patches.nbytes + sw.sim_ap.nbytes + sw.sim_an.nbytes),
                "d2h_bytes_per_step": int(J * 12 + 4)},
        "gpu_launches": int(launches),
    }
    if not args.no_cpu_baseline and rank == 0:
        import oracle
        sample = 2
        t0 = time.perf_counter()
        cands = np.concatenate([sw.centres[:sample], sw.sides[:sample, None]], axis=1)
        oracle.select_feature(sw.patches, cands, sw.sim_ap, sw.sim_an, sw.tau)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": sample / dt, "unit": "candidates/s", "cores": 1,
                                "kind": "oracle", "host": host_cpu(),
                                "sample": f"{sample} candidates over all {n} triplets, single-threaded C, "
                                          f"{dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    torch.cuda.synchronize()
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["plain", "large", "batch", "train", "select"],
                    default="plain")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-workloads", action="store_true",
                    help="the default (plain) run skips the records of the other workloads")
    ap.add_argument("--no-components", action="store_true",
                    help="skip the per-stage component measurements")
    ap.add_argument("--batch-config", default=None,
                    help="the fields of bd_batch_config (bad_kp_per_item,ctas_per_sm,hs_first"
                         "[,hs_kp_per_item[,proj_fused[,bad_shared[,proj_half]]]]) for the "
                         "persistent kernel instead of the autotuner's pick")
    ap.add_argument("--match", choices=["auto", "tensor", "popc", "fused"], default="auto",
                    help="matching: tensor cores (bd_match_tc), POPC (bd_match_batch), fused into "
                         "the describing launch (bd_batch_set_matches), or auto (tensor cores from "
                         "2^24 query-train pairs up, else fused)")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--ref-sample-kp", type=int, default=250)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "train":
        run_train(args)
    elif args.workload == "select":
        run_select(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
