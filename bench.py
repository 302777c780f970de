"""Benchmark of the MAFOD hot path on GB300.

A step is one pass of the whole hot path over one batch: for every image,
scale selection, then M cycles of (tensor build, FED cycle of n steps).
Metric: Mpixel-FED-steps/s = sum_images(w h) * M * n / time.

Default workload "batch64_fundus": 64 seeded fundus-like images (circular field
of view, radial vignetting, dark vessel tree of depth 6 with radii 8 -> 1 px,
noise sd 0.1), square sides drawn from 512..2048 (123 Mpixel in total),
8 scales log-spaced over 1..8 px, valley mode, 5 FED cycles of 20 steps
(T = 35, tau_max = 0.05), lambda = 0.005, rho = 0.5, beta = 0.5.  The inputs
(0.5 GB of images, 2 GB of tensor field) are larger than L2.

--impl reference times the FP64 CPU oracle (the method's reference
implementation written from the paper) on the host cores on a bounded sample
of the same workload.

Multi-GPU (torchrun): each rank filters its own batch (seeds offset by rank),
no collective on the data path; value = all ranks' pixel-steps / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpixel-steps/s, batched+learned vs plain GB300, at stated FP64-oracle error"
UNIT = "Mpixel-steps/s"


def _gen_one(args):
    seed, side = args
    from paper_1611_06906_gb300 import synth
    return synth.fundus_like(seed, side)


def make_workload(name: str, rank: int, limit: int = 0):
    """Returns (list of float32 images, config dict)."""
    from paper_1611_06906_gb300 import synth
    wl = dict(synth.WORKLOADS[name])
    if name == "batch64_fundus":
        sides = synth.batch_sides(3000 + 1000 * rank)
        if limit:
            sides = sides[:limit]
        seeds = [3000 + 1000 * rank + i for i in range(len(sides))]
        with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
            imgs = pool.map(_gen_one, list(zip(seeds, sides)))
    elif name == "tree_1024":
        imgs = [synth.vessel_tree(2000 + rank, 1024, 1024)]
    elif name == "tree16_4096":
        n_img = limit or 16
        imgs = [synth.vessel_tree(5000 + 100 * rank + i, 4096, 4096, depth=8, r0=12.0, r1=0.75,
                                  noise=0.15, polarity_mix=True) for i in range(n_img)]
    else:
        raise SystemExit("unknown workload " + name)
    return imgs, wl


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms (read-only)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", "fd4_clocks_%d_%d.csv" % (os.getpid(), gpu_index))

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


MODES = {"ridge": 0, "valley": 1, "both": 2}


class Image:
    def __init__(self, img, dev, fd4, torch):
        self.h, self.w = img.shape
        self.npx = self.h * self.w
        self.u_in = fd4.to_device(img, dev)
        self.pitch = self.u_in.shape[1]
        self.out = torch.empty_like(self.u_in)
        self.idx = torch.zeros((self.h, self.pitch), dtype=torch.uint8, device=dev)
        self.ten = torch.empty((self.h, self.pitch, 4), dtype=torch.float32, device=dev)


def oracle_sample(imgs, wl, mode, max_images=2):
    """Oracle (FP64, host cores) on the smallest images of the batch: the CPU
    baseline sample and the parity reference.  Returns (list of (i, out, idx), secs, cores, pxsteps)."""
    from oracle import oracle as O
    order = sorted(range(len(imgs)), key=lambda i: imgs[i].size)[:max_images]
    tau, _, _ = O.fed_taus(wl["T"], wl["M"], 0.05, n=wl["n"])
    res = []
    t0 = time.perf_counter()
    for i in order:
        out, idx = O.filter_image(imgs[i], wl["sigmas"], tau, wl["M"], mode=mode)
        res.append((i, out, idx))
    secs = time.perf_counter() - t0
    pxsteps = sum(imgs[i].size for i in order) * wl["M"] * wl["n"]
    return res, secs, O.num_threads(), pxsteps


def run_fd4(args, rank, world, local_rank):
    imgs, wl = make_workload(args.workload, rank, args.limit)  # before CUDA init (spawn pool)
    import torch
    from paper_1611_06906_gb300 import fd4
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
    sig, M, n, T = wl["sigmas"], wl["M"], wl["n"], wl["T"]
    K = len(sig)
    mode = MODES[wl["mode"]]
    prm = fd4.params(mode=mode)
    tau, kappa = fd4.fed_taus(T, M, 0.05, n=n)
    ims = [Image(im, dev, fd4, torch) for im in imgs]
    big = max(ims, key=lambda b: b.h * b.pitch)
    ws = fd4.workspace(fd4.OP_FILTER, big.pitch, max(b.h for b in ims), K, dev)
    stream = torch.cuda.current_stream()
    px_steps = sum(b.npx for b in ims) * M * n
    launches_per_step = sum((K + 1) + M * (K + 1 + n) for _ in ims)

    def step(ev=None):
        for b in ims:
            if ev is not None:
                e = [torch.cuda.Event(enable_timing=True) for _ in range(2 + 2 * M)]
                e[0].record(stream)
            fd4.select_scales(b.u_in, b.w, sig, prm, ws=ws, idx=b.idx)
            b.out.copy_(b.u_in)
            if ev is not None:
                e[1].record(stream)
            for k in range(M):
                fd4.build_tensor(b.out, b.w, b.idx, sig, prm, out=b.ten, ws=ws)
                if ev is not None:
                    e[2 + 2 * k].record(stream)
                fd4.fed_cycle(b.out, b.w, b.ten, tau, ws=ws)
                if ev is not None:
                    e[3 + 2 * k].record(stream)
            if ev is not None:
                ev.append((b, e))

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    barrier()
    evs = []
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        t_start.record(stream)
        for _ in range(args.steps):
            step(evs)
        t_end.record(stream)
        barrier()
    ms = t_start.elapsed_time(t_end)
    fed_ms = sel_ms = ten_ms = 0.0
    fed_bytes = 0
    for b, e in evs:
        sel_ms += e[0].elapsed_time(e[1])
        prev = e[1]
        for k in range(M):
            ten_ms += prev.elapsed_time(e[2 + 2 * k])
            fed_ms += e[2 + 2 * k].elapsed_time(e[3 + 2 * k])
            prev = e[3 + 2 * k]
        fed_bytes += 24 * b.npx * n * M
    if dist is not None:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * px_steps * args.steps / (ms * 1e-3) / 1e6

    # end to end through the public entry point, host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        hin = [b.u_in.cpu().pin_memory() for b in ims]
        hout = [torch.empty_like(h).pin_memory() for h in hin]
        def e2e_step():
            for b, hi, ho in zip(ims, hin, hout):
                b.u_in.copy_(hi, non_blocking=True)
                fd4.filter_image(b.u_in, b.w, sig, T, M, n, prm, out=b.out, ws=ws, keep_idx=False)
                ho.copy_(b.out, non_blocking=True)
        for _ in range(max(1, min(args.warmup, 2))):
            e2e_step()
        barrier()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            e2e_step()
        z.record(stream)
        barrier()
        ems = a.elapsed_time(z)
        if dist is not None:
            t = torch.tensor([ems], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ems = float(t.item())
        nbytes = sum(h.numel() * 4 for h in hin)
        e2e = {"value": world * px_steps * args.steps / (ems * 1e-3) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "ms_per_step": ems / args.steps}

    if rank != 0:
        return
    peak, peak_kind = load_peaks()
    achieved = fed_bytes / (fed_ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": args.traffic, "kernel": "k_fed_step",
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (%s)" % peak_kind,
            "bytes_per_px_step": 24, "avg_launch_us": fed_ms * 1e3 / (len(evs) * M * n)}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": args.workload, "images": len(ims),
                      "mpixel": round(sum(b.npx for b in ims) / 1e6, 3), "sigmas": K, "mode": wl["mode"],
                      "M": M, "n": n, "T": T, "kappa": kappa, "path": "plain",
                      "l2": "inputs larger than L2 (images %.2f GB, tensor field %.2f GB per pass)" % (
                          sum(b.npx for b in ims) * 4e-9, sum(b.npx for b in ims) * 16e-9)},
           "roofline": roof, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
           "clocks": clk.summary(),
           "stages_ms_per_step": {"select": sel_ms / args.steps, "tensor": ten_ms / args.steps,
                                  "fed": fed_ms / args.steps}}
    if world == 1 and not args.no_cpu_baseline:
        res, secs, cores, pxs = oracle_sample(imgs, wl, mode)
        errs, agree, errs_inj = [], [], []
        for i, ref, idx_o in res:
            b = ims[i]
            got = b.out[:, :b.w].cpu().numpy().astype(np.float64)
            errs.append(float(np.abs(got - ref).max()))
            agree.append(float((b.idx[:, :b.w].cpu().numpy() == idx_o).mean()))
            idx_in = torch.zeros_like(b.idx)
            idx_in[:, :b.w] = torch.from_numpy(idx_o).to(dev)
            o2, _ = fd4.filter_image(b.u_in, b.w, sig, T, M, n, prm, sigma_idx=idx_in, ws=ws)
            errs_inj.append(float(np.abs(o2[:, :b.w].cpu().numpy() - ref).max()))
        sample = "oracle full filter of the %d smallest batch images (%s px)" % (
            len(res), ", ".join("%dx%d" % imgs[i].shape[::-1] for i, _, _ in res))
        out["cpu_baseline"] = {"value": pxs / secs / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": sample, "seconds": secs}
        out["parity"] = {"vs": "FP64 oracle", "images": sample, "max_abs": max(errs),
                         "max_abs_oracle_sigma": max(errs_inj), "sigma_agreement": min(agree),
                         "tolerance": 1e-4}
    print(json.dumps(out), flush=True)


def run_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_1611_06906_gb300 import synth
    wl = dict(synth.WORKLOADS[args.workload])
    mode = MODES[wl["mode"]]
    if args.workload == "batch64_fundus":
        sides = synth.batch_sides(3000)
        i = int(np.argmin(sides))
        img = synth.fundus_like(3000 + i, sides[i])
    else:
        imgs, _ = make_workload(args.workload, 0, 1)
        img = imgs[0]
    O.build()
    tau, _, _ = O.fed_taus(wl["T"], wl["M"], 0.05, n=wl["n"])
    pxs = img.size * wl["M"] * wl["n"]

    def step():
        O.filter_image(img, wl["sigmas"], tau, wl["M"], mode=mode)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    secs = time.perf_counter() - t0
    value = pxs * args.steps / secs / 1e6
    sample = "oracle full filter of the smallest batch image (%dx%d px), one image per step" % img.shape[::-1]
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": args.workload, "sample": sample, "sigmas": len(wl["sigmas"]),
                      "mode": wl["mode"], "M": wl["M"], "n": wl["n"], "T": wl["T"]},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fd4", choices=["fd4", "reference"])
    ap.add_argument("--workload", default="batch64_fundus",
                    choices=["batch64_fundus", "tree_1024", "tree16_4096"])
    ap.add_argument("--limit", type=int, default=0, help="use only the first N images (profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per FED launch from an ncu capture of the current kernel")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    run_fd4(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
