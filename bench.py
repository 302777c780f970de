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

from paper_1611_06906_gb300.dist import max_over_ranks as _max_over_ranks, rank_seed  # noqa: E402

# DRAM bytes (read + write) per pixel and launch of k_fed_tma<2,2> (two quads per
# thread), from an ncu capture of one launch over the first 8 batch64_fundus
# images (303.40 + 47.16 MB over 15.13 Mpixel); the roofline's `traffic` scales it
# to the launch timed here.  Re-measured (or set to None: the field null)
# whenever that kernel changes.
TMA2_DRAM_B_PER_PX = 23.17
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
        base = rank_seed(3000, rank)  # weak scaling: every rank filters its own batch
        sides = synth.batch_sides(base)
        if limit:
            sides = sides[:limit]
        seeds = [base + i for i in range(len(sides))]
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


def _timed(fn, steps, stream, torch):
    """CUDA-event time (ms) of `steps` calls of fn on `stream`."""
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        fn()
    z.record(stream)
    z.synchronize()
    return a.elapsed_time(z)


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
    ims = [Image(im, dev, fd4, torch) for im in imgs]
    npx = sum(b.npx for b in ims)
    px_steps = npx * M * n
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def max_over_ranks(ms):
        return _max_over_ranks(ms, dev)

    # batched path: one launch per stage across the batch, replayed as a CUDA graph
    lst = fd4.image_list([b.u_in for b in ims], [b.w for b in ims], [b.out for b in ims], [b.idx for b in ims])
    ws = fd4.batch_workspace(lst, K, dev)
    if args.fed_steps:
        best, tune_ms = args.fed_steps, None
    else:
        best, tune_ms = fd4.autotune_batched(lst, sig, T, M, n, fd4.params(mode=mode), ws=ws)
    prm = fd4.params(mode=mode, fed_steps_per_launch=best)
    if args.only_graph:  # profiling: warm-up and timed replays of the full graph only
        g = fd4.Graph(lst, sig, T, M, n, prm, ws=ws)
        for _ in range(args.warmup + args.steps):
            g.launch()
        torch.cuda.synchronize()
        g.close()
        return
    g_one = fd4.Graph(lst, sig, T, M, n, prm, ws=ws)
    g_all = fd4.Graph(lst, sig, T, M, n, prm, ws=ws, stages=fd4.STAGES_ALL | fd4.GRAPH_TWO_STREAMS) \
        if (args.two_streams and len(ims) > 1) else g_one
    g_sel = fd4.Graph(lst, sig, T, M, n, prm, ws=ws, stages=fd4.STAGE_SELECT)
    g_ten = fd4.Graph(lst, sig, T, M, n, prm, ws=ws, stages=fd4.STAGE_TENSOR)
    g_fed = fd4.Graph(lst, sig, T, M, n, prm, ws=ws, stages=fd4.STAGE_FED)
    L = -(-n // best) if best > 1 else n          # FED launches per cycle
    fed_launches = M * L
    launches_per_step = g_all.kernel_count()      # kernel nodes of the captured graph

    for _ in range(args.warmup):
        g_all.launch()
    barrier()
    with ClockSampler(local_rank) as clk:
        ms = _timed(g_all.launch, args.steps, stream, torch)
        barrier()
    ms = max_over_ranks(ms)
    value = world * px_steps * args.steps / (ms * 1e-3) / 1e6
    one_stream_ms = _timed(g_one.launch, args.steps, stream, torch) / args.steps
    # stage split and the FED kernel alone (each graph replays one stage of the same schedule)
    sel_ms = _timed(g_sel.launch, args.steps, stream, torch) / args.steps
    ten_ms = _timed(g_ten.launch, args.steps, stream, torch) / args.steps
    fed_ms = _timed(g_fed.launch, args.steps, stream, torch) / args.steps

    # the scale image selected again on the current image before every cycle
    # (reselect_each_cycle); its outputs on the oracle sample are kept for parity
    resel = None
    if not args.no_reselect:
        g_re = fd4.Graph(lst, sig, T, M, n, fd4.params(mode=mode, fed_steps_per_launch=best,
                                                          reselect_each_cycle=1), ws=ws)
        g_re.launch()
        barrier()
        re_ms = max_over_ranks(_timed(g_re.launch, args.steps, stream, torch)) / args.steps
        order = sorted(range(len(ims)), key=lambda i: ims[i].npx)[:2]
        resel = {"value": world * px_steps / (re_ms * 1e-3) / 1e6, "ms_per_step": re_ms,
                 "gpu_launches_per_step": g_re.kernel_count(),
                 "path": "batched graph, scale image re-selected on u^k before every cycle",
                 "_out": {i: (ims[i].out[:, :ims[i].w].cpu().numpy().astype(np.float64),
                              ims[i].idx[:, :ims[i].w].cpu().numpy()) for i in order}}
        g_re.close()

    # the scale image post-processed after its selection (Sec. 3.3), at the
    # paper's fundus threshold theta = 0.13; outputs kept for parity as above
    post = None
    if not args.no_postprocess:
        theta = float(np.float32(0.13))
        g_po = fd4.Graph(lst, sig, T, M, n, fd4.params(mode=mode, fed_steps_per_launch=best,
                                                          postprocess_scales=1, theta=theta), ws=ws)
        g_po.launch()
        barrier()
        po_ms = max_over_ranks(_timed(g_po.launch, args.steps, stream, torch)) / args.steps
        order = sorted(range(len(ims)), key=lambda i: ims[i].npx)[:2]
        post = {"value": world * px_steps / (po_ms * 1e-3) / 1e6, "ms_per_step": po_ms, "theta": theta,
                "gpu_launches_per_step": g_po.kernel_count(),
                "path": "batched graph, scale image post-processed after the selection",
                "_out": {i: (ims[i].out[:, :ims[i].w].cpu().numpy().astype(np.float64),
                             ims[i].idx[:, :ims[i].w].cpu().numpy()) for i in order}}
        g_po.close()

    # the IFOD comparator of Eq. 2 (sigma 1, the paper's setting) on the same batch
    ifod = None
    if not args.no_ifod:
        g_if = fd4.Graph(lst, sig, T, M, n, fd4.params(mode=mode, fed_steps_per_launch=best,
                                                          model=fd4.MODEL_IFOD, ifod_sigma=1.0), ws=ws)
        g_if.launch()
        barrier()
        if_ms = max_over_ranks(_timed(g_if.launch, args.steps, stream, torch)) / args.steps
        order = sorted(range(len(ims)), key=lambda i: ims[i].npx)[:2]
        ifod = {"value": world * px_steps / (if_ms * 1e-3) / 1e6, "ms_per_step": if_ms, "sigma": 1.0,
                "gpu_launches_per_step": g_if.kernel_count(),
                "path": "batched graph, IFOD tensor (1, 0, g, g) rebuilt every cycle, same FED cycles",
                "_out": {i: ims[i].out[:, :ims[i].w].cpu().numpy().astype(np.float64) for i in order}}
        g_if.close()
    g_all.launch()  # leave the outputs of a complete filter pass in place
    barrier()

    # plain path: per-image calls, one launch per FED step
    plain_prm = fd4.params(mode=mode, fed_steps_per_launch=1)
    ws_plain = fd4.workspace(fd4.OP_FILTER, max(b.pitch for b in ims), max(b.h for b in ims), K, dev)
    outs_plain = [torch.empty_like(b.u_in) for b in ims]

    def plain_step():
        for b, o in zip(ims, outs_plain):
            fd4.filter_image(b.u_in, b.w, sig, T, M, n, plain_prm, out=o, ws=ws_plain, keep_idx=False)

    plain_step()
    barrier()
    plain_ms = max_over_ranks(_timed(plain_step, max(1, min(args.steps, 3)), stream, torch) / max(1, min(args.steps, 3)))
    plain_value = world * px_steps / (plain_ms * 1e-3) / 1e6
    diff_plain = max(float((o[:, :b.w] - b.out[:, :b.w]).abs().max()) for o, b in zip(outs_plain, ims))

    # end to end through the public API: pinned host buffers, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        hin = [b.u_in.cpu().pin_memory() for b in ims]
        hout = [torch.empty_like(h).pin_memory() for h in hin]

        def e2e_step():
            for b, hi in zip(ims, hin):
                b.u_in.copy_(hi, non_blocking=True)
            g_all.launch()
            for b, ho in zip(ims, hout):
                ho.copy_(b.out, non_blocking=True)

        e2e_step()
        barrier()
        ems = max_over_ranks(_timed(e2e_step, args.steps, stream, torch))
        nbytes = sum(h.numel() * 4 for h in hin)
        e2e = {"value": world * px_steps * args.steps / (ems * 1e-3) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "ms_per_step": ems / args.steps,
               "path": "pinned host images -> fd4_graph_launch (batched filter) -> pinned host results"}

    if rank != 0:
        return
    peak, peak_kind = load_peaks()
    fed_bytes = 24 * npx * M * n  # algorithmic bytes of the FED steps of one pass
    achieved = fed_bytes / (fed_ms * 1e-3) / 1e9
    # the FED kernel the schedule runs: the TMA-staged quad kernel for 2 and 4 steps per launch
    # (fd4_fed_tma.cu), the scalar fused kernel for 3, one launch per step for 1 (fd4_fed.cu)
    kname = {1: "k_fed_step", 2: "k_fed_tma<2,2>", 3: "k_fed_fused<3>", 4: "k_fed_tma<4,2>"}[best]
    default_kernels = not any(os.environ.get(v) for v in ("FD4_FED_PIPELINE", "FD4_FED_QUAD_ROWS", "FD4_FED_FUSE",
                                                          "FD4_FED_QUADS"))
    traffic = args.traffic
    if traffic is None and kname == "k_fed_tma<2,2>" and default_kernels and TMA2_DRAM_B_PER_PX is not None:
        traffic = TMA2_DRAM_B_PER_PX * npx
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_unit": "bytes per launch", "kernel": kname,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (%s)" % peak_kind,
            "bytes_per_px_step": 24, "steps_per_launch": best,
            "avg_launch_us": fed_ms * 1e3 / fed_launches,
            "algorithmic_bytes_per_launch": fed_bytes / fed_launches}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": args.workload, "images": len(ims), "mpixel": round(npx / 1e6, 3),
                      "sigmas": K, "mode": wl["mode"], "M": M, "n": n, "T": T,
                      "path": "batched (one persistent launch per stage) + CUDA graph" + (
                          ", two image groups on two streams" if g_all is not g_one else ""),
                      "one_stream_graph_ms_per_step": one_stream_ms,
                      "fed_steps_per_launch": best, "autotune_ms": tune_ms,
                      "l2": "inputs larger than L2 (images %.2f GB, tensor field %.2f GB per pass)" % (
                          npx * 4e-9, npx * 16e-9)},
           "roofline": roof, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
           "clocks": clk.summary(),
           "stages_ms_per_step": {"select": sel_ms, "tensor": ten_ms, "fed": fed_ms},
           "plain": {"value": plain_value, "ms_per_step": plain_ms,
                     "path": "per-image fd4_filter calls, one launch per FED step",
                     "speedup_of_batched": value / plain_value, "max_abs_diff_to_batched": diff_plain}}
    if not args.no_learned:
        out["learned"] = learned_variant(args, ims, sig, T, M, n, mode, best, stream, torch, fd4)
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
            o2, _ = fd4.filter_image(b.u_in, b.w, sig, T, M, n, prm, sigma_idx=idx_in, ws=ws_plain)
            errs_inj.append(float(np.abs(o2[:, :b.w].cpu().numpy() - ref).max()))
        sample = "oracle full filter of the %d smallest batch images (%s px)" % (
            len(res), ", ".join("%dx%d" % imgs[i].shape[::-1] for i, _, _ in res))
        out["cpu_baseline"] = {"value": pxs / secs / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": sample, "seconds": secs}
        out["parity"] = {"vs": "FP64 oracle", "images": sample, "max_abs": max(errs),
                         "max_abs_oracle_sigma": max(errs_inj), "sigma_agreement": min(agree),
                         "tolerance": 1e-4}
        if resel is not None:
            from oracle import oracle as O
            tau_o, _, _ = O.fed_taus(T, M, 0.05, n=n)
            r_err, r_agree = [], []
            for i, (got, gidx) in resel["_out"].items():
                ref, ridx = O.filter_image(imgs[i], sig, tau_o, M, mode=mode, reselect=True)
                r_err.append(float(np.abs(got - ref).max()))
                r_agree.append(float((gidx == ridx).mean()))
            resel["parity"] = {"vs": "FP64 oracle, re-selecting schedule", "images": sample,
                               "max_abs": max(r_err), "last_sigma_agreement": min(r_agree), "tolerance": 1e-4}
        if post is not None:
            from oracle import oracle as O
            tau_o, _, _ = O.fed_taus(T, M, 0.05, n=n)
            p_err, p_agree, p_inj = [], [], []
            for i, (got, gidx) in post["_out"].items():
                ref, ridx = O.filter_image(imgs[i], sig, tau_o, M, mode=mode, postprocess=True,
                                           theta=post["theta"])
                p_err.append(float(np.abs(got - ref).max()))
                p_agree.append(float((gidx == ridx).mean()))
                # the same filter at the oracle's post-processed scale image
                b = ims[i]
                idx_in = torch.zeros_like(b.idx)
                idx_in[:, :b.w] = torch.from_numpy(ridx).to(dev)
                o2, _ = fd4.filter_image(b.u_in, b.w, sig, T, M, n, prm, sigma_idx=idx_in, ws=ws_plain)
                p_inj.append(float(np.abs(o2[:, :b.w].cpu().numpy() - ref).max()))
            post["parity"] = {"vs": "FP64 oracle, post-processed scale image", "images": sample,
                              "max_abs": max(p_err), "max_abs_oracle_sigma": max(p_inj),
                              "sigma_agreement": min(p_agree), "tolerance": 1e-4}
        if ifod is not None:
            from oracle import oracle as O
            tau_o, _, _ = O.fed_taus(T, M, 0.05, n=n)
            errs_if = [float(np.abs(got - O.filter_ifod(imgs[i], tau_o, M, sigma=1.0, lam=0.005)).max())
                       for i, got in ifod["_out"].items()]
            ifod["parity"] = {"vs": "FP64 oracle IFOD filter", "images": sample, "max_abs": max(errs_if),
                              "tolerance": 1e-4}
    if ifod is not None:
        ifod.pop("_out", None)
        out["ifod"] = ifod
    if world == 1 and not args.no_creases and args.workload == "batch64_fundus":
        out["creases"] = crease_leg(args, ims, mode, stream, torch, fd4)
    if resel is not None:
        resel.pop("_out", None)
        out["reselect"] = resel
    if post is not None:
        post.pop("_out", None)
        out["postprocess"] = post
    for g in {id(x): x for x in (g_all, g_one, g_sel, g_ten, g_fed)}.values():
        g.close()
    print(json.dumps(out), flush=True)


def crease_leg(args, ims, mode, stream, torch, fd4):
    """Crease extraction (Sec. 4) timed over the filtered batch, and the accuracy
    of Sec. 5 (E, p against the generator's centre lines inside the field of
    view, 6-pixel neighbourhood) of the creases of the input and of the
    filtered output of the two smallest images."""
    import ctypes
    from paper_1611_06906_gb300 import creases, synth
    sigma_d = 1.0
    maxw = max(b.w for b in ims)
    maxh = max(b.h for b in ims)
    cap = 2 * (maxw - 1) * (maxh - 1)
    segs = torch.empty((cap, 4), dtype=torch.float32, device=ims[0].out.device)
    keys = torch.empty(cap, dtype=torch.int32, device=segs.device)
    count = torch.zeros(1, dtype=torch.int32, device=segs.device)
    ws = fd4.workspace(fd4.OP_CREASES, max(b.pitch for b in ims), maxh, 0, segs.device)

    def run_all():
        for b in ims:
            rc = fd4.lib().fd4_extract_creases(ctypes.c_void_p(b.out.data_ptr()), b.w, b.h, b.pitch, sigma_d, mode,
                                               ctypes.c_void_p(segs.data_ptr()), ctypes.c_void_p(keys.data_ptr()),
                                               cap, ctypes.c_void_p(count.data_ptr()),
                                               ctypes.c_void_p(ws.data_ptr()), ws.numel(), None)
            if rc != 0:
                raise fd4.Fd4Error(rc, "fd4_extract_creases")

    run_all()
    torch.cuda.synchronize()
    ms = _timed(run_all, 3, stream, torch) / 3
    base = rank_seed(3000, 0)
    sides = synth.batch_sides(base)
    order = sorted(range(len(ims)), key=lambda i: ims[i].npx)[:2]
    acc = []
    for i in order:
        side = sides[i]
        c = (side - 1) / 2.0
        gt = [g for g in synth.vessel_tree_centrelines(base + i, side, side, depth=6, noise=0.0)
              if max(math.hypot(g[0] - c, g[1] - c), math.hypot(g[2] - c, g[3] - c)) < 0.9 * 0.48 * side]
        s_in, _ = fd4.extract_creases(ims[i].u_in, ims[i].w, sigma_d, mode)
        s_out, _ = fd4.extract_creases(ims[i].out, ims[i].w, sigma_d, mode)
        e_in, p_in = creases.evaluate(s_in, gt)
        e_out, p_out = creases.evaluate(s_out, gt)
        acc.append({"image": "%dx%d" % (ims[i].w, ims[i].h), "E_input": e_in, "p_input": p_in,
                    "E_filtered": e_out, "p_filtered": p_out, "segments_input": int(len(s_in)),
                    "segments_filtered": int(len(s_out)), "truth_segments": len(gt)})
    return {"sigma": sigma_d, "ms_per_batch": ms, "mpixel_per_s": sum(b.npx for b in ims) / (ms * 1e-3) / 1e6,
            "path": "fd4_extract_creases per filtered image (field + marching squares)", "accuracy": acc}


def learned_variant(args, ims, sig, T, M, n, mode, best, stream, torch, fd4):
    """Batched + learned path: the selector is trained here with the library's own
    kernels (seeded 256^2 crops labelled by the plain selection), then a step is
    the learned selection with plain fallback on low-confidence tiles, followed by
    the batched filter with those scales given, replayed as a CUDA graph."""
    from paper_1611_06906_gb300 import selector_train as ST
    t0 = time.perf_counter()
    crops, labels = ST.make_training_set(args.sel_crops, sig, mode)
    sel = fd4.Selector()
    sel.init(1)
    losses = ST.train(sel, crops, labels, epochs=2, batch=32, lr=2e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del crops, labels
    prm = fd4.params(mode=mode, fed_steps_per_launch=best)
    idx_l = [torch.zeros_like(b.idx) for b in ims]
    outs_l = [torch.empty_like(b.u_in) for b in ims]
    lst = fd4.image_list([b.u_in for b in ims], [b.w for b in ims], outs_l, idx_l)
    ws = fd4.batch_workspace(lst, len(sig))
    g = fd4.Graph(lst, sig, T, M, n, prm, sigma_given=True, ws=ws)
    big = max(ims, key=lambda b: b.h * b.pitch)
    wsl = torch.empty(int(fd4.lib().fd4_select_learned_workspace_bytes(big.pitch, big.h, big.pitch, len(sig))),
                      dtype=torch.uint8, device=big.u_in.device)
    thr = args.sel_threshold

    def step():
        for b, ix in zip(ims, idx_l):
            sel.select_learned(b.u_in, b.w, sig, prm, conf_threshold=thr, idx=ix, ws=wsl)
        g.launch()

    step()
    torch.cuda.synchronize()
    ms = _timed(step, max(1, min(args.steps, 3)), stream, torch) / max(1, min(args.steps, 3))
    px_steps = sum(b.npx for b in ims) * M * n
    agree = sum(int((a[:, :b.w] == b.idx[:, :b.w]).sum().item()) for a, b in zip(idx_l, ims)) / sum(
        b.npx for b in ims)
    fb = 0
    for b, ix in zip(ims, idx_l):
        _, _, nfb = sel.select_learned(b.u_in, b.w, sig, prm, conf_threshold=thr, idx=ix, ws=wsl)
        fb += int(nfb.item())
    tiles = sum(((b.w + 31) // 32) * ((b.h + 63) // 64) for b in ims)
    diff = max(float((o[:, :b.w] - b.out[:, :b.w]).abs().max()) for o, b in zip(outs_l, ims))
    # the network alone (no fallback) for its agreement and time
    def net_only():
        for b, ix in zip(ims, idx_l):
            sel.predict(b.u_in, b.w, idx=ix, ws=wsl)
    net_ms = _timed(net_only, 1, stream, torch)
    agree_net = sum(int((a[:, :b.w] == b.idx[:, :b.w]).sum().item()) for a, b in zip(idx_l, ims)) / sum(
        b.npx for b in ims)
    g.close()
    return {"value": px_steps / (ms * 1e-3) / 1e6, "ms_per_step": ms, "conf_threshold": thr,
            "sigma_agreement_with_plain": agree, "fallback_tile_fraction": fb / tiles,
            "max_abs_diff_to_plain_batched": diff, "network_only_sigma_agreement": agree_net,
            "network_only_ms": net_ms, "train": {"crops": args.sel_crops, "epochs": 2, "steps": len(losses),
                                                 "loss_first": losses[0], "loss_last": float(np.mean(losses[-10:])),
                                                 "seconds": train_s}}


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
    ap.add_argument("--fed-steps", type=int, default=0, help="FED steps per launch (0: autotune)")
    ap.add_argument("--no-learned", action="store_true", help="skip the batched+learned variant")
    ap.add_argument("--no-reselect", action="store_true", help="skip the per-cycle re-selection variant")
    ap.add_argument("--no-postprocess", action="store_true", help="skip the scale post-processing variant")
    ap.add_argument("--no-ifod", action="store_true", help="skip the IFOD comparator")
    ap.add_argument("--no-creases", action="store_true", help="skip the crease extraction and its accuracy")
    ap.add_argument("--two-streams", type=int, default=0, help="headline graph on two streams (1) or one (0)")
    ap.add_argument("--sel-crops", type=int, default=4096, help="training crops of the learned selector")
    ap.add_argument("--sel-threshold", type=float, default=0.5, help="fallback confidence threshold")
    ap.add_argument("--only-graph", action="store_true", help="replay the full graph only (profiling)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per FED launch from an ncu capture of the current kernel "
                         "(default: the stored per-pixel figure of k_fed_quad<2,64>, else null)")
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
