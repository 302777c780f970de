"""Benchmark of the MAFOD hot path on GB300.

A step is one pass of the whole hot path over one batch: for every image,
scale selection, then M cycles of (tensor build, FED cycle of n steps).
Metric: Mpixel-FED-steps/s = sum_images(w h) * M * n / time.

Default workload "tree16_4096": 16 seeded 4096^2 synthetic vessel trees (depth
8, radii 12 -> 0.75 px, each branch a ridge or a valley, noise sd 0.15;
268 Mpixel), 12 scales log-spaced over 0.75..12 px (kernel radii up to 48),
both creases enhanced, 10 FED cycles of 25 steps (T = 325/3, tau_max = 0.05),
lambda = 0.005, rho = 0.5, beta = 0.5.  The inputs (1.07 GB of images, 4.3 GB
of tensor field) are larger than L2.  "batch64_fundus" (64 fundus-like images
of 512^2..2048^2, 8 scales, valley mode, 5 x 20) and "tree_1024" are the other
workloads.

`value` is the batched path (one persistent launch per stage over the whole
batch, the schedule replayed as a CUDA graph, the FED kernel schedule picked by
the autotuner) with the plain vesselness selection; `plain` times the same
filter as per-image fd4_filter calls at the library's default FED fusion and
at one launch per FED step; `learned` is the batched path with the learned
selector (its network trained in the run on 10,000 seeded 256^2 crops).

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

# DRAM bytes (read + write) per pixel and launch of the FED kernel the
# autotuner picks, keyed by its schedule (steps, region rows, quads per thread),
# from an ncu capture of one launch on a smaller case of the same workload
# (profiles/); the roofline's `traffic` scales it to the launch timed here.
# Entries are removed (the field is then null) whenever that kernel changes.
FED_DRAM_B_PER_PX = {
    # k_fed_tma<2,2,64,true>: one launch over one 4096^2 image of the workload, 268.53 MB
    # read + 50.76 MB written over 16.78 Mpixel (profiles/k_fed_tma_tree16_4096.md)
    (2, 64, 2): 19.03,
}
# Algorithmic bytes of one FED step per pixel: u read (4) and written (4), and
# the three FED coefficient planes the filter's tensor build leaves for the
# kernel (mu3, q cos 2t, q sin 2t: 12).
FED_B_PER_PX_STEP = 20
METRIC = "Mpixel-steps/s, batched+learned vs plain GB300, at stated FP64-oracle error"
UNIT = "Mpixel-steps/s"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms (read-only)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    _count = 0

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        ClockSampler._count += 1  # one file per sampler: several may be summarised late
        self.path = os.path.join("/tmp", "fd4_clocks_%d_%d_%d.csv" % (os.getpid(), gpu_index, ClockSampler._count))

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


def _gen_fundus(args):
    seed, side = args
    from paper_1611_06906_gb300 import synth
    return synth.fundus_like(seed, side)


def _gen_tree16(seed):
    from paper_1611_06906_gb300 import synth
    return synth.tree16(seed)


def tree16_seed(rank: int, i: int) -> int:
    return 5000 + 100 * rank + i


def make_workload(name: str, rank: int, limit: int = 0):
    """Returns (list of float32 images, config dict)."""
    from paper_1611_06906_gb300 import synth
    wl = dict(synth.WORKLOADS[name])
    pool_n = min(16, os.cpu_count() or 1)
    if name == "batch64_fundus":
        base = rank_seed(3000, rank)  # weak scaling: every rank filters its own batch
        sides = synth.batch_sides(base)
        if limit:
            sides = sides[:limit]
        seeds = [base + i for i in range(len(sides))]
        with mp.get_context("spawn").Pool(pool_n) as pool:
            imgs = pool.map(_gen_fundus, list(zip(seeds, sides)))
    elif name == "tree_1024":
        imgs = [synth.vessel_tree(2000 + rank, 1024, 1024)]
    elif name == "tree16_4096":
        seeds = [tree16_seed(rank, i) for i in range(limit or 16)]
        with mp.get_context("spawn").Pool(pool_n) as pool:
            imgs = pool.map(_gen_tree16, seeds)
    else:
        raise SystemExit("unknown workload " + name)
    return imgs, wl


def center_crop(img, side):
    h, w = img.shape
    side = min(side, h, w)
    y0, x0 = (h - side) // 2, (w - side) // 2
    return np.ascontiguousarray(img[y0:y0 + side, x0:x0 + side])


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return "unknown"


def oracle_samples(imgs, wl, mode):
    """The two samples the oracle (FP64, host cores) is run on: the all-core
    sample (also the parity reference of the main path) and the smaller
    single-core one.  tree16_4096: central 512^2 and 256^2 crops of the first
    image; the other workloads: the smallest image and its central 256^2 crop."""
    if wl.get("name") == "tree16_4096" or imgs[0].shape == (4096, 4096):
        big = center_crop(imgs[0], 512)
        what = "central 512x512 crop of the first 4096x4096 image"
    else:
        k = min(range(len(imgs)), key=lambda i: imgs[i].size)
        big = imgs[k]
        what = "the smallest image (%dx%d)" % big.shape[::-1]
    small = center_crop(big, 256)
    return big, what, small


def oracle_timed(img, wl, mode, threads=0, **kw):
    """One oracle filter of img with the workload's parameters; returns (out, idx, seconds)."""
    from oracle import oracle as O
    tau, _, _ = O.fed_taus(wl["T"], wl["M"], 0.05, n=wl["n"])
    t0 = time.perf_counter()
    out, idx = O.filter_image(img, wl["sigmas"], tau, wl["M"], mode=mode, **kw)
    return out, idx, time.perf_counter() - t0


class Image:
    def __init__(self, img, dev, fd4, torch):
        self.h, self.w = img.shape
        self.npx = self.h * self.w
        self.u_in = fd4.to_device(img, dev)
        self.pitch = self.u_in.shape[1]
        self.out = torch.empty_like(self.u_in)
        self.idx = torch.zeros((self.h, self.pitch), dtype=torch.uint8, device=dev)


def _timed(fn, steps, stream, torch):
    """CUDA-event time (ms) of `steps` calls of fn on `stream`."""
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        fn()
    z.record(stream)
    z.synchronize()
    return a.elapsed_time(z)


def fed_kernel_name(sch) -> str:
    s, r, q = sch.steps_per_launch, sch.tile_rows, sch.quads_per_thread
    if s == 1:
        return "k_fed_step"
    if s == 3:
        return "k_fed_fused<3>"
    # the filter's tensor builds leave the FED coefficient planes for this kernel (SOA)
    return "k_fed_tma<%d,%d,%d,true>" % (s, q or 2, r or 64)


def run_fd4(args, rank, world, local_rank):
    imgs, wl = make_workload(args.workload, rank, args.limit)  # before CUDA init (spawn pool)
    wl["name"] = args.workload
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

    if args.only_selector:  # profiling: the learned selector's prediction over the batch's stack only
        if len({(b.h, b.pitch) for b in ims}) != 1:
            raise SystemExit("--only-selector needs images of one size")
        sel = fd4.Selector()
        sel.init(1)  # the kernels' work does not depend on the weights
        stack = torch.stack([b.u_in for b in ims])
        idx = torch.zeros(stack.shape, dtype=torch.uint8, device=dev)
        conf = torch.zeros(stack.shape, dtype=torch.float32, device=dev)
        wss = fd4.Selector.workspace(len(ims), ims[0].w, ims[0].h, ims[0].pitch, dev, infer=True)
        for _ in range(args.warmup):
            sel.predict(stack, ims[0].w, n_bins=K, idx=idx, conf=conf, ws=wss)
        ms = _timed(lambda: sel.predict(stack, ims[0].w, n_bins=K, idx=idx, conf=conf, ws=wss), args.steps,
                    stream, torch) / args.steps
        print(json.dumps({"only_selector": True, "images": len(ims), "ms_per_prediction": ms,
                          "gpx_per_s": npx / (ms * 1e-3) / 1e9}))
        return

    # batched path: one launch per stage across the batch, replayed as a CUDA graph
    lst = fd4.image_list([b.u_in for b in ims], [b.w for b in ims], [b.out for b in ims], [b.idx for b in ims])
    ws = fd4.batch_workspace(lst, K, dev)
    tried = []
    if args.fed_steps:
        sched = fd4.FedSchedule(args.fed_steps, 0, 0, 0.0)
    else:
        sched, tried = fd4.autotune_batched(lst, sig, T, M, n, fd4.params(mode=mode), ws=ws)
    prm = fd4.params(mode=mode, **sched.as_params())
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
    S = sched.steps_per_launch
    fed_launches = M * (-(-n // S))               # FED kernel launches per pass
    launches_per_step = g_all.kernel_count()      # kernel nodes of the captured graph

    for _ in range(args.warmup):
        g_all.launch()
    barrier()
    with ClockSampler(local_rank) as clk:
        ms = _timed(g_all.launch, args.steps, stream, torch)
        barrier()
    ms = max_over_ranks(ms)
    value = world * px_steps * args.steps / (ms * 1e-3) / 1e6

    # end to end through the public API: pinned host buffers, copies inside the
    # timed region; timed right after the device-resident steps, in the same
    # thermal and clock state (clocks sampled over it as well)
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
        with ClockSampler(local_rank) as clk_e2e:
            ems = max_over_ranks(_timed(e2e_step, args.steps, stream, torch))
            barrier()
        nbytes = sum(h.numel() * 4 for h in hin)
        serial = {"value": world * px_steps * args.steps / (ems * 1e-3) / 1e6, "ms_per_step": ems / args.steps,
                  "path": "pinned host images -> fd4_graph_launch -> pinned host results, one stream"}
        # streamed: two device buffer sets and two graphs (one workspace: each
        # replay writes its own tables); the copies of steps k + 1 (in) and k (out)
        # run on a copy stream while step k's graph runs
        dev_b = [(torch.empty_like(b.u_in), torch.empty_like(b.out), torch.zeros_like(b.idx)) for b in ims]
        lst_b = fd4.image_list([x[0] for x in dev_b], [b.w for b in ims], [x[1] for x in dev_b],
                               [x[2] for x in dev_b])
        g_b = fd4.Graph(lst_b, sig, T, M, n, prm, ws=ws)
        sets = [([b.u_in for b in ims], [b.out for b in ims], g_all), ([x[0] for x in dev_b], [x[1] for x in dev_b], g_b)]
        cs = torch.cuda.Stream()

        def streamed(K):
            ev_in = [torch.cuda.Event(), torch.cuda.Event()]
            ev_done = [torch.cuda.Event(), torch.cuda.Event()]
            ev_free = [None, None]
            start = torch.cuda.Event()
            start.record(stream)
            cs.wait_event(start)
            with torch.cuda.stream(cs):
                for d, hi in zip(sets[0][0], hin):
                    d.copy_(hi, non_blocking=True)
                ev_in[0].record(cs)
            for k in range(K):
                S, S1 = k % 2, (k + 1) % 2
                stream.wait_event(ev_in[S])
                sets[S][2].launch()
                ev_done[S].record(stream)
                with torch.cuda.stream(cs):
                    if k + 1 < K:
                        if ev_free[S1] is not None:
                            cs.wait_event(ev_free[S1])
                        for d, hi in zip(sets[S1][0], hin):
                            d.copy_(hi, non_blocking=True)
                        ev_in[S1].record(cs)
                    cs.wait_event(ev_done[S])
                    for ho, o in zip(hout, sets[S][1]):
                        ho.copy_(o, non_blocking=True)
                    ev_free[S] = torch.cuda.Event()
                    ev_free[S].record(cs)
            stream.wait_event(ev_free[(K - 1) % 2])

        streamed(2)
        barrier()
        with ClockSampler(local_rank) as clk_st:
            sms = max_over_ranks(_timed(lambda: streamed(args.steps), 1, stream, torch))
            barrier()
        g_b.close()
        del dev_b, lst_b
        e2e = {"value": world * px_steps * args.steps / (sms * 1e-3) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes, "ms_per_step": sms / args.steps,
               "path": "pinned host images -> fd4_graph_launch (batched filter) -> pinned host results; two "
                       "device buffer sets, the copies of the neighbouring steps on a copy stream during each "
                       "step's graph",
               "clocks": clk_st.summary(), "serial": dict(serial, clocks=clk_e2e.summary())}
    one_stream_ms = _timed(g_one.launch, args.steps, stream, torch) / args.steps
    # stage split and the FED kernel alone (each graph replays one stage of the same schedule)
    sel_ms = _timed(g_sel.launch, args.steps, stream, torch) / args.steps
    ten_ms = _timed(g_ten.launch, args.steps, stream, torch) / args.steps
    fed_ms = _timed(g_fed.launch, args.steps, stream, torch) / args.steps
    # the FED kernel's own launches (events around each launch of the FED-only graph
    # would split it; the graph's FED launches are all of one kernel, plus one
    # copy-back after the last cycle when the pass's launch count is odd: the cycles
    # alternate between u and the FED plane)
    fed_copy_backs = (M * ((-(-n // S)) if S > 1 else n)) % 2

    variants = {}
    crop_px_steps = None
    # the scale image selected again on the current image before every cycle
    # (reselect_each_cycle); the scale image post-processed after its selection
    # (Sec. 3.3) at the paper's fundus threshold theta = 0.13; the IFOD comparator
    # of Eq. 2 (sigma 1, the paper's setting) -- each on the same batch
    theta = float(np.float32(0.13))
    legs = []
    if not args.no_reselect:
        legs.append(("reselect", dict(reselect_each_cycle=1),
                     "batched graph, scale image re-selected on u^k before every cycle"))
    if not args.no_postprocess:
        legs.append(("postprocess", dict(postprocess_scales=1, theta=theta),
                     "batched graph, scale image post-processed after the selection"))
    if not args.no_ifod:
        legs.append(("ifod", dict(model=fd4.MODEL_IFOD, ifod_sigma=1.0),
                     "batched graph, IFOD tensor (1, 0, g, g) rebuilt every cycle, same FED cycles"))
    for name, kw, path in legs:
        g_v = fd4.Graph(lst, sig, T, M, n, fd4.params(mode=mode, **sched.as_params(), **kw), ws=ws)
        g_v.launch()
        barrier()
        v_ms = max_over_ranks(_timed(g_v.launch, args.steps, stream, torch)) / args.steps
        variants[name] = {"value": world * px_steps / (v_ms * 1e-3) / 1e6, "ms_per_step": v_ms,
                          "gpu_launches_per_step": g_v.kernel_count(), "path": path, "_kw": kw}
        g_v.close()
    if "postprocess" in variants:
        variants["postprocess"]["theta"] = theta
    if "ifod" in variants:
        variants["ifod"]["sigma"] = 1.0
    g_all.launch()  # leave the outputs of a complete filter pass in place
    barrier()

    # plain GPU path: per-image fd4_filter calls, at the library's default FED
    # schedule (2 steps fused per launch) and at one launch per FED step
    ws_plain = fd4.workspace(fd4.OP_FILTER, max(b.pitch for b in ims), max(b.h for b in ims), K, dev)
    outs_plain = [torch.empty_like(b.u_in) for b in ims]
    plain = {}
    n_plain = max(1, min(args.steps, 3))
    for key, kw, path in (("default_fusion", {}, "per-image fd4_filter calls, library default FED schedule "
                                                 "(2 steps per launch)"),
                          ("one_launch_per_step", dict(fed_steps_per_launch=1),
                           "per-image fd4_filter calls, one launch per FED step")):
        pp = fd4.params(mode=mode, **kw)

        def plain_step(pp=pp):
            for b, o in zip(ims, outs_plain):
                fd4.filter_image(b.u_in, b.w, sig, T, M, n, pp, out=o, ws=ws_plain, keep_idx=False)

        plain_step()
        barrier()
        p_ms = max_over_ranks(_timed(plain_step, n_plain, stream, torch) / n_plain)
        plain[key] = {"value": world * px_steps / (p_ms * 1e-3) / 1e6, "ms_per_step": p_ms, "path": path,
                      "max_abs_diff_to_batched": max(float((o[:, :b.w] - b.out[:, :b.w]).abs().max())
                                                     for o, b in zip(outs_plain, ims))}
    plain["speedup_of_batched"] = value / plain["default_fusion"]["value"]
    plain["speedup_of_fusion"] = plain["default_fusion"]["value"] / plain["one_launch_per_step"]["value"]
    plain["speedup_of_batched_over_one_launch_per_step"] = value / plain["one_launch_per_step"]["value"]

    learned = None
    if not args.no_learned:
        learned = learned_variant(args, ims, wl, sig, T, M, n, mode, sched, stream, torch, fd4)

    if rank != 0:
        return
    peak, peak_kind = load_peaks()
    fed_bytes = FED_B_PER_PX_STEP * npx * M * n  # algorithmic bytes of the FED steps of one pass
    fed_kernel_ms = fed_ms  # includes the copy-back launch, if any (one memory copy of u per pass)
    achieved = fed_bytes / (fed_kernel_ms * 1e-3) / 1e9
    key = (sched.steps_per_launch, sched.tile_rows, sched.quads_per_thread)
    traffic = args.traffic
    if traffic is None and key in FED_DRAM_B_PER_PX:
        traffic = FED_DRAM_B_PER_PX[key] * npx
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_unit": "bytes per launch", "kernel": fed_kernel_name(sched),
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (%s)" % peak_kind,
            "bytes_per_px_step": FED_B_PER_PX_STEP, "steps_per_launch": S,
            "avg_launch_us": fed_kernel_ms * 1e3 / fed_launches, "copy_back_launches_per_pass": fed_copy_backs,
            "algorithmic_bytes_per_launch": fed_bytes / fed_launches}
    # the selection stage is FP32-FMA bound: its algorithmic FMAs per pass (row and
    # column pass of 3 fields at every scale, radius ceil(4 sigma)) against the
    # FMA rate measured on this GPU
    fma_sel = sum(6 * (2 * math.ceil(4 * sg) + 1) for sg in sig) * npx
    fma_scalar, fma_pair = fd4.measure_fma_rate()
    fma_peak = max(fma_scalar, fma_pair)
    alu = {"fp32_fma_rate_measured_tfma": {"scalar": fma_scalar, "packed_pairs": fma_pair},
           "selection_stage": {"algorithmic_fma_per_pass": fma_sel,
                               "achieved_tfma": fma_sel / (sel_ms * 1e-3) / 1e12,
                               "frac_of_measured_fma_rate": fma_sel / (sel_ms * 1e-3) / 1e12 / fma_peak}}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "value_path": "batched (one persistent launch per stage over the batch's tiles) + CUDA graph, "
                         "plain vesselness selection (the learned selector's number is `learned`)",
           "config": {"workload": args.workload, "images": len(ims), "mpixel": round(npx / 1e6, 3),
                      "sigmas": K, "mode": wl["mode"], "M": M, "n": n, "T": T,
                      "path": "batched (one persistent launch per stage) + CUDA graph" + (
                          ", two image groups on two streams" if g_all is not g_one else ""),
                      "one_stream_graph_ms_per_step": one_stream_ms,
                      "fed_schedule": sched.as_dict(),
                      "autotune": [c.as_dict() for c in tried],
                      "l2": "inputs larger than L2 (images %.2f GB, tensor field %.2f GB per pass)" % (
                          npx * 4e-9, npx * 16e-9)},
           "roofline": roof, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
           "clocks": clk.summary(),
           "stages_ms_per_step": {"select": sel_ms, "tensor": ten_ms, "fed": fed_ms}, "alu": alu,
           "plain": plain}
    if learned is not None:
        out["learned"] = learned
    if world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        O.build()
        big, what, small = oracle_samples(imgs, wl, mode)
        cores = O.num_threads()
        ref, ridx, secs = oracle_timed(big, wl, mode)
        O.set_num_threads(1)
        _, _, secs1 = oracle_timed(small, wl, mode)
        O.set_num_threads(cores)
        rate = big.size * M * n / secs / 1e6
        rate1 = small.size * M * n / secs1 / 1e6
        full_h = px_steps / (rate * 1e6) / 3600
        out["cpu_baseline"] = {
            "value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "oracle full filter (the workload's scales, mode, M x n) of the %s, all %d threads"
                      % (what, cores),
            "seconds": secs, "cpu_model": cpu_model(),
            "single_thread": {"value": rate1, "unit": UNIT, "cores": 1, "seconds": secs1,
                              "sample": "central %dx%d crop of that sample, one thread" % small.shape[::-1]},
            "extrapolation": "the whole workload (%.1f G pixel-steps) at the all-thread rate: %.2f h; "
                             "at the one-thread rate: %.1f h" % (px_steps / 1e9, full_h,
                                                                 px_steps / (rate1 * 1e6) / 3600)}
        # parity on the same sample: the library's per-image filter with the bench's schedule
        u_s = fd4.to_device(big, dev)
        w_s = big.shape[1]
        o_s, i_s = fd4.filter_image(u_s, w_s, sig, T, M, n, prm)
        agree = float((i_s[:, :w_s].cpu().numpy() == ridx).mean())
        err = float(np.abs(o_s[:, :w_s].cpu().numpy() - ref).max())
        idx_in = torch.zeros_like(i_s)
        idx_in[:, :w_s] = torch.from_numpy(ridx).to(dev)
        o2, _ = fd4.filter_image(u_s, w_s, sig, T, M, n, prm, sigma_idx=idx_in)
        err_inj = float(np.abs(o2[:, :w_s].cpu().numpy() - ref).max())
        out["parity"] = {"vs": "FP64 oracle", "images": what, "tolerance": 1e-4,
                         "max_abs": err_inj,
                         "max_abs_is": "the filter's output from the oracle's scale image (every FP32 operation "
                                       "of the GPU path against FP64)",
                         "sigma_agreement": agree,
                         "sigma_disagreements": _tie_report(O, big, sig, mode, i_s[:, :w_s].cpu().numpy(), ridx),
                         "max_abs_own_selection": err}
        # the learned selector's scale image on the same sample: the filter's
        # distance from the oracle's (the method with the plain selection)
        if learned is not None and "_sel" in learned:
            i_n, _ = learned["_sel"].predict(u_s, w_s, n_bins=K)
            o_n, _ = fd4.filter_image(u_s, w_s, sig, T, M, n, prm, sigma_idx=i_n)
            dn = np.abs(o_n[:, :w_s].cpu().numpy() - ref)
            learned["network_only"]["vs_oracle"] = {
                "images": what, "max_abs": float(dn.max()), "mean_abs": float(dn.mean()),
                "sigma_agreement_with_oracle": float((i_n[:, :w_s].cpu().numpy() == ridx).mean())}
        # the variant legs against the oracle's variant on the 256^2 crop
        sm = center_crop(big, 256)
        u_sm = fd4.to_device(sm, dev)
        for name, leg in variants.items():
            kw = leg["_kw"]
            pv = fd4.params(mode=mode, **sched.as_params(), **kw)
            o_v, i_v = fd4.filter_image(u_sm, 256, sig, T, M, n, pv)
            got = o_v[:, :256].cpu().numpy()
            if name == "ifod":
                tau_o, _, _ = O.fed_taus(T, M, 0.05, n=n)
                ref_v = O.filter_ifod(sm, tau_o, M, sigma=1.0, lam=0.005)
                leg["parity"] = {"vs": "FP64 oracle IFOD filter", "images": "central 256x256 crop of the sample",
                                 "max_abs": float(np.abs(got - ref_v).max()), "tolerance": 1e-4}
                continue
            okw = dict(reselect=True) if name == "reselect" else dict(postprocess=True, theta=theta)
            ref_v, ridx_v, _ = oracle_timed(sm, wl, mode, **okw)
            par = {"vs": "FP64 oracle, %s" % ("re-selecting schedule" if name == "reselect"
                                              else "post-processed scale image"),
                   "images": "central 256x256 crop of the sample", "max_abs": float(np.abs(got - ref_v).max()),
                   "sigma_agreement": float((i_v[:, :256].cpu().numpy() == ridx_v).mean()), "tolerance": 1e-4}
            if name == "postprocess":
                idx_v = torch.zeros_like(i_v)
                idx_v[:, :256] = torch.from_numpy(ridx_v).to(dev)
                o3, _ = fd4.filter_image(u_sm, 256, sig, T, M, n, prm, sigma_idx=idx_v)
                par["max_abs_own_selection"] = par["max_abs"]
                par["max_abs"] = float(np.abs(o3[:, :256].cpu().numpy() - ref_v).max())
                par["max_abs_is"] = "the cycles from the oracle's post-processed scale image"
            else:
                par["max_abs_is"] = "the re-selecting schedule as it runs (no scale image can be given)"
            leg["parity"] = par
    for name, leg in variants.items():
        leg.pop("_kw", None)
        out[name] = leg
    if world == 1 and not args.no_creases:
        out["creases"] = crease_leg(args, ims, wl, mode, stream, torch, fd4,
                                    learned.get("_sel") if learned is not None else None, prm)
    if learned is not None:
        learned.pop("_sel", None)
    for g in {id(x): x for x in (g_all, g_one, g_sel, g_ten, g_fed)}.values():
        g.close()
    print(json.dumps(out), flush=True)


def _tie_report(O, img, sig, mode, idx_gpu, idx_oracle):
    """Where the GPU's FP32 selection picks another scale than the oracle's: how
    many pixels, and how far the oracle's own V at the GPU's scale is below its
    V at the oracle's scale (relative): a near-tie within FP32 rounding makes
    both selections valid, and the filter then legitimately differs there."""
    mism = idx_gpu != idx_oracle
    rep = {"pixels": int(mism.sum())}
    if mism.any():
        _, _, vall, _ = O.select_scales(img, sig, mode)
        yy, xx = np.nonzero(mism)
        v_best = vall[idx_oracle[yy, xx], yy, xx]
        v_gpu = vall[idx_gpu[yy, xx], yy, xx]
        gap = (v_best - v_gpu) / np.maximum(v_best, 1e-30)
        rep.update({"max_relative_V_gap": float(gap.max()), "all_within_1e-3": bool((gap <= 1e-3).all())})
    return rep


def _clip_split(gt, lo, hi, shift, max_len=32.0):
    """Ground-truth centre-line pieces clipped to the square [lo, hi]^2 (then
    shifted by -shift) and cut into pieces of at most max_len pixels: a chain
    of the reconstruction is matched piece by piece, so a branch hundreds of
    pixels long is scored along its whole length."""
    out = []
    for g in gt:
        ax, ay, bx, by = g[0], g[1], g[2], g[3]
        t0, t1 = 0.0, 1.0
        ok = True
        for p, q in ((-(bx - ax), ax - lo), (bx - ax, hi - ax), (-(by - ay), ay - lo), (by - ay, hi - ay)):
            if p == 0.0:
                if q < 0.0:
                    ok = False
                continue
            r = q / p
            if p < 0.0:
                t0 = max(t0, r)
            else:
                t1 = min(t1, r)
        if not ok or t1 <= t0:
            continue
        x0, y0 = ax + t0 * (bx - ax), ay + t0 * (by - ay)
        x1, y1 = ax + t1 * (bx - ax), ay + t1 * (by - ay)
        k = max(1, int(math.ceil(math.hypot(x1 - x0, y1 - y0) / max_len)))
        for i in range(k):
            f0, f1 = i / k, (i + 1) / k
            out.append((x0 + f0 * (x1 - x0) - shift, y0 + f0 * (y1 - y0) - shift,
                        x0 + f1 * (x1 - x0) - shift, y0 + f1 * (y1 - y0) - shift) + tuple(g[4:]))
    return out


def crease_leg(args, ims, wl, mode, stream, torch, fd4, sel=None, prm=None):
    """Crease extraction (Sec. 4) timed over the filtered batch, and the accuracy
    of Sec. 5 (E, p against the generator's centre lines, 6-pixel
    neighbourhood) of the creases of the input, of the filtered output and of
    the output filtered from the learned selector's scales: on the two smallest
    images of the fundus batch (pieces inside the field of view), or on the
    central 1024^2 window of the first 4096^2 tree; the centre lines are cut
    into pieces of at most 32 px."""
    import ctypes
    from paper_1611_06906_gb300 import creases, synth
    sigma_d = 1.0
    sig, M, n, T = wl["sigmas"], wl["M"], wl["n"], wl["T"]
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
    del segs, keys

    def learned_out(b):
        if sel is None:
            return None
        idx, _ = sel.predict(b.u_in, b.w, n_bins=len(sig))
        o, _ = fd4.filter_image(b.u_in, b.w, sig, T, M, n, prm, sigma_idx=idx)
        return o

    acc = []
    if wl["name"] == "batch64_fundus":
        base = rank_seed(3000, 0)
        sides = synth.batch_sides(base)
        order = sorted(range(len(ims)), key=lambda i: ims[i].npx)[:2]
        for i in order:
            side = sides[i]
            c = (side - 1) / 2.0
            gt = [g for g in synth.vessel_tree_centrelines(base + i, side, side, depth=6, noise=0.0)
                  if max(math.hypot(g[0] - c, g[1] - c), math.hypot(g[2] - c, g[3] - c)) < 0.9 * 0.48 * side]
            gt = _clip_split(gt, 0.0, side - 1.0, 0.0)
            pairs = [(ims[i].u_in, ims[i].w), (ims[i].out, ims[i].w)]
            lo = learned_out(ims[i])
            if lo is not None:
                pairs.append((lo, ims[i].w))
            acc.append(_crease_accuracy(fd4, creases, pairs, gt, sigma_d, mode, "%dx%d" % (ims[i].w, ims[i].h)))
    elif wl["name"] == "tree16_4096":
        win, y0 = 1024, (4096 - 1024) // 2
        gt = _clip_split(synth.vessel_tree_centrelines(tree16_seed(0, 0), 4096, 4096, depth=8, r0=12.0, r1=0.75,
                                                       noise=0.15), y0 + 8.0, y0 + win - 9.0, float(y0))
        pairs = []
        lo = learned_out(ims[0])
        for t in (ims[0].u_in, ims[0].out) + ((lo,) if lo is not None else ()):
            crop = fd4.empty_image(win, win, device=t.device)
            crop[:, :win] = t[y0:y0 + win, y0:y0 + win]
            pairs.append((crop, win))
        acc.append(_crease_accuracy(fd4, creases, pairs, gt, sigma_d, mode,
                                    "central %dx%d window of image 0" % (win, win)))
    return {"sigma": sigma_d, "ms_per_batch": ms, "mpixel_per_s": sum(b.npx for b in ims) / (ms * 1e-3) / 1e6,
            "path": "fd4_extract_creases per filtered image (field + marching squares)", "accuracy": acc}


def _crease_accuracy(fd4, creases, pairs, gt, sigma_d, mode, label):
    res = {"image": label, "truth_segments": len(gt)}
    for name, (u, w) in zip(("input", "filtered", "filtered_learned_scales"), pairs):
        s_, _ = fd4.extract_creases(u, w, sigma_d, mode)
        e, p = creases.evaluate(s_, gt)
        res["E_" + name] = e
        res["p_" + name] = p
        res["segments_" + name] = int(len(s_))
    return res


def learned_reselect(sel, ims, src, wss, ws, sig, T, M, n, mode, sched, K, stream, torch, fd4, reps):
    """Scales re-selected before every cycle by the network (SURVEY NEXT-2 with
    the learned selector): M times, the network's prediction on u^k over the
    image stack (one launch per layer), then one FED cycle with those scales
    (a one-cycle graph, scales given; the cycle's steps are those of T / M).
    Compared with the plain re-selecting schedule (reselect_each_cycle) on the
    same batch: its rate, and the distance between the two outputs.  src: the
    input stack; wss, ws: the selector's and the batch's workspaces (reused)."""
    dev = ims[0].u_in.device
    nb, w = len(ims), ims[0].w
    shape = (nb,) + tuple(ims[0].u_in.shape)
    buf = [torch.empty(shape, dtype=torch.float32, device=dev) for _ in range(2)]
    idx = torch.zeros(shape, dtype=torch.uint8, device=dev)
    prm = fd4.params(mode=mode, **sched.as_params())

    def lst(a, b):
        return fd4.image_list([a[k] for k in range(nb)], [w] * nb, [b[k] for k in range(nb)],
                              [idx[k] for k in range(nb)])

    lists = [lst(src, buf[0]), lst(buf[0], buf[1]), lst(buf[1], buf[0])]
    graphs = [fd4.Graph(l, sig, T / M, 1, n, prm, sigma_given=True, ws=ws) for l in lists]
    net_ms = [0.0]

    def step():
        cur = src
        for c in range(M):
            sel.predict(cur, w, n_bins=K, idx=idx, ws=wss)
            g = 0 if c == 0 else (1 if c % 2 else 2)
            graphs[g].launch()
            cur = buf[0] if g != 1 else buf[1]
        return cur

    out = step()
    torch.cuda.synchronize()
    ms = _timed(step, reps, stream, torch) / reps
    net_ms = _timed(lambda: sel.predict(src, w, n_bins=K, idx=idx, ws=wss), reps, stream, torch) / reps
    # the network's scale agreement with the plain selection on the same u^k, cycle by cycle
    agree = []
    cur = src
    wsel = fd4.workspace(fd4.OP_SELECT_SCALES, ims[0].pitch, ims[0].h, K, dev)
    idx_plain = torch.zeros(ims[0].u_in.shape, dtype=torch.uint8, device=dev)
    for c in range(M):
        sel.predict(cur, w, n_bins=K, idx=idx, ws=wss)
        a = 0
        for k in range(nb):
            fd4.select_scales(cur[k], w, sig, fd4.params(mode=mode), ws=wsel, idx=idx_plain)
            a += int((idx[k, :, :w] == idx_plain[:, :w]).sum())
        agree.append(a / (nb * ims[0].npx))
        g = 0 if c == 0 else (1 if c % 2 else 2)
        graphs[g].launch()
        cur = buf[0] if g != 1 else buf[1]
    out = cur
    torch.cuda.synchronize()
    # the plain re-selecting schedule on the same inputs
    outp = torch.empty(shape, dtype=torch.float32, device=dev)
    idxp = torch.zeros(shape, dtype=torch.uint8, device=dev)
    lp = fd4.image_list([src[k] for k in range(nb)], [w] * nb, [outp[k] for k in range(nb)],
                        [idxp[k] for k in range(nb)])
    gp = fd4.Graph(lp, sig, T, M, n, fd4.params(mode=mode, reselect_each_cycle=1, **sched.as_params()), ws=ws)
    gp.launch()
    torch.cuda.synchronize()
    d = (out[:, :, :w] - outp[:, :, :w]).abs()
    res = {"value": nb * ims[0].npx * M * n / (ms * 1e-3) / 1e6, "ms_per_step": ms,
           "network_ms_per_cycle": net_ms,
           "path": "per cycle: the network's prediction on u^k (one launch per layer over the stack), then a "
                   "one-cycle batched graph with those scales; M cycles",
           "sigma_agreement_per_cycle": agree,
           "vs_plain_reselect": {"max_abs": float(d.max()), "mean_abs": float(d.double().mean())}}
    for g in graphs + [gp]:
        g.close()
    return res


def learned_variant(args, ims, wl, sig, T, M, n, mode, sched, stream, torch, fd4):
    """The batched filter with the learned selector.  The network (n_bins = the
    workload's scales) is trained here with the library's own kernels on seeded
    256^2 crops labelled by the plain selection (sources disjoint from the
    batch), then timed and compared with the plain selection on the batch:

      * network only: its scale images (one launch per layer over the whole
        batch when the images have one size), then the batched filter graph
        with those scales given -- its rate, its scale agreement with the plain
        selection and its output's distance from the plain filter's;
      * network with the plain fallback: every 32 x 64 tile holding a pixel
        below the confidence threshold is selected again by the plain sweep
        (with the threshold at 1 every tile is, and the result is the plain
        filter's)."""
    from paper_1611_06906_gb300 import selector_train as ST
    K = len(sig)
    kind = "tree16" if wl["name"] == "tree16_4096" else "fundus"
    t0 = time.perf_counter()
    crops, labels = ST.make_training_set(args.sel_crops, sig, mode, kind=kind)
    t_set = time.perf_counter() - t0
    sel = fd4.Selector()
    sel.init(1)
    t0 = time.perf_counter()
    losses = ST.train(sel, crops, labels, K, epochs=args.sel_epochs, batch=32, lr=2e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del crops, labels
    prm = fd4.params(mode=mode, **sched.as_params())
    npx = sum(b.npx for b in ims)
    px_steps = npx * M * n
    same = len({(b.h, b.pitch) for b in ims}) == 1
    idx_l = [torch.zeros_like(b.idx) for b in ims]
    outs_l = [torch.empty_like(b.u_in) for b in ims]
    lst = fd4.image_list([b.u_in for b in ims], [b.w for b in ims], outs_l, idx_l)
    ws = fd4.batch_workspace(lst, K)
    g = fd4.Graph(lst, sig, T, M, n, prm, sigma_given=True, ws=ws)
    if same:  # one stack: every layer is one launch over the whole batch
        stack = torch.stack([b.u_in for b in ims])
        idx_stack = torch.zeros(stack.shape, dtype=torch.uint8, device=stack.device)
        wss = fd4.Selector.workspace(len(ims), ims[0].w, ims[0].h, ims[0].pitch, stack.device, infer=True)

        def net_select():
            sel.predict(stack, ims[0].w, n_bins=K, idx=idx_stack, ws=wss)
            for k, ix in enumerate(idx_l):
                ix.copy_(idx_stack[k])
    else:
        big = max(ims, key=lambda b: b.h * b.pitch)
        wsp = fd4.Selector.workspace(1, big.pitch, big.h, big.pitch, big.u_in.device, infer=True)

        def net_select():
            for b, ix in zip(ims, idx_l):
                sel.predict(b.u_in, b.w, n_bins=K, idx=ix, ws=wsp)

    def net_step():
        net_select()
        g.launch()

    net_step()
    torch.cuda.synchronize()
    reps = max(1, min(args.steps, 3))
    net_sel_ms = _timed(net_select, reps, stream, torch) / reps
    net_ms = _timed(net_step, reps, stream, torch) / reps
    agree_net = sum(int((a[:, :b.w] == b.idx[:, :b.w]).sum().item()) for a, b in zip(idx_l, ims)) / npx
    diff = [(o[:, :b.w] - b.out[:, :b.w]).abs() for o, b in zip(outs_l, ims)]
    net_out = {"value": px_steps / (net_ms * 1e-3) / 1e6, "ms_per_step": net_ms, "selection_ms": net_sel_ms,
               "sigma_agreement_with_plain": agree_net,
               "max_abs_diff_to_plain_filter": max(float(d.max()) for d in diff),
               "mean_abs_diff_to_plain_filter": sum(float(d.double().sum()) for d in diff) / npx,
               "launches_per_layer": 1 if same else len(ims)}
    # the fallback path: the network's confident tiles, the plain sweep on the rest
    thr = args.sel_threshold
    big = max(ims, key=lambda b: b.h * b.pitch)
    wsl = torch.empty(int(fd4.lib().fd4_select_learned_workspace_bytes(big.pitch, big.h, big.pitch, K)),
                      dtype=torch.uint8, device=big.u_in.device)
    nfb_l = []

    def exact_step():
        nfb_l.clear()
        for b, ix in zip(ims, idx_l):
            nfb_l.append(sel.select_learned(b.u_in, b.w, sig, prm, conf_threshold=thr, idx=ix, ws=wsl)[2])
        g.launch()

    exact_step()
    torch.cuda.synchronize()
    ex_ms = _timed(exact_step, reps, stream, torch) / reps
    fb = sum(int(x.item()) for x in nfb_l)
    tiles = sum(((b.w + 31) // 32) * ((b.h + 63) // 64) for b in ims)
    agree = sum(int((a[:, :b.w] == b.idx[:, :b.w]).sum().item()) for a, b in zip(idx_l, ims)) / npx
    fallback = {"value": px_steps / (ex_ms * 1e-3) / 1e6, "ms_per_step": ex_ms, "conf_threshold": thr,
             "sigma_agreement_with_plain": agree, "fallback_tile_fraction": fb / tiles,
             "max_abs_diff_to_plain_filter": max(float((o[:, :b.w] - b.out[:, :b.w]).abs().max())
                                                 for o, b in zip(outs_l, ims))}
    g.close()
    rs = None
    if same and not args.no_reselect:
        # a second network for re-selection before every cycle, trained on the
        # images of every cycle of the plain re-selecting schedule
        t0 = time.perf_counter()
        crops, labels = ST.make_training_set(args.sel_crops, sig, mode, kind=kind, cycles=(T, M, n))
        t_set_rs = time.perf_counter() - t0
        sel_rs = fd4.Selector()
        sel_rs.init(2)
        t0 = time.perf_counter()
        losses_rs = ST.train(sel_rs, crops, labels, K, epochs=args.sel_epochs, batch=32, lr=2e-3)
        torch.cuda.synchronize()
        train_rs = time.perf_counter() - t0
        del crops, labels
        rs = learned_reselect(sel_rs, ims, stack, wss, ws, sig, T, M, n, mode, sched, K, stream, torch, fd4, reps)
        rs["train"] = {"crops": args.sel_crops, "source": kind + ", every cycle of the re-selecting schedule",
                       "epochs": args.sel_epochs, "steps": len(losses_rs), "loss_first": losses_rs[0],
                       "loss_last": float(np.mean(losses_rs[-10:])), "set_seconds": t_set_rs,
                       "train_seconds": train_rs}
    return {"value": net_out["value"], "ms_per_step": net_ms, "reselect": rs,
            "value_is": "network-only scale selection + the batched filter graph (an approximation of the "
                        "method: see its agreement and its distance from the plain filter and the oracle)",
            "bins": K, "network_only": net_out, "with_fallback": fallback, "_sel": sel,
            "train": {"crops": args.sel_crops, "source": kind, "epochs": args.sel_epochs, "steps": len(losses),
                      "loss_first": losses[0], "loss_last": float(np.mean(losses[-10:])),
                      "set_seconds": t_set, "train_seconds": train_s}}


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle, as it stands, on the host cores; each
    step is one full filter of the bench's oracle sample of the workload."""
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_1611_06906_gb300 import synth
    wl = dict(synth.WORKLOADS[args.workload])
    wl["name"] = args.workload
    mode = MODES[wl["mode"]]
    if args.workload == "batch64_fundus":
        sides = synth.batch_sides(3000)
        i = int(np.argmin(sides))
        imgs = [synth.fundus_like(3000 + i, sides[i])]
    elif args.workload == "tree16_4096":
        imgs = [synth.tree16(tree16_seed(0, 0))]
    else:
        imgs, _ = make_workload(args.workload, 0, 1)
    O.build()
    big, what, _ = oracle_samples(imgs, wl, mode)
    pxs = big.size * wl["M"] * wl["n"]
    for _ in range(args.warmup):
        oracle_timed(big, wl, mode)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_timed(big, wl, mode)
    secs = time.perf_counter() - t0
    value = pxs * args.steps / secs / 1e6
    sample = "oracle full filter of the %s, one sample per step, all %d threads" % (what, O.num_threads())
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": args.workload, "sample": sample, "sigmas": len(wl["sigmas"]),
                      "mode": wl["mode"], "M": wl["M"], "n": wl["n"], "T": wl["T"]},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                            "sample": sample, "cpu_model": cpu_model()},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fd4", choices=["fd4", "reference"])
    ap.add_argument("--workload", default="tree16_4096",
                    choices=["tree16_4096", "batch64_fundus", "tree_1024"])
    ap.add_argument("--limit", type=int, default=0, help="use only the first N images (profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--fed-steps", type=int, default=0,
                    help="FED steps per launch with the default region and quads (0: autotune the schedule)")
    ap.add_argument("--no-learned", action="store_true", help="skip the batched+learned variant")
    ap.add_argument("--no-reselect", action="store_true", help="skip the per-cycle re-selection variant")
    ap.add_argument("--no-postprocess", action="store_true", help="skip the scale post-processing variant")
    ap.add_argument("--no-ifod", action="store_true", help="skip the IFOD comparator")
    ap.add_argument("--no-creases", action="store_true", help="skip the crease extraction and its accuracy")
    ap.add_argument("--two-streams", type=int, default=0, help="headline graph on two streams (1) or one (0)")
    ap.add_argument("--sel-crops", type=int, default=10000, help="training crops (256^2) of the learned selector")
    ap.add_argument("--sel-epochs", type=int, default=4, help="training epochs of the learned selector")
    ap.add_argument("--sel-threshold", type=float, default=0.5, help="fallback confidence threshold")
    ap.add_argument("--only-graph", action="store_true", help="replay the full graph only (profiling)")
    ap.add_argument("--only-selector", action="store_true",
                    help="time the learned selector's prediction over the batch only (profiling)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per FED launch from an ncu capture of the kernel the schedule runs "
                         "(default: the stored per-pixel figure of that schedule, else null)")
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
