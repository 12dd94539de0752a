"""Benchmark of the fused rounded-KLT hot path (forward + zonal + inverse + PSNR).

Workload (default, "roofline_4096"): 16 synthetic AR(1) uint8 images of
4096 x 4096 (rho = 0.95, seeds 2000..2015); block sizes N in {4, 8, 16, 32}
with the RKLT for rho = 0.95 and alpha_N = 2 sqrt(N/8); r = N^2/8.  One step
runs the fused kernel once per N over the 16 images and produces, per N, the
compact zig-zag coefficients, the rounded 8-bit reconstruction and per-image
SSE / PSNR.  Inputs (268 MB) exceed the 129 MB L2, so no flush is needed.

Metric: Mpixel/s of fused fwd+zonal+inv+PSNR (pixels counted once per N).
Under torchrun each rank processes its own 16 images (weak scaling, no
collective on the data path; the max over ranks of the timed region is used).

`--impl reference` times the FP64 CPU oracle (the reference arm of this
build) on a bounded sample of the same workload, on the host cores.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NS = (4, 8, 16, 32)
RHO = 0.95
NIMG, SIDE = 16, 4096

# DRAM traffic per launch from ncu (dram__bytes_read.sum + dram__bytes_write.sum),
# keyed by kernel; None until a capture of the current kernel exists.
# The fused kernel instantiation the library picks for r = N^2/8 (variant 0: one thread
# per block; 4: tensor cores, one warp per 32 x 32 block or region).
# (N = 4, 8: the register path with the error by Parseval, pars_kernel<N, D, OUT> with
# D the diagonal bound of r = N^2/8 and OUT = 3 (coefficients and reconstruction);
# N = 16, 32: the tensor-core variant of fused_kernel.)
KERNEL = {4: "pars_kernel<4, 2, 3>", 8: "pars_kernel<8, 4, 3>", 16: "fused_kernel<16, 4>", 32: "fused_kernel<32, 4>"}
TRAFFIC = {
    # dram__bytes_read.sum + dram__bytes_write.sum of one launch per kernel of the 16 x 4096^2
    # step, from the full ncu captures (profiles/pars_kernel_n4_n8_4096x16.md,
    # profiles/fused_kernel_tc_n16_n32_4096x16_full.md)
    "pars_kernel<4, 2, 3>": 268489216 + 342649088,
    "pars_kernel<8, 4, 3>": 268519168 + 344211712,
    "fused_kernel<16, 4>": 268546048 + 343022848,
    "fused_kernel<32, 4>": 268663552 + 343248896,
}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.skip = 0
        self.path = None

    def __enter__(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix=f"rklt_clocks_gpu{self.gpu}_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            # the timed region starts once nvidia-smi is producing samples
            t0 = time.time()
            while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
            self.f.flush()
            with open(self.path) as f:
                self.skip = sum(1 for _ in f)  # samples taken before the timed region
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        s = self._summary()
        try:
            if self.path:
                os.unlink(self.path)
        except OSError:
            pass
        return s

    def _summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            lines = f.readlines()
        body = lines[self.skip:] if len(lines) > self.skip else lines
        for ln in body:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_images(rank: int = 0):
    """This rank's 16 images: seeds 2000 + 16*rank + i (rank 0 = the single-GPU workload).
    Imports only the input generators, so the oracle arm never loads the CUDA library."""
    import synth_inputs as si
    return si.roofline_batch(NIMG, SIDE, si.rank_seeds(2000, NIMG, rank)[0])


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline leg)
# ---------------------------------------------------------------------------
def oracle_sample(imgs, budget_s: float = 15.0):
    """Time the FP64 oracle on a bounded sample: image 0 (then 1, 2, ...) for every
    N until about budget_s of CPU work; returns (Mpixel/s, cores, sample text)."""
    import oracle
    oracle.build()
    plans = {n: oracle.Plan(n, RHO) for n in NS}
    px = 0
    t0 = time.perf_counter()
    used = 0
    for i in range(imgs.shape[0]):
        for n in NS:
            oracle.pipeline(n, plans[n].That, imgs[i], n * n // 8)
            px += imgs[i].size
        used = i + 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    cores = oracle.max_threads()
    return px / dt / 1e6, cores, (f"{used} of {imgs.shape[0]} images x N in {NS}, {SIDE}x{SIDE}, "
                                  f"r = N^2/8, FP64 C oracle with OpenMP over blocks ({dt:.1f} s)")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    imgs = make_images()
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; steps below are timed as they are
    vals = []
    cores, sample = None, None
    for _ in range(max(1, args.steps)):
        v, cores, sample = oracle_sample(imgs, budget_s=args.ref_budget)
        vals.append(v)
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": "Mpixel/s fwd+zonal+inv+PSNR", "value": value, "unit": "Mpixel/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        # the time one whole step (16 images x 4 block sizes) takes at the sampled rate
        "ms_per_step": len(NS) * NIMG * SIDE * SIDE / (value * 1e6) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic AR(1) uint8",
        "config": {"workload": "roofline_4096: 16 x 4096x4096 AR(1) rho=0.95, N in {4,8,16,32}, r=N^2/8",
                   "impl_detail": "FP64 CPU oracle (oracle/rklt_oracle.c)",
                   "ms_per_step": "extrapolated from the sampled rate (each step times a bounded sample)"},
        "cpu_baseline": {"value": value, "unit": "Mpixel/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    global NS
    NS = tuple(int(x) for x in args.block_sizes.split(","))
    import paper_2111_14239_gb300 as rk

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    imgs_np = make_images(rank)
    H = W = SIDE
    plans = {n: rk.rklt_make(n, RHO) for n in NS}
    rs = {n: n * n // 8 for n in NS}
    dev = torch.device("cuda", local)
    d_img = torch.from_numpy(imgs_np).to(dev)
    outs = {}
    for n in NS:
        nblk = (H // n) * (W // n)
        outs[n] = dict(
            zc=torch.empty((NIMG, nblk, rs[n]), dtype=torch.float32, device=dev),
            rec=torch.empty((NIMG, H, W), dtype=torch.uint8, device=dev),
            sse=torch.empty(NIMG, dtype=torch.float64, device=dev),
            ps=torch.empty(NIMG, dtype=torch.float32, device=dev))
    stream = torch.cuda.current_stream(dev)

    def one_pass(ev=None):
        for n in NS:
            o = outs[n]
            if ev is not None:
                ev[n][0].record(stream)
            rk.rklt_fused_batched(plans[n], d_img, rs[n], o["sse"], o["ps"], zcoef=o["zc"], recon=o["rec"],
                                  stream=stream)
            if ev is not None:
                ev[n][1].record(stream)

    # one step = `passes` passes over the 16 images, chosen so that the K timed steps
    # last at least --min-timed-s on the device (steadier kernel times, several clock
    # samples); the per-kernel events bracket the first pass of every step
    for _ in range(3):
        one_pass()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(5):
        one_pass()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    pass_ms = e0.elapsed_time(e1) / 5
    passes = max(1, math.ceil(args.min_timed_s * 1e3 / (args.steps * pass_ms)))
    if dist:  # every rank runs the same number of passes
        t = torch.tensor([passes], dtype=torch.int64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        passes = int(t.item())

    def step(ev=None):
        for p in range(passes):
            one_pass(ev if p == 0 else None)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    rk.rklt_device_status()

    # ---- device-resident timed region
    evs = [{n: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for n in NS}
           for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        start.record(stream)
        for k in range(args.steps):
            step(evs[k])
        stop.record(stream)
        torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    ms = start.elapsed_time(stop)
    kern_ms = {n: statistics.mean(e[n][0].elapsed_time(e[n][1]) for e in evs) for n in NS}
    from paper_2111_14239_gb300 import replicas
    ms = replicas.max_over_ranks(ms, dev)
    rk.rklt_device_status()

    px_step = len(NS) * NIMG * H * W * passes
    value = replicas.job_throughput(px_step * args.steps, world, ms / 1e3) / 1e6

    # ---- end to end through the C ABI with host buffers
    pin_in = torch.from_numpy(imgs_np).pin_memory()
    pin_out = {n: dict(zc=torch.empty(outs[n]["zc"].shape, dtype=torch.float32).pin_memory(),
                       rec=torch.empty(outs[n]["rec"].shape, dtype=torch.uint8).pin_memory(),
                       ps=torch.empty(NIMG, dtype=torch.float32).pin_memory()) for n in NS}

    # image by image on four streams, so that one image's copies overlap the others'
    # kernels and copies (the link carries ~200 GB/s each way, ~330 GB/s both ways)
    side = [torch.cuda.Stream(dev) for _ in range(4)]
    joins = [torch.cuda.Event() for _ in side]

    def e2e_step():
        go = torch.cuda.Event()
        go.record(stream)
        for s_ in side:
            s_.wait_event(go)
        for i in range(NIMG):
            s_ = side[i % len(side)]
            with torch.cuda.stream(s_):
                d_img[i].copy_(pin_in[i], non_blocking=True)
                for n in NS:
                    o = outs[n]
                    rk.rklt_fused(plans[n], d_img[i], rs[n], o["sse"][i:i + 1], o["ps"][i:i + 1], zcoef=o["zc"][i],
                                  recon=o["rec"][i], stream=s_)
                    pin_out[n]["zc"][i].copy_(o["zc"][i], non_blocking=True)
                    pin_out[n]["rec"][i].copy_(o["rec"][i], non_blocking=True)
                    pin_out[n]["ps"][i:i + 1].copy_(o["ps"][i:i + 1], non_blocking=True)
        for s_, j in zip(side, joins):
            j.record(s_)
            stream.wait_event(j)

    e2e_steps = 0 if args.no_e2e else max(2, min(args.steps, 10))
    for _ in range(2 if e2e_steps else 0):
        e2e_step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    s2, t2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s2.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    t2.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = replicas.max_over_ranks(s2.elapsed_time(t2), dev)
    h2d = imgs_np.nbytes
    d2h = sum(pin_out[n]["zc"].numel() * 4 + pin_out[n]["rec"].numel() + NIMG * 4 for n in NS)
    px_pass = len(NS) * NIMG * H * W
    e2e_val = px_pass * e2e_steps * world / (e2e_ms / 1e3) / 1e6 if e2e_steps else None

    psnr = {n: [round(float(x), 4) for x in outs[n]["ps"].cpu().tolist()[:2]] for n in NS}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (longest launch)
    hbm, hbm_src = peaks()
    per_n = {}
    for n in NS:
        r = rs[n]
        alg_bytes = NIMG * H * W * (1.0 + 4.0 * r / (n * n) + 1.0)
        gbs = alg_bytes / (kern_ms[n] / 1e3) / 1e9
        per_n[str(n)] = {"kernel": KERNEL[n], "ms": round(kern_ms[n], 4), "alg_bytes": alg_bytes,
                         "GB/s": round(gbs, 1), "frac_of_measured_hbm": round(gbs / hbm, 4)}
    dom = max(NS, key=lambda n: kern_ms[n])
    dk = per_n[str(dom)]
    traffic = TRAFFIC.get(dk["kernel"])
    cpu = None
    if not args.no_cpu_baseline:
        v, cores, sample = oracle_sample(imgs_np, budget_s=args.ref_budget)
        cpu = {"value": v, "unit": "Mpixel/s", "cores": cores, "kind": "oracle", "sample": sample}

    workloads = {}
    if world == 1 and not args.no_extras:
        for name, fn in (("single_512", lambda: leg_single(rk, dev, stream)),
                         ("psnr_only_4096", lambda: leg_psnr_only(rk, d_img, dev, stream)),
                         ("comparison_klt_dct_4096", lambda: leg_comparison(rk, d_img, dev, stream)),
                         ("quant_jpeg_like_4096", lambda: leg_quant(rk, d_img, dev, stream)),
                         ("mssim_4096", lambda: leg_mssim(rk, d_img, dev, stream)),
                         ("r_sweep_256x512", lambda: leg_sweep(rk, dev, stream)),
                         ("batch_2000_uneven", lambda: leg_batch(rk, dev, stream, args.batch_images)),
                         ("serving", lambda: leg_serve(rk, dev, args.serve_seconds))):
            if args.legs and name not in args.legs.split(","):
                continue
            try:
                workloads[name] = fn()
            except Exception as e:  # report, do not lose the main line
                workloads[name] = {"error": repr(e)}
        rk.rklt_device_status()

    line = {
        "metric": "Mpixel/s fwd+zonal+inv+PSNR",
        "value": value, "unit": "Mpixel/s", "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup),
        "ms_per_step": ms / args.steps, "ms_per_pass": ms / (args.steps * passes),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": ("u8 in / int-exact T-stage / f32 inverse (N = 16, 32: tensor-core inverse on two binary16 "
                  "digits per operand, about 22 significant bits, f32 accumulation)"),
        "data": "synthetic AR(1) uint8 (seeded)",
        "config": {"workload": "roofline_4096: 16 x 4096x4096 AR(1) rho=0.95, N in {4,8,16,32}, r=N^2/8, "
                               "outputs: compact coeffs + uint8 recon + PSNR",
                   "images_per_gpu": NIMG, "side": SIDE, "block_sizes": list(NS), "r": [rs[n] for n in NS],
                   "l2": "inputs 268 MB > 129 MB L2 (no flush needed)", "parallelism": f"replicas x{world}",
                   "passes_per_step": passes, "timed_ms": round(ms, 2),
                   "step": "passes_per_step passes of the fused call over the 16 images for every N"},
        "roofline": {"bound": "hbm", "achieved": dk["GB/s"], "peak": hbm, "unit": "GB/s",
                     "frac": round(dk["GB/s"] / hbm, 4), "traffic": traffic,
                     "kernel": dk["kernel"], "peak_source": f"{hbm_src} hbm_gbs (MEASURED_PEAKS.json)"},
        "per_block_size": per_n,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "Mpixel/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        # per pass and N: the fused kernel and the per-image finalize kernel (plus a
        # memset of the error accumulators on the register path)
        "gpu_launches": 2 * len(NS) * args.steps * passes,
        "clocks": clk.summary(),
        "psnr_sample_db": psnr,
        "workloads": workloads,
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()



# ---------------------------------------------------------------------------
# Extra workloads, measured after the main timed region (single GPU only)
# ---------------------------------------------------------------------------
def _time_ms(fn, reps, stream):
    import torch
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def leg_single(rk, dev, stream):
    """One 512 x 512 image (rho 0.95, seed 0), N = 8, r = 10: per-call latency."""
    import torch
    import synth_inputs as si
    img = torch.from_numpy(si.single_512()).to(dev)
    plan = rk.rklt_make(8, 0.95)
    zc = torch.empty((64 * 64, 10), device=dev)
    rec = torch.empty_like(img)
    sse = torch.empty(1, dtype=torch.float64, device=dev)
    ps = torch.empty(1, device=dev)
    ms = _time_ms(lambda: rk.rklt_fused(plan, img, 10, sse, ps, zcoef=zc, recon=rec, stream=stream), 200, stream)
    # the same call captured 100 times in a CUDA graph: the device-side latency without
    # the host's per-call issue cost (about 10 us of argument checks, descriptors, launches)
    gs = torch.cuda.Stream(dev)
    with torch.cuda.stream(gs):
        for _ in range(3):
            rk.rklt_fused(plan, img, 10, sse, ps, zcoef=zc, recon=rec, stream=gs)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gs):
        for _ in range(100):
            rk.rklt_fused(plan, img, 10, sse, ps, zcoef=zc, recon=rec, stream=gs)
    gms = _time_ms(graph.replay, 5, stream) / 100
    return {"workload": "1 x 512x512, N=8, rho=0.95, r=10, fwd+zonal+inv+PSNR", "us_per_image": ms * 1e3,
            "mpixel_per_s": 512 * 512 / (ms / 1e3) / 1e6, "graph_us_per_image": gms * 1e3,
            "graph_mpixel_per_s": 512 * 512 / (gms / 1e3) / 1e6, "psnr_db": round(float(ps.item()), 4)}


def leg_psnr_only(rk, d_img, dev, stream):
    """The 16 x 4096^2 workload with PSNR as the only product (no coefficients, no
    reconstruction): 1.0 B/px of algorithmic traffic, per N."""
    import torch
    nimg, H, W = d_img.shape
    hbm, _ = peaks()
    out = {"workload": f"{nimg} x {H}x{W} AR(1) rho={RHO}, N in {{4,8,16,32}}, r=N^2/8, PSNR only (1 B/px)"}
    for n in NS:
        plan = rk.rklt_make(n, RHO)
        sse = torch.empty(nimg, dtype=torch.float64, device=dev)
        ps = torch.empty(nimg, device=dev)
        ms = _time_ms(lambda: rk.rklt_fused_batched(plan, d_img, n * n // 8, sse, ps, stream=stream), 10, stream)
        gbs = nimg * H * W * 1.0 / (ms / 1e3) / 1e9
        # N <= 8 with T T^T diagonal: the error by Parseval in integers, no inverse
        pars = plan.kind == 0 and plan.orthogonal and (n == 4 or (n == 8 and n * n // 8 <= 15))
        kern = (f"pars_kernel<{n}, {zz_bound(n, n * n // 8)}, 0>" if pars else
                f"fused_kernel<{n}, 4>")
        out[str(n)] = {"ms": round(ms, 4), "GB/s": round(gbs, 1), "frac_of_measured_hbm": round(gbs / hbm, 4),
                       "psnr_db_img0": round(float(ps[0].item()), 4),
                       "error_by": "parseval (integers)" if pars else "inverse transform",
                       "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                                    "frac": round(gbs / hbm, 4), "traffic": None, "kernel": kern,
                                    "bytes_per_px": 1.0}}
    return out


def zz_bound(n, r):
    """Diagonal bound D of the first r zig-zag positions (every kept (i, j) has i + j < D)."""
    d, cnt = 0, 0
    while cnt < r:
        cnt += min(d, 2 * n - 2 - d) + 1
        d += 1
    return d


def leg_comparison(rk, d_img, dev, stream):
    """The paper's comparison transforms (exact KLT, DCT-II; FP32 dense) against the
    RKLT through the same fused pass on the 16 x 4096^2 workload, N = 8, r = 8: time,
    bandwidth and PSNR of image 0 for each."""
    import torch
    n, r = 8, 8
    nimg, H, W = d_img.shape
    nblk = (H // n) * (W // n)
    zc = torch.empty((nimg, nblk, r), device=dev)
    rec = torch.empty_like(d_img)
    sse = torch.empty(nimg, dtype=torch.float64, device=dev)
    ps = torch.empty(nimg, device=dev)
    out = {"workload": f"{nimg} x {H}x{W} AR(1) rho={RHO}, N=8, r=8; outputs as the main line"}
    hbm, _ = peaks()
    for name, plan in (("rklt", rk.rklt_make(n, RHO)), ("exact_klt", rk.rklt_make_klt(n, RHO)),
                       ("dct", rk.rklt_make_dct(n))):
        ms = _time_ms(lambda: rk.rklt_fused_batched(plan, d_img, r, sse, ps, zcoef=zc, recon=rec, stream=stream),
                      10, stream)
        gbs = nimg * H * W * 2.5 / (ms / 1e3) / 1e9
        out[name] = {"ms": round(ms, 4), "GB/s": round(gbs, 1), "frac_of_measured_hbm": round(gbs / hbm, 4),
                     "psnr_db_img0": round(float(ps[0].item()), 4)}
    return out


def leg_quant(rk, d_img, dev, stream):
    """JPEG-like quantisation with S absorbed (Appendix) on the 16 x 4096^2 workload,
    N = 8, every coefficient quantised (r = 64) with a frequency ramp Q = 2 + 3 (i + j):
    time, bandwidth (1 B read + 4 B/coefficient int32 + 1 B reconstruction per pixel)
    and PSNR of image 0."""
    import numpy as np
    import torch
    n, r = 8, 64
    nimg, H, W = d_img.shape
    nblk = (H // n) * (W // n)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    Q = 2.0 + 3.0 * (i + j)
    plan = rk.rklt_make(n, RHO)
    qc = torch.empty(nimg * nblk * r, dtype=torch.int32, device=dev)
    rec = torch.empty_like(d_img)
    sse = torch.empty(nimg, dtype=torch.float64, device=dev)
    ps = torch.empty(nimg, device=dev)
    ms = _time_ms(lambda: rk.rklt_fused_quant(plan, d_img, r, Q, sse, ps, qcoef=qc, recon=rec, stream=stream), 10,
                  stream)
    bytes_px = 1.0 + 4.0 * r / (n * n) + 1.0
    gbs = nimg * H * W * bytes_px / (ms / 1e3) / 1e9
    hbm, _ = peaks()
    out = {"workload": f"{nimg} x {H}x{W} AR(1) rho={RHO}, N=8, r=64, Q = 2 + 3 (i + j), int32 coefficients",
           "ms": round(ms, 4), "GB/s": round(gbs, 1), "frac_of_measured_hbm": round(gbs / hbm, 4),
           "bytes_per_px": bytes_px, "psnr_db_img0": round(float(ps[0].item()), 4)}
    # N = 32 at r = N^2/8 on the tensor cores, same ramp
    n, r = 32, 128
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    plan = rk.rklt_make(n, RHO)
    qc = torch.empty(nimg * (H // n) * (W // n) * r, dtype=torch.int32, device=dev)
    ms = _time_ms(lambda: rk.rklt_fused_quant(plan, d_img, r, 2.0 + 3.0 * (i + j), sse, ps, qcoef=qc, recon=rec,
                                              stream=stream), 10, stream)
    bytes_px = 1.0 + 4.0 * r / (n * n) + 1.0
    gbs = nimg * H * W * bytes_px / (ms / 1e3) / 1e9
    out["n32_r128"] = {"ms": round(ms, 4), "GB/s": round(gbs, 1), "frac_of_measured_hbm": round(gbs / hbm, 4),
                       "bytes_per_px": bytes_px, "psnr_db_img0": round(float(ps[0].item()), 4)}
    return out


def fp32_peak_tflops(dev, sm_mhz=None):
    """FP32 FMA peak from the unit counts and the maximum SM clock: the device's SM
    count (cudaGetDeviceProperties) x 128 FP32 lanes x 2 flop x clock (default: the
    maximum SM clock recorded in MEASURED_PEAKS.json, else 2070 MHz)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    if sm_mhz is None:
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                sm_mhz = float(json.load(f)["sm_max_mhz"])
        except Exception:
            sm_mhz = 2070.0
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12, sms, sm_mhz


def leg_mssim(rk, d_img, dev, stream):
    """MSSIM (Sec. 4.1) of the 16 x 4096^2 originals against their 8-bit RKLT
    reconstructions (N = 8, r = 8): time of the MSSIM pass alone (2 B/px read) and
    the MSSIM of image 0."""
    import torch
    n, r = 8, 8
    nimg, H, W = d_img.shape
    plan = rk.rklt_make(n, RHO)
    rec = torch.empty_like(d_img)
    sse = torch.empty(nimg, dtype=torch.float64, device=dev)
    ps = torch.empty(nimg, device=dev)
    rk.rklt_fused_batched(plan, d_img, r, sse, ps, recon=rec, stream=stream)
    out = torch.empty(nimg, dtype=torch.float64, device=dev)
    ms = _time_ms(lambda: rk.rklt_mssim(d_img, rec, out, stream=stream), 10, stream)
    gbs = nimg * H * W * 2.0 / (ms / 1e3) / 1e9
    hbm, _ = peaks()
    # ALU roofline: the separable window costs 4 sums x (11 + 11) taps x 2 flop = 176
    # FP32 flop per output position; peak = 152 SMs x 128 FP32 lanes x 2 flop x SM clock
    npos = nimg * (H - 10) * (W - 10)
    tflops = npos * 176.0 / (ms / 1e3) / 1e12
    fp32_peak, sms, mhz = fp32_peak_tflops(dev)
    # the fused pass with MSSIM in one launch, against the fused pass + this pass
    fused_ms = _time_ms(lambda: rk.rklt_fused_batched(plan, d_img, r, sse, ps, recon=rec, stream=stream), 10, stream)
    ms2 = torch.empty_like(out)
    one_rec = _time_ms(lambda: rk.rklt_fused_mssim(plan, d_img, r, sse, ps, ms2, recon=rec, stream=stream), 10,
                       stream)
    one_norec = _time_ms(lambda: rk.rklt_fused_mssim(plan, d_img, r, sse, ps, ms2, stream=stream), 10, stream)
    torch.cuda.synchronize()
    fused_vs_two = float((ms2 - out).abs().max().item())
    return {"workload": f"{nimg} x {H}x{W}: original vs 8-bit RKLT reconstruction (N=8, r=8)",
            "ms": round(ms, 4), "GB/s": round(gbs, 1), "frac_of_measured_hbm": round(gbs / hbm, 4),
            "fused_then_mssim_ms": round(fused_ms + ms, 4),
            "fused_mssim_one_launch_ms": round(one_rec, 4),
            "fused_mssim_one_launch_no_recon_ms": round(one_norec, 4),
            "one_launch_vs_two_pass_max_abs_mssim_diff": fused_vs_two,
            "roofline": {"bound": "alu", "achieved": round(tflops, 2), "peak": round(fp32_peak, 1),
                         "unit": "TFLOP/s", "frac": round(tflops / fp32_peak, 4),
                         "flop_per_position": 176,
                         "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz (device properties)"},
            "mssim_img0": round(float(out[0].item()), 6), "psnr_db_img0": round(float(ps[0].item()), 4)}


def leg_sweep(rk, dev, stream):
    """256 images of 512 x 512 (rho ~ U(0.80, 0.98)), N = 8 plans for the 10 grid rho,
    PSNR for every r = 1..64."""
    import torch
    import synth_inputs as si
    imgs, _ = si.sweep_batch(256, 512, 1000)
    d = torch.from_numpy(imgs).to(dev)
    plans = [rk.rklt_make(8, rho) for rho in si.GRID_RHOS]
    ps = torch.empty((256, len(plans), 64), device=dev)
    ms = _time_ms(lambda: rk.rklt_rsweep(plans, d, None, ps, stream=stream), 10, stream)
    return {"workload": "256 x 512x512 AR(1), 10 plans (4 distinct T), r = 1..64", "ms_per_sweep": ms,
            "mpixel_per_s": imgs.size / (ms / 1e3) / 1e6,
            "psnr_values_per_s": 256 * len(plans) * 64 / (ms / 1e3),
            "l2": "input 67 MB is L2-resident between repetitions",
            "psnr_db_img0_T4_r10": round(float(ps[0, 9, 9].item()), 4)}


def leg_batch(rk, dev, stream, n_images=2000):
    """2000 AR(1) crops, sides U{64..4096 step 8}, rho ~ U(0.5, 0.98) -> nearest of the
    10 grid RKLTs, N = 8, r ~ U{1..64}: one graph-replayed persistent batch against
    one fused launch per image."""
    import numpy as np
    import torch
    import synth_inputs as si
    items = si.mixed_items(n_images)
    need = sorted({si.nearest_grid_rho(it.rho) for it in items})
    bases = si.base_fields(need, 4096, 6000)
    hosts = si.mixed_batch(items, bases)
    plans = [rk.rklt_make(8, rho) for rho in si.GRID_RHOS]
    pidx = {rho: k for k, rho in enumerate(si.GRID_RHOS)}
    bufs, entries = [], []
    for it, h in zip(items, hosts):
        d = torch.from_numpy(np.ascontiguousarray(h)).to(dev)
        rec = torch.empty_like(d)
        zc = torch.empty((it.h // 8) * (it.w // 8) * it.r, device=dev)
        bufs.append((d, rec, zc))
        entries.append((d, pidx[si.nearest_grid_rho(it.rho)], it.r, zc, rec))
    item_arr = rk.make_items(entries)
    sse_b = torch.empty(n_images, dtype=torch.float64, device=dev)
    ps_b = torch.empty(n_images, device=dev)
    batch = rk.rklt_batch_create(item_arr, plans, sse_b, ps_b, autotune=True)
    ms_batch = _time_ms(lambda: batch.run(stream), 5, stream)
    sse_p = torch.empty(n_images, dtype=torch.float64, device=dev)
    ps_p = torch.empty(n_images, device=dev)

    def plain():
        for k, (it, (d, rec, zc)) in enumerate(zip(items, bufs)):
            rk.rklt_fused(plans[entries[k][1]], d, it.r, sse_p[k:k + 1], ps_p[k:k + 1], zcoef=zc, recon=rec,
                          stream=stream)
    ms_plain = _time_ms(plain, 2, stream)
    a, b = sse_b.cpu().numpy(), sse_p.cpu().numpy()
    rel = float(np.max(np.abs(a - b) / np.maximum(b, 1e-30)))
    px = sum(it.h * it.w for it in items)
    info = batch.info()
    batch.close()
    # algorithmic bytes: per image 1 B read + 4 r / 64 B coefficients + 1 B reconstruction per pixel
    alg = sum(it.h * it.w * (2.0 + 4.0 * it.r / 64.0) for it in items)
    hbm, _ = peaks()
    gbs = alg / (ms_batch / 1e3) / 1e9
    return {"workload": f"{n_images} AR(1) crops, sides U{{64..4096/8}}, N=8, r~U{{1..64}}, nearest of 10 RKLTs",
            "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(gbs / hbm, 4), "traffic": None, "alg_bytes": alg},
            "gpixel": px / 1e9, "graph_batch_ms": ms_batch, "plain_launches_ms": ms_plain,
            "graph_batch_mpixel_per_s": px / (ms_batch / 1e3) / 1e6,
            "plain_mpixel_per_s": px / (ms_plain / 1e3) / 1e6, "speedup": ms_plain / ms_batch,
            "max_rel_sse_diff_vs_plain": rel, "autotuned": info}


def leg_serve(rk, dev, duration_s=60.0, rate=2000.0, stress_s=10.0):
    """Config 5: Poisson 2000 req/s for 60 s (about 120 000 requests); lognormal sides
    (median 768, sigma 0.5); rho in {0.5, 0.8, 0.9, 0.95}; r ~ U{1..64}; 8 GB budget.
    The library's native request loop, continuous batching against one request at
    a time (the latter run twice on the same trace); then a 4x stress rate."""
    import synth_inputs as si
    from paper_2111_14239_gb300 import serve
    rhos = (0.5, 0.8, 0.9, 0.95)
    bases = si.base_fields(rhos, 4096, 6100)
    pool = si.serving_pool(96, bases)
    srv = serve.Server(rhos, budget_bytes=8 << 30, streams=4)
    out = {"workload": f"Poisson arrivals, lognormal sides (median 768, sigma 0.5), N=8, "
                       f"rho in {{0.5,0.8,0.9,0.95}}, r~U{{1..64}}, 8 GB budget; nominal {rate:.0f} req/s "
                       f"for {duration_s:.0f} s and a 4x stress rate for {stress_s:.0f} s; native request loop",
           "latency": "arrival to results (reconstruction, coefficients, SSE, PSNR) in pinned host memory"}
    for tag, rr, dur, plain_runs in (("nominal", rate, duration_s, 2), ("stress_4x", 4 * rate, stress_s, 1)):
        cont = srv.run(serve.make_trace(rr, dur, pool, seed=5000, rhos=rhos))
        plains = [srv.run(serve.make_trace(rr, dur, pool, seed=5000, rhos=rhos), mode=serve.PLAIN)
                  for _ in range(plain_runs)]
        out[tag] = {"rate_req_per_s": rr, "continuous_batching": cont,
                    "plain_per_request": plains[0] if plain_runs == 1 else plains}
    srv.close()
    return out

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-budget", type=float, default=15.0, help="seconds of oracle work per sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--block-sizes", default="4,8,16,32", help="subset of N (profiling runs)")
    ap.add_argument("--no-extras", action="store_true", help="skip the single/sweep/batch/serving legs")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--min-timed-s", type=float, default=1.0,
                    help="lower bound on the device-timed region (passes per step scale to reach it)")
    ap.add_argument("--legs", default="", help="comma-separated subset of the extra legs (profiling runs)")
    ap.add_argument("--batch-images", type=int, default=2000,
                    help="images of the uneven-batch leg (fewer only for profiling runs)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
