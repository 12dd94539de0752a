"""Serving loop: compress + decompress + PSNR requests with continuous batching.

Requests (one uint8 image, a plan, r) arrive on a trace.  The server admits a
waiting request as soon as its device buffers (input, reconstruction, compact
coefficients) fit in the device-memory budget, copies it in, and launches every
admitted request of the current tick together with one `rklt_fused_items`
call.  Batches go round-robin onto several CUDA streams, so a batch admitted
while earlier ones are still on the GPU overlaps with them (copies and
kernels); results (PSNR, reconstruction, coefficients) are copied back into
pinned host memory and a request completes when its stream event has fired.
Plans are built once at start-up and travel with each launch as kernel
parameters, so no per-request table upload exists.

`serve_plain` is the reference point: one `rklt_fused` launch per request,
strictly one request at a time, each with its own copies and a synchronisation.
Both take the same trace and report p50/p99 latency (arrival to results on the
host) and throughput.
"""
from __future__ import annotations

import bisect
import contextlib
import gc
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import Plan, make_items, rklt_fused, rklt_fused_items, rklt_make


@contextlib.contextmanager
def frozen_heap():
    """Move every object alive on entry into the collector's permanent generation
    until exit.  A full collection during a request loop then scans only objects
    made inside the loop; scanning the whole heap (the trace, the image pool,
    torch's objects) stalls the loop for tens of milliseconds, which lands in
    the latency of every request waiting meanwhile.  A heap that was already
    partly frozen on entry stays frozen on exit (no partial unfreeze exists)."""
    was_frozen = gc.get_freeze_count() > 0
    gc.collect()
    gc.freeze()
    try:
        yield
    finally:
        if not was_frozen:
            gc.unfreeze()


def _align(x: int, a: int = 256) -> int:
    return (x + a - 1) // a * a


class Arena:
    """First-fit allocator over one preallocated buffer (offsets in bytes)."""

    def __init__(self, nbytes: int):
        self.size = nbytes
        self.free = [(0, nbytes)]   # sorted (offset, length)
        self.used = 0

    def alloc(self, n: int):
        n = _align(n)
        for k, (off, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(k)
                else:
                    self.free[k] = (off + n, ln - n)
                self.used += n
                return off
        return None

    def release(self, off: int, n: int):
        n = _align(n)
        self.used -= n
        k = bisect.bisect_left(self.free, (off, 0))
        self.free.insert(k, (off, n))
        # coalesce with neighbours
        if k + 1 < len(self.free) and self.free[k][0] + self.free[k][1] == self.free[k + 1][0]:
            self.free[k] = (self.free[k][0], self.free[k][1] + self.free[k + 1][1])
            self.free.pop(k + 1)
        if k > 0 and self.free[k - 1][0] + self.free[k - 1][1] == self.free[k][0]:
            self.free[k - 1] = (self.free[k - 1][0], self.free[k - 1][1] + self.free[k][1])
            self.free.pop(k)


@dataclass
class Request:
    rid: int
    arrival: float          # seconds from the start of the trace
    image: np.ndarray       # uint8 H x W (host)
    plan: int
    r: int
    # filled by the server
    done: float = -1.0
    psnr: float = float("nan")
    sse: float = float("nan")
    recon: np.ndarray | None = None
    coef: np.ndarray | None = None
    _slots: dict = field(default_factory=dict)


def bytes_needed(h: int, w: int, r: int, n: int = 8) -> tuple:
    """(input, reconstruction, coefficients) bytes of one request."""
    ld = _align(w, 16)
    return h * ld, h * ld, (h // n) * (w // n) * r * 4


class Server:
    def __init__(self, rhos, n: int = 8, budget_bytes: int = 8 << 30, streams: int = 3, device="cuda"):
        self.n = n
        self.plans: list = [rklt_make(n, rho) for rho in rhos]
        self.dev = torch.device(device)
        self.budget = budget_bytes
        self.d_arena = torch.empty(budget_bytes, dtype=torch.uint8, device=self.dev)
        self.h_arena = torch.empty(budget_bytes, dtype=torch.uint8).pin_memory()
        self.alloc = Arena(budget_bytes)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(streams)]
        self.next_stream = 0
        self.rejected = 0
        # pinned result slots (per batch: PSNR and SSE of up to max_batch requests)
        self.nslots = 64
        self.max_batch = 256
        self.ps_slots = torch.empty((self.nslots, self.max_batch), dtype=torch.float32).pin_memory()
        self.sse_slots = torch.empty((self.nslots, self.max_batch), dtype=torch.float64).pin_memory()
        self.d_ps = torch.empty((self.nslots, self.max_batch), dtype=torch.float32, device=self.dev)
        self.d_sse = torch.empty((self.nslots, self.max_batch), dtype=torch.float64, device=self.dev)
        self.free_slots = list(range(self.nslots))
        self.warm_up()

    def warm_up(self):
        """Load every kernel variant once (r = 1..N*N) so that no request pays for
        module loading."""
        img = torch.zeros((self.n * 4, 256), dtype=torch.uint8, device=self.dev)
        rec = torch.empty_like(img)
        rs = list(range(0, self.n * self.n + 1))
        zc = [torch.empty((self.n * 4 // self.n) * (256 // self.n) * max(r, 1), device=self.dev) for r in rs]
        entries = [(img, 0, r, zc[k], rec) for k, r in enumerate(rs)]
        for lo in range(0, len(entries), 16):
            chunk = entries[lo:lo + 16]
            rklt_fused_items(make_items(chunk), self.plans, self.d_sse[0, :len(chunk)], self.d_ps[0, :len(chunk)])
        torch.cuda.synchronize(self.dev)

    # ---- buffers --------------------------------------------------------------
    def _views(self, req: Request, base: int):
        """Device and pinned-host views of a request's buffers.  Images use a 16-byte
        row pitch; the host<->device copies move whole padded rows, so every copy is
        one contiguous transfer from pinned memory (a strided view would make the
        copy go through a pageable temporary and block the loop)."""
        h, w = req.image.shape
        ld = _align(w, 16)
        bi, br, bc = bytes_needed(h, w, req.r, self.n)
        oi, orc, oc = base, base + _align(bi), base + _align(bi) + _align(br)
        d_in = self.d_arena[oi:oi + bi].view(h, ld)
        d_rec = self.d_arena[orc:orc + br].view(h, ld)
        d_coef = self.d_arena[oc:oc + bc].view(torch.float32) if bc else None
        h_in = self.h_arena[oi:oi + bi].view(h, ld)
        h_rec = self.h_arena[orc:orc + br].view(h, ld)
        h_coef = self.h_arena[oc:oc + bc].view(torch.float32) if bc else None
        return d_in, d_rec, d_coef, h_in, h_rec, h_coef

    def _total(self, req: Request) -> int:
        h, w = req.image.shape
        bi, br, bc = bytes_needed(h, w, req.r, self.n)
        return _align(bi) + _align(br) + _align(bc)

    # ---- continuous batching --------------------------------------------------
    def run(self, trace: list, keep_outputs: bool = False, max_batch: int = 256) -> dict:
        """Replay `trace` (list of Request, sorted by arrival) in real time."""
        with frozen_heap():
            return self._run(trace, keep_outputs, max_batch)

    def _run(self, trace: list, keep_outputs: bool, max_batch: int) -> dict:
        max_batch = min(max_batch, self.max_batch)
        pending = list(trace)
        waiting: list = []
        inflight: list = []          # (event, [requests], psnr_host, sse_host)
        t0 = time.perf_counter()
        k = 0
        completed = 0
        while completed < len(trace):
            now = time.perf_counter() - t0
            while k < len(pending) and pending[k].arrival <= now:
                waiting.append(pending[k])
                k += 1
            # admission by budget (FIFO; a request larger than the whole budget is rejected)
            batch = []
            while waiting and len(batch) < max_batch and self.free_slots:
                req = waiting[0]
                need = self._total(req)
                if need > self.budget:
                    waiting.pop(0)
                    req.done = now
                    self.rejected += 1
                    completed += 1
                    continue
                off = self.alloc.alloc(need)
                if off is None:
                    break
                waiting.pop(0)
                req._slots = {"off": off, "need": need, "views": self._views(req, off)}
                batch.append(req)
            if batch:
                s = self.streams[self.next_stream]
                self.next_stream = (self.next_stream + 1) % len(self.streams)
                nb = len(batch)
                slot = self.free_slots.pop()
                sse, ps = self.d_sse[slot, :nb], self.d_ps[slot, :nb]
                entries = []
                with torch.cuda.stream(s):
                    for req in batch:
                        d_in, d_rec, d_coef, h_in, h_rec, h_coef = req._slots["views"]
                        w = req.image.shape[1]
                        h_in[:, :w].copy_(torch.from_numpy(req.image))
                        d_in.copy_(h_in, non_blocking=True)          # whole padded rows: contiguous
                        entries.append((d_in[:, :w], req.plan, req.r, d_coef, d_rec[:, :w]))
                    rklt_fused_items(make_items(entries), self.plans, sse, ps, stream=s)
                    for req in batch:
                        d_in, d_rec, d_coef, h_in, h_rec, h_coef = req._slots["views"]
                        h_rec.copy_(d_rec, non_blocking=True)
                        if d_coef is not None:
                            h_coef.copy_(d_coef, non_blocking=True)
                    ps_h = self.ps_slots[slot, :nb]
                    sse_h = self.sse_slots[slot, :nb]
                    ps_h.copy_(ps, non_blocking=True)
                    sse_h.copy_(sse, non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(s)
                inflight.append((ev, batch, ps_h, sse_h, sse, ps, slot))
            # completions
            still = []
            for item in inflight:
                ev, reqs, ps_h, sse_h = item[0], item[1], item[2], item[3]
                if ev.query():
                    tdone = time.perf_counter() - t0
                    for j, req in enumerate(reqs):
                        req.done = tdone
                        req.psnr = float(ps_h[j])
                        req.sse = float(sse_h[j])
                        if keep_outputs:
                            _, _, _, h_in, h_rec, h_coef = req._slots["views"]
                            req.recon = h_rec[:, :req.image.shape[1]].numpy().copy()
                            req.coef = h_coef.numpy().copy() if h_coef is not None else np.zeros(0, np.float32)
                        self.alloc.release(req._slots["off"], req._slots["need"])
                        req._slots = {}
                        completed += 1
                    self.free_slots.append(item[6])
                else:
                    still.append(item)
            inflight = still
            if not batch and not inflight:
                # idle: sleep until just before the next arrival
                if k < len(pending):
                    gap = pending[k].arrival - (time.perf_counter() - t0)
                    if gap > 0.0003:
                        time.sleep(gap - 0.0002)
        wall = time.perf_counter() - t0
        return summarize(trace, wall, self.rejected)


def serve_plain(plans: list, trace: list, device="cuda", keep_outputs: bool = False) -> dict:
    """One request at a time: copy in, one rklt_fused launch, copy out, synchronise.
    Staging and device buffers are preallocated for the largest request."""
    with frozen_heap():
        return _serve_plain(plans, trace, device, keep_outputs)


def _serve_plain(plans: list, trace: list, device, keep_outputs: bool) -> dict:
    dev = torch.device(device)
    s = torch.cuda.Stream(dev)
    n = plans[0].N
    wh, ww = 4 * n, 256                      # warm-up image
    wblk = (wh // n) * (ww // n)
    max_px = max(max(r.image.size for r in trace), wh * ww)
    max_coef = max(max((r.image.shape[0] // n) * (r.image.shape[1] // n) * max(r.r, 1) for r in trace),
                   wblk * n * n)
    h_in = torch.empty(max_px, dtype=torch.uint8).pin_memory()
    h_rec = torch.empty(max_px, dtype=torch.uint8).pin_memory()
    h_coef = torch.empty(max_coef, dtype=torch.float32).pin_memory()
    h_res = torch.empty(2, dtype=torch.float64).pin_memory()
    d_in = torch.empty(max_px, dtype=torch.uint8, device=dev)
    d_rec = torch.empty(max_px, dtype=torch.uint8, device=dev)
    d_coef = torch.empty(max_coef, dtype=torch.float32, device=dev)
    sse = torch.empty(1, dtype=torch.float64, device=dev)
    ps = torch.empty(1, dtype=torch.float32, device=dev)
    for r in range(0, n * n + 1):   # load every kernel variant before the trace starts
        rklt_fused(plans[0], d_in[:wh * ww].view(wh, ww), r, sse, ps, zcoef=d_coef[:max(wblk * r, 1)],
                   recon=d_rec[:wh * ww].view(wh, ww), stream=s)
    s.synchronize()
    t0 = time.perf_counter()
    for req in trace:
        now = time.perf_counter() - t0
        if req.arrival > now:
            time.sleep(req.arrival - now)
        h, w = req.image.shape
        npx, nc = h * w, (h // n) * (w // n) * req.r
        h_in[:npx].view(h, w).copy_(torch.from_numpy(req.image))
        with torch.cuda.stream(s):
            d_in[:npx].copy_(h_in[:npx], non_blocking=True)
            rklt_fused(plans[req.plan], d_in[:npx].view(h, w), req.r, sse, ps, zcoef=d_coef[:max(nc, 1)],
                       recon=d_rec[:npx].view(h, w), stream=s)
            h_rec[:npx].copy_(d_rec[:npx], non_blocking=True)
            if nc:
                h_coef[:nc].copy_(d_coef[:nc], non_blocking=True)
            h_res[0:1].copy_(sse, non_blocking=True)
            h_res[1:2].copy_(ps.double(), non_blocking=True)
        s.synchronize()
        req.done = time.perf_counter() - t0
        req.sse, req.psnr = float(h_res[0]), float(h_res[1])
        if keep_outputs:
            req.recon = h_rec[:npx].view(h, w).numpy().copy()
            req.coef = h_coef[:nc].numpy().copy()
    wall = time.perf_counter() - t0
    return summarize(trace, wall, 0)


def summarize(trace: list, wall: float, rejected: int) -> dict:
    lat = np.array([r.done - r.arrival for r in trace if r.done >= 0]) * 1e3
    px = sum(r.image.size for r in trace)
    return {"requests": len(trace), "rejected": rejected, "wall_s": wall,
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "mean_ms": float(lat.mean()) if lat.size else None,
            "mpixel_per_s": px / wall / 1e6, "offered_mpixel": px / 1e6}


def make_trace(rate_hz: float, duration_s: float, pool: list, seed: int = 5000, rhos=(0.5, 0.8, 0.9, 0.95),
               r_max: int = 64) -> list:
    """Poisson arrivals; each request takes an image from `pool` (list of uint8 arrays,
    e.g. lognormal-size AR(1) images), a plan index into `rhos` and r ~ U{1..r_max}."""
    g = np.random.Generator(np.random.PCG64(seed))
    t, out, i = 0.0, [], 0
    while True:
        t += g.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        img = pool[int(g.integers(0, len(pool)))]
        out.append(Request(i, t, img, int(g.integers(0, len(rhos))), int(g.integers(1, r_max + 1))))
        i += 1
    return out
