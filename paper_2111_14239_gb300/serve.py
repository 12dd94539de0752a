"""Serving: compress + decompress + PSNR requests through the library's request loop.

The loop itself is native (rklt_server_run in the C ABI): it replays a trace of
timed arrivals in real time, admits requests against a device-memory budget and
either batches them continuously (every request admitted in one pass of the loop
goes out in one rklt_fused_items launch on the next of several streams, so batches
overlap on the device) or serves them one at a time (copy in, rklt_fused, copy
out, synchronise).  This module builds traces, hands them to the loop and
summarises latencies; it does no per-request work of its own.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import NativeServer, RklTRequest, rklt_make

CONTINUOUS, PLAIN = 0, 1


def _align(x: int, a: int = 256) -> int:
    return (x + a - 1) // a * a


def bytes_needed(h: int, w: int, r: int, n: int = 8) -> tuple:
    """(input, reconstruction, coefficients) bytes of one request in the server's
    arena (rows padded to 16 bytes)."""
    ld = _align(w, 16)
    return h * ld, h * ld, (h // n) * (w // n) * r * 4


@dataclass
class Request:
    rid: int
    arrival: float          # seconds from the start of the trace
    image: np.ndarray       # uint8 H x W (host, C-contiguous)
    plan: int
    r: int
    # filled by a run
    admit: float = -1.0
    done: float = -1.0
    psnr: float = float("nan")
    sse: float = float("nan")
    status: int = -1
    recon: np.ndarray | None = None
    coef: np.ndarray | None = None


class Server:
    """Plans for `rhos` (block size n) and a native request loop over a budget."""

    def __init__(self, rhos, n: int = 8, budget_bytes: int = 8 << 30, streams: int = 4, max_batch: int = 256):
        self.n = n
        self.plans: list = [rklt_make(n, rho) for rho in rhos]
        self.native = NativeServer(self.plans, budget_bytes, streams, max_batch)

    def run(self, trace: list, keep_outputs: bool = False, mode: int = CONTINUOUS) -> dict:
        """Replay `trace` (list of Request sorted by arrival) in real time."""
        n = len(trace)
        reqs = (RklTRequest * max(n, 1))()
        for k, q in enumerate(trace):
            assert q.image.dtype == np.uint8 and q.image.flags.c_contiguous
            h, w = q.image.shape
            reqs[k].arrival_s, reqs[k].h_img = q.arrival, q.image.ctypes.data
            reqs[k].H, reqs[k].W, reqs[k].plan, reqs[k].r = h, w, q.plan, q.r
        recon = coef = None
        if keep_outputs:
            recon = [np.empty(q.image.shape, np.uint8) for q in trace]
            coef = [np.empty((q.image.shape[0] // self.n) * (q.image.shape[1] // self.n) * q.r, np.float32)
                    for q in trace]
        res, wall = self.native.run(reqs, mode, recon, coef)
        rejected = 0
        for k, q in enumerate(trace):
            q.done, q.admit, q.sse, q.psnr, q.status = (res[k].done_s, res[k].admit_s, res[k].sse, res[k].psnr,
                                                        res[k].status)
            if q.status != 0:
                rejected += 1
                q.sse = q.psnr = float("nan")
            if keep_outputs:
                q.recon, q.coef = recon[k], coef[k]
        return summarize(trace, wall, rejected)

    def close(self):
        self.native.close()


def summarize(trace: list, wall: float, rejected: int) -> dict:
    lat = np.array([r.done - r.arrival for r in trace if r.done >= 0]) * 1e3
    queued = np.array([r.admit - r.arrival for r in trace if r.admit >= 0]) * 1e3
    px = sum(r.image.size for r in trace)
    return {"requests": len(trace), "rejected": rejected, "wall_s": wall,
            "p50_ms": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_ms": float(np.percentile(lat, 99)) if lat.size else None,
            "p99_until_launch_ms": float(np.percentile(queued, 99)) if queued.size else None,
            "max_ms": float(lat.max()) if lat.size else None,
            "mean_ms": float(lat.mean()) if lat.size else None,
            "mpixel_per_s": px / wall / 1e6 if wall > 0 else None, "offered_mpixel": px / 1e6}


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
        img = np.ascontiguousarray(pool[int(g.integers(0, len(pool)))])
        out.append(Request(i, t, img, int(g.integers(0, len(rhos))), int(g.integers(1, r_max + 1))))
        i += 1
    return out
