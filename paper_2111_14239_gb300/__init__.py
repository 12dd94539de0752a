"""Python binding of the GB300 rounded-KLT library (librklt.so, C ABI in include/rklt.h).

Argument marshalling only: every step of the transform runs in the library's CUDA
kernels.  PyTorch supplies device memory and streams.  There is no CPU fallback:
if the library cannot be built or loaded, importing this package raises.

Names follow the C ABI: rklt_make, rklt_forward, rklt_zonal, rklt_inverse,
rklt_psnr, rklt_fused, rklt_fused_batched, ...  Functions take torch tensors
(device tensors for d_* arguments) and an optional torch.cuda.Stream (default:
the current stream).
"""
from __future__ import annotations

import ctypes
import os
import re

from . import _build

__all__ = [
    "RklTError", "Plan", "lib", "header_symbols", "rklt_make", "rklt_make_alpha", "rklt_make_from_matrix",
    "rklt_make_klt", "rklt_make_dct", "rklt_design_sweep", "rklt_figures", "rklt_plan_info", "rklt_forward_int", "rklt_forward", "rklt_zonal", "rklt_inverse", "rklt_psnr",
    "rklt_fused", "rklt_fused_batched", "rklt_fused_quant", "rklt_mssim", "rklt_fused_mssim", "rklt_fused_noalloc", "rklt_device_status", "RklTItem", "make_items",
    "rklt_fused_items", "Batch", "rklt_batch_create", "rklt_rsweep", "rklt_set_wait_timeout_us",
    "rklt_set_transport", "rklt_set_tensor_engine", "rklt_debug_inject_stall", "rklt_version", "default_alpha", "nblocks",
    "RklTRequest", "RklTResult", "NativeServer", "rklt_server_create",
]

STATUS = {0: "RKLT_OK", 1: "RKLT_ERR_ARG", 2: "RKLT_ERR_SHAPE", 3: "RKLT_ERR_DEGENERATE", 4: "RKLT_ERR_CUDA",
          5: "RKLT_ERR_OOM", 6: "RKLT_ERR_BUDGET", 7: "RKLT_ERR_TIMEOUT", 8: "RKLT_ERR_UNSUPPORTED"}

_HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(_HERE), "include", "rklt.h")


class RklTItem(ctypes.Structure):
    """rklt_item of include/rklt.h."""
    _fields_ = [("d_img", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int), ("ld", ctypes.c_int64),
                ("plan", ctypes.c_int), ("r", ctypes.c_int), ("d_zcoef", ctypes.c_void_p),
                ("d_recon", ctypes.c_void_p), ("ld_recon", ctypes.c_int64)]


class RklTRequest(ctypes.Structure):
    """rklt_request of include/rklt.h."""
    _fields_ = [("arrival_s", ctypes.c_double), ("h_img", ctypes.c_void_p), ("H", ctypes.c_int),
                ("W", ctypes.c_int), ("plan", ctypes.c_int), ("r", ctypes.c_int)]


class RklTResult(ctypes.Structure):
    """rklt_result of include/rklt.h."""
    _fields_ = [("done_s", ctypes.c_double), ("admit_s", ctypes.c_double), ("sse", ctypes.c_double),
                ("psnr", ctypes.c_float), ("status", ctypes.c_int)]


class RklTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _load() -> ctypes.CDLL:
    path = _build.build()
    return ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)


lib = _load()

_P, _I, _D, _L, _U32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_uint32
_SIGS = {
    "rklt_last_error": (ctypes.c_char_p, []),
    "rklt_status_string": (ctypes.c_char_p, [_I]),
    "rklt_version": (_I, []),
    "rklt_make": (_I, [_I, _D, ctypes.POINTER(_P)]),
    "rklt_make_alpha": (_I, [_I, _D, _D, ctypes.POINTER(_P)]),
    "rklt_make_from_matrix": (_I, [_I, _P, ctypes.POINTER(_P)]),
    "rklt_make_klt": (_I, [_I, _D, ctypes.POINTER(_P)]),
    "rklt_make_dct": (_I, [_I, ctypes.POINTER(_P)]),
    "rklt_plan_kind": (_I, [_P]),
    "rklt_plan_matrix": (_I, [_P, _P]),
    "rklt_design_sweep": (_I, [_I, _D, _D, _I, _P, _P, _P, ctypes.POINTER(_I)]),
    "rklt_figures": (_I, [_P, _D, _P, _P, _P, _P]),
    "rklt_destroy": (None, [_P]),
    "rklt_plan_info": (_I, [_P, _P, _P, _P, _P, _P, _P]),
    "rklt_forward_int": (_I, [_P, _P, _I, _I, _L, _P, _P]),
    "rklt_forward": (_I, [_P, _P, _I, _I, _L, _P, _P]),
    "rklt_zonal": (_I, [_P, _P, _L, _I, _P, _P]),
    "rklt_inverse": (_I, [_P, _P, _I, _I, _I, _P, _L, _P]),
    "rklt_psnr": (_I, [_P, _L, _P, _L, _I, _I, _P, _P, _P]),
    "rklt_fused": (_I, [_P, _P, _I, _I, _L, _I, _P, _P, _L, _P, _P, _P]),
    "rklt_fused_batched": (_I, [_P, _P, _I, _I, _I, _L, _L, _I, _P, _P, _L, _L, _P, _P, _P]),
    "rklt_fused_quant": (_I, [_P, _P, _I, _I, _I, _L, _L, _I, _P, _P, _P, _L, _L, _P, _P, _P]),
    "rklt_mssim": (_I, [_P, _P, _I, _I, _I, _L, _L, _L, _L, _P, _P]),
    "rklt_fused_mssim": (_I, [_P, _P, _I, _I, _I, _L, _L, _I, _P, _P, _L, _L, _P, _P, _P, _P]),
    "rklt_fused_noalloc": (_I, [_P, _P, _I, _I, _L, _I, _P, _P, _L, _P, _P, _P]),
    "rklt_device_status": (_I, []),
    "rklt_fused_items": (_I, [_P, _I, _P, _I, _P, _P, _P]),
    "rklt_batch_create": (_I, [_P, _I, _P, _I, _P, _P, _I, ctypes.POINTER(_P)]),
    "rklt_batch_run": (_I, [_P, _P]),
    "rklt_batch_info": (_I, [_P, _P, _P, _P, _P, _P]),
    "rklt_batch_candidates": (_I, [_P, _P, _P, _P, _P, _I, _P]),
    "rklt_batch_destroy": (None, [_P]),
    "rklt_rsweep": (_I, [_P, _I, _P, _I, _I, _I, _L, _L, _P, _P, _P]),
    "rklt_server_create": (_I, [_P, _I, ctypes.c_size_t, _I, _I, ctypes.POINTER(_P)]),
    "rklt_server_run": (_I, [_P, _P, _I, _I, _P, _P, _P, ctypes.POINTER(_D)]),
    "rklt_server_destroy": (None, [_P]),
    "rklt_arena_selftest": (_I, [ctypes.c_uint, _I]),
    "rklt_copypool_selftest": (_I, [ctypes.c_uint, _I]),
    "rklt_set_wait_timeout_us": (None, [_U32]),
    "rklt_set_transport": (None, [_I]),
    "rklt_set_tensor_engine": (None, [_I]),
    "rklt_debug_inject_stall": (None, [_I]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def header_symbols() -> list:
    """Function names declared in include/rklt.h."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rklt_[a-z0-9_]+)\s*\(", text)))


def _check(status: int):
    if status != 0:
        raise RklTError(status, lib.rklt_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def default_alpha(n: int) -> float:
    return 2.0 * (n / 8.0) ** 0.5


def nblocks(n: int, h: int, w: int) -> int:
    return (h // n) * (w // n)


class Plan:
    """Owns an rklt_plan handle (host tables; the library frees it on close)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)
        n = ctypes.c_int()
        a = ctypes.c_double()
        rho = ctypes.c_double()
        o = ctypes.c_int()
        _check(lib.rklt_plan_info(self._h, None, None, ctypes.byref(o), ctypes.byref(n), ctypes.byref(a),
                                  ctypes.byref(rho)))
        self.N, self.alpha, self.rho, self.orthogonal = n.value, a.value, rho.value, bool(o.value)
        self.kind = lib.rklt_plan_kind(self._h)   # 0 rounded KLT, 1 exact KLT, 2 DCT-II

    @property
    def handle(self):
        return self._h

    def info(self):
        """(T int8 numpy [N,N], s float64 numpy [N], orthogonal)."""
        import numpy as np
        T = np.zeros((self.N, self.N), np.int8)
        s = np.zeros(self.N, np.float64)
        o = ctypes.c_int()
        _check(lib.rklt_plan_info(self._h, T.ctypes.data, s.ctypes.data, ctypes.byref(o), None, None, None))
        return T, s, bool(o.value)

    def matrix(self):
        """The analysis matrix (float64 [N,N]): T-hat = S T, or the exact KLT / DCT."""
        import numpy as np
        M = np.zeros((self.N, self.N), np.float64)
        _check(lib.rklt_plan_matrix(self._h, M.ctypes.data))
        return M

    def close(self):
        if self._h and self._h.value:
            lib.rklt_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rklt_make(n: int, rho: float) -> Plan:
    h = ctypes.c_void_p()
    _check(lib.rklt_make(n, rho, ctypes.byref(h)))
    return Plan(h.value)


def rklt_make_alpha(n: int, rho: float, alpha: float) -> Plan:
    h = ctypes.c_void_p()
    _check(lib.rklt_make_alpha(n, rho, alpha, ctypes.byref(h)))
    return Plan(h.value)


def rklt_make_from_matrix(n: int, T) -> Plan:
    import numpy as np
    T = np.ascontiguousarray(T, dtype=np.int8)
    h = ctypes.c_void_p()
    _check(lib.rklt_make_from_matrix(n, T.ctypes.data, ctypes.byref(h)))
    return Plan(h.value)


def rklt_make_klt(n: int, rho: float) -> Plan:
    """The exact KLT of the Markov-1 model as a plan (FP32 kernels, S = I)."""
    h = ctypes.c_void_p()
    _check(lib.rklt_make_klt(n, rho, ctypes.byref(h)))
    return Plan(h.value)


def rklt_make_dct(n: int) -> Plan:
    """The orthonormal DCT-II as a plan (FP32 kernels, S = I)."""
    h = ctypes.c_void_p()
    _check(lib.rklt_make_dct(n, ctypes.byref(h)))
    return Plan(h.value)


def rklt_design_sweep(n: int, alpha: float, step: float, max_out: int = 64):
    """Algorithm 1 (Sec. 3): list of (T int8 [N,N], rho_first, rho_last)."""
    import numpy as np
    T = np.zeros((max_out, n, n), np.int8)
    lo = np.zeros(max_out)
    hi = np.zeros(max_out)
    cnt = ctypes.c_int()
    _check(lib.rklt_design_sweep(n, alpha, step, max_out, T.ctypes.data, lo.ctypes.data, hi.ctypes.data,
                                 ctypes.byref(cnt)))
    return [(T[k].copy(), float(lo[k]), float(hi[k])) for k in range(cnt.value)]


def rklt_figures(plan: Plan, rho: float) -> dict:
    """Figures of merit of the plan's matrix for the Markov-1 model (Sec. 3.1)."""
    v = [ctypes.c_double() for _ in range(4)]
    _check(lib.rklt_figures(plan.handle, rho, *[ctypes.byref(x) for x in v]))
    return dict(cg=v[0].value, eta=v[1].value, mse=v[2].value, eps=v[3].value)


def rklt_plan_info(plan: Plan):
    return plan.info()


def _img_args(img):
    """(ptr, H, W, ld) of a 2-D uint8 tensor with unit column stride."""
    assert img.dim() == 2 and img.stride(1) == 1, "image must be 2-D with contiguous rows"
    return img.data_ptr(), img.shape[0], img.shape[1], img.stride(0)


def rklt_forward_int(plan: Plan, img, C, stream=None):
    p, H, W, ld = _img_args(img)
    _check(lib.rklt_forward_int(plan.handle, p, H, W, ld, _ptr(C), _stream(stream)))


def rklt_forward(plan: Plan, img, coef, stream=None):
    p, H, W, ld = _img_args(img)
    _check(lib.rklt_forward(plan.handle, p, H, W, ld, _ptr(coef), _stream(stream)))


def rklt_zonal(plan: Plan, coef, nblk: int, r: int, out, stream=None):
    _check(lib.rklt_zonal(plan.handle, _ptr(coef), nblk, r, _ptr(out), _stream(stream)))


def rklt_inverse(plan: Plan, zcoef, r: int, H: int, W: int, recon, stream=None):
    ld = recon.stride(0) if recon is not None and hasattr(recon, "stride") else W
    _check(lib.rklt_inverse(plan.handle, _ptr(zcoef), r, H, W, _ptr(recon), ld, _stream(stream)))


def rklt_psnr(img, recon, sse, psnr, stream=None):
    p, H, W, ld = _img_args(img)
    _check(lib.rklt_psnr(p, ld, _ptr(recon), recon.stride(0), H, W, _ptr(sse), _ptr(psnr), _stream(stream)))


def rklt_fused(plan: Plan, img, r: int, sse, psnr, zcoef=None, recon=None, stream=None):
    p, H, W, ld = _img_args(img)
    ldr = recon.stride(0) if recon is not None else 0
    _check(lib.rklt_fused(plan.handle, p, H, W, ld, r, _ptr(zcoef), _ptr(recon), ldr, _ptr(sse), _ptr(psnr),
                          _stream(stream)))


def rklt_fused_noalloc(plan: Plan, img, r: int, sse, psnr, zcoef=None, recon=None, stream=None):
    """rklt_fused without any allocation (scratch in the library's fixed device array)."""
    p, H, W, ld = _img_args(img)
    ldr = recon.stride(0) if recon is not None else 0
    _check(lib.rklt_fused_noalloc(plan.handle, p, H, W, ld, r, _ptr(zcoef), _ptr(recon), ldr, _ptr(sse),
                                  _ptr(psnr), _stream(stream)))


def rklt_fused_batched(plan: Plan, imgs, r: int, sse, psnr, zcoef=None, recon=None, stream=None):
    """imgs: uint8 tensor [nimg, H, W] (rows contiguous); recon likewise or None."""
    assert imgs.dim() == 3 and imgs.stride(2) == 1
    nimg, H, W = imgs.shape
    ld, istr = imgs.stride(1), imgs.stride(0)
    if recon is not None:
        ldr, rstr = recon.stride(1), recon.stride(0)
    else:
        ldr, rstr = 0, 0
    _check(lib.rklt_fused_batched(plan.handle, imgs.data_ptr(), nimg, H, W, ld, istr, r, _ptr(zcoef), _ptr(recon),
                                  ldr, rstr, _ptr(sse), _ptr(psnr), _stream(stream)))


def rklt_fused_quant(plan: Plan, imgs, r: int, Q, sse, psnr, qcoef=None, recon=None, stream=None):
    """JPEG-like quantisation with S absorbed (Appendix).  imgs: uint8 [H, W] or [nimg, H, W];
    Q: N x N positive values (host); qcoef: int32 [nimg * nblk * r] or None; recon like imgs or None."""
    import numpy as np
    if imgs.dim() == 2:
        imgs = imgs.unsqueeze(0)
        recon = recon.unsqueeze(0) if recon is not None else None
    assert imgs.dim() == 3 and imgs.stride(2) == 1
    nimg, H, W = imgs.shape
    Qh = np.ascontiguousarray(np.asarray(Q, dtype=np.float64).reshape(-1))
    ldr, rstr = (recon.stride(1), recon.stride(0)) if recon is not None else (0, 0)
    _check(lib.rklt_fused_quant(plan.handle, imgs.data_ptr(), nimg, H, W, imgs.stride(1), imgs.stride(0), r,
                                Qh.ctypes.data, _ptr(qcoef), _ptr(recon), ldr, rstr, _ptr(sse), _ptr(psnr),
                                _stream(stream)))


def rklt_fused_mssim(plan: Plan, imgs, r: int, sse, psnr, mssim, zcoef=None, recon=None, stream=None):
    """rklt_fused_batched plus the MSSIM of each image against its reconstruction, in
    one pass.  imgs: uint8 [H, W] or [nimg, H, W]; mssim: float64 [nimg]."""
    if imgs.dim() == 2:
        imgs = imgs.unsqueeze(0)
        recon = recon.unsqueeze(0) if recon is not None else None
    assert imgs.dim() == 3 and imgs.stride(2) == 1
    nimg, H, W = imgs.shape
    ldr, rstr = (recon.stride(1), recon.stride(0)) if recon is not None else (0, 0)
    _check(lib.rklt_fused_mssim(plan.handle, imgs.data_ptr(), nimg, H, W, imgs.stride(1), imgs.stride(0), r,
                                _ptr(zcoef), _ptr(recon), ldr, rstr, _ptr(sse), _ptr(psnr), _ptr(mssim),
                                _stream(stream)))


def rklt_mssim(x, y, out, stream=None):
    """Mean SSIM (Sec. 4.1) of uint8 images x, y: [H, W] or [nimg, H, W]; out: float64 [nimg]."""
    if x.dim() == 2:
        x, y = x.unsqueeze(0), y.unsqueeze(0)
    assert x.shape == y.shape and x.stride(2) == 1 and y.stride(2) == 1
    nimg, H, W = x.shape
    _check(lib.rklt_mssim(x.data_ptr(), y.data_ptr(), nimg, H, W, x.stride(1), x.stride(0), y.stride(1),
                          y.stride(0), _ptr(out), _stream(stream)))


def make_items(entries):
    """entries: iterable of (img 2-D uint8 tensor, plan_index, r, zcoef tensor|None, recon tensor|None)."""
    entries = list(entries)
    arr = (RklTItem * len(entries))()
    for k, (img, plan, r, zc, rec) in enumerate(entries):
        assert img.dim() == 2 and img.stride(1) == 1
        arr[k].d_img = img.data_ptr()
        arr[k].H, arr[k].W = img.shape
        arr[k].ld = img.stride(0)
        arr[k].plan = plan
        arr[k].r = r
        arr[k].d_zcoef = zc.data_ptr() if zc is not None else None
        arr[k].d_recon = rec.data_ptr() if rec is not None else None
        arr[k].ld_recon = rec.stride(0) if rec is not None else 0
    return arr


def _plan_array(plans):
    arr = (ctypes.c_void_p * len(plans))()
    for k, p in enumerate(plans):
        arr[k] = p.handle.value
    return arr


def rklt_fused_items(items, plans, sse, psnr, stream=None):
    """items: make_items(...) array; plans: list of Plan."""
    _check(lib.rklt_fused_items(ctypes.cast(items, ctypes.c_void_p), len(items),
                                ctypes.cast(_plan_array(plans), ctypes.c_void_p), len(plans),
                                _ptr(sse), _ptr(psnr), _stream(stream)))


class Batch:
    """rklt_batch: a graph-captured, autotuned batch over fixed device buffers."""

    def __init__(self, items, plans, sse, psnr, autotune=True):
        self._plans = list(plans)   # keep plans alive for the batch's lifetime
        self._items = items
        h = ctypes.c_void_p()
        _check(lib.rklt_batch_create(ctypes.cast(items, ctypes.c_void_p), len(items),
                                     ctypes.cast(_plan_array(self._plans), ctypes.c_void_p), len(self._plans),
                                     _ptr(sse), _ptr(psnr), 1 if autotune else 0, ctypes.byref(h)))
        self._h = h

    def run(self, stream=None):
        _check(lib.rklt_batch_run(self._h, _stream(stream)))

    def info(self):
        t, c, g, us, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
        _check(lib.rklt_batch_info(self._h, ctypes.byref(t), ctypes.byref(c), ctypes.byref(g), ctypes.byref(us),
                                   ctypes.byref(m)))
        n = ctypes.c_int()
        md, th, cs, ts = (ctypes.c_int * 16)(), (ctypes.c_int * 16)(), (ctypes.c_int * 16)(), (ctypes.c_double * 16)()
        _check(lib.rklt_batch_candidates(self._h, md, th, cs, ts, 16, ctypes.byref(n)))
        cands = [{"mode": "queue" if md[k] else "grouped", "threads": th[k], "ctas_per_sm": cs[k],
                  "us": round(ts[k], 1)} for k in range(min(n.value, 16))]
        return {"mode": "one queue launch" if m.value else "grouped launches", "threads": t.value,
                "ctas_per_sm": c.value, "groups": g.value, "tuned_us": us.value, "candidates": cands}

    def matrix(self):
        """The analysis matrix (float64 [N,N]): T-hat = S T, or the exact KLT / DCT."""
        import numpy as np
        M = np.zeros((self.N, self.N), np.float64)
        _check(lib.rklt_plan_matrix(self._h, M.ctypes.data))
        return M

    def close(self):
        if self._h and self._h.value:
            lib.rklt_batch_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rklt_batch_create(items, plans, sse, psnr, autotune=True) -> Batch:
    return Batch(items, plans, sse, psnr, autotune)


def rklt_rsweep(plans, imgs, sse, psnr, stream=None):
    """imgs: uint8 tensor [nimg, H, W]; psnr (and sse, or None): [nimg, nplans, N*N]."""
    assert imgs.dim() == 3 and imgs.stride(2) == 1
    nimg, H, W = imgs.shape
    _check(lib.rklt_rsweep(ctypes.cast(_plan_array(plans), ctypes.c_void_p), len(plans), imgs.data_ptr(), nimg, H, W,
                           imgs.stride(1), imgs.stride(0), _ptr(sse), _ptr(psnr), _stream(stream)))


def rklt_device_status():
    _check(lib.rklt_device_status())


def rklt_set_wait_timeout_us(us: int):
    lib.rklt_set_wait_timeout_us(us)


def rklt_set_transport(mode: int):
    lib.rklt_set_transport(mode)


def rklt_set_tensor_engine(mode: int):
    """N = 32 with r <= 136: 0 warp-level mma.sync (default), 1 tcgen05 with TMEM accumulators."""
    lib.rklt_set_tensor_engine(mode)


def rklt_debug_inject_stall(on: bool):
    lib.rklt_debug_inject_stall(1 if on else 0)


def rklt_version() -> int:
    return lib.rklt_version()


class NativeServer:
    """rklt_server: the library's request loop (continuous batching, or one request at
    a time) over a device-memory budget; runs a trace in real time on the calling
    thread."""

    def __init__(self, plans, budget_bytes: int = 8 << 30, streams: int = 4, max_batch: int = 256):
        self._plans = list(plans)
        self._arr = _plan_array(self._plans)
        h = ctypes.c_void_p()
        _check(lib.rklt_server_create(ctypes.cast(self._arr, ctypes.c_void_p), len(self._plans), budget_bytes, streams,
                                      max_batch, ctypes.byref(h)))
        self._h = h

    def run(self, reqs, mode: int = 0, recon=None, coef=None):
        """reqs: RklTRequest array; recon / coef: optional lists of host arrays (numpy,
        contiguous) receiving each request's outputs.  Returns (RklTResult array, wall_s)."""
        n = len(reqs)
        res = (RklTResult * max(n, 1))()
        wall = ctypes.c_double()
        pr = pc = None
        if recon is not None:
            pr = (ctypes.c_void_p * n)(*[a.ctypes.data if a is not None else None for a in recon])
        if coef is not None:
            pc = (ctypes.c_void_p * n)(*[a.ctypes.data if a is not None else None for a in coef])
        _check(lib.rklt_server_run(self._h, ctypes.cast(reqs, ctypes.c_void_p), n, mode,
                                   ctypes.cast(pr, ctypes.c_void_p) if pr is not None else None,
                                   ctypes.cast(pc, ctypes.c_void_p) if pc is not None else None,
                                   ctypes.cast(res, ctypes.c_void_p), ctypes.byref(wall)))
        return res, wall.value

    def close(self):
        if self._h:
            lib.rklt_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rklt_server_create(plans, budget_bytes: int = 8 << 30, streams: int = 4, max_batch: int = 256) -> NativeServer:
    return NativeServer(plans, budget_bytes, streams, max_batch)
