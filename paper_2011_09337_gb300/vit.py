"""Python binding of libvit (include/vit.h): argument marshalling only.

Every step of decoding runs in the library's CUDA kernels; this module checks
shapes, allocates outputs and scratch with torch on the caller's device and
passes raw pointers plus ``torch.cuda.current_stream()``.  The library is
loaded on first use; a missing build raises ``RuntimeError``.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import torch

from . import build_lib

STREAM, TERMINATED, FREE_START = 0, 1, 2
DECODER_AUTO, DECODER_TILES, DECODER_SHARED, DECODER_SPREAD = 0, 1, 2, 3
BATCH_GRAPH, BATCH_PERSISTENT, BATCH_HOST = 1, 4, 8
PT_STORED, PT_RANDOM = 0, 1

_lib = None


class VitError(RuntimeError):
    pass


def lib_path() -> str:
    return build_lib.LIB


def load(path: str | None = None):
    """Loads libvit.so (built by ``build_lib.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or lib_path()
    if not os.path.exists(p):
        raise RuntimeError(f"libvit.so not built at {p}: run __graft_entry__.build() or "
                           "python -m paper_2011_09337_gb300.build_lib")
    L = ctypes.CDLL(p)
    i32, i64, vp, sz = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t
    sig = {
        "vit_create": (i32, [ctypes.POINTER(vp), i32, i32, vp, i64, i64]),
        "vit_set_overlaps": (i32, [vp, i64, i64]),
        "vit_set_puncture": (i32, [vp, vp, i32]),
        "vit_set_termination": (i32, [vp, i32]),
        "vit_destroy": (None, [vp]),
        "vit_llr_count": (i64, [vp, i64]),
        "vit_output_bits": (i64, [vp, i64]),
        "vit_decode_workspace": (sz, [vp, i64]),
        "vit_decode_ws": (i32, [vp, vp, i64, vp, vp, sz, vp]),
        "vit_decode": (i32, [vp, vp, i64, vp, vp]),
        "vit_encode": (i32, [vp, vp, i64, vp, vp]),
        "vit_last_error": (ctypes.c_char_p, []),
        "vit_code_supported": (i32, [i32, i32, vp]),
        "vit_set_parallel_traceback": (i32, [vp, i64, i32, ctypes.c_uint64]),
        "vit_hard_llr": (i32, [vp, i64, vp, vp]),
        "vit_set_decoder": (i32, [vp, i32]),
    }
    optional = {
        "vit_batch_plan": (i32, [ctypes.POINTER(vp), vp, i32, i32]),
        "vit_batch_run": (i32, [vp, vp]),
        "vit_batch_destroy": (None, [vp]),
        "vit_decode_batch": (i32, [vp, i32, vp]),
        "vit_metric_workspace": (sz, [vp, i32, i64, ctypes.c_float, i32]),
        "vit_metric_fwd": (i32, [vp, vp, i32, i64, ctypes.c_float, i32, vp, vp, sz, vp]),
        "vit_metric_bwd": (i32, [vp, vp, vp, i32, i64, ctypes.c_float, i32, vp, sz, vp, vp]),
        "vit_probe_rate": (i32, [i32, i32, i32, i32, vp, ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    }
    for name, (res, args) in list(sig.items()) + list(optional.items()):
        if not hasattr(L, name):
            if name in sig:
                raise RuntimeError(f"libvit.so lacks {name}")
            continue
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(rc: int):
    if rc != 0:
        msg = load().vit_last_error().decode(errors="replace")
        raise VitError(f"libvit status {rc}: {msg}")


def _stream(device: torch.device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _u32(polys: Sequence[int]) -> ctypes.Array:
    return (ctypes.c_uint32 * len(polys))(*polys)


class Code:
    """A convolutional code and its tiling (vit_create / vit_set_*)."""

    def __init__(self, K: int, beta: int, polys: Sequence[int], f: int = 0, v: int = 0,
                 v1: int | None = None, v2: int | None = None, mode: int = STREAM,
                 puncture: Sequence[Sequence[int]] | None = None, pt_f0: int = 0, pt_rule: int = 0,
                 pt_seed: int = 0, decoder: int = DECODER_AUTO):
        """pt_f0 > 0 selects the parallel traceback with subframes of pt_f0
        stages (pt_rule: PT_STORED or PT_RANDOM, pt_seed: SplitMix64 key);
        decoder: DECODER_AUTO, DECODER_TILES, DECODER_SHARED or DECODER_SPREAD
        (vit_set_decoder)."""
        L = load()
        self.K, self.beta, self.polys = K, beta, tuple(int(p) for p in polys)
        self.f = f
        self.v1 = v if v1 is None else v1
        self.v2 = v if v2 is None else v2
        self.mode = mode
        h = ctypes.c_void_p()
        _check(L.vit_create(ctypes.byref(h), K, beta, ctypes.cast(_u32(self.polys), ctypes.c_void_p), f, v))
        self._h = h
        if v1 is not None or v2 is not None:
            _check(L.vit_set_overlaps(h, self.v1, self.v2))
        if mode != STREAM:
            _check(L.vit_set_termination(h, mode))
        self.puncture = None
        if puncture is not None:
            import numpy as np
            m = np.ascontiguousarray(np.asarray(puncture, dtype=np.uint8))
            if m.ndim != 2 or m.shape[0] != beta:
                raise ValueError("puncturing mask must be beta x period")
            self.puncture = m
            _check(L.vit_set_puncture(h, m.ctypes.data_as(ctypes.c_void_p), m.shape[1]))
        self.pt = (pt_f0, pt_rule, pt_seed)
        if pt_f0:
            _check(L.vit_set_parallel_traceback(h, pt_f0, pt_rule, pt_seed))
        if decoder != DECODER_AUTO:
            _check(L.vit_set_decoder(h, decoder))

    @property
    def handle(self):
        return self._h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.vit_destroy(h)
            self._h = None

    def llr_count(self, n: int) -> int:
        return int(load().vit_llr_count(self._h, n))

    def output_bits(self, n: int) -> int:
        return int(load().vit_output_bits(self._h, n))

    def workspace_bytes(self, n: int) -> int:
        return int(load().vit_decode_workspace(self._h, n))


def supported(K: int, beta: int, polys: Sequence[int]) -> bool:
    return bool(load().vit_code_supported(K, beta, ctypes.cast(_u32(polys), ctypes.c_void_p)))


def decode(code: Code, llr: torch.Tensor, n: int | None = None, out: torch.Tensor | None = None,
           workspace: torch.Tensor | None = None) -> torch.Tensor:
    """Decodes one frame.  ``llr``: int8 CUDA tensor of code.llr_count(n) values
    (stage-major).  Returns packed bits (uint8, LSB-first)."""
    if not (llr.is_cuda and llr.dtype == torch.int8 and llr.is_contiguous()):
        raise ValueError("llr must be a contiguous int8 CUDA tensor")
    if n is None:
        if code.puncture is not None:
            raise ValueError("n is required with puncturing")
        n = llr.numel() // code.beta
    if llr.numel() != code.llr_count(n):
        raise ValueError(f"expected {code.llr_count(n)} LLRs for {n} stages, got {llr.numel()}")
    nbytes = (code.output_bits(n) + 7) // 8
    if out is None:
        out = torch.empty(nbytes, dtype=torch.uint8, device=llr.device)
    elif out.numel() < nbytes or out.dtype != torch.uint8 or not out.is_cuda:
        raise ValueError("out too small")
    need = code.workspace_bytes(n)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=llr.device)
    _check(load().vit_decode_ws(code.handle, llr.data_ptr(), n, out.data_ptr(), workspace.data_ptr(), need,
                                _stream(llr.device)))
    return out


def encode(code: Code, bits: torch.Tensor) -> torch.Tensor:
    """Eq. 1 encoder on the GPU: uint8 bits (n,) -> coded bits (n, beta)."""
    if not (bits.is_cuda and bits.dtype == torch.uint8 and bits.is_contiguous()):
        raise ValueError("bits must be a contiguous uint8 CUDA tensor")
    n = bits.numel()
    out = torch.empty((n, code.beta), dtype=torch.uint8, device=bits.device)
    _check(load().vit_encode(code.handle, bits.data_ptr(), n, out.data_ptr(), _stream(bits.device)))
    return out


def hard_llr(bits: torch.Tensor, count: int) -> torch.Tensor:
    """Hard-decision input: packed received bits (uint8 CUDA tensor, LSB-first)
    -> int8 LLRs of +1 (bit 0) / -1 (bit 1), ``count`` of them."""
    if not (bits.is_cuda and bits.dtype == torch.uint8 and bits.is_contiguous()):
        raise ValueError("bits must be a contiguous uint8 CUDA tensor")
    if bits.numel() * 8 < count:
        raise ValueError("fewer packed bits than count")
    out = torch.empty(count, dtype=torch.int8, device=bits.device)
    _check(load().vit_hard_llr(bits.data_ptr(), count, out.data_ptr(), _stream(bits.device)))
    return out


class _Frame(ctypes.Structure):
    _fields_ = [("code", ctypes.c_void_p), ("llr", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("mode", ctypes.c_int), ("bits_out", ctypes.c_void_p)]


class Batch:
    """A planned batch of frames (vit_batch_plan): decodes the same device
    buffers every time ``run()`` is called; ``graph=True`` replays one
    captured CUDA graph.  Code groups run as concurrent launches, or with
    ``persistent=True`` (two groups with a compiled two-code kernel) as one
    persistent launch over a shared task queue.  With ``host=True``
    (VIT_BATCH_HOST) the tensors are pinned CPU tensors: each run copies the
    LLRs in, decodes and copies the bits back, pipelined over ``chunks``
    chunks (0 = library default)."""

    def __init__(self, frames, graph: bool = True, warps: int = 0, persistent: bool = False,
                 host: bool = False, chunks: int = 0, device=None):
        """frames: iterable of (code, llr, n, mode, out) with CUDA tensors
        (pinned CPU tensors with host=True); warps: CTA size in warps (1..8,
        0 = library default); device: the CUDA device of a host batch
        (default: the current one)."""
        L = load()
        self._keep = []
        arr = (_Frame * len(frames))()
        for i, (code, llr, n, mode, out) in enumerate(frames):
            if host:
                if not (not llr.is_cuda and llr.is_pinned() and llr.dtype == torch.int8 and llr.is_contiguous()):
                    raise ValueError("host batch: llr must be a contiguous pinned int8 CPU tensor")
                if not (not out.is_cuda and out.is_pinned() and out.dtype == torch.uint8 and out.is_contiguous()):
                    raise ValueError("host batch: out must be a contiguous pinned uint8 CPU tensor")
            elif not (llr.is_cuda and llr.dtype == torch.int8 and llr.is_contiguous()):
                raise ValueError("llr must be a contiguous int8 CUDA tensor")
            if llr.numel() != code.llr_count(n):
                raise ValueError(f"frame {i}: expected {code.llr_count(n)} LLRs, got {llr.numel()}")
            nb = n - (code.K - 1) if mode == TERMINATED else n
            if out.numel() < (nb + 7) // 8:
                raise ValueError(f"frame {i}: output too small")
            arr[i] = _Frame(code.handle.value, llr.data_ptr(), n, mode, out.data_ptr())
            self._keep.append((code, llr, out))
        h = ctypes.c_void_p()
        flags = ((BATCH_GRAPH if graph else 0) | (BATCH_PERSISTENT if persistent else 0) | (BATCH_HOST if host else 0)
                 | ((int(warps) & 0xFF) << 8) | ((int(chunks) & 0xFF) << 16))
        _check(L.vit_batch_plan(ctypes.byref(h), arr, len(frames), flags))
        self._h = h
        if host:
            self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        else:
            self.device = frames[0][1].device

    def run(self):
        _check(load().vit_batch_run(self._h, _stream(self.device)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.vit_batch_destroy(h)
            self._h = None


def metric_workspace(code: Code, nframes: int, n: int, tau: float, C: int) -> int:
    return int(load().vit_metric_workspace(code.handle, nframes, n, float(tau), C))


def metric_fwd(code: Code, llr: torch.Tensor, tau: float, C: int, out: torch.Tensor, ws: torch.Tensor) -> None:
    """vit_metric_fwd on caller-allocated tensors: llr float32 [F, n, beta],
    out float32 [F], ws uint8 of at least metric_workspace(...) bytes (kept for
    the matching metric_bwd)."""
    F, n, _ = llr.shape
    _check(load().vit_metric_fwd(code.handle, llr.data_ptr(), F, n, float(tau), C, out.data_ptr(),
                                 ws.data_ptr(), ws.numel(), _stream(llr.device)))


def metric_bwd(code: Code, llr: torch.Tensor, grad_metric: torch.Tensor, tau: float, C: int, ws: torch.Tensor,
               grad_llr: torch.Tensor) -> None:
    """vit_metric_bwd on caller-allocated tensors: grad_metric float32 [F],
    grad_llr float32 [F, n, beta], ws as left by metric_fwd."""
    F, n, _ = llr.shape
    _check(load().vit_metric_bwd(code.handle, llr.data_ptr(), grad_metric.data_ptr(), F, n, float(tau), C,
                                 ws.data_ptr(), ws.numel(), grad_llr.data_ptr(), _stream(llr.device)))


class ViterbiMetric(torch.autograd.Function):
    """Best-path metric of zero-terminated frames (tau == 0) or its
    temperature-tau log-sum-exp relaxation (tau > 0), with a hand-written
    backward (vit_metric_fwd / vit_metric_bwd).

    llr: float32 CUDA tensor [F, n, beta]; returns float32 [F].
    """

    @staticmethod
    def forward(ctx, llr: torch.Tensor, code: Code, tau: float = 0.0, C: int = 64):
        if not (llr.is_cuda and llr.dtype == torch.float32 and llr.dim() == 3 and llr.shape[2] == code.beta):
            raise ValueError("llr must be a float32 CUDA tensor [F, n, beta]")
        x = llr.contiguous()
        F, n, _ = x.shape
        ws = torch.empty(max(metric_workspace(code, F, n, tau, C), 1), dtype=torch.uint8, device=x.device)
        out = torch.empty(F, dtype=torch.float32, device=x.device)
        metric_fwd(code, x, tau, C, out, ws)
        ctx.save_for_backward(x)
        ctx.ws, ctx.code, ctx.tau, ctx.C = ws, code, float(tau), C
        return out

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (x,) = ctx.saved_tensors
        g = grad_out.contiguous().to(torch.float32)
        grad = torch.empty_like(x)
        metric_bwd(ctx.code, x, g, ctx.tau, ctx.C, ctx.ws, grad)
        return grad, None, None, None


def path_metric(llr: torch.Tensor, code: Code, tau: float = 0.0, C: int = 64) -> torch.Tensor:
    return ViterbiMetric.apply(llr, code, tau, C)


PROBE_KINDS = {"iadd": 0, "vmax16": 1, "imad": 2, "prmt": 3, "lop3": 4, "fadd": 5, "fmax": 6, "ex2": 7, "lg2": 8}


def probe_rate(kind: str, ctas_per_sm: int = 4, warps: int = 8, iters: int = 2000, device=None):
    """Instruction-rate microbenchmark (include/vit_probe.h): returns
    (warp instructions of class ``kind`` per SM clock per SM, launch ms, SM count)."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    rate, ms, sms = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(load().vit_probe_rate(PROBE_KINDS[kind], ctas_per_sm, warps, iters, _stream(dev), ctypes.byref(rate),
                                 ctypes.byref(ms), ctypes.byref(sms)))
    return rate.value, ms.value, sms.value
