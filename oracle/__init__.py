"""CPU oracle for the soft-decision Viterbi hot path (arxiv 2011.09337).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product library never calls it and shares no code with it: the arithmetic lives
in ``vit_oracle.c`` (plain C99, int64 metrics, FP64 for the metric forms), and
this module only marshals numpy arrays through ``ctypes``.

Functions and the passage each one follows:

* :func:`encode`            Eq. 1 and Fig. 1 (convolutional encoder).
* :func:`depuncture`        Sec. "De-puncturing" (zero LLR at removed symbols).
* :func:`viterbi_blocked`   Eq. 2-4 with Alg. 1 (forward) and Alg. 2 (traceback),
                            run on the overlapped tiles of Fig. relworks;
                            ``f=0`` is the full-frame decoder.
* :func:`viterbi_blocked_pt` the same tiles with the first parallel traceback
                            of Sec. "Parallel Traceback Algorithm" (Fig. pt1):
                            subframes of ``f0`` stages, each traced back from
                            ``v2`` stages to its right, starting at the stored
                            argmax state or at a SplitMix64 state.
* :func:`viterbi_window`    one window with an explicit traceback start state.
* :func:`splitmix64`        the counter-based generator of the random start.
* :func:`viterbi_full`      the same with one tile.
* :func:`brute_force_ml`    exhaustive maximum-likelihood search (pin only).
* :func:`metric_hard`,
  :func:`metric_lse`        best-path metric and its temperature relaxation with
                            gradients; the paper does not define these, the
                            definitions are stated in the C source.

Parity status: the traceback-start rule of the tiles (argmax of the window's
last stage, ties to the lowest state; zero initial metrics for windows that do
not start at stage 0) and the LLR quantisation are conventions, not facts the
paper fixes -- "parity unpinned" beyond the special cases the tests check
(single tile == full frame, noiseless recovery, brute force).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Sequence

import numpy as np

STREAM, TERMINATED, FREE_START = 0, 1, 2
M_DEFAULT = 8192

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vit_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``vit_oracle.c`` into ``oracle/_build/liboracle.so`` (gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
            lib.orc_encode.argtypes = [i32, i32, vp, vp, i64, vp]
            lib.orc_depuncture.argtypes = [vp, i64, i64, i32, vp, i32, vp]
            lib.orc_depuncture.restype = i64
            lib.orc_viterbi_blocked.argtypes = [i32, i32, vp, vp, i64, i64, i64, i64, i32, i64, i64, i64, vp, vp]
            lib.orc_viterbi_blocked_pt.argtypes = [i32, i32, vp, vp, i64, i64, i64, i64, i64, i32,
                                                   ctypes.c_uint64, i32, i64, i64, i64, vp]
            lib.orc_viterbi_window.argtypes = [i32, i32, vp, vp, i64, i64, i32, i64, i32, i64, i64, vp]
            lib.orc_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.orc_splitmix64.restype = ctypes.c_uint64
            lib.orc_brute_force.argtypes = [i32, i32, vp, vp, i32, i32, vp, vp, vp]
            lib.orc_metric_hard.argtypes = [i32, i32, vp, vp, i64, vp, vp]
            lib.orc_metric_lse.argtypes = [i32, i32, vp, vp, i64, ctypes.c_double, vp, vp]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _polys(K: int, beta: int, polys: Sequence[int]) -> np.ndarray:
    p = np.asarray(list(polys), dtype=np.uint32)
    if p.shape != (beta,):
        raise ValueError("need one generator polynomial per coded bit")
    return p


def _check(rc: int, what: str):
    if rc < 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def encode(K: int, beta: int, polys: Sequence[int], bits: np.ndarray) -> np.ndarray:
    """Eq. 1: coded bits, shape (n, beta), for input bits starting in state 0."""
    lib = _load()
    x = np.ascontiguousarray(bits, dtype=np.uint8)
    out = np.empty((x.size, beta), dtype=np.uint8)
    p = _polys(K, beta, polys)
    _check(lib.orc_encode(K, beta, _ptr(p), _ptr(x), x.size, _ptr(out)), "encode")
    return out


def depuncture(rx: np.ndarray, n: int, beta: int, mask: np.ndarray) -> np.ndarray:
    """De-puncture kept int8 symbols into an (n, beta) stream with zeros."""
    lib = _load()
    r = np.ascontiguousarray(rx, dtype=np.int8)
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    if m.ndim != 2 or m.shape[0] != beta:
        raise ValueError("mask must be beta x P")
    out = np.empty((n, beta), dtype=np.int8)
    k = lib.orc_depuncture(_ptr(r), r.size, n, beta, _ptr(m), m.shape[1], _ptr(out))
    _check(k, "depuncture")
    if k != r.size:
        raise ValueError(f"punctured stream has {r.size} symbols, {k} used")
    return out


def viterbi_blocked(K: int, beta: int, polys: Sequence[int], llr: np.ndarray, f: int, v1: int, v2: int,
                    mode: int = STREAM, M: int = M_DEFAULT, blocks: tuple[int, int] | None = None,
                    return_metrics: bool = False):
    """Blocked decoder.  ``llr`` is stage-major int8, shape (n, beta) or flat.

    Returns one decoded bit per stage (uint8, length n; stages outside the
    decoded blocks are left 0).  ``blocks=(b0, b1)`` decodes that block range.
    """
    lib = _load()
    x = np.ascontiguousarray(llr, dtype=np.int8).reshape(-1)
    if x.size % beta:
        raise ValueError("LLR count is not a multiple of beta")
    n = x.size // beta
    p = _polys(K, beta, polys)
    bits = np.zeros(n, dtype=np.uint8)
    fb = n if (f == 0 or f > n) else f
    nb = (n + fb - 1) // fb if n else 0
    b0, b1 = (0, nb) if blocks is None else blocks
    metrics = np.zeros(max(b1 - b0, 1), dtype=np.int64)
    _check(lib.orc_viterbi_blocked(K, beta, _ptr(p), _ptr(x), n, f, v1, v2, mode, M, b0, b1, _ptr(bits),
                                   _ptr(metrics)), "viterbi_blocked")
    if return_metrics:
        return bits, metrics[: b1 - b0]
    return bits


PT_STORED, PT_RANDOM = 0, 1


def viterbi_blocked_pt(K: int, beta: int, polys: Sequence[int], llr: np.ndarray, f: int, v1: int, v2: int,
                       f0: int, start: int = PT_STORED, seed: int = 0, mode: int = STREAM, M: int = M_DEFAULT,
                       blocks: tuple[int, int] | None = None):
    """Blocked decoder with the parallel traceback (subframes of ``f0`` stages,
    overlap ``v2``; ``start`` = PT_STORED or PT_RANDOM).  Returns one bit per
    stage like :func:`viterbi_blocked`."""
    lib = _load()
    x = np.ascontiguousarray(llr, dtype=np.int8).reshape(-1)
    if x.size % beta:
        raise ValueError("LLR count is not a multiple of beta")
    n = x.size // beta
    p = _polys(K, beta, polys)
    bits = np.zeros(n, dtype=np.uint8)
    fb = n if (f == 0 or f > n) else f
    nb = (n + fb - 1) // fb if n else 0
    b0, b1 = (0, nb) if blocks is None else blocks
    _check(lib.orc_viterbi_blocked_pt(K, beta, _ptr(p), _ptr(x), n, f, v1, v2, f0, start, seed, mode, M, b0, b1,
                                      _ptr(bits)), "viterbi_blocked_pt")
    return bits


def viterbi_window(K: int, beta: int, polys: Sequence[int], llr: np.ndarray, t0: int, t1: int, known: bool,
                   end_state: int = -1, emit: tuple[int, int] | None = None, M: int = M_DEFAULT) -> np.ndarray:
    """One window [t0, t1) of the stream (Alg. 1 + Alg. 2) with an explicit
    traceback start state (-1: argmax).  Returns n bits; only ``emit``
    (default: the whole window) is written."""
    lib = _load()
    x = np.ascontiguousarray(llr, dtype=np.int8).reshape(-1)
    n = x.size // beta
    p = _polys(K, beta, polys)
    bits = np.zeros(n, dtype=np.uint8)
    e0, e1 = (t0, t1) if emit is None else emit
    _check(lib.orc_viterbi_window(K, beta, _ptr(p), _ptr(x), t0, t1, int(known), M, end_state, e0, e1, _ptr(bits)),
           "viterbi_window")
    return bits


def splitmix64(seed: int, i: int) -> int:
    """Output ``i`` (0-based) of SplitMix64 seeded with ``seed``."""
    return int(_load().orc_splitmix64(seed, i))


def viterbi_full(K: int, beta: int, polys: Sequence[int], llr: np.ndarray, mode: int = STREAM,
                 M: int = M_DEFAULT):
    """Full-frame Viterbi (Alg. 1 + Alg. 2).  Returns (bits per stage, metric)."""
    bits, m = viterbi_blocked(K, beta, polys, llr, 0, 0, 0, mode, M, return_metrics=True)
    return bits, int(m[0])


def brute_force_ml(K: int, beta: int, polys: Sequence[int], llr: np.ndarray, n_info: int, mode: int = STREAM):
    """Exhaustive ML over all messages: (best metric, #maximisers, lowest maximiser's bits)."""
    lib = _load()
    x = np.ascontiguousarray(llr, dtype=np.int8).reshape(-1)
    p = _polys(K, beta, polys)
    n = n_info + (K - 1 if mode == TERMINATED else 0)
    if x.size != n * beta:
        raise ValueError("LLR length does not match the message length")
    best = np.zeros(1, dtype=np.int64)
    cnt = np.zeros(1, dtype=np.int64)
    bits = np.zeros(max(n, 1), dtype=np.uint8)
    _check(lib.orc_brute_force(K, beta, _ptr(p), _ptr(x), n_info, mode, _ptr(best), _ptr(cnt), _ptr(bits)),
           "brute_force")
    return int(best[0]), int(cnt[0]), bits[:n]


def metric_hard(K: int, beta: int, polys: Sequence[int], llr: np.ndarray, grad: bool = True):
    """Best 0-rooted, 0-terminated path metric per frame and its +-1 subgradient.

    ``llr`` has shape (F, n, beta) (float); returns (metric (F,), grad (F, n, beta)).
    """
    lib = _load()
    x = np.ascontiguousarray(llr, dtype=np.float64)
    F, n, b = x.shape
    p = _polys(K, beta, polys)
    met = np.zeros(F, dtype=np.float64)
    g = np.zeros_like(x) if grad else None
    for i in range(F):
        mi = np.zeros(1, dtype=np.float64)
        _check(lib.orc_metric_hard(K, beta, _ptr(p), _ptr(x[i]), n, _ptr(mi),
                                   _ptr(g[i]) if grad else None), "metric_hard")
        met[i] = mi[0]
    return met, g


def metric_lse(K: int, beta: int, polys: Sequence[int], llr: np.ndarray, tau: float, grad: bool = True):
    """Temperature-tau log-sum-exp path metric per frame and its gradient (FP64)."""
    lib = _load()
    x = np.ascontiguousarray(llr, dtype=np.float64)
    F, n, b = x.shape
    p = _polys(K, beta, polys)
    met = np.zeros(F, dtype=np.float64)
    g = np.zeros_like(x) if grad else None
    for i in range(F):
        mi = np.zeros(1, dtype=np.float64)
        _check(lib.orc_metric_lse(K, beta, _ptr(p), _ptr(x[i]), n, float(tau), _ptr(mi),
                                  _ptr(g[i]) if grad else None), "metric_lse")
        met[i] = mi[0]
    return met, g
