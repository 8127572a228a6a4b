"""Autotuner for batched decoding: tiling (f, v) per code and CTA size.

The decoded bits of a tile depend on f and v (the tiling of Fig. relworks),
so the tuner treats them as a quality/speed trade-off: for every code in the
batch it times the candidate tilings on that code's frames and keeps the
fastest whose output differs from the full-frame (f = 0, Alg. 1 + 2) decode
of the same frames on at most ``max_disagree`` of the bits.  The CTA size
(warps per block) is then timed on the whole batch.  All timing uses CUDA
events around planned, graph-captured batch runs; every decode runs in the
library's kernels.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import vit


@dataclass
class Choice:
    f: int
    v: int
    ms: float
    disagree: float


def _time(batch: "vit.Batch", reps: int) -> float:
    batch.run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        batch.run()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def _run(frames, code_of, warps=0, graph=True, reps=3):
    """frames: list of (code_key, llr, n, mode); code_of: key -> vit.Code.
    Returns (ms per run, one uint8 tensor holding every frame's packed bits)."""
    sizes = [(code_of[key].output_bits(n) + 7) // 8 for key, _, n, _ in frames]
    buf = torch.empty(sum(sizes), dtype=torch.uint8, device=frames[0][1].device)
    specs, off = [], 0
    for (key, llr, n, mode), sz in zip(frames, sizes):
        specs.append((code_of[key], llr, n, mode, buf[off:off + sz]))
        off += sz
    b = vit.Batch(specs, graph=graph, warps=warps)
    ms = _time(b, reps)
    return ms, buf


def _disagree(a: torch.Tensor, b: torch.Tensor, nbits: int) -> float:
    """Fraction of differing decoded bits between two packed outputs."""
    import numpy as np
    x = torch.bitwise_xor(a, b).cpu().numpy()
    return float(np.unpackbits(x).sum()) / max(nbits, 1)


def default_candidates(K: int):
    fs = [256, 512, 1024, 2048, 0]
    vs = [7 * (K - 1), 10 * (K - 1), 14 * (K - 1)]
    return [(f, v) for f in fs for v in vs if not (f == 0 and v != vs[0])]


def pick(rows, max_disagree: float):
    """The fastest timed tiling whose disagreement with the full-frame decode
    is at most ``max_disagree`` (rows: dicts with f, v, ms, disagree), or
    None when no row qualifies."""
    best = None
    for r in rows:
        if r["disagree"] <= max_disagree and (best is None or r["ms"] < best.ms):
            best = Choice(r["f"], r["v"], r["ms"], r["disagree"])
    return best


def _make_code(K, beta, polys, f, v, mode):
    return vit.Code(K, beta, polys, f=f, v=v, mode=mode)


def tune(frames, codes, candidates=None, max_disagree: float = 2e-4, warps_options=(2, 4, 8), reps: int = 3,
         runner=None, make_code=None):
    """frames: list of (code_index, llr CUDA int8 tensor, n, mode);
    codes: list of (K, beta, polys).  Returns ({code_index: Choice}, warps, report).

    ``runner(frames, code_map, warps=.., reps=..) -> (ms, packed bits)`` and
    ``make_code(K, beta, polys, f, v, mode)`` default to timed, graph-captured
    batch runs of the library and ``vit.Code``; they are parameters so that
    the selection logic can be exercised with a cost table."""
    runner = runner or _run
    make_code = make_code or _make_code
    chosen = {}
    report = {}
    for ci, (K, beta, polys) in enumerate(codes):
        sub = [(ci, llr, n, mode) for c, llr, n, mode in frames if c == ci]
        if not sub:
            continue
        modes = {m for _, _, _, m in sub}
        mode = modes.pop() if len(modes) == 1 else vit.STREAM

        def code_for(f, v):
            return {ci: make_code(K, beta, polys, f, v, mode)}

        _, ref_out = runner(sub, code_for(0, 0), reps=1)
        rows = []
        for f, v in (candidates or default_candidates(K)):
            cmap = code_for(f, v)
            ms, out = runner(sub, cmap, reps=reps)
            nbits = sum(cmap[ci].output_bits(n) for _, _, n, _ in sub)
            dis = 0.0 if f == 0 else _disagree(out, ref_out, nbits)
            rows.append({"f": f, "v": v, "ms": ms, "disagree": dis})
        chosen[ci] = pick(rows, max_disagree)
        if chosen[ci] is None:
            raise ValueError(f"no candidate tiling of code {ci} is within max_disagree={max_disagree}")
        report[ci] = rows
    code_objs = {ci: make_code(*codes[ci], chosen[ci].f, chosen[ci].v,
                               next(m for c, _, _, m in frames if c == ci)) for ci in chosen}
    wbest, wms = None, None
    for w in warps_options:
        ms, _ = runner(frames, code_objs, warps=w, reps=reps)
        report.setdefault("warps", []).append({"warps": w, "ms": ms})
        if wms is None or ms < wms:
            wbest, wms = w, ms
    return chosen, wbest, report
