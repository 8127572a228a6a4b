"""Bit-error-rate tools (Sec. "Experimental results", Tables II and III).

* :func:`distance_spectrum` and :func:`union_bound` — the code's own union
  bound on the bit error rate of maximum-likelihood soft decoding, which
  stands in for the MATLAB bertool curves the paper compares against:
  ``P_b <= sum_d c_d Q(sqrt(2 d R Eb/N0))`` with ``c_d`` the number of input
  ones on the paths that leave state 0 and first return with output weight d.
* :func:`ber` — the measured bit error rate of the GPU decoder on a
  synthetic BPSK/AWGN stream (noise drawn on the GPU), for any tiling and
  traceback variant.
* :func:`table_ii` / :func:`table_iii` — the paper's two parameter sweeps:
  BER against the tile length f and the overlap v2 (serial traceback), and
  against the subframe length f0 and v2 (parallel traceback).

Run ``python -m paper_2011_09337_gb300.ber`` for the tables.
"""
from __future__ import annotations

import math
from typing import Sequence

import torch

from . import vit


def _parity(x: int) -> int:
    return bin(x).count("1") & 1


def distance_spectrum(K: int, beta: int, polys: Sequence[int], dmax: int) -> dict[int, tuple[int, int]]:
    """{d: (a_d, c_d)} for every output weight d <= dmax: a_d paths leave state
    0 and first return to it with output weight d, carrying c_d input ones in
    total.  Found by a breadth-first walk of the state diagram (Eq. 1 outputs,
    state = the K-1 previous inputs, newest in the top bit)."""
    S = 1 << (K - 1)
    out_w = [sum(_parity(g & R) for g in polys) for R in range(2 * S)]
    # frontier: (state, weight) -> [paths, input ones], paths not yet back in 0
    first = 1 << (K - 1)
    frontier = {(first >> 1, out_w[first]): [1, 1]} if out_w[first] <= dmax else {}
    spec: dict[int, list[int]] = {}
    for _ in range(S * (dmax + 1) + K):
        if not frontier:
            break
        nxt: dict[tuple[int, int], list[int]] = {}
        for (s, w), (n, ones) in frontier.items():
            for b in (0, 1):
                R = (b << (K - 1)) | s
                w2 = w + out_w[R]
                if w2 > dmax:
                    continue
                j = R >> 1
                if j == 0:
                    e = spec.setdefault(w2, [0, 0])
                    e[0] += n
                    e[1] += ones + b * n
                else:
                    e = nxt.setdefault((j, w2), [0, 0])
                    e[0] += n
                    e[1] += ones + b * n
        frontier = nxt
    else:
        raise ValueError("the state diagram has a zero-weight cycle (catastrophic code)")
    return {d: (v[0], v[1]) for d, v in sorted(spec.items())}


def _q(x: float) -> float:
    return 0.5 * math.erfc(x / math.sqrt(2.0))


def union_bound(K: int, beta: int, polys: Sequence[int], ebn0_db: float, rate: float | None = None,
                terms: int = 8) -> float:
    """Union bound on the bit error rate at Eb/N0 (dB) from the first `terms`
    nonzero spectrum lines; rate defaults to 1/beta."""
    R = rate if rate is not None else 1.0 / beta
    g = 10.0 ** (ebn0_db / 10.0)
    dmax = 2 * (K - 1) * beta + 8
    while True:
        spec = distance_spectrum(K, beta, polys, dmax)
        if len(spec) >= terms:
            break
        dmax += 4
    lines = list(spec.items())[:terms]
    return sum(c * _q(math.sqrt(2.0 * d * R * g)) for d, (_, c) in lines)


def _channel_llr(coded: torch.Tensor, ebn0_db: float, rate: float, gen: torch.Generator) -> torch.Tensor:
    """BPSK x = 1 - 2c over AWGN with sigma^2 = 1 / (2 R Eb/N0); int8 LLRs
    q = clip(sign(L) floor(16 |L| + 1/2), +-127), L = 2 y / sigma^2."""
    sigma = math.sqrt(1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0)))
    x = 1.0 - 2.0 * coded.to(torch.float32)
    y = x + sigma * torch.randn(x.shape, generator=gen, device=x.device, dtype=torch.float32)
    L = 2.0 * y / (sigma * sigma)
    q = torch.sign(L) * torch.floor(L.abs() * 16.0 + 0.5)
    return q.clamp_(-127, 127).to(torch.int8)


def ber(code: "vit.Code", ebn0_db: float, nbits: int = 1 << 22, seed: int = 0, device: str = "cuda") -> float:
    """Measured bit error rate of `code` (its tiling, termination mode and
    traceback variant) on a random `nbits`-bit STREAM message."""
    if code.puncture is not None:
        raise ValueError("BER sweeps here use unpunctured codes")
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    msg = torch.randint(0, 2, (nbits,), generator=gen, device=device, dtype=torch.uint8)
    coded = vit.encode(code, msg).reshape(-1)
    llr = _channel_llr(coded, ebn0_db, 1.0 / code.beta, gen)
    out = vit.decode(code, llr, nbits)
    bits = torch.stack([(out >> k) & 1 for k in range(8)], dim=1).reshape(-1)[:nbits]
    return float((bits != msg).sum().item()) / nbits


def table_ii(K: int, beta: int, polys: Sequence[int], ebn0_db: float, fs: Sequence[int], v2s: Sequence[int],
             v1: int = 21, nbits: int = 1 << 22) -> dict[tuple[int, int], float]:
    """BER against tile length f and right overlap v2 (serial traceback)."""
    res = {}
    for f in fs:
        for v2 in v2s:
            code = vit.Code(K, beta, polys, f=f, v1=v1, v2=v2)
            res[(f, v2)] = ber(code, ebn0_db, nbits, seed=1)
    return res


def table_iii(K: int, beta: int, polys: Sequence[int], ebn0_db: float, f0s: Sequence[int], v2s: Sequence[int],
              f: int = 296, v1: int = 21, rule: int = 0, nbits: int = 1 << 22) -> dict[tuple[int, int], float]:
    """BER against subframe length f0 and overlap v2 (parallel traceback,
    rule PT_STORED or PT_RANDOM)."""
    res = {}
    for f0 in f0s:
        for v2 in v2s:
            code = vit.Code(K, beta, polys, f=f, v1=v1, v2=v2, pt_f0=f0, pt_rule=rule, pt_seed=7)
            res[(f0, v2)] = ber(code, ebn0_db, nbits, seed=1)
    return res


def bound_ebn0_at(K: int, beta: int, polys: Sequence[int], target: float, rate: float | None = None) -> float:
    """Eb/N0 (dB) at which the union bound equals `target` (bisection; the
    bound falls monotonically with Eb/N0)."""
    lo, hi = -2.0, 15.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if union_bound(K, beta, polys, mid, rate) > target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def ebn0_at(points: Sequence[tuple[float, float]], target: float) -> float | None:
    """Eb/N0 at which a measured BER curve crosses `target`: linear in
    log10(BER) between the two measured points around the crossing; None if
    the points do not bracket it."""
    pts = sorted(p for p in points if p[1] > 0)
    for (e0, b0), (e1, b1) in zip(pts, pts[1:]):
        if b0 >= target >= b1:
            if b0 == b1:
                return e0
            t = (math.log10(b0) - math.log10(target)) / (math.log10(b0) - math.log10(b1))
            return e0 + t * (e1 - e0)
    return None


def curve(code: "vit.Code", target: float, ebn0s: Sequence[float], nbits: int, seed: int = 1):
    """BER at increasing Eb/N0 until it is below target / 3 (a measured
    BER under 100 / nbits is not used).  Returns [(Eb/N0, BER)]."""
    pts = []
    for e in ebn0s:
        b = ber(code, e, nbits, seed=seed)
        pts.append((e, b))
        if b < target / 3 or b * nbits < 100:
            break
    return pts


GAP_TARGET = 1e-4
GAP_EBN0 = (2.0, 2.5, 3.0, 3.5, 4.0, 4.5, 5.0, 5.5, 6.0, 6.5)


def gap_db(code: "vit.Code", K: int, beta: int, polys: Sequence[int], ref_ebn0: float, nbits: int,
           target: float = GAP_TARGET):
    """The paper's BER metric (Sec. "BER Performance"): how much more Eb/N0
    the decoder needs than a reference curve to reach the target BER, here
    both the code's union bound and a measured reference decoder.
    Returns (gap to the union bound, gap to the reference, points)."""
    pts = curve(code, target, GAP_EBN0, nbits)
    e = ebn0_at(pts, target)
    if e is None:
        return None, None, pts
    return e - bound_ebn0_at(K, beta, polys, target), e - ref_ebn0, pts


def reference_ebn0(K: int, beta: int, polys: Sequence[int], nbits: int, target: float = GAP_TARGET) -> float:
    """Eb/N0 at which the tiled decoder with a very long overlap (f = 2048,
    v1 = v2 = 256: the traceback has merged with the maximum-likelihood path
    long before it reaches the emitted stages) reaches the target BER."""
    code = vit.Code(K, beta, polys, f=2048, v=256)
    return ebn0_at(curve(code, target, GAP_EBN0, nbits), target)


def table_ii_gaps(K, beta, polys, fs, v2s, v1=21, nbits=1 << 24, target=GAP_TARGET):
    """Table II: dB gap of the serial-traceback decoder for every (f, v2)."""
    ref = reference_ebn0(K, beta, polys, nbits, target)
    out = {"target_ber": target, "nbits_per_point": nbits, "v1": v1, "reference_ebn0": ref,
           "bound_ebn0": bound_ebn0_at(K, beta, polys, target), "cells": {}}
    for f in fs:
        for v2 in v2s:
            code = vit.Code(K, beta, polys, f=f, v1=v1, v2=v2)
            gb, gr, pts = gap_db(code, K, beta, polys, ref, nbits, target)
            out["cells"][f"f={f},v2={v2}"] = {"f": f, "v2": v2, "gap_to_union_bound_db": gb,
                                              "gap_to_reference_db": gr, "points": pts}
    return out


def table_iii_gaps(K, beta, polys, f0s, v2s, f=296, v1=21, rule=0, nbits=1 << 24, target=GAP_TARGET):
    """Table III: dB gap of the parallel-traceback decoder for every (f0, v2)."""
    ref = reference_ebn0(K, beta, polys, nbits, target)
    out = {"target_ber": target, "nbits_per_point": nbits, "f": f, "v1": v1, "rule": rule, "reference_ebn0": ref,
           "bound_ebn0": bound_ebn0_at(K, beta, polys, target), "cells": {}}
    for f0 in f0s:
        for v2 in v2s:
            code = vit.Code(K, beta, polys, f=f, v1=v1, v2=v2, pt_f0=f0, pt_rule=rule, pt_seed=7)
            gb, gr, pts = gap_db(code, K, beta, polys, ref, nbits, target)
            out["cells"][f"f0={f0},v2={v2}"] = {"f0": f0, "v2": v2, "gap_to_union_bound_db": gb,
                                                "gap_to_reference_db": gr, "points": pts}
    return out


def _print_grid(title, res, rows, cols, rname, cname):
    print(title)
    print(f"{rname:>6s} \\ {cname:<4s}" + "".join(f"{c:>10d}" for c in cols))
    for r in rows:
        print(f"{r:>11d}" + "".join(f"{res[(r, c)]:10.2e}" for c in cols))


def _print_gaps(title, tab, rows, cols, rkey, ckey):
    print(title)
    print(f"{ckey:>6s} \\ {rkey:<4s}" + "".join(f"{r:>9d}" for r in rows))
    for c in cols:
        vals = []
        for r in rows:
            g = tab["cells"][f"{rkey}={r},{ckey}={c}"]["gap_to_union_bound_db"]
            vals.append(f"{g:9.3f}" if g is not None else f"{'-':>9s}")
        print(f"{c:>11d}" + "".join(vals))


if __name__ == "__main__":
    import argparse
    import json
    from . import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--ebn0", type=float, default=3.0)
    ap.add_argument("--bits", type=int, default=1 << 22)
    ap.add_argument("--gaps", metavar="JSON", help="compute the dB-gap grids of Tables II and III and write them")
    a = ap.parse_args()
    if a.gaps:
        K, beta, polys = synth.CODE_K7_R12
        t2 = table_ii_gaps(K, beta, polys, [32, 64, 128, 256, 512], [10, 20, 30, 40], nbits=a.bits)
        t3 = table_iii_gaps(K, beta, polys, [8, 16, 24, 32, 40, 48, 56], [25, 30, 35, 40, 45], nbits=a.bits)
        t3r = table_iii_gaps(K, beta, polys, [32], [25, 35, 45], rule=1, nbits=a.bits)
        _print_gaps("Table II: dB gap to the union bound at BER 1e-4 (columns f, rows v2)", t2,
                    [32, 64, 128, 256, 512], [10, 20, 30, 40], "f", "v2")
        _print_gaps("Table III: dB gap, parallel traceback, f=296 (columns f0, rows v2)", t3,
                    [8, 16, 24, 32, 40, 48, 56], [25, 30, 35, 40, 45], "f0", "v2")
        with open(a.gaps, "w") as fh:
            json.dump({"code": "K=7 (171,133) r1/2, int8 LLRs x16, BPSK/AWGN, STREAM",
                       "table_ii": t2, "table_iii": t3, "table_iii_random_start": t3r}, fh, indent=1)
        raise SystemExit(0)
    K, beta, polys = synth.CODE_K7_R12
    print("union bound, K=7 (171,133):",
          ", ".join(f"{e} dB: {union_bound(K, beta, polys, e):.2e}" for e in (2, 3, 4, 5, 6)))
    fs, v2s = [64, 128, 256, 512, 1024], [9, 21, 33, 45]
    _print_grid(f"BER, serial traceback, Eb/N0 {a.ebn0} dB (rows f, columns v2)",
                table_ii(K, beta, polys, a.ebn0, fs, v2s, nbits=a.bits), fs, v2s, "f", "v2")
    f0s = [8, 16, 24, 32, 40, 48, 56]
    _print_grid(f"BER, parallel traceback, f=296, Eb/N0 {a.ebn0} dB (rows f0, columns v2)",
                table_iii(K, beta, polys, a.ebn0, f0s, v2s, nbits=a.bits), f0s, v2s, "f0", "v2")
