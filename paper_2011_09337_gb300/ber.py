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


def _print_grid(title, res, rows, cols, rname, cname):
    print(title)
    print(f"{rname:>6s} \\ {cname:<4s}" + "".join(f"{c:>10d}" for c in cols))
    for r in rows:
        print(f"{r:>11d}" + "".join(f"{res[(r, c)]:10.2e}" for c in cols))


if __name__ == "__main__":
    import argparse
    from . import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--ebn0", type=float, default=3.0)
    ap.add_argument("--bits", type=int, default=1 << 22)
    a = ap.parse_args()
    K, beta, polys = synth.CODE_K7_R12
    print("union bound, K=7 (171,133):",
          ", ".join(f"{e} dB: {union_bound(K, beta, polys, e):.2e}" for e in (2, 3, 4, 5, 6)))
    fs, v2s = [64, 128, 256, 512, 1024], [9, 21, 33, 45]
    _print_grid(f"BER, serial traceback, Eb/N0 {a.ebn0} dB (rows f, columns v2)",
                table_ii(K, beta, polys, a.ebn0, fs, v2s, nbits=a.bits), fs, v2s, "f", "v2")
    f0s = [8, 16, 24, 32, 40, 48, 56]
    _print_grid(f"BER, parallel traceback, f=296, Eb/N0 {a.ebn0} dB (rows f0, columns v2)",
                table_iii(K, beta, polys, a.ebn0, f0s, v2s, nbits=a.bits), f0s, v2s, "f0", "v2")
