"""Seeded synthetic inputs: the transmitter and channel of the paper's
verification system (Sec. "BER Performance", Fig. verifSys).

Uniform random message bits, a caller-supplied convolutional encoder,
optional puncturing of the coded bits, BPSK over AWGN, and LLR formation /
int8 quantisation.  This module holds none of the decoder's arithmetic: the
encoder is passed in (the tests pass the oracle's, the benchmark the
library's), so the same generators serve both sides.  numpy only.

Channel reading (the paper's noise formula is garbled): BPSK x = 1 - 2c,
y = x + sigma * N(0, 1) with sigma^2 = 1 / (2 R 10^(EbN0/10)), R the code
rate after puncturing; L = 2 y / sigma^2.  int8 LLRs are
clip(sign(L) * floor(16 |L| + 1/2), -127, 127) (round half away from zero).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, Sequence

import numpy as np

LLR_SCALE = 16.0
LLR_CLIP = 127

# generator polynomials used by the workloads (octal literals)
CODE_K7_R12 = (7, 2, (0o171, 0o133))
CODE_K7_R13 = (7, 3, (0o133, 0o171, 0o165))
CODE_K9_R12 = (9, 2, (0o561, 0o753))
PUNCT_R34 = np.array([[1, 1, 0], [1, 0, 1]], dtype=np.uint8)  # rows: coded stream, cols: stage mod 3
PUNCT_R23 = np.array([[1, 1], [1, 0]], dtype=np.uint8)
PUNCT_R56 = np.array([[1, 1, 0, 1, 0], [1, 0, 1, 0, 1]], dtype=np.uint8)

Encoder = Callable[[np.ndarray], np.ndarray]  # bits (n,) -> coded bits (n, beta)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def info_bits(n: int, g: np.random.Generator) -> np.ndarray:
    return g.integers(0, 2, size=n, dtype=np.uint8)


def noise_sigma(ebn0_db: float, rate: float) -> float:
    return float(np.sqrt(1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0))))


def bpsk_awgn(coded: np.ndarray, sigma: float, g: np.random.Generator) -> np.ndarray:
    c = np.asarray(coded, dtype=np.float64).reshape(-1)
    return (1.0 - 2.0 * c) + sigma * g.standard_normal(c.size)


def llr_from_channel(y: np.ndarray, sigma: float) -> np.ndarray:
    return 2.0 * y / (sigma * sigma)


def quantize_llr(L: np.ndarray, scale: float = LLR_SCALE) -> np.ndarray:
    mag = np.floor(np.abs(L) * scale + 0.5)
    q = np.sign(L) * np.minimum(mag, LLR_CLIP)
    return q.astype(np.int8)


def puncture(coded: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """Keep coded symbols where mask[b, t mod P] == 1, stage-major order."""
    c = np.asarray(coded)
    n, beta = c.shape
    m = np.asarray(mask, dtype=bool)
    P = m.shape[1]
    keep = m[:, np.arange(n) % P].T  # (n, beta)
    return c[keep]


def kept_symbols(n: int, mask: np.ndarray) -> int:
    m = np.asarray(mask, dtype=np.int64)
    P = m.shape[1]
    per = m.sum(axis=0)
    return int(per.sum() * (n // P) + per[: n % P].sum())


def punctured_rate(mask: np.ndarray) -> float:
    m = np.asarray(mask)
    return m.shape[1] / float(m.sum())


@dataclass
class Stream:
    bits: np.ndarray           # message bits, one per trellis stage (uint8)
    llr: np.ndarray            # int8 (punctured stream if mask given, else (n, beta))
    ebn0_db: float
    sigma: float


def make_stream(encode: Encoder, beta: int, n: int, ebn0_db: float, seed: int, mask: np.ndarray | None = None,
                tail: int = 0, quantize: bool = True) -> Stream:
    """Message of n - tail random bits (+ tail zeros), encoded, punctured, sent over BPSK/AWGN."""
    g = rng(seed)
    bits = np.zeros(n, dtype=np.uint8)
    bits[: n - tail] = info_bits(n - tail, g)
    coded = encode(bits)
    if mask is not None:
        sym = puncture(coded, mask)
        rate = punctured_rate(mask)  # info bits per transmitted symbol
    else:
        sym = coded.reshape(-1)
        rate = 1.0 / beta
    sigma = noise_sigma(ebn0_db, rate)
    L = llr_from_channel(bpsk_awgn(sym, sigma, g), sigma)
    if quantize:
        llr = quantize_llr(L)
    else:
        llr = L.astype(np.float32)
    if mask is None:
        llr = llr.reshape(n, beta)
    return Stream(bits=bits, llr=llr, ebn0_db=ebn0_db, sigma=sigma)


@dataclass
class FrameSpec:
    code: int        # index into the code list of the batch
    n_info: int
    ebn0_db: float
    seed: int


def mixed_batch_spec(nframes: int, seed: int, lo: int = 40, hi: int = 6144, ebn0=(1.0, 5.0)) -> list[FrameSpec]:
    """Uneven-length frames: half on code 0, half on code 1, in shuffled order.

    Info lengths are uniform in [lo, hi]; Eb/N0 uniform in the given range."""
    g = rng(seed)
    lens = g.integers(lo, hi + 1, size=nframes)
    snr = g.uniform(ebn0[0], ebn0[1], size=nframes)
    codes = np.array([0] * (nframes // 2) + [1] * (nframes - nframes // 2))
    g.shuffle(codes)
    return [FrameSpec(int(codes[i]), int(lens[i]), float(snr[i]), seed * 1_000_003 + i) for i in range(nframes)]


def float_frames(encode: Encoder, beta: int, K: int, nframes: int, n_info: int, ebn0_db: float,
                 seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Zero-terminated frames with FP32 LLRs L = 2y/sigma^2: (bits (F, n), llr (F, n, beta))."""
    n = n_info + K - 1
    bits = np.zeros((nframes, n), dtype=np.uint8)
    llr = np.zeros((nframes, n, beta), dtype=np.float32)
    for i in range(nframes):
        s = make_stream(encode, beta, n, ebn0_db, seed * 1_000_003 + i, tail=K - 1, quantize=False)
        bits[i] = s.bits
        llr[i] = s.llr.reshape(n, beta)
    return bits, llr


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """LSB-first packing: bit t -> byte t >> 3, bit t & 7."""
    return np.packbits(np.asarray(bits, dtype=np.uint8), bitorder="little")


def unpack_bits(packed: np.ndarray, n: int) -> np.ndarray:
    return np.unpackbits(np.asarray(packed, dtype=np.uint8), bitorder="little")[:n]
