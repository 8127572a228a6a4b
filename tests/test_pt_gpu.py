"""The parallel traceback (Sec. "Parallel Traceback Algorithm", Fig. pt1) on
the GPU against the oracle's parallel-traceback mode, bit for bit: stored
argmax and SplitMix64 starts, stream, terminated and free-start frames,
batches, and the 2^24-bit stream workload on sampled tiles."""
import numpy as np
import pytest
import torch

import oracle
from paper_2011_09337_gb300 import synth

pytestmark = pytest.mark.gpu

CODES = {"k7": synth.CODE_K7_R12, "k7r13": synth.CODE_K7_R13, "k5": (5, 2, (0o23, 0o35)), "k3": (3, 2, (0o7, 0o5))}


@pytest.fixture(scope="module")
def vit():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2011_09337_gb300 import vit as v
    v.load()
    return v


def _stream(key, n, seed, ebn0=1.5, tail=0):
    K, beta, polys = CODES[key]
    return synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, n, ebn0, seed, tail=tail)


@pytest.mark.parametrize("key", list(CODES))
def test_parallel_traceback_matches_oracle(vit, key):
    K, beta, polys = CODES[key]
    cases = [(70_000, 1024, 48, 48, vit.STREAM, 32, 0), (70_000, 1024, 48, 45, vit.STREAM, 32, 1),
             (4102, 0, 0, 21, vit.TERMINATED, 64, 0), (30_001, 256, 20, 9, vit.FREE_START, 8, 1),
             (77_777, 512, 33, 0, vit.TERMINATED, 56, 0), (25_000, 64, 3, 3, vit.STREAM, 16, 1),
             (9000, 200, 30, 20, vit.STREAM, 400, 1)]
    for i, (n, f, v1, v2, mode, f0, rule) in enumerate(cases):
        tail = K - 1 if mode == vit.TERMINATED else 0
        s = _stream(key, n, 100 + i, tail=tail)
        seed = 0xC0FFEE + 7 * i
        code = vit.Code(K, beta, polys, f=f, v1=v1, v2=v2, mode=mode, pt_f0=f0, pt_rule=rule, pt_seed=seed)
        got = vit.decode(code, torch.from_numpy(s.llr.reshape(-1)).cuda(), n)
        torch.cuda.synchronize()
        nout = n - tail
        want = oracle.viterbi_blocked_pt(K, beta, polys, s.llr, f, v1, v2, f0, rule, seed=seed, mode=mode)[:nout]
        np.testing.assert_array_equal(synth.unpack_bits(got.cpu().numpy(), nout), want, err_msg=f"case {i}")


def test_parallel_traceback_in_a_batch(vit):
    """Two codes, each with its own subframe length and start rule, in one
    planned batch (concurrent launches, graph replay)."""
    dev = torch.device("cuda")
    specs, checks = [], []
    for ci, (key, f0, rule, seed) in enumerate((("k7", 32, 0, 0), ("k7r13", 24, 1, 99))):
        K, beta, polys = CODES[key]
        code = vit.Code(K, beta, polys, f=512, v=40, mode=vit.TERMINATED, pt_f0=f0, pt_rule=rule, pt_seed=seed)
        for j, n in enumerate((5000, 1234, 20_000)):
            s = _stream(key, n, 200 + 10 * ci + j, tail=K - 1)
            x = torch.from_numpy(s.llr.reshape(-1)).to(dev)
            o = torch.full(((n - K + 1 + 7) // 8,), 0xAA, dtype=torch.uint8, device=dev)
            specs.append((code, x, n, vit.TERMINATED, o))
            want = oracle.viterbi_blocked_pt(K, beta, polys, s.llr, 512, 40, 40, f0, rule, seed=seed,
                                             mode=oracle.TERMINATED)[: n - K + 1]
            checks.append((o, n - K + 1, want))
    b = vit.Batch(specs, graph=True)
    b.run()
    b.run()
    torch.cuda.synchronize()
    for o, nout, want in checks:
        np.testing.assert_array_equal(synth.unpack_bits(o.cpu().numpy(), nout), want)


def test_parallel_traceback_full_size_sampled(vit):
    """2^24-bit K=7 stream, f=1024, v=48, subframes of 32: tiles sampled
    across the stream (first, last, and spread) against the oracle."""
    K, beta, polys = CODES["k7"]
    n = 1 << 24
    code = vit.Code(K, beta, polys, f=1024, v=48, pt_f0=32)
    msg = synth.info_bits(n, synth.rng(7))
    coded = vit.encode(code, torch.from_numpy(msg).cuda()).cpu().numpy()
    sigma = synth.noise_sigma(2.0, 0.5)
    llr = synth.quantize_llr(synth.llr_from_channel(synth.bpsk_awgn(coded.reshape(-1), sigma, synth.rng(8)), sigma))
    got = synth.unpack_bits(vit.decode(code, torch.from_numpy(llr).cuda(), n).cpu().numpy(), n)
    nb = n // 1024
    for b in [0, 1, 2, 63, 64, 4095, 8191, nb // 2 + 17, nb - 2, nb - 1]:
        want = oracle.viterbi_blocked_pt(K, beta, polys, llr, 1024, 48, 48, 32, blocks=(b, b + 1))
        np.testing.assert_array_equal(got[b * 1024:(b + 1) * 1024], want[b * 1024:(b + 1) * 1024],
                                      err_msg=f"tile {b}")
