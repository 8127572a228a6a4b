"""Parity of the CUDA decoder (through the C ABI) with the CPU oracle:
bit-exact decoded bits on seeded inputs, every frame mode, tilings that span
several warps with ragged tails, punctured streams and extreme LLRs."""
import numpy as np
import pytest
import torch

import oracle
from paper_2011_09337_gb300 import synth

pytestmark = pytest.mark.gpu

CODES = {
    "k7": synth.CODE_K7_R12,
    "k7swap": (7, 2, (0o133, 0o171)),
    "k7r13": synth.CODE_K7_R13,
    "k5": (5, 2, (0o23, 0o35)),
    "k5b3": (5, 3, (0o25, 0o33, 0o37)),
    "k3": (3, 2, (0o7, 0o5)),
    "k4b4": (4, 4, (0o13, 0o15, 0o17, 0o11)),
    "k6asym": (6, 2, (0o53, 0o46)),
    "k9": synth.CODE_K9_R12,
}


@pytest.fixture(scope="module")
def vit():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2011_09337_gb300 import vit as v
    v.load()
    return v


def _enc(code):
    K, beta, polys = code
    return lambda x: oracle.encode(K, beta, polys, x)


def _gpu_decode(vit, code, llr, f, v, mode, n, puncture=None, v1=None, v2=None):
    K, beta, polys = code
    c = vit.Code(K, beta, polys, f=f, v=v, v1=v1, v2=v2, mode=mode, puncture=puncture)
    x = torch.from_numpy(np.ascontiguousarray(llr).reshape(-1)).cuda()
    out = vit.decode(c, x, n=n)
    torch.cuda.synchronize()
    return synth.unpack_bits(out.cpu().numpy(), c.output_bits(n))


def test_encoder_matches_oracle(vit):
    for key in ("k7", "k7r13", "k4b4", "k6asym"):
        K, beta, polys = CODES[key]
        bits = synth.info_bits(10007, synth.rng(3))
        c = vit.Code(K, beta, polys)
        got = vit.encode(c, torch.from_numpy(bits).cuda()).cpu().numpy()
        np.testing.assert_array_equal(got, oracle.encode(K, beta, polys, bits))


@pytest.mark.parametrize("key", list(CODES))
@pytest.mark.parametrize("mode", [oracle.STREAM, oracle.TERMINATED, oracle.FREE_START])
def test_decode_matches_oracle(vit, key, mode):
    K, beta, polys = CODES[key]
    tail = K - 1 if mode == oracle.TERMINATED else 0
    cases = [(9000, 1024, 48, 1.0), (70 * 64 + 13, 64, 20, 0.0), (5000, 0, 0, 3.0), (300, 8, 40, 2.0),
             (4096 + 6, 512, 7, 6.0)]
    for i, (n, f, v, ebn0) in enumerate(cases):
        s = synth.make_stream(_enc(CODES[key]), beta, n, ebn0, seed=100 * i + mode, tail=tail)
        want = oracle.viterbi_blocked(K, beta, polys, s.llr, f, v, v, mode)[: n - tail]
        got = _gpu_decode(vit, CODES[key], s.llr, f, v, mode, n)
        np.testing.assert_array_equal(got, want, err_msg=f"{key} mode={mode} n={n} f={f} v={v}")


def test_asymmetric_overlaps_and_tiny_frames(vit):
    K, beta, polys = CODES["k7"]
    for n, f, v1, v2 in ((1, 8, 3, 3), (2, 0, 0, 0), (7, 8, 0, 0), (64, 16, 0, 40), (1000, 32, 100, 5),
                         (2049, 2048, 64, 64)):
        s = synth.make_stream(_enc(CODES["k7"]), beta, n, 1.5, seed=n)
        want = oracle.viterbi_blocked(K, beta, polys, s.llr, f, v1, v2, oracle.STREAM)
        got = _gpu_decode(vit, CODES["k7"], s.llr, f, 0, oracle.STREAM, n, v1=v1, v2=v2)
        np.testing.assert_array_equal(got, want, err_msg=f"n={n} f={f} v1={v1} v2={v2}")


@pytest.mark.parametrize("key", ["k7", "k7r13", "k4b4"])
def test_extreme_llrs_and_ties(vit, key):
    # saturated LLRs maximise the metric spread; all-zero and +-1 LLRs force ties
    K, beta, polys = CODES[key]
    g = synth.rng(77)
    n = 20000
    llrs = [np.where(g.random((n, beta)) < 0.5, -127, 127).astype(np.int8),
            np.zeros((n, beta), np.int8),
            g.integers(-1, 2, size=(n, beta)).astype(np.int8),
            np.full((n, beta), -127, np.int8)]
    for llr in llrs:
        for f, v in ((1024, 48), (0, 0), (40, 17)):
            want = oracle.viterbi_blocked(K, beta, polys, llr, f, v, v)
            got = _gpu_decode(vit, CODES[key], llr, f, v, oracle.STREAM, n)
            np.testing.assert_array_equal(got, want, err_msg=f"f={f} v={v}")


def test_punctured_rate_three_quarters(vit):
    K, beta, polys = CODES["k7"]
    mask = synth.PUNCT_R34
    for n, f, v in ((30000, 2048, 64), (3001, 256, 10), (5000, 0, 0)):
        s = synth.make_stream(_enc(CODES["k7"]), beta, n, 4.0, seed=n, mask=mask)
        dep = oracle.depuncture(s.llr, n, beta, mask)
        want = oracle.viterbi_blocked(K, beta, polys, dep, f, v, v)
        got = _gpu_decode(vit, CODES["k7"], s.llr, f, v, oracle.STREAM, n, puncture=mask)
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("key", ["k7", "k9", "k7r13", "k5"])
@pytest.mark.parametrize("mask_name", ["PUNCT_R23", "PUNCT_R34", "PUNCT_R56", "drop_third"])
def test_arbitrary_puncturing_masks(vit, key, mask_name):
    """Rate 2/3, 3/4, 5/6 and a mask that removes every third coded bit of a
    rate-1/3 code, for K = 5, 7, 9; each decoded like the oracle's
    de-punctured stream (phase by global stage index, any f and v)."""
    K, beta, polys = CODES[key]
    if mask_name == "drop_third":
        mask = np.ones((beta, 3), np.uint8)
        mask[beta - 1, 1] = 0
        mask[0, 2] = 0
    else:
        mask = getattr(synth, mask_name)
        if mask.shape[0] != beta:
            pytest.skip("mask for rate-1/2 codes")
    for n, f, v in ((20000, 2048, 8 * (K - 1)), (3001, 256, 10), (1500, 0, 0)):
        s = synth.make_stream(_enc(CODES[key]), beta, n, 5.0, seed=n + K, mask=mask)
        dep = oracle.depuncture(s.llr, n, beta, mask)
        want = oracle.viterbi_blocked(K, beta, polys, dep, f, v, v)
        got = _gpu_decode(vit, CODES[key], s.llr, f, v, oracle.STREAM, n, puncture=mask)
        np.testing.assert_array_equal(got, want, err_msg=f"n={n} f={f} v={v}")


def test_config0_terminated_frame(vit):
    # one zero-terminated frame of 4096 info bits + 6 tail bits, Eb/N0 3 dB, full-frame decode
    K, beta, polys = CODES["k7"]
    s = synth.make_stream(_enc(CODES["k7"]), beta, 4102, 3.0, seed=0, tail=6)
    want, _ = oracle.viterbi_full(K, beta, polys, s.llr, oracle.TERMINATED)
    got = _gpu_decode(vit, CODES["k7"], s.llr, 0, 0, oracle.TERMINATED, 4102)
    np.testing.assert_array_equal(got, want[:4096])


def test_config1_full_size_sampled(vit):
    # 2^24-bit stream, f=1024, v=48 at 0 dB (most decision ties and path merges
    # happen at low SNR); tiles compared with the oracle on a sample
    K, beta, polys = CODES["k7"]
    n = 1 << 24
    s = synth.make_stream(_enc(CODES["k7"]), beta, n, 0.0, seed=1)
    got = _gpu_decode(vit, CODES["k7"], s.llr, 1024, 48, oracle.STREAM, n)
    g = synth.rng(5)
    ntiles = n // 1024
    sample = np.unique(np.concatenate([[0, 1, ntiles - 2, ntiles - 1], g.integers(0, ntiles, 60)]))
    for b in sample:
        want = oracle.viterbi_blocked(K, beta, polys, s.llr, 1024, 48, 48, blocks=(int(b), int(b) + 1))
        np.testing.assert_array_equal(got[b * 1024:(b + 1) * 1024], want[b * 1024:(b + 1) * 1024],
                                      err_msg=f"tile {b}")
    # statistical sanity against the transmitted message: at 0 dB a rate-1/2
    # K=7 code is still above its waterfall (BER near 0.15)
    assert np.mean(got != s.bits) < 0.25


def test_config4_k9_stream_sampled(vit):
    # K=9 (561,753) stream, f=2048, v=96, Eb/N0 4 dB: tiles sampled against the oracle
    K, beta, polys = CODES["k9"]
    n = 1 << 22
    s = synth.make_stream(_enc(CODES["k9"]), beta, n, 4.0, seed=4)
    got = _gpu_decode(vit, CODES["k9"], s.llr, 2048, 96, oracle.STREAM, n)
    ntiles = n // 2048
    sample = np.unique(np.concatenate([[0, 1, ntiles - 1], synth.rng(8).integers(0, ntiles, 20)]))
    for b in sample:
        want = oracle.viterbi_blocked(K, beta, polys, s.llr, 2048, 96, 96, blocks=(int(b), int(b) + 1))
        np.testing.assert_array_equal(got[b * 2048:(b + 1) * 2048], want[b * 2048:(b + 1) * 2048],
                                      err_msg=f"tile {b}")
    assert np.mean(got != s.bits) < 1e-3


def test_config4_k7_punctured_sampled(vit):
    # K=7 (171,133) punctured to rate 3/4 with [110;101], f=2048, v=64, 4 dB
    K, beta, polys = CODES["k7"]
    n = 1 << 22
    mask = synth.PUNCT_R34
    s = synth.make_stream(_enc(CODES["k7"]), beta, n, 4.0, seed=5, mask=mask)
    got = _gpu_decode(vit, CODES["k7"], s.llr, 2048, 64, oracle.STREAM, n, puncture=mask)
    dep = oracle.depuncture(s.llr, n, beta, mask)
    ntiles = n // 2048
    sample = np.unique(np.concatenate([[0, 1, ntiles - 1], synth.rng(9).integers(0, ntiles, 20)]))
    for b in sample:
        want = oracle.viterbi_blocked(K, beta, polys, dep, 2048, 64, 64, blocks=(int(b), int(b) + 1))
        np.testing.assert_array_equal(got[b * 2048:(b + 1) * 2048], want[b * 2048:(b + 1) * 2048],
                                      err_msg=f"tile {b}")


@pytest.mark.parametrize("key", ["k7", "k9", "k7r13"])
def test_hard_decision_input(vit, key):
    """vit_hard_llr expands packed received bits to +-1 LLRs; decoding them
    matches the oracle on the same +-1 LLRs (stream and punctured)."""
    K, beta, polys = CODES[key]
    for n, f, v, mask in ((50_000, 1024, 48, None), (7001, 256, 30, synth.PUNCT_R34 if beta == 2 else None)):
        s = synth.make_stream(_enc(CODES[key]), beta, n, 5.0, seed=n + K, mask=mask, quantize=False)
        rx = (s.llr.reshape(-1) < 0).astype(np.uint8)  # hard decisions of the kept symbols
        packed = torch.from_numpy(synth.pack_bits(rx)).cuda()
        llr = vit.hard_llr(packed, rx.size)
        np.testing.assert_array_equal(llr.cpu().numpy(), np.where(rx == 1, -1, 1).astype(np.int8))
        code = vit.Code(K, beta, polys, f=f, v=v, puncture=mask)
        got = synth.unpack_bits(vit.decode(code, llr, n).cpu().numpy(), n)
        pm = np.where(rx == 1, -1, 1).astype(np.int8)
        dep = pm.reshape(n, beta) if mask is None else oracle.depuncture(pm, n, beta, mask)
        np.testing.assert_array_equal(got, oracle.viterbi_blocked(K, beta, polys, dep, f, v, v))
