"""Codes with no compiled kernel: any generators for every K in [3, 9] and
beta in [2, 4] (Eq. 1, Fig. 1 define the decoder for any (beta, 1, K) code).

Such codes are decoded by kernels that take the generators at run time: one
warp per tile with decisions in global memory (frames of more than 1024
tiles, windows longer than 6144 stages, K = 8, 9, batches) and, for K <= 7,
the single-frame warp-per-tile decoder with decisions in shared memory.  Each
seeded random generator set below goes through both (where both exist), in
every frame mode, and the decoded bits are compared with the oracle element
by element.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2011_09337_gb300 import synth

pytestmark = pytest.mark.gpu

COMPILED = {(7, 2, (0o171, 0o133)), (7, 2, (0o133, 0o171)), (7, 3, (0o133, 0o171, 0o165)),
            (9, 2, (0o561, 0o753)), (3, 2, (0o7, 0o5)), (5, 2, (0o23, 0o35)), (4, 4, (0o13, 0o15, 0o17, 0o11)),
            (6, 2, (0o53, 0o46)), (5, 3, (0o25, 0o33, 0o37))}


def _random_codes():
    g = synth.rng(2024)
    out = []
    for K in range(3, 10):
        for beta in (2, 3, 4):
            if (K - 1) * beta > 32:
                continue
            while True:
                polys = tuple(int(x) for x in g.integers(1, 1 << K, size=beta))
                if (K, beta, polys) not in COMPILED:
                    break
            out.append((K, beta, polys))
    return out


CODES = _random_codes()


@pytest.fixture(scope="module")
def vit():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2011_09337_gb300 import vit as v
    v.load()
    return v


def _decode(vit, code, llr, n, f, v, mode, puncture=None):
    K, beta, polys = code
    c = vit.Code(K, beta, polys, f=f, v=v, mode=mode, puncture=puncture)
    x = torch.from_numpy(np.ascontiguousarray(llr).reshape(-1)).cuda()
    out = vit.decode(c, x, n=n)
    torch.cuda.synchronize()
    return synth.unpack_bits(out.cpu().numpy(), c.output_bits(n))


@pytest.mark.parametrize("code", CODES, ids=lambda c: f"K{c[0]}b{c[1]}_" + "_".join(oct(p)[2:] for p in c[2]))
def test_runtime_code_matches_oracle(vit, code):
    K, beta, polys = code
    assert vit.supported(K, beta, polys)
    # (n, f, v, mode, Eb/N0): > 1024 tiles and a window longer than 6144
    # stages take the decoder with decisions in global memory; 12 tiles and
    # the short full frame take the shared-memory decoder when K <= 7
    cases = [(9001, 8, 12, oracle.STREAM, 1.0), (3000, 256, 20, oracle.TERMINATED, 2.0),
             (2000, 0, 0, oracle.FREE_START, 3.0), (7000, 0, 0, oracle.TERMINATED, 1.5),
             (16 * 1100 + 7, 16, 5, oracle.FREE_START, 0.5)]
    for i, (n, f, v, mode, ebn0) in enumerate(cases):
        tail = K - 1 if mode == oracle.TERMINATED else 0
        s = synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, n, ebn0, seed=10 * i + K, tail=tail)
        want = oracle.viterbi_blocked(K, beta, polys, s.llr, f, v, v, mode)[: n - tail]
        got = _decode(vit, code, s.llr, n, f, v, mode)
        np.testing.assert_array_equal(got, want, err_msg=f"case {i}: n={n} f={f} v={v} mode={mode}")
    # saturated LLRs over a window of 9000 stages (metric renormalisation)
    g = synth.rng(K * 7 + beta)
    llr = np.where(g.random((9000, beta)) < 0.5, -127, 127).astype(np.int8)
    want = oracle.viterbi_blocked(K, beta, polys, llr, 0, 0, 0, oracle.STREAM)
    np.testing.assert_array_equal(_decode(vit, code, llr, 9000, 0, 0, oracle.STREAM), want)


def test_runtime_codes_in_a_batch_and_punctured(vit):
    """A planned batch mixing two runtime codes (K = 8 and K = 6) with a
    compiled code, graph-replayed; and a punctured runtime code."""
    codes = [(8, 2, (0o247, 0o371)), (6, 3, (0o45, 0o71, 0o13)), (7, 2, (0o171, 0o133))]
    frames, checks = [], []
    for i in range(24):
        K, beta, polys = codes[i % 3]
        n = 500 + 97 * i
        mode = (oracle.TERMINATED, oracle.STREAM)[i % 2]
        tail = K - 1 if mode == oracle.TERMINATED else 0
        s = synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, n, 2.0, seed=300 + i, tail=tail)
        c = vit.Code(K, beta, polys, f=128, v=30, mode=mode)
        o = torch.zeros((c.output_bits(n) + 7) // 8, dtype=torch.uint8, device="cuda")
        frames.append((c, torch.from_numpy(s.llr.reshape(-1)).cuda(), n, mode, o))
        checks.append((o, c.output_bits(n), oracle.viterbi_blocked(K, beta, polys, s.llr, 128, 30, 30, mode)))
    b = vit.Batch(frames, graph=True)
    for _ in range(2):
        b.run()
    torch.cuda.synchronize()
    for j, (o, nb, want) in enumerate(checks):
        np.testing.assert_array_equal(synth.unpack_bits(o.cpu().numpy(), nb), want[:nb], err_msg=f"frame {j}")
    # rate 3/4 from a runtime K = 8 code
    K, beta, polys = codes[0]
    n = 20001
    s = synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, n, 5.0, seed=77, mask=synth.PUNCT_R34)
    dep = oracle.depuncture(s.llr, n, beta, synth.PUNCT_R34)
    want = oracle.viterbi_blocked(K, beta, polys, dep, 512, 48, 48)
    got = _decode(vit, codes[0], s.llr, n, 512, 48, oracle.STREAM, puncture=synth.PUNCT_R34)
    np.testing.assert_array_equal(got, want)
