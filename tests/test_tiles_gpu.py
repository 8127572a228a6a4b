"""Parity of the 64-tiles-per-warp tile decoder with the CPU oracle for every
compiled code.

Single frames of at most 1024 tiles go to the warp-per-tile decoder, so the
frames here are cut into more than 1024 tiles (f = 8 or 16): every case
below runs a tile decoder (Alg. 1 + Alg. 2 on the overlapped tiles of Fig.
relworks), including warp tasks whose last tiles are missing, a short last
tile, windows clipped at both frame ends, asymmetric overlaps, saturated and
all-zero LLRs, and an LLR buffer that starts at an odd address (byte loads
instead of the 32-bit word loads).  The K=7 rate-1/2 codes run both their
two-tiles-per-lane decoder and their spread decoder (four lanes per tile
pair).  Decoded bits are compared with ``oracle.viterbi_blocked`` element by
element.
"""
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


SPREAD = ("k7", "k7swap")  # codes with a compiled spread tile decoder


def _decoders(vit, key):
    return [vit.DECODER_TILES] + ([vit.DECODER_SPREAD] if key in SPREAD else [])


def _decode(vit, key, llr, n, f, v1, v2, mode, offset=0, decoder=None):
    """Decodes through vit_decode_ws; ``offset`` places the LLRs that many
    bytes into a larger device buffer."""
    K, beta, polys = CODES[key]
    c = vit.Code(K, beta, polys, f=f, v=v1, v1=v1, v2=v2, mode=mode,
                 decoder=vit.DECODER_TILES if decoder is None else decoder)
    flat = np.ascontiguousarray(llr).reshape(-1)
    buf = torch.zeros(flat.size + 16, dtype=torch.int8, device="cuda")
    buf[offset:offset + flat.size] = torch.from_numpy(flat).cuda()
    x = buf[offset:offset + flat.size]
    assert (x.data_ptr() % 4 == 0) == (offset % 4 == 0)
    out = vit.decode(c, x, n=n)
    torch.cuda.synchronize()
    return synth.unpack_bits(out.cpu().numpy(), c.output_bits(n))


# (n, f, v1, v2): more than 1024 tiles each, ragged last tiles and tasks
CASES = [(9001, 8, 12, 12), (16 * 1100 + 5, 16, 40, 9), (8 * 1500, 8, 0, 30)]


@pytest.mark.parametrize("key", list(CODES))
@pytest.mark.parametrize("mode", [oracle.STREAM, oracle.TERMINATED, oracle.FREE_START])
def test_tile_decoder_matches_oracle(vit, key, mode):
    K, beta, polys = CODES[key]
    tail = K - 1 if mode == oracle.TERMINATED else 0
    for i, (n, f, v1, v2) in enumerate(CASES):
        assert (n + f - 1) // f > 1024
        s = synth.make_stream(_enc(CODES[key]), beta, n, 1.0 + i, seed=1000 * i + 10 * mode + K, tail=tail)
        want = oracle.viterbi_blocked(K, beta, polys, s.llr, f, v1, v2, mode)[: n - tail]
        for d in _decoders(vit, key):
            got = _decode(vit, key, s.llr, n, f, v1, v2, mode, decoder=d)
            np.testing.assert_array_equal(got, want,
                                          err_msg=f"{key} mode={mode} n={n} f={f} v1={v1} v2={v2} decoder={d}")


@pytest.mark.parametrize("key", list(CODES))
def test_tile_decoder_extreme_llrs(vit, key):
    """Saturated +-127 LLRs (the widest metric spread the renormalisation
    must hold), all-zero LLRs and +-1 LLRs (every comparison a tie)."""
    K, beta, polys = CODES[key]
    g = synth.rng(91 + K)
    n, f, v = 8 * 1200 + 3, 8, 2 * (K - 1)
    llrs = [np.where(g.random((n, beta)) < 0.5, -127, 127).astype(np.int8),
            np.zeros((n, beta), np.int8),
            g.integers(-1, 2, size=(n, beta)).astype(np.int8)]
    for j, llr in enumerate(llrs):
        want = oracle.viterbi_blocked(K, beta, polys, llr, f, v, v)
        for d in _decoders(vit, key):
            got = _decode(vit, key, llr, n, f, v, v, oracle.STREAM, decoder=d)
            np.testing.assert_array_equal(got, want, err_msg=f"{key} llr set {j} decoder={d}")


@pytest.mark.parametrize("key", ["k7", "k7swap", "k7r13", "k9", "k4b4"])
@pytest.mark.parametrize("offset", [1, 2, 3])
def test_tile_decoder_unaligned_llrs(vit, key, offset):
    """LLRs at an address that is not a multiple of 4: the warp tasks cannot
    use 32-bit word loads and fall back to byte loads."""
    K, beta, polys = CODES[key]
    n, f, v = 16 * 1030 + 11, 16, 3 * (K - 1)
    s = synth.make_stream(_enc(CODES[key]), beta, n, 2.5, seed=offset + 7 * K)
    want = oracle.viterbi_blocked(K, beta, polys, s.llr, f, v, v)
    for d in _decoders(vit, key):
        got = _decode(vit, key, s.llr, n, f, v, v, oracle.STREAM, offset=offset, decoder=d)
        np.testing.assert_array_equal(got, want, err_msg=f"decoder={d}")


@pytest.mark.parametrize("key", ["k7", "k7r13", "k5", "k6asym"])
def test_decoder_choice(vit, key):
    """vit_set_decoder: the shared-memory warp-per-tile decoder on a frame of
    more than 1024 tiles, the tile decoder on a frame of a few tiles; both
    match the oracle.  A window longer than 6144 stages cannot use the
    shared-memory decoder."""
    K, beta, polys = CODES[key]
    for n, f, v, which in ((9001, 8, 12, vit.DECODER_SHARED), (3000, 256, 20, vit.DECODER_TILES),
                           (5000, 0, 0, vit.DECODER_TILES), (2049 * 16, 16, 30, vit.DECODER_SHARED)):
        s = synth.make_stream(_enc(CODES[key]), beta, n, 2.0, seed=n + K)
        c = vit.Code(K, beta, polys, f=f, v=v, decoder=which)
        got = synth.unpack_bits(vit.decode(c, torch.from_numpy(s.llr.reshape(-1)).cuda(), n=n).cpu().numpy(), n)
        np.testing.assert_array_equal(got, oracle.viterbi_blocked(K, beta, polys, s.llr, f, v, v),
                                      err_msg=f"n={n} f={f} decoder={which}")
    c = vit.Code(K, beta, polys, f=0, v=0, decoder=vit.DECODER_SHARED)
    x = torch.zeros(7000 * beta, dtype=torch.int8, device="cuda")
    with pytest.raises(vit.VitError):
        vit.decode(c, x, n=7000)
    if key not in SPREAD:  # no spread decoder compiled
        c = vit.Code(K, beta, polys, f=64, v=20, decoder=vit.DECODER_SPREAD)
        with pytest.raises(vit.VitError):
            vit.decode(c, x, n=7000)


def test_auto_picks_the_spread_decoder_for_few_tiles(vit):
    """A 2^21-stage K=7 stream at f=1024 has 32 warp tasks of 64 tiles; the
    automatic choice gives it the spread decoder (128 tasks of 16 tiles) and
    the bits match the oracle on sampled tiles; workspace follows the
    choice (the spread slab rounds windows to 6 stages instead of 2)."""
    K, beta, polys = CODES["k7"]
    n = 1 << 21
    s = synth.make_stream(_enc(CODES["k7"]), beta, n, 1.0, seed=21)
    x = torch.from_numpy(s.llr.reshape(-1)).cuda()
    outs = {}
    for d in (vit.DECODER_AUTO, vit.DECODER_TILES, vit.DECODER_SPREAD):
        c = vit.Code(K, beta, polys, f=1024, v=48, decoder=d)
        outs[d] = (synth.unpack_bits(vit.decode(c, x, n=n).cpu().numpy(), n), c.workspace_bytes(n))
    assert outs[vit.DECODER_AUTO][1] == outs[vit.DECODER_SPREAD][1] != outs[vit.DECODER_TILES][1]
    np.testing.assert_array_equal(outs[vit.DECODER_AUTO][0], outs[vit.DECODER_TILES][0])
    np.testing.assert_array_equal(outs[vit.DECODER_SPREAD][0], outs[vit.DECODER_TILES][0])
    for b in (0, 1, 777, 2047):
        want = oracle.viterbi_blocked(K, beta, polys, s.llr, 1024, 48, 48, blocks=(b, b + 1))
        np.testing.assert_array_equal(outs[vit.DECODER_AUTO][0][b * 1024:(b + 1) * 1024], want[b * 1024:(b + 1) * 1024])


@pytest.mark.parametrize("key", ["k7", "k9"])
def test_slab_slots_reused_beyond_one_wave(vit, key):
    """A frame with more warp tasks than the tile decoder keeps resident: the
    warps stride over the tasks and reuse their survivor-slab slots, so the
    scratch stops growing with n, and the bits still match the oracle."""
    K, beta, polys = CODES[key]
    f, v = 8, 2 * (K - 1)
    tpt = 64 if K <= 7 else 16
    n = f * tpt * 3000 + 5  # 3000 warp tasks, more than any GB300 keeps resident
    c = vit.Code(K, beta, polys, f=f, v=v)
    per_task = ((f + 2 * v + 7) // 8 * 8) * 32 * 16
    assert c.workspace_bytes(n) < 3000 * per_task
    assert c.workspace_bytes(2 * n) == c.workspace_bytes(n)
    s = synth.make_stream(_enc(CODES[key]), beta, n, 2.0, seed=K)
    want = oracle.viterbi_blocked(K, beta, polys, s.llr, f, v, v)
    got = _decode(vit, key, s.llr, n, f, v, v, oracle.STREAM)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("key,tasks", [("k7", 700), ("k9", 1000), ("k7r13", 1300)])
def test_balanced_cta_launch(vit, key, tasks):
    """Single frames whose warp tasks fill one wave unevenly with 4-warp CTAs
    (on 152 SMs: 700 tasks -> 5-warp CTAs, 1000 K=9 tasks -> 7-warp CTAs,
    1300 -> 9-warp CTAs) decode with one larger CTA per SM; every bit matches
    the oracle."""
    K, beta, polys = CODES[key]
    f, v = 8, 2 * (K - 1)
    tpt = 64 if K <= 7 else 16
    n = f * tpt * tasks - 3  # the last task one tile short, the last tile ragged
    s = synth.make_stream(_enc(CODES[key]), beta, n, 2.0, seed=40 + K)
    want = oracle.viterbi_blocked(K, beta, polys, s.llr, f, v, v)
    got = _decode(vit, key, s.llr, n, f, v, v, oracle.STREAM)
    np.testing.assert_array_equal(got, want)
