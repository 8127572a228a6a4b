"""Pins of the oracle's parallel-traceback mode (Sec. "Parallel Traceback
Algorithm", Fig. pt1): its subframe bookkeeping is checked against the
window decoder (itself pinned by brute force in test_oracle_pins.py), its
degenerate cases against the serial blocked decoder, its random start against
the published SplitMix64 outputs, and the paper's BER trends (Table III,
Fig. ber:sp) on fixed seeds.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_2011_09337_gb300 import synth

CODES = {
    "k3": (3, 2, (0o7, 0o5)),
    "k5": (5, 2, (0o23, 0o35)),
    "k7": synth.CODE_K7_R12,
    "k7r13": synth.CODE_K7_R13,
    "k9": synth.CODE_K9_R12,
}


def _noisy(key, n, seed, ebn0=2.0):
    K, beta, polys = CODES[key]
    s = synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, n, ebn0, seed)
    return s


def _windows(n, f, v1, v2, f0):
    """Blocks, subframes and traceback starts of the parallel traceback."""
    fb = n if f == 0 or f > n else f
    sub = fb if f0 == 0 or f0 > fb else f0
    out = []
    for b in range((n + fb - 1) // fb):
        e0, e1 = b * fb, min(n, (b + 1) * fb)
        t0, t1 = max(0, e0 - v1), min(n, e1 + v2)
        for s0 in range(e0, e1, sub):
            s1 = min(s0 + sub, e1)
            out.append((t0, t1, s0, s1, min(s1 + v2, t1) - 1))
    return out


def test_splitmix64_published_outputs():
    # first three outputs of SplitMix64 seeded with 0 (Steele, Lea and Flood,
    # OOPSLA 2014; the reference splitmix64.c sequence)
    assert oracle.splitmix64(0, 0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(0, 1) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64(0, 2) == 0x06C45D188009454F


@pytest.mark.parametrize("key", ["k3", "k7", "k9"])
@pytest.mark.parametrize("mode", [oracle.STREAM, oracle.TERMINATED, oracle.FREE_START])
def test_one_subframe_is_the_serial_traceback(key, mode):
    K, beta, polys = CODES[key]
    s = _noisy(key, 1500, 11)
    for f, v in [(256, 5 * (K - 1)), (100, 7), (0, 0)]:
        ref = oracle.viterbi_blocked(K, beta, polys, s.llr, f, v, v, mode)
        for f0 in (0, f if f else 1500, 10_000):
            for start in (oracle.PT_STORED, oracle.PT_RANDOM):
                got = oracle.viterbi_blocked_pt(K, beta, polys, s.llr, f, v, v, f0, start, seed=3, mode=mode)
                np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("key", ["k5", "k7", "k7r13"])
def test_subframes_are_windows_from_their_stored_argmax(key):
    """Subframe k's bits are the window [t0, u] decoded with Alg. 2's argmax
    start at its last stage u, emitting [s0, s1)."""
    K, beta, polys = CODES[key]
    n = 900
    s = _noisy(key, n, 5, ebn0=1.0)
    for f, v1, v2, f0 in [(256, 30, 21, 32), (200, 0, 9, 48), (128, 17, 0, 8), (300, 42, 45, 7)]:
        got = oracle.viterbi_blocked_pt(K, beta, polys, s.llr, f, v1, v2, f0, oracle.PT_STORED)
        for t0, t1, s0, s1, u in _windows(n, f, v1, v2, f0):
            want = oracle.viterbi_window(K, beta, polys, s.llr, t0, u + 1, t0 == 0, -1, (s0, s1))
            np.testing.assert_array_equal(got[s0:s1], want[s0:s1], err_msg=f"subframe {s0}..{s1}")


@pytest.mark.parametrize("key", ["k5", "k7", "k9"])
def test_subframes_start_at_the_splitmix_state(key):
    """With the random start, subframe k starts in the top K-1 bits of
    SplitMix64 output u (u = its first traceback stage), except where u is
    the window's last stage."""
    K, beta, polys = CODES[key]
    n = 700
    s = _noisy(key, n, 8, ebn0=1.0)
    for f, v1, v2, f0, seed in [(256, 30, 21, 32, 0), (160, 11, 5, 16, 12345), (350, 0, 64, 50, 2**63 + 7)]:
        got = oracle.viterbi_blocked_pt(K, beta, polys, s.llr, f, v1, v2, f0, oracle.PT_RANDOM, seed=seed)
        for t0, t1, s0, s1, u in _windows(n, f, v1, v2, f0):
            st = -1 if u == t1 - 1 else oracle.splitmix64(seed, u) >> (64 - (K - 1))
            want = oracle.viterbi_window(K, beta, polys, s.llr, t0, u + 1, t0 == 0, st, (s0, s1))
            np.testing.assert_array_equal(got[s0:s1], want[s0:s1], err_msg=f"subframe {s0}..{s1}")


@pytest.mark.parametrize("key", ["k3", "k7", "k9"])
def test_noiseless_recovery(key):
    """Noiseless +-127 LLRs: the stored argmax is the transmitted state, so
    every subframe decodes exactly for any f0 and v2; from a random state the
    survivor merges with the transmitted path within 6(K-1) stages."""
    K, beta, polys = CODES[key]
    n = 1200
    for seed in range(4):
        msg = synth.info_bits(n, synth.rng(seed))
        llr = ((1 - 2 * oracle.encode(K, beta, polys, msg).astype(np.int64)) * 127).astype(np.int8)
        for f0, v2 in [(1, 0), (8, 3), (32, 21), (100, 0)]:
            got = oracle.viterbi_blocked_pt(K, beta, polys, llr, 256, K, v2, f0, oracle.PT_STORED)
            np.testing.assert_array_equal(got, msg)
        got = oracle.viterbi_blocked_pt(K, beta, polys, llr, 256, K, 6 * (K - 1), 16, oracle.PT_RANDOM, seed=seed)
        np.testing.assert_array_equal(got, msg)


def test_terminated_frame_end_uses_state_zero():
    K, beta, polys = CODES["k7"]
    n = 600
    s = synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, n, 1.0, 4, tail=K - 1)
    got = oracle.viterbi_blocked_pt(K, beta, polys, s.llr, 256, 20, 30, 40, oracle.PT_STORED,
                                    mode=oracle.TERMINATED)
    for t0, t1, s0, s1, u in _windows(n, 256, 20, 30, 40):
        end = 0 if u == n - 1 else -1
        want = oracle.viterbi_window(K, beta, polys, s.llr, t0, u + 1, t0 == 0, end, (s0, s1))
        np.testing.assert_array_equal(got[s0:s1], want[s0:s1])


def test_ber_trends_of_table_iii_and_fig_ber_sp():
    """Fixed seeds, K=7 at 3 dB: the BER of the parallel traceback falls as
    v2 grows (Table III), and the random start is worse than the stored
    argmax start at the same v2 (Fig. ber:sp)."""
    K, beta, polys = CODES["k7"]
    n = 60_000
    s = synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, n, 3.0, 21)

    def ber(v2, start, f0=32):
        b = oracle.viterbi_blocked_pt(K, beta, polys, s.llr, 300, 21, v2, f0, start, seed=9)
        return float(np.mean(b != s.bits))

    stored = [ber(v2, oracle.PT_STORED) for v2 in (3, 9, 21, 45)]
    assert stored[0] > stored[1] > stored[3]
    assert ber(9, oracle.PT_RANDOM) > 2 * stored[1]
    assert ber(45, oracle.PT_RANDOM) >= stored[3]
