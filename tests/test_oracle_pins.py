"""Pins of the CPU oracle against facts other than itself: the paper's printed
encoder (Fig. 1 / Eq. 1), textbook distance spectra, exhaustive
maximum-likelihood search, noiseless recovery, closed forms and the
special cases that reduce one mode to another.  CPU only."""
import itertools
import os
from collections import defaultdict

import numpy as np
import pytest
from scipy.special import logsumexp

import oracle
from paper_2011_09337_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CODES = {
    "k3": (3, 2, (0o7, 0o5)),
    "k5": (5, 2, (0o23, 0o35)),
    "k7": synth.CODE_K7_R12,
    "k7r13": synth.CODE_K7_R13,
    "k9": synth.CODE_K9_R12,
    "k4b4": (4, 4, (0o13, 0o15, 0o17, 0o11)),
}


def _load_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- encoder
def test_encoder_impulse_response_matches_fig1():
    rows = _load_table("encoder_impulse_171_133.txt")
    want = np.array([[int(r[1]), int(r[2])] for r in rows], dtype=np.uint8)
    K, beta, polys = synth.CODE_K7_R12
    x = np.zeros(12, dtype=np.uint8)
    x[0] = 1
    out = oracle.encode(K, beta, polys, x)
    np.testing.assert_array_equal(out[: len(want)], want)
    assert not out[len(want):].any()  # the register empties after K stages


def test_encoder_linearity_and_shift_invariance():
    K, beta, polys = synth.CODE_K7_R12
    g = synth.rng(11)
    a, b = synth.info_bits(200, g), synth.info_bits(200, g)
    np.testing.assert_array_equal(oracle.encode(K, beta, polys, a ^ b),
                                  oracle.encode(K, beta, polys, a) ^ oracle.encode(K, beta, polys, b))
    shifted = np.concatenate([np.zeros(5, np.uint8), a])
    np.testing.assert_array_equal(oracle.encode(K, beta, polys, shifted)[5:], oracle.encode(K, beta, polys, a))


def _branch_table(K, beta, polys):
    """Output weight and next state for (state, input), using the oracle's encoder
    driven into each state (state = previous K-1 inputs, newest at the MSB)."""
    S = 1 << (K - 1)
    w = np.zeros((S, 2), dtype=int)
    nxt = np.zeros((S, 2), dtype=int)
    for s in range(S):
        prev = [(s >> m) & 1 for m in range(K - 1)]  # oldest input first (bit 0 = oldest)
        for u in (0, 1):
            c = oracle.encode(K, beta, polys, np.array(prev + [u], dtype=np.uint8))
            w[s, u] = int(c[-1].sum())
            # the state after this input, read back from an all-zero continuation
            nxt[s, u] = (u << (K - 2)) | (s >> 1)
    return w, nxt


def _spectrum(K, beta, polys, dmax):
    w, nxt = _branch_table(K, beta, polys)
    a, c = defaultdict(int), defaultdict(int)
    frontier = defaultdict(int)
    frontier[(nxt[0, 1], w[0, 1], 1)] = 1
    while frontier:
        nf = defaultdict(int)
        for (s, ow, iw), cnt in frontier.items():
            if s == 0:
                a[ow] += cnt
                c[ow] += cnt * iw
                continue
            for u in (0, 1):
                o2 = ow + w[s, u]
                if o2 <= dmax:
                    nf[(nxt[s, u], o2, iw + u)] += cnt
        frontier = nf
    return a, c


def test_encoder_state_convention_consistent():
    # the next-state rule used by the spectrum search agrees with the encoder:
    # continuing from state s with zeros must produce the zero-input response
    K, beta, polys = synth.CODE_K7_R12
    w, nxt = _branch_table(K, beta, polys)
    assert nxt[0, 0] == 0 and w[0, 0] == 0


@pytest.mark.parametrize("key", ["7 2 171,133", "9 2 561,753", "7 3 133,171,165"])
def test_distance_spectrum_textbook(key):
    rows = [r for r in _load_table("distance_spectra.txt") if " ".join(r[:3]) == key]
    K, beta = int(rows[0][0]), int(rows[0][1])
    polys = tuple(int(p, 8) for p in rows[0][2].split(","))
    dmax = max(int(r[3]) for r in rows)
    a, c = _spectrum(K, beta, polys, dmax)
    dfree = min(d for d in a if a[d] > 0)
    assert dfree == int(rows[0][3])
    for r in rows:
        d, ad, cd = int(r[3]), int(r[4]), int(r[5])
        if ad >= 0:
            assert a[d] == ad, (d, a[d])
        if cd >= 0:
            assert c[d] == cd, (d, c[d])


# ------------------------------------------------------------ brute force
def _correlate(K, beta, polys, bits, llr, start_state=0):
    """sum_t sum_b (-1)^c llr for the path of `bits` from `start_state`."""
    prev = [(start_state >> m) & 1 for m in range(K - 1)]
    c = oracle.encode(K, beta, polys, np.array(prev + list(bits), dtype=np.uint8))[K - 1:]
    sgn = 1 - 2 * c.astype(np.int64)
    return int((sgn * llr.reshape(-1, beta).astype(np.int64)).sum())


@pytest.mark.parametrize("key", ["k3", "k5", "k7", "k4b4"])
@pytest.mark.parametrize("mode", [oracle.STREAM, oracle.TERMINATED, oracle.FREE_START])
def test_full_frame_is_maximum_likelihood(key, mode):
    K, beta, polys = CODES[key]
    g = synth.rng(100 + K + 10 * mode)
    n_info = 8 if (mode == oracle.FREE_START and K >= 7) else 10
    trials = 6 if K >= 7 else 12
    for trial in range(trials):
        n = n_info + (K - 1 if mode == oracle.TERMINATED else 0)
        amp = [2, 3, 20, 127][trial % 4]  # small magnitudes force ties
        llr = g.integers(-amp, amp + 1, size=(n, beta)).astype(np.int8)
        best, nbest, bb = oracle.brute_force_ml(K, beta, polys, llr, n_info, mode)
        bits, metric = oracle.viterbi_full(K, beta, polys, llr, mode)
        assert metric == best
        if mode != oracle.FREE_START:
            assert _correlate(K, beta, polys, bits, llr) == best
        else:
            # some start state reproduces the metric along the decoded bits
            S = 1 << (K - 1)
            assert max(_correlate(K, beta, polys, bits, llr, s) for s in range(S)) == best
        if mode == oracle.TERMINATED:
            assert not bits[n_info:].any()
        if nbest == 1:
            np.testing.assert_array_equal(bits[:n_info], bb[:n_info])


def test_all_zero_llr_ties_decode_to_zero():
    # every comparison ties, so every decision is the lower predecessor and the
    # traceback starts at state 0 (the lowest index): the output is all zeros
    for key in ["k3", "k7", "k9"]:
        K, beta, polys = CODES[key]
        llr = np.zeros((300, beta), dtype=np.int8)
        for mode in (oracle.STREAM, oracle.TERMINATED, oracle.FREE_START):
            bits, metric = oracle.viterbi_full(K, beta, polys, llr, mode)
            assert not bits.any() and metric == 0
            assert not oracle.viterbi_blocked(K, beta, polys, llr, 64, 16, 16, mode).any()


def test_lower_predecessor_wins_a_constructed_tie():
    # K=3 (7,5): make the two paths into state 0 at the last stage tie exactly.
    # Message A = 0,0,0 and message B = 1,0,0 differ in the first bit; choose LLRs
    # so both have the same correlation and beat every other path.  The paths
    # merge in state 0 at the last stage, A arriving from state 0 and B from
    # state 1; the lower-predecessor rule keeps A.
    K, beta, polys = CODES["k3"]
    a = np.array([0, 0, 0], np.uint8)
    b = np.array([1, 0, 0], np.uint8)
    ca, cb = oracle.encode(K, beta, polys, a), oracle.encode(K, beta, polys, b)
    llr = np.where(ca == cb, np.where(ca == 0, 40, -40), 0).astype(np.int8)
    best, nbest, _ = oracle.brute_force_ml(K, beta, polys, llr, 1, oracle.TERMINATED)
    assert nbest == 2
    bits, metric = oracle.viterbi_full(K, beta, polys, llr, oracle.TERMINATED)
    assert metric == best
    np.testing.assert_array_equal(bits, a)


# -------------------------------------------------------- noiseless recovery
@pytest.mark.parametrize("key", ["k3", "k7", "k7r13", "k9", "k4b4"])
def test_noiseless_recovery_full_and_blocked(key):
    K, beta, polys = CODES[key]
    g = synth.rng(7 * K + beta)
    n = 3000
    bits = synth.info_bits(n, g)
    c = oracle.encode(K, beta, polys, bits)
    for amp in (1, 5, 127):
        llr = (amp * (1 - 2 * c.astype(np.int16))).astype(np.int8)
        dec, metric = oracle.viterbi_full(K, beta, polys, llr, oracle.STREAM)
        np.testing.assert_array_equal(dec, bits)
        assert metric == amp * beta * n
        for f, v in ((256, 48), (100, 7), (1, 30)):
            np.testing.assert_array_equal(oracle.viterbi_blocked(K, beta, polys, llr, f, v, v), bits)


def test_self_consistency_reencode():
    K, beta, polys = synth.CODE_K7_R12
    s = synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, 5000, 1.0, seed=5)
    bits, metric = oracle.viterbi_full(K, beta, polys, s.llr, oracle.STREAM)
    assert _correlate(K, beta, polys, bits, s.llr) == metric


def test_finite_minus_infinity_is_exact():
    # a finite "-infinity" M > 2 (K-1) beta 127 gives the same decoded bits and
    # metrics as an effectively infinite one
    for key in ["k7", "k9", "k4b4"]:
        K, beta, polys = CODES[key]
        g = synth.rng(3 + K)
        llr = np.where(g.random((2000, beta)) < 0.5, -127, 127).astype(np.int8)
        llr[::7] = g.integers(-127, 128, size=llr[::7].shape)
        for mode in (oracle.STREAM, oracle.TERMINATED):
            b1, m1 = oracle.viterbi_full(K, beta, polys, llr, mode, M=8192)
            b2, m2 = oracle.viterbi_full(K, beta, polys, llr, mode, M=1 << 50)
            np.testing.assert_array_equal(b1, b2)
            assert m1 == m2
        for f, v in ((128, 20), (7, 3)):
            np.testing.assert_array_equal(oracle.viterbi_blocked(K, beta, polys, llr, f, v, v, M=8192),
                                          oracle.viterbi_blocked(K, beta, polys, llr, f, v, v, M=1 << 50))


# ------------------------------------------------------------ blocking
def test_single_block_equals_full_frame():
    K, beta, polys = synth.CODE_K7_R12
    s = synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, 4000, 0.5, seed=9)
    full, _ = oracle.viterbi_full(K, beta, polys, s.llr)
    for f in (0, 4000, 10000):
        np.testing.assert_array_equal(oracle.viterbi_blocked(K, beta, polys, s.llr, f, 48, 48), full)


def test_blocks_are_windowed_viterbi():
    # each block equals a full-frame decode of its window: known start when the
    # window begins at stage 0, otherwise free start, traceback from the argmax
    K, beta, polys = synth.CODE_K7_R12
    s = synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, 3000, 0.0, seed=4)
    n, f, v1, v2 = 3000, 256, 40, 24
    got = oracle.viterbi_blocked(K, beta, polys, s.llr, f, v1, v2)
    for b in range((n + f - 1) // f):
        e0, e1 = b * f, min(n, (b + 1) * f)
        t0, t1 = max(0, e0 - v1), min(n, e1 + v2)
        mode = oracle.STREAM if t0 == 0 else oracle.FREE_START
        w, _ = oracle.viterbi_full(K, beta, polys, s.llr[t0:t1], mode)
        np.testing.assert_array_equal(got[e0:e1], w[e0 - t0:e1 - t0])


def test_block_range_argument_matches_whole_run():
    K, beta, polys = synth.CODE_K7_R12
    s = synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, 5000, 2.0, seed=12)
    whole = oracle.viterbi_blocked(K, beta, polys, s.llr, 512, 48, 48)
    part = np.zeros_like(whole)
    for b0, b1 in ((0, 3), (3, 4), (4, 10)):
        part |= oracle.viterbi_blocked(K, beta, polys, s.llr, 512, 48, 48, blocks=(b0, b1))
    np.testing.assert_array_equal(part, whole)


def test_long_overlap_converges_to_full_frame():
    # statistical: with v2 well beyond the convergence depth almost every bit
    # agrees with the full-frame ML decision (BER-level differences only)
    K, beta, polys = synth.CODE_K7_R12
    s = synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, 40000, 2.0, seed=21)
    full, _ = oracle.viterbi_full(K, beta, polys, s.llr)
    blk = oracle.viterbi_blocked(K, beta, polys, s.llr, 1024, 96, 96)
    assert np.mean(full != blk) < 2e-4


# ------------------------------------------------------------ puncturing
def test_depuncture_inverts_puncture_with_zeros():
    g = synth.rng(1)
    n, beta = 1001, 2
    x = g.integers(-127, 128, size=(n, beta)).astype(np.int8)
    rx = synth.puncture(x, synth.PUNCT_R34)
    assert rx.size == synth.kept_symbols(n, synth.PUNCT_R34)
    y = oracle.depuncture(rx, n, beta, synth.PUNCT_R34)
    keep = synth.PUNCT_R34.astype(bool)[:, np.arange(n) % 3].T
    np.testing.assert_array_equal(y[keep], x[keep])
    assert not y[~keep].any()
    # transmission order is stage-major: c0(3k), c1(3k), c0(3k+1), c1(3k+2)
    np.testing.assert_array_equal(rx[:4], [x[0, 0], x[0, 1], x[1, 0], x[2, 1]])


def test_punctured_noiseless_recovery_and_free_distance():
    K, beta, polys = synth.CODE_K7_R12
    g = synth.rng(2)
    bits = synth.info_bits(3000, g)
    c = oracle.encode(K, beta, polys, bits)
    rx = synth.puncture((127 * (1 - 2 * c.astype(np.int16))).astype(np.int8), synth.PUNCT_R34)
    llr = oracle.depuncture(rx, 3000, beta, synth.PUNCT_R34)
    np.testing.assert_array_equal(oracle.viterbi_full(K, beta, polys, llr)[0], bits)
    np.testing.assert_array_equal(oracle.viterbi_blocked(K, beta, polys, llr, 2048, 64, 64), bits)
    # Free distance of the rate-3/4 punctured code, searched over all nonzero
    # messages of up to 12 bits with a zero tail, at every puncturing phase.
    # Textbook pin: the IEEE 802.11a assignment (row [110] on generator 133,
    # row [101] on generator 171) has free distance 5.  The workload's literal
    # row order ([110] on 171, [101] on 133) gives 4.
    def dfree(pol, mask=synth.PUNCT_R34):
        P = mask.shape[1]
        best = 99
        for m in range(1, 1 << 12):
            msg = np.array([(m >> t) & 1 for t in range(12)] + [0] * (K - 1), dtype=np.uint8)
            cm = oracle.encode(K, beta, pol, msg)
            for ph in range(P):
                keep = mask.astype(bool)[:, (np.arange(cm.shape[0]) + ph) % P].T
                best = min(best, int(cm[keep].sum()))
        return best
    assert dfree((0o133, 0o171)) == 5
    assert dfree((0o171, 0o133)) == 4
    # the IEEE 802.11 rate-2/3 and rate-5/6 patterns on (133, 171): free
    # distances 6 and 4 (textbook values for these punctured codes)
    assert dfree((0o133, 0o171), synth.PUNCT_R23) == 6
    assert dfree((0o133, 0o171), synth.PUNCT_R56) == 4


# ------------------------------------------------------- path-metric forms
def _all_paths(K, beta, polys, n_info):
    """Every zero-terminated message and its +-1 branch symbols (for brute force)."""
    n = n_info + K - 1
    msgs = np.array(list(itertools.product([0, 1], repeat=n_info)), dtype=np.uint8)[:, ::-1]
    msgs = np.concatenate([msgs, np.zeros((msgs.shape[0], K - 1), np.uint8)], axis=1)
    sym = np.stack([1.0 - 2.0 * oracle.encode(K, beta, polys, m) for m in msgs])  # (P, n, beta)
    return msgs, sym


@pytest.mark.parametrize("key", ["k3", "k5"])
def test_metric_hard_matches_brute_force(key):
    K, beta, polys = CODES[key]
    g = synth.rng(31 + K)
    n_info = 9
    _, sym = _all_paths(K, beta, polys, n_info)
    llr = g.standard_normal((4, n_info + K - 1, beta)) * 3.0
    met, grad = oracle.metric_hard(K, beta, polys, llr)
    for i in range(4):
        scores = (sym * llr[i]).sum(axis=(1, 2))
        k = int(np.argmax(scores))
        assert met[i] == pytest.approx(scores[k], abs=1e-9)
        np.testing.assert_array_equal(grad[i], sym[k])  # continuous LLRs: unique maximiser


@pytest.mark.parametrize("key", ["k3", "k5"])
@pytest.mark.parametrize("tau", [0.5, 1.0, 2.0])
def test_metric_lse_matches_brute_force(key, tau):
    K, beta, polys = CODES[key]
    g = synth.rng(41 + K)
    n_info = 9
    _, sym = _all_paths(K, beta, polys, n_info)
    llr = g.standard_normal((3, n_info + K - 1, beta)) * 2.0
    met, grad = oracle.metric_lse(K, beta, polys, llr, tau)
    for i in range(3):
        scores = (sym * llr[i]).sum(axis=(1, 2)) / tau
        assert met[i] == pytest.approx(tau * logsumexp(scores), rel=1e-12, abs=1e-12)
        p = np.exp(scores - logsumexp(scores))
        np.testing.assert_allclose(grad[i], np.einsum("p,pnb->nb", p, sym), rtol=1e-10, atol=1e-12)


def test_metric_lse_limits_and_finite_differences():
    K, beta, polys = synth.CODE_K7_R12
    g = synth.rng(51)
    llr = g.standard_normal((2, 40, beta)) * 4.0
    hard, hgrad = oracle.metric_hard(K, beta, polys, llr)
    small, sgrad = oracle.metric_lse(K, beta, polys, llr, 1e-3)
    np.testing.assert_allclose(small, hard, atol=0.05)
    assert np.mean(np.abs(sgrad - hgrad) < 1e-3) > 0.99
    # log-sum-exp upper-bounds the max and exceeds it by at most tau*log(#paths)
    for tau in (0.5, 2.0):
        m, gr = oracle.metric_lse(K, beta, polys, llr, tau)
        assert np.all(m >= hard - 1e-9) and np.all(m <= hard + tau * 34 * np.log(2) + 1e-9)
        assert np.all(np.abs(gr) <= 1 + 1e-12)
        # central differences on a few coordinates
        eps = 1e-6
        for (i, t, b) in ((0, 3, 0), (1, 17, 1), (0, 39, 1)):
            lp, lm = llr.copy(), llr.copy()
            lp[i, t, b] += eps
            lm[i, t, b] -= eps
            fd = (oracle.metric_lse(K, beta, polys, lp[i:i + 1], tau, grad=False)[0][0]
                  - oracle.metric_lse(K, beta, polys, lm[i:i + 1], tau, grad=False)[0][0]) / (2 * eps)
            assert fd == pytest.approx(gr[i, t, b], rel=1e-5, abs=1e-7)


# ------------------------------------------------------------ synthetic inputs
def test_llr_quantiser_rounds_half_away_and_clips():
    L = np.array([0.0, 1 / 32, -1 / 32, 3 / 32, -3 / 32, 7.96875, 100.0, -100.0, 0.01])
    np.testing.assert_array_equal(synth.quantize_llr(L), [0, 1, -1, 2, -2, 127, 127, -127, 0])


def test_channel_noise_variance():
    sigma = synth.noise_sigma(3.0, 0.5)
    assert sigma ** 2 == pytest.approx(1 / (2 * 0.5 * 10 ** 0.3))
    y = synth.bpsk_awgn(np.zeros(200000, np.uint8), sigma, synth.rng(0))
    assert np.mean(y) == pytest.approx(1.0, abs=0.01)
    assert np.std(y) == pytest.approx(sigma, rel=0.01)


def test_punctured_stream_noise_uses_the_punctured_rate():
    """Eb/N0 is energy per information bit: a rate-3/4 stream carries 3/4 of a
    bit per transmitted symbol, so sigma^2 = 1 / (2 * 3/4 * Eb/N0)."""
    mask = np.array(synth.PUNCT_R34)
    assert synth.punctured_rate(mask) == pytest.approx(0.75)
    s = synth.make_stream(lambda x: np.zeros((x.size, 2), np.uint8), 2, 3000, 4.0, seed=1, mask=mask)
    assert s.sigma ** 2 == pytest.approx(1 / (2 * 0.75 * 10 ** 0.4))
    assert s.llr.size == synth.kept_symbols(3000, mask) == 4000


# ------------------------------------------------------ hard-decision input
def test_hard_decision_is_minimum_hamming_distance_decoding():
    """+-1 LLRs from received bits: the full-frame decoder returns a message
    whose codeword is at minimum Hamming distance from the received bits
    (exhaustive search over all 2^10 terminated messages)."""
    for key in ("k3", "k5", "k7"):
        K, beta, polys = CODES[key]
        g = synth.rng(40 + K)
        n_info = 10
        msgs = np.array([[(m >> t) & 1 for t in range(n_info)] + [0] * (K - 1) for m in range(1 << n_info)],
                        dtype=np.uint8)
        words = np.stack([oracle.encode(K, beta, polys, m) for m in msgs])  # (2^10, n, beta)
        for trial in range(6):
            rx = words[g.integers(0, 1 << n_info)].copy()
            flips = g.random(rx.shape) < 0.12
            rx ^= flips.astype(np.uint8)
            llr = np.where(rx == 1, -1, 1).astype(np.int8)
            bits, _ = oracle.viterbi_full(K, beta, polys, llr, oracle.TERMINATED)
            dist = (words != rx[None]).reshape(len(msgs), -1).sum(axis=1)
            got = oracle.encode(K, beta, polys, bits)
            assert int((got != rx).sum()) == int(dist.min())


def test_soft_decision_gain_of_about_two_db():
    """Sec. "Hard-decision vs. Soft-decision": soft decisions lower the BER by
    about 2.3 dB.  Fixed seeds, K=7 (171,133), f=1024, v=48: the hard-input
    BER at x + 1.5 dB is still above the soft BER at x, and at x + 3 dB below
    it (x = 3 dB)."""
    K, beta, polys = CODES["k7"]
    n = 120_000

    def ber(ebn0, hard):
        s = synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, n, ebn0, seed=3, quantize=False)
        llr = np.where(s.llr < 0, -1, 1).astype(np.int8) if hard else synth.quantize_llr(s.llr)
        return float(np.mean(oracle.viterbi_blocked(K, beta, polys, llr, 1024, 48, 48) != s.bits))

    soft3 = ber(3.0, False)
    assert 0 < soft3 < 2e-3
    assert ber(4.5, True) > soft3
    assert ber(6.0, True) < soft3
