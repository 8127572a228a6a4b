"""The batch autotuner (paper_2011_09337_gb300.tune).

CPU: the selection logic on a cost table -- the chosen tiling is the fastest
candidate whose decoded bits disagree with the full-frame decode on at most
``max_disagree`` of the bits, faster candidates beyond the limit are passed
over, and the CTA size is the fastest timed one.
GPU: the tuner run on a small mixed-code batch; the plan built from its
choice decodes every frame bit-exactly like the oracle at the chosen (f, v).
"""
import numpy as np
import pytest
import torch

from paper_2011_09337_gb300 import tune


class _FakeCode:
    def __init__(self, K, beta, polys, f, v, mode):
        self.K, self.beta, self.polys, self.f, self.v, self.mode = K, beta, polys, f, v, mode

    def output_bits(self, n):
        return n


def _fake_runner(table, flips, warp_ms):
    """Costs from ``table[(f, v)]``; the output of (f, v) differs from the
    full-frame output in ``flips[(f, v)]`` bits; warps w costs warp_ms[w]."""
    nbits = 8000

    def run(frames, code_map, warps=0, reps=1):
        codes = list(code_map.values())
        if warps:
            return warp_ms[warps], None
        c = codes[0]
        k = flips.get((c.f, c.v), 0)
        bits = np.zeros(nbits, np.uint8)
        bits[:k] = 1
        out = torch.from_numpy(np.packbits(bits, bitorder="little"))
        return table.get((c.f, c.v), 0.0), out

    return run, nbits


def test_tuner_picks_fastest_within_disagreement_limit():
    cands = [(256, 42), (512, 42), (1024, 48), (0, 0)]
    table = {(256, 42): 0.5, (512, 42): 0.7, (1024, 48): 0.9, (0, 0): 3.0}
    flips = {(256, 42): 5, (512, 42): 1, (1024, 48): 0}
    run, nbits = _fake_runner(table, flips, {2: 1.3, 4: 1.1, 8: 1.2})
    frames = [(0, None, nbits, 0)]
    codes = [(7, 3, (0o133, 0o171, 0o165))]
    # 5 / 8000 = 6.25e-4 > 2e-4: the fastest candidate is passed over
    chosen, warps, report = tune.tune(frames, codes, candidates=cands, max_disagree=2e-4, runner=run,
                                      make_code=_FakeCode)
    assert (chosen[0].f, chosen[0].v) == (512, 42)
    assert chosen[0].disagree == pytest.approx(1 / nbits)
    assert warps == 4
    assert [r["f"] for r in report[0]] == [c[0] for c in cands]
    # a looser limit admits it
    chosen, _, _ = tune.tune(frames, codes, candidates=cands, max_disagree=1e-3, runner=run,
                             make_code=_FakeCode)
    assert (chosen[0].f, chosen[0].v) == (256, 42)
    # a limit of zero leaves only the exact tilings; the full frame is slowest
    chosen, _, _ = tune.tune(frames, codes, candidates=cands, max_disagree=0.0, runner=run,
                             make_code=_FakeCode)
    assert (chosen[0].f, chosen[0].v) == (1024, 48)


def test_pick_rejects_when_nothing_qualifies():
    rows = [{"f": 256, "v": 10, "ms": 1.0, "disagree": 0.1}]
    assert tune.pick(rows, 1e-3) is None
    rows.append({"f": 512, "v": 10, "ms": 2.0, "disagree": 0.0})
    best = tune.pick(rows, 1e-3)
    assert (best.f, best.v, best.ms) == (512, 10, 2.0)


def test_default_candidates_are_valid_tilings():
    for K in (3, 5, 7, 9):
        for f, v in tune.default_candidates(K):
            assert f == 0 or (f > 0 and f % 8 == 0)
            assert v >= 0
        assert (0, 7 * (K - 1)) in tune.default_candidates(K)


@pytest.mark.gpu
def test_tuned_plan_matches_oracle():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import oracle
    from paper_2011_09337_gb300 import synth, vit

    codes = [synth.CODE_K7_R13, synth.CODE_K9_R12]
    g = synth.rng(31)
    frames, truth = [], []
    for i in range(48):
        ci = i % 2
        K, beta, polys = codes[ci]
        n = int(g.integers(200, 3000)) + K - 1
        s = synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, n, float(g.uniform(1.5, 4.0)),
                              seed=500 + i, tail=K - 1)
        frames.append((ci, torch.from_numpy(s.llr.reshape(-1)).cuda(), n, vit.TERMINATED))
        truth.append(s)
    chosen, warps, _ = tune.tune(frames, codes, candidates=[(256, 42), (512, 60), (0, 0)], reps=2)
    assert warps in (2, 4, 8)
    cobj = {ci: vit.Code(*codes[ci], f=chosen[ci].f, v=chosen[ci].v, mode=vit.TERMINATED) for ci in chosen}
    outs = [torch.zeros((cobj[ci].output_bits(n) + 7) // 8, dtype=torch.uint8, device="cuda")
            for ci, _, n, _ in frames]
    vit.Batch([(cobj[ci], llr, n, vit.TERMINATED, o) for (ci, llr, n, _), o in zip(frames, outs)],
              graph=True, warps=warps).run()
    torch.cuda.synchronize()
    for (ci, _, n, _), o, s in zip(frames, outs, truth):
        K, beta, polys = codes[ci]
        ch = chosen[ci]
        want = oracle.viterbi_blocked(K, beta, polys, s.llr, ch.f, ch.v, ch.v, oracle.TERMINATED)[: n - K + 1]
        np.testing.assert_array_equal(synth.unpack_bits(o.cpu().numpy(), n - K + 1), want)
