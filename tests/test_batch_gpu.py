"""Batched decoding (vit_batch_plan / vit_batch_run) against the oracle:
mixed codes and uneven frame lengths as concurrent per-code launches or one
persistent launch, graph replay, CTA sizes, and agreement with per-frame
launches."""
import numpy as np
import pytest
import torch

import oracle
from paper_2011_09337_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vit():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2011_09337_gb300 import vit as v
    v.load()
    return v


def _mixed_frames(nframes, hi, seed):
    spec = synth.mixed_batch_spec(nframes, seed, lo=40, hi=hi)
    codes = [synth.CODE_K7_R13, synth.CODE_K9_R12]
    frames = []
    for fs in spec:
        K, beta, polys = codes[fs.code]
        n = fs.n_info + K - 1
        s = synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, n, fs.ebn0_db, fs.seed, tail=K - 1)
        frames.append((fs.code, n, s))
    return codes, frames


@pytest.mark.parametrize("tiling", [((256, 48), (256, 64)), ((0, 0), (0, 0)), ((512, 40), (1024, 72))])
def test_mixed_codes_one_launch(vit, tiling):
    codes, frames = _mixed_frames(150, 2500, seed=2)
    cobj = [vit.Code(*codes[i], f=tiling[i][0], v=tiling[i][1], mode=vit.TERMINATED) for i in range(2)]
    dev = torch.device("cuda")
    ins, outs, specs = [], [], []
    for ci, n, s in frames:
        c = cobj[ci]
        x = torch.from_numpy(s.llr.reshape(-1)).to(dev)
        o = torch.zeros((c.output_bits(n) + 7) // 8, dtype=torch.uint8, device=dev)
        ins.append(x)
        outs.append(o)
        specs.append((c, x, n, vit.TERMINATED, o))
    for warps, persistent in ((4, False), (1, False), (8, False), (4, True), (2, True)):
        for o in outs:
            o.fill_(0xAA)
        b = vit.Batch(specs, graph=True, warps=warps, persistent=persistent)
        b.run()
        b.run()  # replay of the captured graph
        # a copy queued right behind the batch on the same stream must see
        # every group's output (the groups after the first are launched as
        # programmatic dependents): clear, run, copy, with no sync between
        torch.cuda.synchronize()
        want_all = torch.cat(outs)
        for o in outs:
            o.fill_(0xAA)
        b.run()
        snap = torch.cat(outs)
        torch.cuda.synchronize()
        assert torch.equal(snap, want_all), (warps, persistent)
        for k, (ci, n, s) in enumerate(frames):
            K, beta, polys = codes[ci]
            f, v = tiling[ci]
            want = oracle.viterbi_blocked(K, beta, polys, s.llr, f, v, v, oracle.TERMINATED)[: n - (K - 1)]
            got = synth.unpack_bits(outs[k].cpu().numpy(), n - (K - 1))
            np.testing.assert_array_equal(got, want, err_msg=f"frame {k} code {ci} n={n} warps={warps} "
                                                             f"persistent={persistent}")
    # per-frame launches give the same bits
    for k, (ci, n, s) in enumerate(frames[:20]):
        one = vit.decode(cobj[ci], ins[k], n)
        torch.cuda.synchronize()
        assert torch.equal(one, outs[k])


def test_single_code_streams_and_puncturing(vit):
    K, beta, polys = synth.CODE_K7_R12
    dev = torch.device("cuda")
    plain = vit.Code(K, beta, polys, f=1024, v=48)
    punct = vit.Code(K, beta, polys, f=2048, v=64, puncture=synth.PUNCT_R34)
    specs, checks = [], []
    for i, n in enumerate((70000, 5000, 123457)):
        s = synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, n, 2.0 + i, seed=30 + i)
        x = torch.from_numpy(s.llr.reshape(-1)).to(dev)
        o = torch.zeros((n + 7) // 8, dtype=torch.uint8, device=dev)
        specs.append((plain, x, n, vit.STREAM, o))
        checks.append((s.llr, n, 1024, 48, o))
    for i, n in enumerate((40000, 3001)):
        s = synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, n, 4.0, seed=40 + i,
                              mask=synth.PUNCT_R34)
        x = torch.from_numpy(s.llr).to(dev)
        o = torch.zeros((n + 7) // 8, dtype=torch.uint8, device=dev)
        specs.append((punct, x, n, vit.STREAM, o))
        checks.append((oracle.depuncture(s.llr, n, beta, synth.PUNCT_R34), n, 2048, 64, o))
    b = vit.Batch(specs, graph=False)
    b.run()
    torch.cuda.synchronize()
    for llr, n, f, v, o in checks:
        want = oracle.viterbi_blocked(K, beta, polys, llr, f, v, v)
        np.testing.assert_array_equal(synth.unpack_bits(o.cpu().numpy(), n), want)
