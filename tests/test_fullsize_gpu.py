"""The benchmark's own step at full size: seven 2^24-bit K=7 (171,133)
streams at Eb/N0 0..6 dB, f = 1024, v1 = v2 = 48, decoded by one planned
batch replayed from a CUDA graph (the launch the headline number times).
Tiles are sampled against the oracle (first, second and last tile of every
stream plus random ones), and the host-staged batch that the end-to-end
number times must give the same bytes."""
import numpy as np
import pytest
import torch

import oracle
from paper_2011_09337_gb300 import synth

pytestmark = pytest.mark.gpu

K, BETA, POLYS = 7, 2, (0o171, 0o133)
N, F, V = 1 << 24, 1024, 48


@pytest.fixture(scope="module")
def vit():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2011_09337_gb300 import vit as v
    v.load()
    return v


def test_benchmark_step_sampled_against_oracle(vit):
    enc = lambda x: oracle.encode(K, BETA, POLYS, x)
    streams = [synth.make_stream(enc, BETA, N, float(e), seed=1000 + e) for e in range(7)]
    code = vit.Code(K, BETA, POLYS, f=F, v=V)
    dev = torch.device("cuda")
    d_llr = [torch.from_numpy(s.llr.reshape(-1)).to(dev) for s in streams]
    d_out = [torch.full((N // 8,), 0xAA, dtype=torch.uint8, device=dev) for _ in streams]
    batch = vit.Batch([(code, d_llr[i], N, vit.STREAM, d_out[i]) for i in range(7)], graph=True)
    batch.run()
    batch.run()  # graph replay
    torch.cuda.synchronize()
    ntiles = N // F
    g = synth.rng(11)
    bers = []
    for i, s in enumerate(streams):
        got = synth.unpack_bits(d_out[i].cpu().numpy(), N)
        sample = np.unique(np.concatenate([[0, 1, ntiles - 1], g.integers(0, ntiles, 8)]))
        for b in sample:
            want = oracle.viterbi_blocked(K, BETA, POLYS, s.llr, F, V, V, blocks=(int(b), int(b) + 1))
            np.testing.assert_array_equal(got[b * F:(b + 1) * F], want[b * F:(b + 1) * F],
                                          err_msg=f"stream {i} tile {b}")
        bers.append(float(np.mean(got != s.bits)))
    # BER falls with Eb/N0: 0 dB is above the waterfall, 6 dB far below it
    assert bers[0] < 0.25 and bers[3] < 5e-3 and bers[6] < 1e-5, bers
    assert all(bers[i + 1] <= bers[i] for i in range(6)), bers

    # the end-to-end path: pinned host buffers through a host-staged batch
    h_llr = [torch.from_numpy(s.llr.reshape(-1)).pin_memory() for s in streams]
    h_out = [torch.zeros(N // 8, dtype=torch.uint8).pin_memory() for _ in streams]
    hb = vit.Batch([(code, h_llr[i], N, vit.STREAM, h_out[i]) for i in range(7)], graph=True, host=True)
    hb.run()
    torch.cuda.synchronize()
    for i in range(7):
        assert torch.equal(h_out[i], d_out[i].cpu()), f"stream {i}"
