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


def test_mixed_batch_full_size_sampled(vit):
    # the benchmark's mixed batch: 4096 zero-terminated frames, info lengths
    # U[40, 6144], half K=7 r1/3, half K=9 r1/2, Eb/N0 U[1, 5] dB, at the
    # tilings its tuner settles on; one graph launch (concurrent per-code
    # launches) and the persistent two-code launch, sampled frames against
    # the oracle
    spec = synth.mixed_batch_spec(4096, 2)
    codes = [synth.CODE_K7_R13, synth.CODE_K9_R12]
    tilings = {0: (256, 42), 1: (256, 80)}
    cobj = {ci: vit.Code(*codes[ci], f=tilings[ci][0], v=tilings[ci][1], mode=vit.TERMINATED) for ci in (0, 1)}
    dev = torch.device("cuda")
    frames, specs = [], []
    for fs in spec:
        K, beta, polys = codes[fs.code]
        n = fs.n_info + K - 1
        s = synth.make_stream(lambda x, K=K, beta=beta, polys=polys: oracle.encode(K, beta, polys, x), beta, n,
                              fs.ebn0_db, fs.seed, tail=K - 1)
        x = torch.from_numpy(s.llr.reshape(-1)).to(dev)
        o = torch.full(((cobj[fs.code].output_bits(n) + 7) // 8,), 0xAA, dtype=torch.uint8, device=dev)
        frames.append((fs.code, n, s, o))
        specs.append((cobj[fs.code], x, n, vit.TERMINATED, o))
    g = synth.rng(21)
    lens = np.array([n for _, n, _, _ in frames])
    sample = np.unique(np.concatenate([[0, len(frames) - 1, int(lens.argmax()), int(lens.argmin())],
                                       g.integers(0, len(frames), 40)]))
    want = {}
    for k in sample:
        ci, n, s, _ = frames[k]
        K, beta, polys = codes[ci]
        f, v = tilings[ci]
        want[k] = oracle.viterbi_blocked(K, beta, polys, s.llr, f, v, v, oracle.TERMINATED)[: n - (K - 1)]
    for persistent in (False, True):
        for _, _, _, o in frames:
            o.fill_(0xAA)
        b = vit.Batch(specs, graph=True, persistent=persistent)
        b.run()
        b.run()
        torch.cuda.synchronize()
        for k in sample:
            ci, n, _, o = frames[k]
            got = synth.unpack_bits(o.cpu().numpy(), n - (codes[ci][0] - 1))
            np.testing.assert_array_equal(got, want[k], err_msg=f"frame {k} code {ci} n={n} persistent={persistent}")


def test_path_metric_full_size_sampled(vit):
    # the benchmark's path-metric workload: 1024 frames x 2054 stages, K=7 r1/2,
    # FP32 LLRs at 2 dB, C = 64; sampled frames against the FP64 oracle
    _, llr = synth.float_frames(lambda x: oracle.encode(K, BETA, POLYS, x), BETA, K, 1024, 2048, 2.0, seed=3)
    code = vit.Code(K, BETA, POLYS, mode=vit.TERMINATED)
    sample = [0, 1, 511, 1023] + [int(i) for i in synth.rng(22).integers(0, 1024, 4)]
    for tau in (0.0, 1.0):
        x = torch.from_numpy(llr).cuda().requires_grad_(True)
        m = vit.path_metric(x, code, tau, 64)
        m.sum().backward()
        torch.cuda.synchronize()
        got_m = m.detach().cpu().numpy().astype(np.float64)[sample]
        got_g = x.grad.cpu().numpy().astype(np.float64)[sample]
        x64 = llr[sample].astype(np.float64)
        if tau == 0.0:
            want_m, want_g = oracle.metric_hard(K, BETA, POLYS, x64)
            np.testing.assert_allclose(got_m, want_m, rtol=1e-5)
            assert np.mean(got_g != want_g) < 1e-3
        else:
            want_m, want_g = oracle.metric_lse(K, BETA, POLYS, x64, tau)
            np.testing.assert_allclose(got_m, want_m, rtol=1e-5)
            np.testing.assert_allclose(got_g, want_g, rtol=1e-3, atol=2e-4)
