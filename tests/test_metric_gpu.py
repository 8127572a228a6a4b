"""The differentiable path metric on the GPU against the FP64 oracle: metric
values, the hard +-1 subgradient and the log-sum-exp gradient, plus central
finite differences of the FP64 oracle metric on tiny frames."""
import numpy as np
import pytest
import torch

import oracle
from paper_2011_09337_gb300 import synth

pytestmark = pytest.mark.gpu
K, BETA, POLYS = synth.CODE_K7_R12


@pytest.fixture(scope="module")
def vit():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2011_09337_gb300 import vit as v
    v.load()
    return v


def _frames(F, n_info, ebn0, seed):
    return synth.float_frames(lambda x: oracle.encode(K, BETA, POLYS, x), BETA, K, F, n_info, ebn0, seed)


def _run(vit, llr, tau, C=64, g=None):
    code = vit.Code(K, BETA, POLYS)
    x = torch.from_numpy(llr).cuda().requires_grad_(True)
    m = vit.path_metric(x, code, tau, C)
    gm = torch.ones_like(m) if g is None else torch.from_numpy(g).cuda()
    (m * gm).sum().backward()
    torch.cuda.synchronize()
    return m.detach().cpu().numpy().astype(np.float64), x.grad.cpu().numpy().astype(np.float64)


def test_hard_metric_and_subgradient(vit):
    _, llr = _frames(64, 2048, 2.0, seed=3)
    m, g = _run(vit, llr, 0.0)
    want_m, want_g = oracle.metric_hard(K, BETA, POLYS, llr.astype(np.float64))
    np.testing.assert_allclose(m, want_m, rtol=1e-5)
    # fp32 sums can break exact near-ties differently from fp64; demand
    # agreement on all but a tiny fraction of symbols
    assert np.mean(g != want_g) < 1e-3


@pytest.mark.parametrize("tau", [0.5, 1.0, 2.0])
def test_soft_metric_and_gradient(vit, tau):
    _, llr = _frames(32, 2048, 2.0, seed=4)
    up = synth.rng(9).standard_normal(32)
    m, g = _run(vit, llr, tau, g=up.astype(np.float32))
    want_m, want_g = oracle.metric_lse(K, BETA, POLYS, llr.astype(np.float64), tau)
    np.testing.assert_allclose(m, want_m, rtol=1e-5)
    np.testing.assert_allclose(g, want_g * up[:, None, None], rtol=1e-3, atol=2e-4)


@pytest.mark.parametrize("C", [2, 7, 64, 4096])
def test_checkpoint_interval_does_not_change_the_gradient(vit, C):
    _, llr = _frames(8, 300, 1.0, seed=5)
    _, g = _run(vit, llr, 1.0, C=C)
    _, want = oracle.metric_lse(K, BETA, POLYS, llr.astype(np.float64), 1.0)
    np.testing.assert_allclose(g, want, rtol=1e-3, atol=2e-4)


@pytest.mark.parametrize("tau", [0.0, 0.5, 1.0, 2.0])
def test_finite_differences_fp64(vit, tau):
    # 8 frames x (64 + 6) stages; FP64 central differences of the oracle metric
    _, llr = _frames(8, 64, 2.0, seed=6)
    _, g = _run(vit, llr, tau)
    x = llr.astype(np.float64)
    rng = synth.rng(11)
    checked = skipped = 0
    for _ in range(40):
        i, t, b = int(rng.integers(8)), int(rng.integers(70)), int(rng.integers(2))
        eps = 1e-6 * max(1.0, abs(x[i, t, b]))
        xp, xm = x[i:i + 1].copy(), x[i:i + 1].copy()
        xp[0, t, b] += eps
        xm[0, t, b] -= eps
        if tau == 0.0:
            mp, gp = oracle.metric_hard(K, BETA, POLYS, xp)
            mm, gm = oracle.metric_hard(K, BETA, POLYS, xm)
            if not np.array_equal(gp, gm):  # a tie within 2 eps: FD undefined here
                skipped += 1
                continue
        else:
            mp = oracle.metric_lse(K, BETA, POLYS, xp, tau, grad=False)[0]
            mm = oracle.metric_lse(K, BETA, POLYS, xm, tau, grad=False)[0]
        fd = (mp[0] - mm[0]) / (2 * eps)
        assert g[i, t, b] == pytest.approx(fd, rel=1e-4, abs=1e-4), (i, t, b, tau)
        checked += 1
    assert checked >= 30, (checked, skipped)


# Codes of every (states per lane, beta) family the kernels are compiled for:
# R = 1 with S < 32 and S = 32, R = 2, 4 and 8; beta = 2, 3, 4.
OTHER_CODES = [
    (3, 2, (0o7, 0o5)),
    (4, 4, (0o13, 0o15, 0o15, 0o17)),
    (5, 3, (0o25, 0o33, 0o37)),
    (6, 2, (0o53, 0o75)),
    (7, 3, (0o133, 0o171, 0o165)),
    (8, 2, (0o247, 0o371)),
    (9, 2, (0o561, 0o753)),
    (9, 4, (0o463, 0o535, 0o733, 0o745)),
]


@pytest.mark.parametrize("code", OTHER_CODES, ids=lambda c: f"K{c[0]}b{c[1]}")
@pytest.mark.parametrize("tau", [0.0, 1.0])
def test_metric_other_codes(vit, code, tau):
    k, beta, polys = code
    _, llr = synth.float_frames(lambda x: oracle.encode(k, beta, polys, x), beta, k, 6, 90, 2.0, seed=12)
    c = vit.Code(k, beta, polys)
    x = torch.from_numpy(llr).cuda().requires_grad_(True)
    m = vit.path_metric(x, c, tau, 16)
    m.sum().backward()
    torch.cuda.synchronize()
    got_m = m.detach().cpu().numpy().astype(np.float64)
    got_g = x.grad.cpu().numpy().astype(np.float64)
    x64 = llr.astype(np.float64)
    if tau == 0.0:
        want_m, want_g = oracle.metric_hard(k, beta, polys, x64)
        np.testing.assert_allclose(got_m, want_m, rtol=1e-5, atol=1e-4)
        assert np.mean(got_g != want_g) < 1e-2
    else:
        want_m, want_g = oracle.metric_lse(k, beta, polys, x64, tau)
        np.testing.assert_allclose(got_m, want_m, rtol=1e-5, atol=1e-4)
        np.testing.assert_allclose(got_g, want_g, rtol=1e-3, atol=2e-4)


def test_soft_gradient_small_tau(vit):
    # tau = 0.05 sharpens the posteriors towards the best path; the reference
    # taken from the forward metric must keep every exponent finite
    _, llr = _frames(4, 256, 2.0, seed=13)
    up = np.ones(4, np.float32)
    m, g = _run(vit, llr, 0.05, g=up)
    want_m, want_g = oracle.metric_lse(K, BETA, POLYS, llr.astype(np.float64), 0.05)
    assert np.all(np.isfinite(g))
    np.testing.assert_allclose(m, want_m, rtol=1e-5)
    np.testing.assert_allclose(g, want_g, rtol=1e-3, atol=2e-3)


@pytest.mark.parametrize("code", [(3, 2, (0o7, 0o5)), (7, 2, (0o171, 0o133))], ids=["K3", "K7"])
@pytest.mark.parametrize("n_info", [1, 9, 26, 40])
@pytest.mark.parametrize("tau,C", [(0.0, 64), (1.0, 2), (1.0, 64)])
def test_metric_short_frames(vit, code, n_info, tau, C):
    # frames shorter than one 32-stage block, or just over one; checkpoint
    # intervals below and above the frame length
    k, beta, polys = code
    _, llr = synth.float_frames(lambda x: oracle.encode(k, beta, polys, x), beta, k, 5, n_info, 1.5, seed=14)
    c = vit.Code(k, beta, polys)
    x = torch.from_numpy(llr).cuda().requires_grad_(True)
    m = vit.path_metric(x, c, tau, C)
    m.sum().backward()
    torch.cuda.synchronize()
    got_m = m.detach().cpu().numpy().astype(np.float64)
    got_g = x.grad.cpu().numpy().astype(np.float64)
    x64 = llr.astype(np.float64)
    if tau == 0.0:
        want_m, want_g = oracle.metric_hard(k, beta, polys, x64)
        np.testing.assert_allclose(got_m, want_m, rtol=1e-5, atol=1e-4)
        assert np.mean(got_g != want_g) < 2e-2
    else:
        want_m, want_g = oracle.metric_lse(k, beta, polys, x64, tau)
        np.testing.assert_allclose(got_m, want_m, rtol=1e-5, atol=1e-4)
        np.testing.assert_allclose(got_g, want_g, rtol=1e-3, atol=2e-4)
