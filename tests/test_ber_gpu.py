"""Measured BER of the GPU decoder against the code's union bound, and the
trends of the paper's parameter sweeps (Table II: longer v2 lowers the BER;
Table III / Fig. ber:sp: the recorded-argmax start beats the random one)."""
import pytest
import torch

from paper_2011_09337_gb300 import ber, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vit():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2011_09337_gb300 import vit as v
    v.load()
    return v


def test_measured_ber_under_the_union_bound(vit):
    K, beta, polys = synth.CODE_K7_R12
    code = vit.Code(K, beta, polys, f=1024, v=48)
    prev = 1.0
    for e in (3.0, 4.0):
        b = ber.ber(code, e, nbits=1 << 23, seed=3)
        bound = ber.union_bound(K, beta, polys, e)
        assert 0 < b < 1.5 * bound, (e, b, bound)
        assert b < prev
        prev = b


def test_sweep_trends(vit):
    K, beta, polys = synth.CODE_K7_R12
    t2 = ber.table_ii(K, beta, polys, 2.5, fs=[256], v2s=[3, 9, 45], nbits=1 << 21)
    assert t2[(256, 3)] > t2[(256, 9)] > t2[(256, 45)]
    stored = ber.table_iii(K, beta, polys, 2.5, f0s=[32], v2s=[9], rule=0, nbits=1 << 21)
    random = ber.table_iii(K, beta, polys, 2.5, f0s=[32], v2s=[9], rule=1, nbits=1 << 21)
    assert random[(32, 9)] > 2 * stored[(32, 9)]
