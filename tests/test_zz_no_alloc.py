"""The allocation-free decode entry point (vit_decode_noalloc).

It exists for callers that cannot allocate device memory while they decode,
such as real-time receive loops that must not call cudaMalloc or plugins that
are handed only their input and output buffers; its scratch is a fixed 16 MiB
array inside the library.  This test calls it through the C ABI on frames
whose decoding uses that scratch -- the tile decoder's survivor slab (a K=7
stream of more than 1024 tiles, a K=9 frame, the parallel traceback) and the
de-punctured LLRs of a punctured frame -- twice in a row, so the second call
finds the first call's leftovers in the shared array, and checks every
output bit against the CPU oracle.  It also checks that an oversized frame is
refused.  The file name sorts last so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2011_09337_gb300 import synth

pytestmark = pytest.mark.gpu

SCRATCH = 16 << 20


def _fn(L):
    fn = L.vit_decode_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


def test_noalloc_decode_uses_its_scratch_and_matches_the_oracle():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2011_09337_gb300 import vit

    L = vit.load()
    fn = _fn(L)
    stream = torch.cuda.current_stream().cuda_stream
    K7, K9 = synth.CODE_K7_R12, synth.CODE_K9_R12
    # (name, code, f, v, mode, n, Eb/N0, seed, puncture, parallel-traceback f0)
    cases = [
        ("k7 stream, 1465 tiles (tile decoder, survivor slab)", K7, 1024, 48, vit.STREAM, 1_500_000, 1.0, 1,
         None, 0),
        ("k9 terminated frame (rotating-slot tile decoder)", K9, 2048, 96, vit.TERMINATED, 200_001, 3.0, 2,
         None, 0),
        ("k7 punctured r3/4 frame (de-punctured LLRs in scratch)", K7, 256, 10, vit.STREAM, 30_001, 4.0, 3,
         synth.PUNCT_R34, 0),
        ("k7 parallel traceback (subframes of 32)", K7, 1024, 48, vit.STREAM, 300_000, 2.0, 4, None, 32),
    ]
    for name, (K, beta, polys), f, v, mode, n, ebn0, seed, mask, f0 in cases:
        code = vit.Code(K, beta, polys, f=f, v=v, mode=mode, puncture=mask, pt_f0=f0)
        need = code.workspace_bytes(n)
        assert 0 < need <= SCRATCH, name
        tail = K - 1 if mode == vit.TERMINATED else 0
        s = synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, n, ebn0, seed, tail=tail,
                              mask=mask)
        dep = s.llr if mask is None else oracle.depuncture(s.llr, n, beta, mask)
        if f0:
            want = oracle.viterbi_blocked_pt(K, beta, polys, dep, f, v, v, f0, mode=mode)
        else:
            want = oracle.viterbi_blocked(K, beta, polys, dep, f, v, v, mode)
        nout = code.output_bits(n)
        want = want[:nout]
        llr = torch.from_numpy(np.ascontiguousarray(s.llr).reshape(-1)).cuda()
        nbytes = (nout + 7) // 8
        for call in range(2):
            got = torch.full((nbytes,), 0xA5, dtype=torch.uint8, device="cuda")
            rc = fn(code.handle, llr.data_ptr(), n, got.data_ptr(), stream)
            assert rc == 0, L.vit_last_error()
            torch.cuda.synchronize()
            np.testing.assert_array_equal(synth.unpack_bits(got.cpu().numpy(), nout), want,
                                          err_msg=f"{name}, call {call + 1}")

    # a frame whose scratch exceeds the fixed array is refused before any work
    code = vit.Code(*K7, f=1024, v=48)
    big = 4_000_000
    assert code.workspace_bytes(big) > SCRATCH
    rc = fn(code.handle, llr.data_ptr(), big, got.data_ptr(), stream)
    assert rc == -1
    assert b"scratch" in L.vit_last_error()
