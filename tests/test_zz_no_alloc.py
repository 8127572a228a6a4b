"""The allocation-free decode entry point (vit_decode_noalloc).

It exists for callers that cannot allocate device memory while they decode,
such as real-time receive loops that must not call cudaMalloc or plugins that
are handed only their input and output buffers; its scratch is a fixed array
inside the library.  This test calls it through the C ABI and checks that two
calls in a row (the second finding the first call's leftovers in the shared
array) give exactly what vit_decode_ws gives with a caller-allocated
workspace, and that an oversized frame is refused.  The file name sorts last
so that a run stopping at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2011_09337_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_decode_matches_workspace_decode():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2011_09337_gb300 import vit

    L = vit.load()
    fn = L.vit_decode_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    K, beta, polys = synth.CODE_K7_R12
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(vit.STREAM, 600000, 1.0, 1), (vit.TERMINATED, 300001, 3.0, 2)]
    for mode, n, ebn0, seed in cases:
        code = vit.Code(K, beta, polys, f=1024, v=48, mode=mode)
        tail = K - 1 if mode == vit.TERMINATED else 0
        s = synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, n, ebn0, seed, tail=tail)
        llr = torch.from_numpy(s.llr.reshape(-1)).cuda()
        want = vit.decode(code, llr, n)  # vit_decode_ws with a torch-allocated workspace
        nbytes = (code.output_bits(n) + 7) // 8
        got = torch.full((nbytes,), 0xA5, dtype=torch.uint8, device="cuda")
        rc = fn(code.handle, llr.data_ptr(), n, got.data_ptr(), stream)
        assert rc == 0, L.vit_last_error()
        torch.cuda.synchronize()
        assert torch.equal(got, want)

    # a frame whose scratch exceeds the fixed array is refused before any work
    code = vit.Code(K, beta, polys, f=1024, v=48)
    big = 4_000_000
    assert code.workspace_bytes(big) > (16 << 20)
    rc = fn(code.handle, llr.data_ptr(), big, got.data_ptr(), stream)
    assert rc == -1
    assert b"scratch" in L.vit_last_error()
