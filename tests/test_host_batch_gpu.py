"""Host-staged batches (VIT_BATCH_HOST): LLRs and output bits in page-locked
host memory, copied in, decoded and copied back in chunks on plan-owned
streams.  Every output is compared with the oracle bit for bit: long
streams cut into many chunks, mixed codes with terminated and punctured
frames, whole-frame tiles (f = 0), a parallel-traceback group, chunk counts
from 1 to 64, graph replay, and a second run after the host inputs changed
(the copies happen every run)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2011_09337_gb300 import synth

pytestmark = pytest.mark.gpu

K7 = (7, 2, (0o171, 0o133))


@pytest.fixture(scope="module")
def vit():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2011_09337_gb300 import vit as v
    v.load()
    return v


def _enc(code):
    K, beta, polys = code
    return lambda x: oracle.encode(K, beta, polys, x)


def _pinned(a: np.ndarray, dtype) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to(dtype).pin_memory()


def _want(code, llr, n, f, v, mode, mask=None):
    K, beta, polys = code
    x = oracle.depuncture(llr, n, beta, mask) if mask is not None else llr
    nout = n - (K - 1) if mode == oracle.TERMINATED else n
    return oracle.viterbi_blocked(K, beta, polys, x, f, v, v, mode)[:nout], nout


def _streams(seed0):
    """Three K=7 streams (one punctured to rate 3/4) and one terminated frame,
    f = 1024, v = 48: several warp tasks each, ragged last tiles."""
    out = []
    for i, (n, mask, mode) in enumerate(((70001, None, oracle.STREAM), (40000, synth.PUNCT_R34, oracle.STREAM),
                                         (65536, None, oracle.STREAM), (9006, None, oracle.TERMINATED))):
        tail = 6 if mode == oracle.TERMINATED else 0
        s = synth.make_stream(_enc(K7), 2, n, 2.0 + i, seed=seed0 + i, mask=mask, tail=tail)
        out.append((n, mask, mode, s))
    return out


@pytest.mark.parametrize("chunks,graph", [(1, True), (3, True), (8, False), (64, True)])
def test_host_batch_matches_oracle(vit, chunks, graph):
    frames = _streams(seed0=100)
    specs, outs, wants = [], [], []
    for n, mask, mode, s in frames:
        c = vit.Code(*K7, f=1024, v=48, mode=mode, puncture=mask)
        llr = _pinned(s.llr, torch.int8)
        want, nout = _want(K7, s.llr, n, 1024, 48, mode, mask)
        out = torch.full(((nout + 7) // 8,), 0xAA, dtype=torch.uint8).pin_memory()
        specs.append((c, llr, n, mode, out))
        outs.append((out, nout))
        wants.append(want)
    b = vit.Batch(specs, graph=graph, host=True, chunks=chunks)
    for rep in range(2):  # with graph=True the second run replays the graph
        for o, _ in outs:
            o.fill_(0xAA)
        b.run()
        torch.cuda.synchronize()
        for k, ((o, nout), want) in enumerate(zip(outs, wants)):
            got = synth.unpack_bits(o.numpy(), nout)
            np.testing.assert_array_equal(got, want, err_msg=f"frame {k} run {rep}")


def test_host_batch_copies_inputs_every_run(vit):
    """The plan records host pointers, not data: new LLRs in the same pinned
    buffers give the new decode."""
    n = 50000
    a = synth.make_stream(_enc(K7), 2, n, 3.0, seed=7)
    bb = synth.make_stream(_enc(K7), 2, n, 1.0, seed=8)
    c = vit.Code(*K7, f=1024, v=48)
    llr = _pinned(a.llr, torch.int8)
    out = torch.zeros((n + 7) // 8, dtype=torch.uint8).pin_memory()
    b = vit.Batch([(c, llr, n, vit.STREAM, out)], graph=True, host=True, chunks=4)
    for s in (a, bb, a):
        llr.copy_(torch.from_numpy(s.llr.reshape(-1)))
        b.run()
        torch.cuda.synchronize()
        want, _ = _want(K7, s.llr, n, 1024, 48, oracle.STREAM)
        np.testing.assert_array_equal(synth.unpack_bits(out.numpy(), n), want)


def test_host_batch_mixed_codes(vit):
    """Two code groups (K=7 r1/3 and K=9 r1/2, terminated frames of uneven
    lengths) chunked round-robin over the groups."""
    spec = synth.mixed_batch_spec(60, seed=5, lo=40, hi=4000)
    codes = [synth.CODE_K7_R13, synth.CODE_K9_R12]
    tiling = [(256, 42), (256, 80)]
    cobj = [vit.Code(*codes[i], f=tiling[i][0], v=tiling[i][1], mode=vit.TERMINATED) for i in range(2)]
    specs, checks = [], []
    for fs in spec:
        K, beta, polys = codes[fs.code]
        n = fs.n_info + K - 1
        s = synth.make_stream(_enc(codes[fs.code]), beta, n, fs.ebn0_db, fs.seed, tail=K - 1)
        f, v = tiling[fs.code]
        want, nout = _want(codes[fs.code], s.llr, n, f, v, oracle.TERMINATED)
        out = torch.full(((nout + 7) // 8,), 0x55, dtype=torch.uint8).pin_memory()
        specs.append((cobj[fs.code], _pinned(s.llr, torch.int8), n, vit.TERMINATED, out))
        checks.append((out, nout, want))
    b = vit.Batch(specs, graph=True, host=True, chunks=6)
    b.run()
    torch.cuda.synchronize()
    for k, (o, nout, want) in enumerate(checks):
        np.testing.assert_array_equal(synth.unpack_bits(o.numpy(), nout), want, err_msg=f"frame {k}")


def test_host_batch_rejects_device_and_pageable_buffers(vit):
    c = vit.Code(*K7, f=1024, v=48)
    n = 4096
    dev_llr = torch.zeros(2 * n, dtype=torch.int8, device="cuda")
    dev_out = torch.zeros(n // 8, dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        vit.Batch([(c, dev_llr, n, vit.STREAM, dev_out)], host=True)
    # the library's own check, past the binding: a device pointer and a
    # pageable host buffer are both refused at plan time
    import ctypes
    L = vit.load()
    page = np.zeros(2 * n, dtype=np.int8)
    pin_out = torch.zeros(n // 8, dtype=torch.uint8).pin_memory()
    for llr_ptr in (dev_llr.data_ptr(), page.ctypes.data):
        arr = (vit._Frame * 1)(vit._Frame(c.handle.value, llr_ptr, n, vit.STREAM, pin_out.data_ptr()))
        h = ctypes.c_void_p()
        assert L.vit_batch_plan(ctypes.byref(h), arr, 1, vit.BATCH_HOST) == -1
        assert b"page-locked" in L.vit_last_error()


def test_host_batch_whole_frames_and_parallel_traceback(vit):
    """Frames decoded whole (f = 0: one tile each, full-frame Viterbi) next to
    a parallel-traceback group (f0 = 32, random starts) in one host-staged
    batch."""
    specs, checks = [], []
    whole = vit.Code(*K7, f=0, v=0, mode=vit.TERMINATED)
    for i, n in enumerate((70, 1030, 4102, 8000)):
        s = synth.make_stream(_enc(K7), 2, n, 3.0, seed=40 + i, tail=6)
        want, _ = oracle.viterbi_full(*K7, s.llr, oracle.TERMINATED)
        out = torch.full(((n - 6 + 7) // 8,), 0xAA, dtype=torch.uint8).pin_memory()
        specs.append((whole, _pinned(s.llr, torch.int8), n, vit.TERMINATED, out))
        checks.append((out, n - 6, np.asarray(want)[: n - 6]))
    pt = vit.Code(*K7, f=1024, v=48, pt_f0=32, pt_rule=vit.PT_RANDOM, pt_seed=9)
    for i, n in enumerate((30000, 12345)):
        s = synth.make_stream(_enc(K7), 2, n, 2.5, seed=50 + i)
        want = oracle.viterbi_blocked_pt(*K7, s.llr, 1024, 48, 48, 32, start=oracle.PT_RANDOM, seed=9)
        out = torch.full(((n + 7) // 8,), 0x55, dtype=torch.uint8).pin_memory()
        specs.append((pt, _pinned(s.llr, torch.int8), n, vit.STREAM, out))
        checks.append((out, n, want))
    b = vit.Batch(specs, graph=True, host=True, chunks=5)
    b.run()
    torch.cuda.synchronize()
    for k, (o, nout, want) in enumerate(checks):
        np.testing.assert_array_equal(synth.unpack_bits(o.numpy(), nout), want, err_msg=f"frame {k}")
