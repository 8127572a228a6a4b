"""CPU pin of the decoder kernel's arithmetic: the lane routine of
vit_acs.cuh, compiled for the host (tests/emu/emu_vit.cpp), runs the kernel's
packed 16-bit path metrics (biased fields, periodic renormalisation, finite
-M start, sign-bit decisions, prmt survivor layout, rotating slot map,
end-aligned windows) and must reproduce the oracle's int64 decisions bit for
bit, including saturated LLRs that maximise the metric spread."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2011_09337_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")

CODES = [("emu_k7_171_133", synth.CODE_K7_R12), ("emu_k7_133_171_165", synth.CODE_K7_R13),
         ("emu_k5_23_35", (5, 2, (0o23, 0o35))), ("emu_k3_7_5", (3, 2, (0o7, 0o5))),
         ("emu_k4_b4", (4, 4, (0o13, 0o15, 0o17, 0o11))), ("emu_k6_asym", (6, 2, (0o53, 0o46)))]


@pytest.fixture(scope="module")
def emu():
    os.makedirs(BUILD, exist_ok=True)
    out = os.path.join(BUILD, "libemu_vit.so")
    src = os.path.join(HERE, "emu", "emu_vit.cpp")
    csrc = os.path.join(os.path.dirname(HERE), "paper_2011_09337_gb300", "csrc")
    deps = [src, os.path.join(csrc, "vit_acs.cuh"), os.path.join(csrc, "vit_pt.cuh")]
    if not os.path.exists(out) or any(os.path.getmtime(d) > os.path.getmtime(out) for d in deps):
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", "-Wno-unknown-pragmas", src,
                               "-o", out + ".tmp"])
        os.replace(out + ".tmp", out)
    return ctypes.CDLL(out)


def _run(emu, fn, code, llr, f, v, mode):
    K, beta, _ = code
    n = llr.shape[0]
    nout = n - (K - 1) if mode == oracle.TERMINATED else n
    out = np.zeros((nout + 7) // 8 + 1, np.uint8)
    x = np.ascontiguousarray(llr, dtype=np.int8)
    f_ = getattr(emu, fn)
    f_.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                   ctypes.c_int, ctypes.c_void_p]
    M = 2 * (K - 1) * 127 * beta + 1
    f_(x.ctypes.data, n, f, v, v, mode, M, out.ctypes.data)
    return synth.unpack_bits(out, nout)


@pytest.mark.parametrize("fn,code", CODES)
def test_lane_routine_matches_oracle(emu, fn, code):
    K, beta, polys = code
    for i, (n, f, v, mode, ebn0) in enumerate([(5000, 1024, 48, 0, 1.0), (4102, 0, 0, 1, 3.0), (3000, 256, 20, 2, 0.0),
                                                (7777, 512, 33, 1, 2.0), (100, 8, 40, 0, 0.5),
                                                (64 * 200 + 13, 96, 16, 0, 6.0), (2500, 64, 3, 0, 2.0),
                                                (32 * 200 + 5, 32, 10, 1, 1.0), (9000, 0, 0, 0, 3.0),
                                                (3000, 40, 2, 1, 0.0), (1000, 512, 512, 2, 1.0)]):
        tail = K - 1 if mode == 1 else 0
        s = synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, n, ebn0, seed=i, tail=tail)
        want = oracle.viterbi_blocked(K, beta, polys, s.llr, f, v, v, mode)[: n - tail]
        np.testing.assert_array_equal(_run(emu, fn, code, s.llr, f, v, mode), want)


@pytest.mark.parametrize("fn,code", CODES)
def test_saturated_llrs_keep_fields_in_range(emu, fn, code):
    K, beta, polys = code
    g = synth.rng(9)
    llr = np.where(g.random((20000, beta)) < 0.5, -127, 127).astype(np.int8)
    for f, v in ((1024, 48), (0, 0), (64, 7)):
        want = oracle.viterbi_blocked(K, beta, polys, llr, f, v, v, 0)
        np.testing.assert_array_equal(_run(emu, fn, code, llr, f, v, 0), want)


PT_CODES = [("emu_pt_k7_171_133", synth.CODE_K7_R12), ("emu_pt_k7_133_171_165", synth.CODE_K7_R13),
            ("emu_pt_k5_23_35", (5, 2, (0o23, 0o35))), ("emu_pt_k3_7_5", (3, 2, (0o7, 0o5)))]


@pytest.mark.parametrize("fn,code", PT_CODES)
def test_parallel_traceback_lane_routine_matches_oracle(emu, fn, code):
    """The parallel-traceback lane routine (argmax capture in the forward
    pass, one traceback per subframe, SplitMix64 starts) against the oracle's
    parallel-traceback mode, bit for bit."""
    K, beta, polys = code
    f_ = getattr(emu, fn)
    f_.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                   ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p]
    M = 2 * (K - 1) * 127 * beta + 1
    cases = [(5000, 1024, 48, 48, 0, 32, 0), (5000, 1024, 48, 45, 0, 32, 1), (4102, 0, 0, 21, 1, 64, 0),
             (3001, 256, 20, 9, 2, 8, 1), (7777, 512, 33, 0, 1, 56, 0), (2500, 64, 3, 3, 0, 16, 1),
             (900, 96, 10, 5, 1, 96, 0), (1200, 200, 30, 20, 0, 400, 1)]
    for i, (n, f, v1, v2, mode, f0, rule) in enumerate(cases):
        tail = K - 1 if mode == 1 else 0
        s = synth.make_stream(lambda x: oracle.encode(K, beta, polys, x), beta, n, 1.5, seed=50 + i, tail=tail)
        seed = 0x5EED0000 + i
        want = oracle.viterbi_blocked_pt(K, beta, polys, s.llr, f, v1, v2, f0, rule, seed=seed, mode=mode)
        nout = n - tail
        out = np.zeros((nout + 7) // 8 + 1, np.uint8)
        x = np.ascontiguousarray(s.llr, dtype=np.int8)
        f_(x.ctypes.data, n, f, v1, v2, mode, M, f0, rule, seed, out.ctypes.data)
        np.testing.assert_array_equal(synth.unpack_bits(out, nout), want[:nout], err_msg=f"case {i}")

