"""CPU checks of the C ABI library: it loads, exports every entry point that
include/vit.h declares, and its host-side argument checking, tiling and
workspace arithmetic behave as documented.  No compute call is made."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2011_09337_gb300 import build_lib
    path = build_lib.build()
    L = ctypes.CDLL(path)
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    L.vit_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, vp, i64, i64]
    L.vit_last_error.restype = ctypes.c_char_p
    L.vit_llr_count.argtypes = [vp, i64]
    L.vit_llr_count.restype = i64
    L.vit_output_bits.argtypes = [vp, i64]
    L.vit_output_bits.restype = i64
    L.vit_decode_workspace.argtypes = [vp, i64]
    L.vit_decode_workspace.restype = ctypes.c_size_t
    L.vit_set_puncture.argtypes = [vp, vp, ctypes.c_int]
    L.vit_set_termination.argtypes = [vp, ctypes.c_int]
    L.vit_set_overlaps.argtypes = [vp, i64, i64]
    L.vit_destroy.argtypes = [vp]
    L.vit_code_supported.argtypes = [ctypes.c_int, ctypes.c_int, vp]
    L.vit_decode_ws.argtypes = [vp, vp, i64, vp, vp, ctypes.c_size_t, vp]
    return L


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        with open(os.path.join(ROOT, "include", h)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(vit_[a-z_]+)\s*\(", src))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "vit_decode" in names and "vit_metric_bwd" in names and "vit_probe_rate" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, f"declared but not exported: {missing}"


def _u32(*p):
    return ctypes.cast((ctypes.c_uint32 * len(p))(*p), ctypes.c_void_p)


def _create(lib, K, beta, polys, f, v):
    h = ctypes.c_void_p()
    rc = lib.vit_create(ctypes.byref(h), K, beta, _u32(*polys), f, v)
    return rc, h


def test_create_validates_arguments(lib):
    rc, h = _create(lib, 7, 2, (0o171, 0o133), 1024, 48)
    assert rc == 0 and h.value
    lib.vit_destroy(h)
    # invalid codes and tilings
    for args in ((2, 2, (3, 1), 0, 0), (10, 2, (1, 1), 0, 0), (7, 5, (1, 1, 1, 1, 1), 0, 0),
                 (7, 2, (0, 0o133), 0, 0), (7, 2, (0o400, 0o133), 0, 0), (9, 5, (1,) * 5, 0, 0),
                 (7, 2, (0o171, 0o133), 1001, 48), (7, 2, (0o171, 0o133), -8, 0), (7, 2, (0o171, 0o133), 8, -1)):
        rc, h = _create(lib, *args)
        assert rc == -1 and not h.value, args
        assert lib.vit_last_error()
    # a valid code with no compiled kernel is decoded by the kernels that take
    # the generators at run time; every valid code is supported
    rc, h = _create(lib, 7, 2, (0o165, 0o133), 0, 0)
    assert rc == 0 and h.value
    lib.vit_destroy(h)
    for K in range(3, 10):
        for beta in (2, 3, 4):
            ok = (K - 1) * beta <= 32
            polys = tuple((1 << (K - 1)) | (b + 1) for b in range(beta))
            assert lib.vit_code_supported(K, beta, _u32(*polys)) == int(ok), (K, beta)
            rc, h = _create(lib, K, beta, polys, 64, 10)
            assert (rc == 0) == ok, (K, beta)
            lib.vit_destroy(h)
    assert lib.vit_code_supported(7, 2, _u32(0o171, 0o133)) == 1
    assert lib.vit_code_supported(7, 2, _u32(0o400, 0o133)) == 0


def test_decoder_choice_is_validated(lib):
    lib.vit_set_decoder.argtypes = [ctypes.c_void_p, ctypes.c_int]
    rc, h = _create(lib, 7, 2, (0o171, 0o133), 1024, 48)
    assert rc == 0
    for which in (0, 1, 2, 3):
        assert lib.vit_set_decoder(h, which) == 0
    assert lib.vit_set_decoder(h, 4) == -1
    assert lib.vit_set_decoder(None, 0) == -1
    lib.vit_destroy(h)


def test_runtime_code_workspace_and_no_parallel_traceback(lib):
    """A code without a compiled kernel: one warp per tile, max(S/32, 1)
    decision words per stage, windows rounded up to 32 stages; the parallel
    traceback needs a compiled kernel."""
    lib.vit_set_parallel_traceback.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64]
    for K, polys, R in ((8, (0o247, 0o371), 4), (9, (0o457, 0o755), 8), (5, (0o27, 0o31), 1)):
        rc, h = _create(lib, K, 2, polys, 1024, 48)
        assert rc == 0
        n = 100_000
        tiles = (n + 1023) // 1024
        want = tiles * ((1120 + 31) // 32 * 32) * R * 4
        assert lib.vit_decode_workspace(h, n) == (want + 255) // 256 * 256
        assert lib.vit_set_parallel_traceback(h, 32, 0, 0) == -2
        lib.vit_destroy(h)


def test_counts_and_workspace(lib):
    rc, h = _create(lib, 7, 2, (0o171, 0o133), 1024, 48)
    assert rc == 0
    assert lib.vit_llr_count(h, 1000) == 2000
    assert lib.vit_output_bits(h, 1000) == 1000
    assert lib.vit_set_termination(h, 1) == 0
    assert lib.vit_output_bits(h, 1000) == 994
    assert lib.vit_set_termination(h, 7) == -1
    # workspace: ceil(tiles / 64) tasks x (window rounded to 2) x 32 lanes x 16 bytes
    n = 1 << 20
    tiles = n // 1024
    want = ((tiles + 63) // 64) * 1120 * 32 * 16
    assert lib.vit_decode_workspace(h, n) == (want + 255) // 256 * 256
    # rate-3/4 puncturing [110;101]: 4 symbols per 3 stages
    mask = (ctypes.c_uint8 * 6)(1, 1, 0, 1, 0, 1)
    assert lib.vit_set_puncture(h, ctypes.cast(mask, ctypes.c_void_p), 3) == 0
    assert lib.vit_llr_count(h, 3000) == 4000
    assert lib.vit_llr_count(h, 3001) == 4002
    assert lib.vit_llr_count(h, 3002) == 4003
    bad = (ctypes.c_uint8 * 6)(1, 0, 0, 1, 0, 0)
    assert lib.vit_set_puncture(h, ctypes.cast(bad, ctypes.c_void_p), 3) == -1
    assert lib.vit_set_overlaps(h, 10, -1) == -1
    lib.vit_destroy(h)


def test_decode_rejects_bad_arguments_before_any_launch(lib):
    rc, h = _create(lib, 7, 2, (0o171, 0o133), 1024, 48)
    fake = ctypes.c_void_p(0x1000)
    # null pointers, empty frame, unaligned or short workspace: all refused on the host
    assert lib.vit_decode_ws(h, None, 100, fake, fake, 1 << 30, None) == -1
    assert lib.vit_decode_ws(h, fake, 0, fake, fake, 1 << 30, None) == -1
    assert lib.vit_decode_ws(h, fake, 100, fake, ctypes.c_void_p(0x1001), 1 << 30, None) == -1
    assert lib.vit_decode_ws(h, fake, 100, fake, fake, 16, None) == -1
    assert b"workspace too small" in lib.vit_last_error()
    assert lib.vit_decode_ws(None, fake, 100, fake, fake, 1 << 30, None) == -1
    lib.vit_destroy(h)


class _VitFrame(ctypes.Structure):
    _fields_ = [("code", ctypes.c_void_p), ("llr", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("mode", ctypes.c_int), ("bits_out", ctypes.c_void_p)]


def test_batch_plan_rejects_bad_arguments_before_any_device_call(lib):
    rc, h = _create(lib, 7, 2, (0o171, 0o133), 1024, 48)
    assert rc == 0
    plan = lib.vit_batch_plan
    plan.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
    out = ctypes.c_void_p()
    fake = 0x1000  # never dereferenced: every check below fails first
    frames = (_VitFrame * 2)(_VitFrame(h.value, fake, 5000, 0, fake), _VitFrame(h.value, fake, 70, 1, fake))
    for flags, msg in ((2, b"flag"), (1 << 24, b"flag"), (9 << 8, b"warps"), (1 << 16, b"VIT_BATCH_HOST"),
                       (8 | (65 << 16), b"chunks"), (8, b"page-locked")):
        assert plan(ctypes.byref(out), ctypes.cast(frames, ctypes.c_void_p), 2, flags) == -1
        assert msg in lib.vit_last_error() and not out.value
    bad = (_VitFrame * 1)(_VitFrame(h.value, fake, 5000, 7, fake))
    assert plan(ctypes.byref(out), ctypes.cast(bad, ctypes.c_void_p), 1, 1) == -1
    assert b"mode" in lib.vit_last_error()
    short = (_VitFrame * 1)(_VitFrame(h.value, fake, 6, 1, fake))
    assert plan(ctypes.byref(out), ctypes.cast(short, ctypes.c_void_p), 1, 1) == -1
    assert plan(ctypes.byref(out), ctypes.cast(frames, ctypes.c_void_p), 0, 1) == -1
    lib.vit_destroy(h)


def test_parallel_traceback_setter_checks(lib):
    f = lib.vit_set_parallel_traceback
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64]
    rc, h = _create(lib, 7, 2, (0o171, 0o133), 1024, 48)
    assert rc == 0
    assert f(h, 32, 0, 0) == 0 and f(h, 0, 0, 0) == 0 and f(h, 64, 1, 2**64 - 1) == 0
    for f0, rule in ((12, 0), (-8, 0), (32, 2)):
        assert f(h, f0, rule, 0) == -1 and lib.vit_last_error()
    # the parallel traceback adds one byte per subframe of every tile to the scratch
    f(h, 0, 0, 0)
    base = lib.vit_decode_workspace(h, 1 << 20)
    f(h, 32, 0, 0)
    assert lib.vit_decode_workspace(h, 1 << 20) - base >= 1024 * 32
    lib.vit_destroy(h)
    rc, h = _create(lib, 9, 2, (0o561, 0o753), 2048, 96)
    assert rc == 0
    assert f(h, 32, 0, 0) == -2 and b"parallel-traceback" in lib.vit_last_error()
    lib.vit_destroy(h)


def test_metric_workspace_layout(lib):
    """vit_metric_workspace per frame: hard form = n stages x ceil(S/32)
    decision words; log-sum-exp form = (checkpoints + C segment rows) x S
    floats, then one fp64 offset per checkpoint and the forward metric; each
    frame's share rounded to 256 bytes; invalid arguments give 0."""
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    lib.vit_metric_workspace.argtypes = [vp, ctypes.c_int, i64, ctypes.c_float, ctypes.c_int]
    lib.vit_metric_workspace.restype = ctypes.c_size_t
    up = lambda x: (x + 255) // 256 * 256
    for K, polys in ((7, (0o171, 0o133)), (9, (0o561, 0o753)), (4, (0o13, 0o15))):
        rc, h = _create(lib, K, 2, polys, 0, 0)
        assert rc == 0
        S = 1 << (K - 1)
        n, F = 2054, 3
        assert lib.vit_metric_workspace(h, F, n, 0.0, 64) == F * up(n * ((S + 31) // 32) * 4)
        for C in (2, 7, 64, 4096):
            nck = (n + C - 1) // C
            assert lib.vit_metric_workspace(h, F, n, 1.0, C) == F * up((nck + C) * S * 4 + (nck + 1) * 8)
        assert lib.vit_metric_workspace(h, F, n, 1.0, 1) == 0       # C below 2
        assert lib.vit_metric_workspace(h, F, n, -1.0, 64) == 0     # negative tau
        assert lib.vit_metric_workspace(h, 0, n, 1.0, 64) == 0      # no frames
        assert lib.vit_metric_workspace(h, F, K - 1, 1.0, 64) == 0  # shorter than K stages
        lib.vit_destroy(h)
