#!/usr/bin/env python
"""Throughput benchmark of the GB300 Viterbi decoder (arxiv 2011.09337).

Workload (one step): the streaming tiled decode of a K=7 rate-1/2 code
(generators 171, 133 octal) with f=1024, v1=v2=48 over seven independent
2^24-bit streams, one per Eb/N0 in 0..6 dB (BPSK/AWGN, int8 LLRs scaled by
16), decoded by one planned batch (one kernel launch, replayed as a CUDA
graph).  Inputs are larger than L2 (235 MB of LLRs per step).

Prints one JSON line: decoded info Mbit/s, the per-frame-launch variant, the
end-to-end number through the C ABI with host buffers, the integer-ALU
roofline of the decode kernel and the CPU oracle baseline.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

K, BETA, POLYS = 7, 2, (0o171, 0o133)
F, V = 1024, 48
NBITS = 1 << 24
EBN0 = [0.0, 1.0, 2.0, 3.0, 4.0, 5.0, 6.0]
WORKLOAD = ("stream K=7 r1/2 (171,133 octal) f=1024 v1=v2=48, 7 streams x 2^24 info bits, "
            "Eb/N0 0..6 dB, int8 LLRs x16")
METRIC = "decoded Mbit/s K=7 r1/2 int8, batched vs per-frame, 1 GB300; % ALU/HBM roofline"
# algorithmic int16 operations one lane performs with one instruction of each
# class: a 32-bit add of two packed 16-bit metrics is two adds, max.u16x2 is a
# compare and a select on each of its two fields
OPS_PER_LANE_INSTR = {"iadd": 2, "imad": 2, "vmax16": 4}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p.get("sm_max_mhz", 2070.0)), float(p.get("hbm_gbs", 6800.0)), "measured"
    except OSError:
        return 2070.0, 6800.0, "fallback"


def alu_peak_leg(vit, device):
    """Measured instruction rates of the decoder's integer classes
    (vit_probe_rate: 32 warps per SM, 8 independent chain pairs per thread),
    in warp instructions per SM clock per SM, and the packed-int16 peak they
    imply: max over classes of rate x 32 lanes x algorithmic ops per lane."""
    rates, sms = {}, None
    for k in ("iadd", "imad", "vmax16", "prmt", "lop3"):
        r, _, sms = vit.probe_rate(k, 4, 8, 2000, device=device)
        rates[k] = r
    best = max(OPS_PER_LANE_INSTR, key=lambda k: rates[k] * 32 * OPS_PER_LANE_INSTR[k])
    per_clk_sm = rates[best] * 32 * OPS_PER_LANE_INSTR[best]
    return {"warp_instr_per_clk_sm": rates, "sms": sms, "int16_ops_per_clk_sm": per_clk_sm, "peak_class": best}


def fp_peak_leg(vit, device):
    """Measured FP32 and MUFU rates (vit_probe_rate), warp instructions per
    SM clock per SM: the denominators of the path-metric kernels."""
    out = {}
    for k in ("fadd", "fmax", "ex2", "lg2"):
        r, _, sms = vit.probe_rate(k, 4, 8, 1000, device=device)
        out[k] = r
    return out


# the sources of the timed kernel (the K=7 tile decoder and its launcher)
HOT_SOURCES = ("vit_acs.cuh", "vit_internal.h", "vit_codes_k7.cu")


def _kernel_source_sha() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2011_09337_gb300", "csrc")
    for name in HOT_SOURCES:
        with open(os.path.join(d, name), "rb") as fh:
            h.update(name.encode() + fh.read())
    return h.hexdigest()[:16]


def _traffic_per_launch():
    """DRAM bytes per decode launch from the committed ncu summary, if it was
    taken on the current kernel sources."""
    p = os.path.join(ROOT, "profiles", "decode_traffic.json")
    try:
        with open(p) as fh:
            t = json.load(fh)
    except OSError:
        return None
    if t.get("source_sha") != _kernel_source_sha():
        return None
    return t.get("dram_bytes_per_launch")


class ClockSampler:
    """SM clock and clock-event reasons sampled during the timed region: NVML
    (read-only queries through ctypes, every 2 ms), else nvidia-smi."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index: int):
        self.idx = cuda_index
        self.samples = []  # (sm_mhz, max_mhz, reasons bitmask)
        self._stop = threading.Event()
        self._nvml = None
        self._dev = None

    def _open_nvml(self):
        import ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
        except OSError:
            return False
        if lib.nvmlInit_v2() != 0:
            return False
        dev = ctypes.c_void_p()
        ok = False
        try:
            import torch
            p = torch.cuda.get_device_properties(self.idx)
            bus = f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0".encode()
            ok = lib.nvmlDeviceGetHandleByPciBusId_v2(ctypes.c_char_p(bus), ctypes.byref(dev)) == 0
        except Exception:
            ok = False
        if not ok:
            ok = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.idx), ctypes.byref(dev)) == 0
        if not ok:
            return False
        self._nvml, self._dev = lib, dev
        return True

    def _poll(self):
        import ctypes
        lib, dev = self._nvml, self._dev
        fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        clk, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            if lib.nvmlDeviceGetClockInfo(dev, 1, ctypes.byref(clk)) == 0 and \
                    lib.nvmlDeviceGetMaxClockInfo(dev, 1, ctypes.byref(mx)) == 0:
                r = rs.value if fn(dev, ctypes.byref(rs)) == 0 else 0
                self.samples.append((float(clk.value), float(mx.value), int(r)))
            time.sleep(0.002)

    def _smi(self):
        fields = ("clocks.sm,clocks.max.sm,clocks_event_reasons.sw_power_cap,clocks_event_reasons.hw_slowdown,"
                  "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.hw_thermal_slowdown")
        try:
            proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={fields}",
                                     "--format=csv,noheader,nounits", "-lms", "100"],
                                    stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            return
        bits = [0x4, 0x8, 0x20, 0x40]
        for line in proc.stdout:
            if self._stop.is_set():
                break
            parts = [x.strip() for x in line.split(",")]
            try:
                r = sum(b for b, v in zip(bits, parts[2:6]) if v.lower() == "active")
                self.samples.append((float(parts[0]), float(parts[1]), r))
            except (ValueError, IndexError):
                continue
        proc.terminate()

    def __enter__(self):
        target = self._poll if self._open_nvml() else self._smi
        self._t = threading.Thread(target=target, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [x[0] for x in self.samples]
        mask = 0
        for x in self.samples:
            mask |= x[2]
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": self.samples[-1][1],
                "reasons": sorted(v for k, v in self.REASONS.items() if mask & k), "samples": len(sm),
                "source": "nvml" if self._nvml is not None else "nvidia-smi"}


def aggregate(total_ms: float, steps: int, bits_per_rank_step: int, world: int, device) -> tuple[float, float]:
    """Whole-job throughput: every rank decodes its own shard (weak scaling);
    the step time is the maximum over ranks, the bits are summed."""
    import torch
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms = total_ms / steps
    return ms, bits_per_rank_step * world / (ms * 1e-3) / 1e6


def make_inputs(vit, code, device, torch, count=len(EBN0)):
    """LLR streams (int8, stage-major), encoded by the library's encoder."""
    from paper_2011_09337_gb300 import synth

    def enc(bits):
        return vit.encode(code, torch.from_numpy(bits).to(device)).cpu().numpy()

    streams = []
    for i, e in enumerate(EBN0[:count]):
        s = synth.make_stream(enc, BETA, NBITS, e, seed=1000 + i)
        streams.append(s)
    return streams


def algorithmic_ops_per_step() -> float:
    """4 integer ops (2 adds, compare, select) per state per processed stage."""
    S = 1 << (K - 1)
    ntiles = NBITS // F
    stages = 0
    for b in range(ntiles):
        e0, e1 = b * F, min((b + 1) * F, NBITS)
        stages += min(NBITS, e1 + V) - max(0, e0 - V)
    return 4.0 * S * stages * len(EBN0)


def cpu_oracle_rate(seconds: float = 12.0):
    """Times the oracle's tiled decoder on a bounded sample of the workload with
    all host cores (ctypes releases the GIL).  Returns (Mbit/s, cores, sample,
    single-core Mbit/s from the 4-tile calibration run on one thread)."""
    import oracle
    from paper_2011_09337_gb300 import synth

    cores = len(os.sched_getaffinity(0))
    n = 256 * F
    s = synth.make_stream(lambda x: oracle.encode(K, BETA, POLYS, x), BETA, n, 3.0, seed=7)
    t0 = time.perf_counter()
    oracle.viterbi_blocked(K, BETA, POLYS, s.llr, F, V, V, blocks=(1, 5))
    per_tile = (time.perf_counter() - t0) / 4
    ntiles = int(max(cores, min(255, seconds * cores / max(per_tile, 1e-6))))
    chunks = np.array_split(np.arange(1, 1 + ntiles), cores)
    t0 = time.perf_counter()
    threads = [threading.Thread(target=oracle.viterbi_blocked,
                                args=(K, BETA, POLYS, s.llr, F, V, V),
                                kwargs={"blocks": (int(c[0]), int(c[-1]) + 1)}) for c in chunks if len(c)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    dt = time.perf_counter() - t0
    return (ntiles * F / dt / 1e6, cores, f"{ntiles} tiles of 1024 bits (f=1024, v=48, 3 dB) on {cores} threads",
            F / per_tile / 1e6)


def other_configs_cpu_rate():
    """One host thread of the oracle's tiled decoder on samples of the other
    workloads: 8 tiles of the 2^26-bit K=9 stream (f=2048, v=96), 8 tiles of
    the K=7 rate-3/4 stream (f=2048, v=64, de-punctured), and 64 frames of the
    mixed batch's lengths at its tuned tilings (f=256, v=42 / 80)."""
    import oracle
    from paper_2011_09337_gb300 import synth
    out = {}
    for name, (k, b, p), f, v, mask in (("k9_stream", synth.CODE_K9_R12, 2048, 96, None),
                                       ("k7_r34_stream", synth.CODE_K7_R12, 2048, 64, synth.PUNCT_R34)):
        n = 10 * f
        st = synth.make_stream(lambda x: oracle.encode(k, b, p, x), b, n, 4.0, seed=11, mask=mask)
        llr = st.llr if mask is None else oracle.depuncture(st.llr, n, b, mask)
        t0 = time.perf_counter()
        oracle.viterbi_blocked(k, b, p, llr, f, v, v, blocks=(1, 9))
        dt = time.perf_counter() - t0
        out[name] = {"value": 8 * f / dt / 1e6, "unit": "Mbit/s", "cores": 1, "sample": f"8 tiles of {f} bits"}
    spec = synth.mixed_batch_spec(64, 2)
    codes = [synth.CODE_K7_R13, synth.CODE_K9_R12]
    fv = [(256, 42), (256, 80)]
    bits, dt = 0, 0.0
    for fs in spec:
        k, b, p = codes[fs.code]
        n = fs.n_info + k - 1
        st = synth.make_stream(lambda x: oracle.encode(k, b, p, x), b, n, fs.ebn0_db, seed=fs.seed, tail=k - 1)
        t0 = time.perf_counter()
        oracle.viterbi_blocked(k, b, p, st.llr, fv[fs.code][0], fv[fs.code][1], fv[fs.code][1], oracle.TERMINATED)
        dt += time.perf_counter() - t0
        bits += fs.n_info
    out["mixed_batch"] = {"value": bits / dt / 1e6, "unit": "Mbit/s", "cores": 1,
                          "sample": "64 frames of the mixed batch's length and code mix"}
    return out


def full_frame_oracle_sample(streams, got_bits, prefix=1 << 17, margin=1024):
    """The oracle's full-frame decoder (Alg. 1 + 2 over the whole prefix, one
    thread) on the first `prefix` stages of every stream: its rate, its BER
    against the transmitted bits, and how often the GPU's tiled decode of the
    whole stream differs from it (compared on the first prefix - margin bits,
    where the prefix's own free end no longer matters)."""
    import oracle
    m = prefix - margin
    out = {"sample": f"first {prefix} stages of each stream, compared on the first {m}", "per_ebn0": {}}
    t0 = time.perf_counter()
    for i, s in enumerate(streams):
        ff = oracle.viterbi_blocked(K, BETA, POLYS, s.llr[:prefix], 0, 0, 0, oracle.STREAM)
        out["per_ebn0"][f"{EBN0[i]:g}dB"] = {
            "full_frame_ber_vs_transmitted": float(np.mean(ff[:m] != s.bits[:m])),
            "tiled_ber_vs_transmitted": float(np.mean(got_bits[i][:m] != s.bits[:m])),
            "tiled_vs_full_frame_disagreement": float(np.mean(got_bits[i][:m] != ff[:m]))}
    dt = time.perf_counter() - t0
    out["rate"] = {"value": prefix * len(streams) / dt / 1e6, "unit": "Mbit/s", "cores": 1}
    return out


def run_reference(args):
    """--impl reference: the CPU oracle on this workload, bounded steps."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2011_09337_gb300 import synth

    cores = len(os.sched_getaffinity(0))
    n = 1024 * F
    s = synth.make_stream(lambda x: oracle.encode(K, BETA, POLYS, x), BETA, n, 3.0, seed=7)
    tiles_per_step = cores * 64
    state = {"next": 1}

    def step():
        # consecutive tiles of the sample stream, split evenly over the host cores
        first = state["next"]
        state["next"] = first + tiles_per_step if first + 2 * tiles_per_step < 1023 else 1
        chunks = np.array_split(np.arange(first, first + tiles_per_step), cores)
        ths = [threading.Thread(target=oracle.viterbi_blocked, args=(K, BETA, POLYS, s.llr, F, V, V),
                                kwargs={"blocks": (int(c[0]), int(c[-1]) + 1)}) for c in chunks if len(c)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = tiles_per_step * F / dt / 1e6
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mbit/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{tiles_per_step} tiles per step"},
        "cpu_baseline": {"value": value, "unit": "Mbit/s", "cores": cores, "kind": "oracle",
                         "sample": f"{tiles_per_step} tiles of 1024 bits per step, {cores} threads"},
        "e2e": {"value": value, "unit": "Mbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


MIX_FRAMES = 4096
MIX_WORKLOAD = ("4096 zero-terminated frames, info lengths U[40, 6144], half K=7 r1/3 (133,171,165), "
                "half K=9 r1/2 (561,753), Eb/N0 U[1, 5] dB, int8 LLRs")


def make_mixed_batch(vit, torch, device, nframes=MIX_FRAMES, seed=2):
    """Frames of the mixed batch, encoded by the library (frames of one code are
    encoded as one message: each K-1 zero tail returns the encoder to state 0)."""
    from paper_2011_09337_gb300 import synth

    spec = synth.mixed_batch_spec(nframes, seed)
    codes = [synth.CODE_K7_R13, synth.CODE_K9_R12]
    g = synth.rng(seed + 17)
    frames = []  # (code index, llr device view, n, bits)
    for ci, (K, beta, polys) in enumerate(codes):
        idx = [i for i, fs in enumerate(spec) if fs.code == ci]
        ns = [spec[i].n_info + K - 1 for i in idx]
        msg = np.zeros(sum(ns), dtype=np.uint8)
        sig = np.zeros(sum(ns) * beta)
        off = 0
        for i, n in zip(idx, ns):
            msg[off:off + spec[i].n_info] = synth.info_bits(spec[i].n_info, g)
            sig[off * beta:(off + n) * beta] = synth.noise_sigma(spec[i].ebn0_db, 1.0 / beta)
            off += n
        code = vit.Code(K, beta, polys)
        coded = vit.encode(code, torch.from_numpy(msg).to(device)).cpu().numpy().reshape(-1)
        y = (1.0 - 2.0 * coded) + sig * g.standard_normal(coded.size)
        llr = torch.from_numpy(synth.quantize_llr(2.0 * y / (sig * sig))).to(device)
        off = 0
        for i, n in zip(idx, ns):
            frames.append((ci, llr[off * beta:(off + n) * beta], n, msg[off:off + n]))
            off += n
    return codes, frames


def frame_latency_leg(vit, torch, device, steps):
    """One 4096-bit frame with its 6-bit zero tail, K=7 (171,133), full-frame
    decoding (f = 0), 3 dB: the latency of one vit_decode_ws call (one launch
    of the tile decoder on one tile), device-resident."""
    from paper_2011_09337_gb300 import synth
    n = 4096 + K - 1
    code = vit.Code(K, BETA, POLYS, f=0, v=0, mode=vit.TERMINATED)

    def enc(bits):
        return vit.encode(code, torch.from_numpy(bits).to(device)).cpu().numpy()

    st = synth.make_stream(enc, BETA, n, 3.0, seed=0, tail=K - 1)
    llr = torch.from_numpy(st.llr.reshape(-1)).to(device)
    ws = torch.empty(code.workspace_bytes(n), dtype=torch.uint8, device=device)
    o = torch.empty((n - K + 1 + 7) // 8, dtype=torch.uint8, device=device)
    for _ in range(3):
        vit.decode(code, llr, n, out=o, workspace=ws)
    torch.cuda.synchronize()
    reps = max(steps, 20)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        vit.decode(code, llr, n, out=o, workspace=ws)
    b.record()
    torch.cuda.synchronize()
    us = a.elapsed_time(b) / reps * 1e3
    got = synth.unpack_bits(o.cpu().numpy(), n - K + 1)
    return {"workload": "4096 info + 6 tail bits, K=7 (171,133), terminated, f=0 (one tile), 3 dB",
            "us_per_frame": us, "value": 4096 / us, "unit": "Mbit/s",
            "bit_errors": int(np.sum(got != st.bits[: n - K + 1]))}


def parallel_traceback_leg(vit, torch, frames_llr, out, steps):
    """The main workload decoded with the parallel traceback (Sec. "Parallel
    Traceback Algorithm"): subframes of 32 stages, each traced back over
    v2 = 48 further stages, starting at the argmax state recorded in the
    forward pass.  Reports its throughput and how many decoded bits differ
    from the serial traceback's."""
    code = vit.Code(K, BETA, POLYS, f=F, v=V, pt_f0=32)
    pt_out = [torch.zeros_like(o) for o in out]
    batch = vit.Batch([(code, x, NBITS, vit.STREAM, o) for x, o in zip(frames_llr, pt_out)], graph=True)
    for _ in range(3):
        batch.run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        batch.run()
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    diff = sum(int(np.unpackbits(torch.bitwise_xor(p, o).cpu().numpy()).sum()) for p, o in zip(pt_out, out))
    nb = NBITS * len(frames_llr)
    return {"f0": 32, "v2": V, "start": "recorded argmax", "value": nb / (ms * 1e-3) / 1e6, "unit": "Mbit/s",
            "ms_per_step": ms, "bits_differing_from_serial_traceback": diff / nb}


def shared_decoder_leg(vit, torch, frames_llr, ref_out, steps):
    """The main workload decoded by the warp-per-tile decoder whose survivor
    decisions stay in shared memory (Sec. "Unified Kernel": one warp per tile,
    9 KB of decision words per 1120-stage window, nothing written to a slab),
    one launch per stream, beside the tile decoder's survivor slab in HBM."""
    code = vit.Code(K, BETA, POLYS, f=F, v=V, decoder=vit.DECODER_SHARED)
    outs = [torch.zeros_like(o) for o in ref_out]
    for _ in range(2):
        for x, o in zip(frames_llr, outs):
            vit.decode(code, x, NBITS, out=o)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        for x, o in zip(frames_llr, outs):
            vit.decode(code, x, NBITS, out=o)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / steps
    same = all(torch.equal(o, r) for o, r in zip(outs, ref_out))
    nb = NBITS * len(frames_llr)
    return {"value": nb / (ms * 1e-3) / 1e6, "unit": "Mbit/s", "ms_per_step": ms, "matches_tile_decoder": same,
            "launches_per_step": len(frames_llr),
            "kernel": "decode_warp_kernel (one warp per tile, decisions in shared memory)"}


def mixed_batch_leg(vit, torch, device, steps):
    from paper_2011_09337_gb300 import tune

    codes, frames = make_mixed_batch(vit, torch, device)
    info_bits = sum(n - (codes[ci][0] - 1) for ci, _, n, _ in frames)
    tf = [(ci, llr, n, vit.TERMINATED) for ci, llr, n, _ in frames]
    chosen, warps, report = tune.tune(tf, codes)
    cobj = {ci: vit.Code(*codes[ci], f=chosen[ci].f, v=chosen[ci].v, mode=vit.TERMINATED) for ci in chosen}
    sizes = [(cobj[ci].output_bits(n) + 7) // 8 for ci, _, n, _ in frames]
    out = torch.zeros(sum(sizes), dtype=torch.uint8, device=device)
    specs, views, off = [], [], 0
    for (ci, llr, n, _), sz in zip(frames, sizes):
        views.append(out[off:off + sz])
        specs.append((cobj[ci], llr, n, vit.TERMINATED, views[-1]))
        off += sz
    batch = vit.Batch(specs, graph=True, warps=warps)
    for _ in range(3):
        batch.run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        batch.run()
    b.record()
    torch.cuda.synchronize()
    ms_batch = a.elapsed_time(b) / steps
    # the same plan as one persistent two-code launch over a shared task queue
    pbatch = vit.Batch(specs, graph=True, warps=warps, persistent=True)
    for _ in range(3):
        pbatch.run()
    torch.cuda.synchronize()
    a.record()
    for _ in range(steps):
        pbatch.run()
    b.record()
    torch.cuda.synchronize()
    ms_persistent = a.elapsed_time(b) / steps
    del pbatch
    # per-frame launches with the same tiling (one vit_decode_ws per frame)
    ws = torch.empty(max(cobj[ci].workspace_bytes(n) for ci, _, n, _ in frames), dtype=torch.uint8, device=device)
    pf_steps = max(1, min(steps, 3))
    for ci, llr, n, _ in frames:
        vit.decode(cobj[ci], llr, n, workspace=ws)
    torch.cuda.synchronize()
    a.record()
    for _ in range(pf_steps):
        for (ci, llr, n, _), v in zip(frames, views):
            vit.decode(cobj[ci], llr, n, out=v, workspace=ws)
    b.record()
    torch.cuda.synchronize()
    ms_pf = a.elapsed_time(b) / pf_steps
    # BER of the batched output against the transmitted bits
    batch.run()
    torch.cuda.synchronize()
    host = out.cpu().numpy()
    err, off = 0, 0
    from paper_2011_09337_gb300 import synth
    for (ci, _, n, bits), sz in zip(frames, sizes):
        nb = n - (codes[ci][0] - 1)
        err += int(np.sum(synth.unpack_bits(host[off:off + sz], nb) != bits[:nb]))
        off += sz
    return {
        "workload": MIX_WORKLOAD, "value": info_bits / (ms_batch * 1e-3) / 1e6, "unit": "Mbit/s",
        "ms_per_step": ms_batch, "per_frame": {"value": info_bits / (ms_pf * 1e-3) / 1e6, "unit": "Mbit/s",
                                               "launches_per_step": len(frames), "ms_per_step": ms_pf},
        "speedup_vs_per_frame": ms_pf / ms_batch,
        "launch": "one CUDA graph: the two code groups as concurrent tile-decoder launches",
        "persistent": {"value": info_bits / (ms_persistent * 1e-3) / 1e6, "unit": "Mbit/s",
                       "ms_per_step": ms_persistent, "launch": "one persistent two-code launch (CUDA graph)"},
        "tuned": {str(ci): {"f": chosen[ci].f, "v": chosen[ci].v, "disagree_vs_full_frame": chosen[ci].disagree}
                  for ci in chosen} | {"warps_per_cta": warps},
        "ber": err / info_bits, "info_bits": info_bits,
        "alu": _mixed_alu(frames, codes, chosen, ms_batch, ms_persistent),
    }


def _window_stages(n: int, f: int, v: int) -> int:
    """Stages processed by the tiles of an n-stage frame (windows clipped to
    the frame; f = 0 is one window)."""
    fb = n if (f == 0 or f > n) else f
    tot = 0
    for b in range((n + fb - 1) // fb):
        e0, e1 = b * fb, min((b + 1) * fb, n)
        tot += min(n, e1 + v) - max(0, e0 - v)
    return tot


def _mixed_alu(frames, codes, chosen, ms_batch, ms_persistent):
    """Algorithmic int16 ops of the mixed batch (4 per state per processed
    stage, overlaps included) over each launch form's step time, against the
    measured peak."""
    ops = 0.0
    for ci, _, n, _ in frames:
        K = codes[ci][0]
        ops += 4.0 * (1 << (K - 1)) * _window_stages(n, chosen[ci].f, chosen[ci].v)
    return {"ops_per_step": ops, "tops_concurrent": ops / (ms_batch * 1e-3) / 1e12,
            "tops_persistent": ops / (ms_persistent * 1e-3) / 1e12}


METRIC_WORKLOAD = ("1024 zero-terminated frames x (2048 + 6) stages, K=7 r1/2 (171,133), FP32 LLRs "
                   "L = 2y/sigma^2 at Eb/N0 2 dB; best-path metric (hard) and log-sum-exp (tau 0.5, 1, 2), "
                   "forward and backward, state metrics checkpointed every 64 stages")


def metric_leg(vit, torch, device, steps, fp_rates, sm_mhz):
    """The differentiable path metric at its workload size: forward and
    backward time per tau, frames/s, and the achieved rate of the unit that
    bounds each form (FP32 adds/max for the hard form, MUFU ex2/lg2 for the
    log-sum-exp form) against the measured per-SM instruction rates."""
    from paper_2011_09337_gb300 import synth
    F, n_info, C = 1024, 2048, 64
    n = n_info + K - 1
    g = synth.rng(3)
    msg = np.zeros((F, n), np.uint8)
    msg[:, :n_info] = g.integers(0, 2, size=(F, n_info), dtype=np.uint8)
    code = vit.Code(K, BETA, POLYS, mode=vit.TERMINATED)
    coded = vit.encode(code, torch.from_numpy(msg.reshape(-1)).to(device)).cpu().numpy().astype(np.float64)
    sigma = synth.noise_sigma(2.0, 1.0 / BETA)
    y = (1.0 - 2.0 * coded) + sigma * g.standard_normal(coded.shape)
    x = torch.from_numpy((2.0 * y / sigma ** 2).astype(np.float32).reshape(F, n, BETA)).to(device)
    S = 1 << (K - 1)
    state_stages = F * n * S
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    out = {"workload": METRIC_WORKLOAD, "frames": F, "stages_per_frame": n, "C": C}
    ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
    def timed(fn, reps):
        torch.cuda.synchronize()
        ev[0].record()
        for _ in range(reps):
            fn()
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / reps

    for tau in (0.0, 0.5, 1.0, 2.0):
        # kernels: the C-ABI calls on preallocated buffers, back to back
        ws = torch.empty(max(vit.metric_workspace(code, F, n, tau, C), 1), dtype=torch.uint8, device=device)
        met = torch.empty(F, dtype=torch.float32, device=device)
        gm = torch.ones(F, dtype=torch.float32, device=device)
        gx = torch.empty_like(x)
        for _ in range(3):
            vit.metric_fwd(code, x, tau, C, met, ws)
            vit.metric_bwd(code, x, gm, tau, C, ws, gx)
        fwd_ms = timed(lambda: vit.metric_fwd(code, x, tau, C, met, ws), max(steps, 20))
        bwd_ms = timed(lambda: vit.metric_bwd(code, x, gm, tau, C, ws, gx), max(steps, 20))
        # the same through torch.autograd (ViterbiMetric), host overhead included
        xr = x.clone().requires_grad_(True)
        for _ in range(2):
            m = vit.path_metric(xr, code, tau, C)
            (ga,) = torch.autograd.grad(m.sum(), xr)
        af_ms = timed(lambda: vit.path_metric(xr, code, tau, C), max(steps, 20))
        m = vit.path_metric(xr, code, tau, C)
        ab_ms = timed(lambda: torch.autograd.grad(m.sum(), xr, retain_graph=True), max(steps, 20))
        key = "hard" if tau == 0.0 else f"tau_{tau:g}"
        r = {"fwd_ms": fwd_ms, "bwd_ms": bwd_ms, "frames_per_s": F / ((fwd_ms + bwd_ms) * 1e-3),
             "autograd_fwd_ms": af_ms, "autograd_bwd_ms": ab_ms,
             "grad_finite": bool(torch.isfinite(gx).all().item()),
             "autograd_matches_kernels": bool(torch.equal(ga, gx))}
        if tau == 0.0:
            # 4 FP32 ops per state per stage (2 adds, compare, select) in the forward pass
            peak = max(fp_rates["fadd"], fp_rates["fmax"]) * 32 * sms * sm_mhz * 1e6
            ach = 4.0 * state_stages / (fwd_ms * 1e-3)
            r["roofline_fwd"] = {"bound": "fp32", "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "Tops/s",
                                 "frac": ach / peak, "ops": "4 FP32 ops per state per stage"}
        else:
            # one exp and one log per state per stage in the forward pass; the
            # backward recomputes the forward (exp, log), runs the beta
            # recursion (exp, log) and forms two branch posteriors (2 exp).
            # The peak of each mix: its MUFU instructions over the cycles they
            # occupy at the measured ex2 and lg2 rates.
            for leg, nex, nlg, ms in (("fwd", 1.0, 1.0, fwd_ms), ("bwd", 4.0, 2.0, bwd_ms)):
                mufu = nex + nlg
                rate = mufu / (nex / fp_rates["ex2"] + nlg / fp_rates["lg2"])
                peak = rate * 32 * sms * sm_mhz * 1e6
                ach = mufu * state_stages / (ms * 1e-3)
                r[f"roofline_{leg}"] = {"bound": "mufu", "achieved": ach / 1e12, "peak": peak / 1e12,
                                        "unit": "Tops/s", "frac": ach / peak,
                                        "ops": f"{nex:g} ex2 + {nlg:g} lg2 per state per stage"}
        out[key] = r
        del xr, m, gx, ga, ws
    return out


def metric_cpu_baseline():
    """The FP64 oracle on the finite-difference subset (8 frames x (64 + 6)
    stages): metric and gradient, hard and log-sum-exp (tau = 1)."""
    import oracle
    from paper_2011_09337_gb300 import synth
    _, llr = synth.float_frames(lambda x: oracle.encode(K, BETA, POLYS, x), BETA, K, 8, 64, 2.0, seed=3)
    x = llr.astype(np.float64)
    t0 = time.perf_counter()
    reps = 0
    while time.perf_counter() - t0 < 2.0:
        oracle.metric_hard(K, BETA, POLYS, x)
        oracle.metric_lse(K, BETA, POLYS, x, 1.0)
        reps += 1
    dt = (time.perf_counter() - t0) / reps
    return {"value": 8 / dt, "unit": "frames/s (hard + lse, fwd + grad)", "cores": 1, "kind": "oracle",
            "sample": "8 frames x 70 stages, FP64, metric and gradient of the hard and tau = 1 forms, one thread"}


LARGE_WORKLOAD = ("2^26-bit streams: K=9 r1/2 (561,753) f=2048 v=96; K=7 (171,133) punctured to r3/4 "
                  "[110;101] f=2048 v=64; K=9 punctured to r3/4 f=2048 v=96; int8 LLRs at Eb/N0 4 dB")


def large_streams_leg(vit, torch, device, steps):
    """The 2^26-bit streams: one decode launch each (plus de-puncturing)."""
    from paper_2011_09337_gb300 import synth

    n = 1 << 26
    out = {}
    cases = [("k9", synth.CODE_K9_R12, 2048, 96, None), ("k7_r34", synth.CODE_K7_R12, 2048, 64, synth.PUNCT_R34),
             ("k9_r34", synth.CODE_K9_R12, 2048, 96, synth.PUNCT_R34)]
    for name, (K, beta, polys), f, v, mask in cases:
        code = vit.Code(K, beta, polys, f=f, v=v, puncture=mask)

        def enc(bits):
            return vit.encode(code, torch.from_numpy(bits).to(device)).cpu().numpy()

        st = synth.make_stream(enc, beta, n, 4.0, seed=4 + len(out), mask=mask)
        llr = torch.from_numpy(st.llr.reshape(-1)).to(device)
        ws = torch.empty(code.workspace_bytes(n), dtype=torch.uint8, device=device)
        o = torch.empty((n + 7) // 8, dtype=torch.uint8, device=device)
        for _ in range(3):
            vit.decode(code, llr, n, out=o, workspace=ws)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            vit.decode(code, llr, n, out=o, workspace=ws)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        S = 1 << (K - 1)
        ops = 4.0 * S * sum(min(n, (t + 1) * f + v) - max(0, t * f - v) for t in range(n // f))
        got = synth.unpack_bits(o.cpu().numpy(), n)
        out[name] = {"value": n / (ms * 1e-3) / 1e6, "unit": "Mbit/s", "ms_per_step": ms,
                     "alu_tops": ops / (ms * 1e-3) / 1e12, "ber": float(np.mean(got != st.bits))}
        del llr, ws, o
    out["workload"] = LARGE_WORKLOAD
    return out


def profile_k9(vit, torch, device, log2_bits=25):
    """Target of the K=9 ncu captures: one 2^log2_bits-bit stream decoded twice."""
    from paper_2011_09337_gb300 import synth
    K9, B9, P9 = synth.CODE_K9_R12
    n = 1 << log2_bits
    code = vit.Code(K9, B9, P9, f=2048, v=96)

    def enc(bits):
        return vit.encode(code, torch.from_numpy(bits).to(device)).cpu().numpy()

    st = synth.make_stream(enc, B9, n, 4.0, seed=9)
    llr = torch.from_numpy(st.llr.reshape(-1)).to(device)
    ws = torch.empty(code.workspace_bytes(n), dtype=torch.uint8, device=device)
    o = torch.empty((n + 7) // 8, dtype=torch.uint8, device=device)
    for _ in range(2):
        vit.decode(code, llr, n, out=o, workspace=ws)
    torch.cuda.synchronize()
    print(json.dumps({"profile_run": "ok", "code": "k9", "bits": n}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-code batch leg")
    ap.add_argument("--no-large", action="store_true", help="skip the 2^26-bit stream leg")
    ap.add_argument("--no-pt", action="store_true", help="skip the parallel-traceback leg")
    ap.add_argument("--no-metric", action="store_true", help="skip the differentiable path-metric leg")
    ap.add_argument("--profile", action="store_true",
                    help="build the workload with --streams streams, run the planned batch twice and exit "
                         "(the target of the ncu captures)")
    ap.add_argument("--streams", type=int, default=len(EBN0))
    ap.add_argument("--profile-code", default="k7", choices=["k7", "k9", "frame", "probe", "metric"],
                    help="with --profile: k7 = the batch above; k9 = one K=9 (561,753) stream (--profile-log2-bits), "
                         "f=2048, v=96, decoded twice; frame = the single-frame latency case, decoded twice; "
                         "probe = the instruction-rate probes of the roofline peak, once each; metric = the "
                         "path-metric workload, forward and backward once per form")
    ap.add_argument("--profile-log2-bits", type=int, default=25,
                    help="with --profile --profile-code k9: the stream's size, 2^N info bits")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2011_09337_gb300 import vit
    if args.profile and args.profile_code == "k9":
        profile_k9(vit, torch, dev, args.profile_log2_bits)
        return
    if args.profile and args.profile_code == "probe":
        print(json.dumps({"profile_run": "ok", "code": "probe", "int": alu_peak_leg(vit, dev),
                          "fp": fp_peak_leg(vit, dev)}))
        return
    if args.profile and args.profile_code == "metric":
        m = metric_leg(vit, torch, dev, 1, fp_peak_leg(vit, dev), _peaks()[0])
        print(json.dumps({"profile_run": "ok", "code": "metric",
                          **{k: m[k] for k in ("hard", "tau_0.5", "tau_1", "tau_2")}}))
        return
    if args.profile and args.profile_code == "frame":
        print(json.dumps({"profile_run": "ok", "code": "frame", **frame_latency_leg(vit, torch, dev, 2)}))
        return
    code = vit.Code(K, BETA, POLYS, f=F, v=V)
    streams = make_inputs(vit, code, dev, torch, args.streams)
    nbytes = (NBITS + 7) // 8
    d_llr = [torch.from_numpy(s.llr.reshape(-1)).to(dev) for s in streams]
    d_out = [torch.zeros(nbytes, dtype=torch.uint8, device=dev) for _ in streams]
    frames = [(code, d_llr[i], NBITS, vit.STREAM, d_out[i]) for i in range(len(streams))]
    batch = vit.Batch(frames, graph=True)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    if args.profile:
        batch.run()
        batch.run()
        barrier()
        print(json.dumps({"profile_run": "ok", "streams": len(streams)}))
        return

    # ---- device-resident timing: one planned batch (one launch) per step
    for _ in range(args.warmup):
        batch.run()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            batch.run()
            ev[i][1].record(stream)
        t_end.record(stream)
        barrier()
    total_ms = t_start.elapsed_time(t_end)
    launch_ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    bits_per_step = NBITS * len(streams)
    ms_per_step, value = aggregate(total_ms, args.steps, bits_per_step, world, dev)

    # BER of this run's output against the transmitted bits, per Eb/N0
    from paper_2011_09337_gb300 import synth
    got_bits = [synth.unpack_bits(o.cpu().numpy(), NBITS) for o in d_out]
    ber_per_ebn0 = {f"{EBN0[i]:g}dB": float(np.mean(g != streams[i].bits)) for i, g in enumerate(got_bits)}

    # ---- per-frame launches (one vit_decode per stream) for comparison
    ws = torch.empty(code.workspace_bytes(NBITS), dtype=torch.uint8, device=dev)
    for _ in range(2):
        for i in range(len(streams)):
            vit.decode(code, d_llr[i], NBITS, out=d_out[i], workspace=ws)
    barrier()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        for i in range(len(streams)):
            vit.decode(code, d_llr[i], NBITS, out=d_out[i], workspace=ws)
    b.record(stream)
    barrier()
    per_frame_value = bits_per_step / (a.elapsed_time(b) / args.steps * 1e-3) / 1e6

    # ---- end to end through the C ABI with pinned host buffers: a host-staged
    # batch (VIT_BATCH_HOST) copies each step's LLRs in and the bits out,
    # pipelined in chunks with the decoding
    h_llr = [torch.from_numpy(s.llr.reshape(-1)).pin_memory() for s in streams]
    h_out = [torch.empty(nbytes, dtype=torch.uint8).pin_memory() for _ in streams]
    h2d = sum(x.numel() for x in h_llr)
    d2h = sum(x.numel() for x in h_out)
    hbatch = vit.Batch([(code, h_llr[i], NBITS, vit.STREAM, h_out[i]) for i in range(len(streams))],
                       graph=True, host=True, device=dev)

    def timed(fn, steps):
        for _ in range(max(2, args.warmup)):
            fn()
        barrier()
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        barrier()
        return a.elapsed_time(b) / steps

    single_ms = timed(hbatch.run, args.steps)
    e2e_ok = all(torch.equal(h_out[i], d_out[i].cpu()) for i in range(len(streams)))

    # double-buffered receiver: a second host-staged plan over its own pinned
    # input and output buffers; consecutive steps alternate between the two
    # plans on two streams, so one step's input copies overlap the previous
    # step's decode.  Every step still copies its 235 MB in and its bits out.
    h_llr2 = [torch.from_numpy(s.llr.reshape(-1)).pin_memory() for s in streams]
    h_out2 = [torch.empty(nbytes, dtype=torch.uint8).pin_memory() for _ in streams]
    hbatch2 = vit.Batch([(code, h_llr2[i], NBITS, vit.STREAM, h_out2[i]) for i in range(len(streams))],
                        graph=True, host=True, device=dev)
    side = [torch.cuda.Stream(dev), torch.cuda.Stream(dev)]
    plans = [hbatch, hbatch2]
    state = {"i": 0}

    def pipelined_step():
        k = state["i"] & 1
        state["i"] += 1
        side[k].wait_stream(stream)
        with torch.cuda.stream(side[k]):
            plans[k].run()
        stream.wait_stream(side[k])

    def pipelined(steps):
        # the caller's stream forks each step to its plan's stream and joins it
        # back only at the end, so steps on the two streams overlap
        ev0 = torch.cuda.Event()
        ev0.record(stream)
        for k in range(steps):
            j = k & 1
            side[j].wait_event(ev0)
            with torch.cuda.stream(side[j]):
                plans[j].run()
        stream.wait_stream(side[0])
        stream.wait_stream(side[1])

    for _ in range(max(2, args.warmup)):
        pipelined_step()
    barrier()
    a.record(stream)
    pipelined(args.steps)
    b.record(stream)
    barrier()
    e2e_ms = a.elapsed_time(b) / args.steps
    e2e_value = bits_per_step * world / (e2e_ms * 1e-3) / 1e6
    e2e_ok = e2e_ok and all(torch.equal(h_out2[i], d_out[i].cpu()) for i in range(len(streams)))

    # the same copies and decode issued one after another on one stream
    def seq_step():
        for i in range(len(streams)):
            d_llr[i].copy_(h_llr[i], non_blocking=True)
        batch.run()
        for i in range(len(streams)):
            h_out[i].copy_(d_out[i], non_blocking=True)

    seq_ms = timed(seq_step, args.steps)

    pt = None if args.no_pt else parallel_traceback_leg(vit, torch, d_llr, d_out, args.steps)
    shared = shared_decoder_leg(vit, torch, d_llr, d_out, max(3, args.steps // 4))
    frame = frame_latency_leg(vit, torch, dev, args.steps)
    mixed = None if args.no_mixed else mixed_batch_leg(vit, torch, dev, args.steps)
    large = None if args.no_large else large_streams_leg(vit, torch, dev, max(3, args.steps // 4))
    fp_rates = fp_peak_leg(vit, dev)
    sm_max_ = _peaks()[0]
    metric = None
    if not args.no_metric:
        metric = metric_leg(vit, torch, dev, max(3, args.steps // 4), fp_rates, sm_max_)
        metric["fp_rates_warp_instr_per_clk_sm"] = fp_rates

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    sm_max, hbm_gbs, peak_src = _peaks()
    ops = algorithmic_ops_per_step()
    probe = alu_peak_leg(vit, dev)
    peak_tops = probe["int16_ops_per_clk_sm"] * probe["sms"] * sm_max * 1e6 / 1e12
    achieved_tops = ops / (launch_ms * 1e-3) / 1e12
    clocks = clk.summary()
    traffic = _traffic_per_launch()
    # algorithmic bytes per launch: int8 LLRs of every window + packed output bits
    alg_bytes = ops / (4 * (1 << (K - 1))) * BETA + bits_per_step / 8
    line = {
        "metric": METRIC, "value": value, "unit": "Mbit/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int16", "data": "synthetic",
        "config": {"workload": WORKLOAD, "frames": len(streams), "info_bits_per_frame": NBITS, "f": F, "v": V,
                   "launch": "one planned batch per step (CUDA graph)",
                   "l2": "inputs larger than L2 (235 MB of LLRs per step)"},
        "per_frame": {"value": per_frame_value, "unit": "Mbit/s", "launches_per_step": len(streams)},
        "e2e": {"value": e2e_value, "unit": "Mbit/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms, "api": "vit_batch_plan(VIT_BATCH_HOST) + vit_batch_run, pinned host buffers, "
                "8 chunks (copies overlapped with decoding); two plans over two pinned buffer sets run on two "
                "streams in turn, so consecutive steps overlap", "matches_device_batch": e2e_ok,
                "single_plan": {"value": bits_per_step * world / (single_ms * 1e-3) / 1e6, "unit": "Mbit/s",
                                "ms_per_step": single_ms, "how": "one host-staged plan, steps one after another"},
                "sequential": {"value": bits_per_step * world / (seq_ms * 1e-3) / 1e6, "unit": "Mbit/s",
                               "ms_per_step": seq_ms, "how": "H2D, decode, D2H in turn on one stream"}},
        "roofline": {"bound": "alu", "achieved": achieved_tops, "peak": peak_tops, "unit": "Tops/s",
                     "frac": achieved_tops / peak_tops, "traffic": traffic,
                     "traffic_over_algorithmic": (traffic / alg_bytes) if traffic else None,
                     "peak_source": (f"alu_peak leg (vit_probe_rate): {probe['peak_class']} at "
                                     f"{probe['warp_instr_per_clk_sm'][probe['peak_class']]:.3f} warp-instr/clk/SM x 32 "
                                     f"lanes x {OPS_PER_LANE_INSTR[probe['peak_class']]} int16 ops x {probe['sms']} SMs "
                                     f"x {sm_max:.0f} MHz ({peak_src} max clock)"),
                     "alu_peak": probe,
                     "kernel": "decode_tiles_kernel<K=7,beta=2>", "launch_ms": launch_ms,
                     "hbm_alg_gbs": alg_bytes / (launch_ms * 1e-3) / 1e9, "hbm_peak_gbs": hbm_gbs},
        "clocks": clocks,
        "gpu_launches": args.steps,
        "parallel_traceback": pt,
        "shared_memory_decoder": shared,
        "frame_latency": frame,
        "batch_mixed": mixed,
        "large_streams": large,
        "metric_leg": metric,
        "ber": {"vs_transmitted": ber_per_ebn0, "bits_per_stream": NBITS},
    }
    if mixed is not None:
        mixed["alu"]["frac_concurrent"] = mixed["alu"]["tops_concurrent"] / peak_tops
        mixed["alu"]["frac_persistent"] = mixed["alu"]["tops_persistent"] / peak_tops
    if large is not None:
        for k, v in large.items():
            if isinstance(v, dict) and "alu_tops" in v:
                v["alu_frac"] = v["alu_tops"] / peak_tops
    if clocks.get("sm_mhz"):
        line["roofline"]["peak_at_sampled_clock"] = peak_tops * clocks["sm_mhz"] / sm_max
        line["roofline"]["frac_at_sampled_clock"] = achieved_tops / (peak_tops * clocks["sm_mhz"] / sm_max)
    if not args.no_cpu_baseline and world == 1 or (world > 1 and rank == 0 and not args.no_cpu_baseline):
        v, cores, sample, v1 = cpu_oracle_rate()
        line["cpu_baseline"] = {"value": v, "unit": "Mbit/s", "cores": cores, "kind": "oracle", "sample": sample,
                                "single_core": {"value": v1, "unit": "Mbit/s", "sample": "4 tiles on 1 thread"}}
        if metric is not None:
            metric["cpu_baseline"] = metric_cpu_baseline()
        line["cpu_baseline"]["full_frame"] = full_frame_oracle_sample(streams, got_bits)
        line["cpu_baseline"]["other_workloads_single_core"] = other_configs_cpu_rate()
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
