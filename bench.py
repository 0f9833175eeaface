#!/usr/bin/env python3
"""Benchmark of the ABFT-protected FP64 GEMM (FT-BLAS, Zhai et al., ICS '21) on GB300.

Workload: FT-DGEMM, column-major, M = N = K = 8192 (a member of the paper's 2048^2-10240^2
DGEMM range), alpha = 1.5, beta = 0.5, A, B, C uniform on [-1, 1) from a fixed seed, one
seeded accumulator bit flip (bits 40-62) per 10 launches. One step = one protected call:
operand staging, fused checksum encode, product, alpha/beta epilogue, verification,
location, correction and the report all run inside it.

Printed (one JSON line, rank 0): FT-GEMM TFLOP/s (2 M N K per step over device time,
inputs resident in HBM), the fraction of the FP64 peak, the ABFT overhead against the same
kernel with protection compiled out (ftblas_dgemm_noabft), with and without injection, the
detected/corrected counts, the error against the CPU oracle on sampled rows, an
end-to-end figure through the host-buffer entry point (copies included), the sampled SM
clocks, and the CPU oracle timed on the host on a bounded sample.

`--impl reference` times the CPU oracle instead (the only reference there is: the paper's
implementation is AVX-512 CPU code that is not available), on bounded samples per step.

Multi-GPU (torchrun): every rank runs its own independent problem (output tiles shard with
no data-path exchange), so scaling is weak; the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "FT-GEMM TFLOP/s, % of peak, ABFT overhead % vs unprotected, at stated error"
UNIT = "TFLOP/s"
SEED = 20210601
TILE = 128  # FP64 verification tile edge at the 8192^3 workload (the oracle's geometry)


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=8192, help="M = N = K")
    ap.add_argument("--engine", choices=["dfma", "dmma"], default="dfma", help="headline FP64 engine")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-second-engine", action="store_true")
    ap.add_argument("--no-bf16", action="store_true", help="skip the BF16 tensor-core measurement")
    ap.add_argument("--no-fp8", action="store_true", help="skip the FP8 (E4M3) tensor-core measurement")
    ap.add_argument("--fp8-size", type=int, default=16384, help="M = N = K of the FP8 measurement")
    ap.add_argument("--bf16-only", action="store_true",
                    help="measure only the BF16 tensor-core form (for profiling); prints its own JSON line")
    ap.add_argument("--soak", type=float, default=0.0, metavar="SECONDS",
                    help="run only the soak (config 5a): back-to-back FT-DGEMM with Poisson-drawn injections")
    ap.add_argument("--soak-rate", type=float, default=5.0, help="injections per second in the soak")
    ap.add_argument("--sweep", action="store_true",
                    help="run only the FP64 size sweep (config 2) and print its own JSON line")
    ap.add_argument("--unfused-only", action="store_true",
                    help="measure only the unfused comparator (ABFT passes around cuBLAS DGEMM)")
    ap.add_argument("--no-unfused", action="store_true", help="skip the unfused comparator")
    ap.add_argument("--no-online", action="store_true", help="skip the online-verification measurement")
    ap.add_argument("--no-emulated", action="store_true", help="skip the emulated FP64 measurement")
    ap.add_argument("--no-large", action="store_true", help="skip the FP64 16384^3 point of the default line")
    ap.add_argument("--no-soak-default", action="store_true", help="skip the 60 s soak of the default line")
    ap.add_argument("--emulated-only", action="store_true", help="measure only the emulated FP64 GEMM")
    ap.add_argument("--no-level3", action="store_true", help="skip the FT-DSYMM / FT-DTRMM measurement")
    ap.add_argument("--level3-only", action="store_true", help="measure only FT-DSYMM / FT-DTRMM")
    ap.add_argument("--linear-only", action="store_true", help="measure only the protected linear layer (config 4)")
    ap.add_argument("--no-linear", action="store_true", help="skip the protected linear layer (config 4)")
    ap.add_argument("--fp8-only", action="store_true",
                    help="measure only the FP8 tensor-core form (for profiling); prints its own JSON line")
    ap.add_argument("--tc-cta-group", type=int, choices=[1, 2], default=None,
                    help="tensor-core product kernel: 1 CTA per tile or a CTA pair (default: the library's)")
    return ap.parse_args()


def peaks():
    """Roofline denominators. MEASURED_PEAKS.json holds the measured HBM copy and BF16 GEMM
    figures (burst and sustained); the FP64 pipe's peak is derived from its unit count and the
    maximum SM clock."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    mp = {}
    if os.path.exists(path):
        with open(path) as f:
            mp = json.load(f)
    bf16 = mp.get("bf16_tflops")
    sm_max = mp.get("sm_max_mhz", 2070.0)
    sms = 152  # GB300; the device's own count when one answers
    try:
        import torch
        if torch.cuda.is_available():
            sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    except Exception:
        pass
    # FP64 FMA pipe: 2 FMA / clock / SM (GB300 nominal 1.25 TFLOP/s at 2070 MHz) x the SMs.
    alu = 2 * 2 * sms * sm_max * 1e6 / 1e12
    if bf16 is not None:
        tensor = bf16 * 1.25 / 2250.0
        tensor_src = f"measured bf16 {bf16} TFLOP/s x nominal FP64/BF16 ratio 1.25/2250"
    else:
        tensor = 1900.0 * 1.25 / 2250.0
        tensor_src = "fallback bf16 1900 TFLOP/s x nominal FP64/BF16 ratio 1.25/2250"
    bf16_peak = bf16 if bf16 is not None else 1900.0
    bf16_src = (f"measured bf16 {bf16} TFLOP/s (burst)" if bf16 is not None
                else "fallback bf16 1900 TFLOP/s (burst)")
    bf16_sus = mp.get("bf16_tflops_sustained") or 1700.0
    return dict(alu=alu, alu_src=f"2 FP64 FMA/clk/SM x {sms} SMs x {sm_max} MHz", tensor=tensor,
                tensor_src=tensor_src, bf16=bf16_peak, bf16_src=bf16_src, bf16_sustained=bf16_sus)


FP64_KERNEL_SOURCES = ("paper_2104_00897_gb300/csrc/ft_dgemm.cu", "paper_2104_00897_gb300/csrc/ft_device.cuh",
                       "paper_2104_00897_gb300/csrc/ft_internal.h")
TC_KERNEL_SOURCES = ("paper_2104_00897_gb300/csrc/ft_gemm_tc.cu", "paper_2104_00897_gb300/csrc/ft_tc_elem.cuh",
                     "paper_2104_00897_gb300/csrc/ft_device.cuh", "paper_2104_00897_gb300/csrc/ft_internal.h",
                     "paper_2104_00897_gb300/csrc/ft_tc.h")


def sources_sha256(paths):
    """SHA-256 of the kernel's code: its sources without comments and blank lines, each
    line stripped. An edit of comments or layout alone keeps a capture's counters valid;
    any change of code voids them."""
    import hashlib
    import re
    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, rel), encoding="utf-8") as f:
            src = f.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for line in src.split("\n"):
            line = line.strip()
            if line:
                h.update(line.encode() + b"\n")
    return h.hexdigest()


def profile_traffic(name, sources):
    """DRAM bytes per launch (read + write) from the committed ncu summary profiles/<name>.md,
    or None when the summary is missing or the kernel's sources changed since the capture
    (the summary records their SHA-256)."""
    import re
    path = os.path.join(ROOT, "profiles", name + ".md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_t = re.search(r"traffic_bytes_per_launch:\s*(\d+)", text)
    m_h = re.search(r"sources_sha256:\s*([0-9a-f]{64})", text)
    if not m_t or not m_h or m_h.group(1) != sources_sha256(sources):
        return None
    return int(m_t.group(1))


def workload_config(n, engine, tile=TILE):
    return {"workload": f"ft_dgemm_fp64_col_major_{n}x{n}x{n}", "M": n, "N": n, "K": n, "alpha": 1.5, "beta": 0.5,
            "layout": "column-major, no transpose", "inputs": "A, B, C uniform[-1,1) from a fixed seed",
            "injection": "one seeded accumulator bit flip (bits 40-62) per 10 launches",
            "verification_tile": f"{tile}x{tile}", "engine": engine, "seed": SEED,
            "seed_per_rank": "seed + rank (each rank solves its own problem)",
            "l2": l2_note(n * n * 8)}


def l2_note(operand_bytes):
    """How the timed steps stand to the 129 MB L2: inputs larger than it, or not, with no flush."""
    mib = operand_bytes / 2**20
    rel = "larger than" if operand_bytes > 129e6 else "within"
    return f"inputs {mib:.0f} MiB per operand, {rel} the 129 MB L2; no flush between steps"


def l2_note_tc(operand_bytes, c_bytes):
    """The same for the tensor-core forms: both operands together, and the FP32 C."""
    rel = "larger than" if operand_bytes + c_bytes > 129e6 else "within"
    return (f"operands {operand_bytes / 2**20:.0f} MiB + C {c_bytes / 2**20:.0f} MiB, {rel} the 129 MB L2; "
            "no flush between steps")


# ------------------------------------------------------------------ multi-rank host logic
# Output problems are independent verification intervals, so N ranks run N independent
# problems (weak scaling) with no data-path exchange; the process group carries only the
# barrier, the maximum of the timed region and the sum of the report counters.

def rank_seed(rank):
    """Input seed of rank `rank`: every rank gets a distinct problem of the same shape."""
    return SEED + rank


def max_over_ranks(x, dist):
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(counts, dist):
    """Element-wise sum over ranks of a dict of integer report counters."""
    if dist is None:
        return dict(counts)
    import torch
    keys = sorted(counts)
    t = torch.tensor([int(counts[k]) for k in keys], dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return {k: int(v) for k, v in zip(keys, t.tolist())}


def or_over_ranks(x, dist):
    """Bitwise OR over ranks (report status bits)."""
    if dist is None:
        return int(x)
    import torch
    t = torch.tensor([int(x)], dtype=torch.int64)
    dist.all_reduce(t, op=dist.ReduceOp.BOR)
    return int(t.item())


def job_tflops(world, flops_per_rank_step, steps, max_ms):
    """Whole-job throughput: the work of all ranks over the slowest rank's time."""
    return world * flops_per_rank_step * steps / (max_ms / 1e3) / 1e12


def gen_inputs(n, seed):
    import synth as S
    A = S.uniform(seed, 0, n * n)   # logical column-major index == storage index (ld = n)
    B = S.uniform(seed, 1, n * n)
    Cin = S.uniform(seed, 2, n * n)
    return A, B, Cin


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(n, A, B, Cin, n_tiles, seed_tiles=7):
    """The CPU oracle (as it stands) on n_tiles seeded 128 x 128 tiles of the workload.
    Returns (flops, seconds, threads)."""
    import oracle as O
    import synth as S
    tr = (n + TILE - 1) // TILE
    tiles = np.unique(S.randint(seed_tiles, 3, n_tiles * 4, 0, tr * tr - 1))[:n_tiles]
    t0 = time.perf_counter()
    O.ft_gemm(O.COL_MAJOR, O.NO_TRANS, O.NO_TRANS, n, n, n, 1.5, A, n, B, n, 0.5, Cin, n, TILE, TILE, 32,
              tiles=tiles, out=np.array(Cin, copy=True))
    dt = time.perf_counter() - t0
    return 2.0 * len(tiles) * TILE * TILE * n, dt, O.num_threads()


# ------------------------------------------------------------------ BF16 tensor-core form
def run_tc(args, dev, kind, n, steps, warmup, fp64_tflops):
    """The tensor-core forms. kind "bf16" (config 3): A, B N(0,1) with rows of A scaled by
    2^u, u in [-8, 8], BF16. kind "fp8" (config 5b): A, B N(0,1) quantised per tensor to
    E4M3 (scale = amax / 448). Both accumulate in FP32 on the tensor cores, store FP32 C and
    compare checksums in FP64. Reports FT and unprotected TFLOP/s, the speedup over FP64
    FT-DGEMM, the error against the FP64 product of the same operands on a sampled block, and
    the fraction of injected output errors 2^p |C| corrected per p."""
    import torch

    import paper_2104_00897_gb300 as fb
    import synth as S

    threads = max(1, min(16, os.cpu_count() or 1))
    fp8 = kind == "fp8"
    seed = SEED + (5 if fp8 else 3)
    A = S.normal_matrix(seed, 0, n, n, threads=threads)
    if not fp8:
        A *= S.pow2_row_scales(seed, 5, n)[:, None]
    B = S.normal_matrix(seed, 1, n, n, threads=threads)
    if fp8:
        sa = float(np.float32(np.max(np.abs(A)) / 448.0))
        sb = float(np.float32(np.max(np.abs(B)) / 448.0))
        # column-major call with A transposed (stored K x M, i.e. A row-major) and B not
        abits = S.map_elementwise(lambda x: S.to_e4m3_bits(x / sa), A, np.uint8, threads)
        bbits_t = S.map_elementwise(lambda x: S.to_e4m3_bits(x / sb), np.ascontiguousarray(B.T), np.uint8, threads)
        dA = torch.from_numpy(abits.ravel()).to(dev)
        dB = torch.from_numpy(bbits_t.ravel()).to(dev)
        dS = torch.tensor([sa, sb], dtype=torch.float32, device=dev)
        dtype, sa_ptr, sb_ptr = fb.R_8F_E4M3, dS.data_ptr(), dS.data_ptr() + 4
        deq = lambda bits, sc: sc * S.e4m3_bits_to_f64(bits)
    else:
        abits = S.map_elementwise(S.to_bf16_bits, A, np.uint16, threads)
        bbits_t = S.map_elementwise(S.to_bf16_bits, np.ascontiguousarray(B.T), np.uint16, threads)
        dA = torch.from_numpy(abits.view(np.int16).ravel()).to(dev)
        dB = torch.from_numpy(bbits_t.view(np.int16).ravel()).to(dev)
        dtype, sa_ptr, sb_ptr = fb.R_16BF, None, None
        deq = lambda bits, sc: S.bf16_bits_to_f64(bits)
        sa = sb = 1.0
    del A, B
    dC = torch.zeros(n * n, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream(dev).cuda_stream
    flops = 2.0 * n ** 3

    def call(protect, rep=None):
        a = (fb.COL_MAJOR, fb.TRANS, fb.NO_TRANS, n, n, n, 1.0, dA.data_ptr(), dtype, n, dB.data_ptr(), dtype, n,
             0.0, dC.data_ptr(), fb.R_32F, n, fb.R_32F, sa_ptr, sb_ptr, st)
        if protect:
            fb.check(fb.ftblas_gemm_ex(*a, rep.data_ptr() if rep is not None else None), "ftblas_gemm_ex")
        else:
            fb.check(fb.ftblas_gemm_ex_noabft(*a), "ftblas_gemm_ex_noabft")

    kernel_ms = {}
    timed_steps = {}

    def timed(protect, inject):
        if inject:
            # output errors of 2^p |C(i,j)|, p far above the rigorous threshold's reach: that
            # threshold scales with the row's sum_k |A(i,k)| max_k sum_j |B(k,j)|, some 30 times
            # a typical |C(i,j)| here, so an unusually small element hides an error of 2^8 |C(i,j)|
            # (G8; the detection map charts the detected fraction per p)
            lo = 18 if fp8 else 16
            fb.ftblas_set_injection(fb.make_injection(seed=seed, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, log2_lo=lo,
                                                      log2_hi=lo + 4, every_n_launches=1, errors_per_launch=1))
        else:
            fb.ftblas_set_injection(None)
        for _ in range(warmup):
            call(protect)
        torch.cuda.synchronize(dev)
        # as many timed calls as cover at least 40 ms (a call takes about a millisecond), so
        # that the host's latency before the first launch is a small part of the region
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call(protect)
        e1.record()
        torch.cuda.synchronize(dev)
        nsteps = max(steps, min(256, int(40.0 / max(e0.elapsed_time(e1), 1e-3)) + 1))
        timed_steps[(protect, inject)] = nsteps
        reps = [fb.new_report(dev) for _ in range(nsteps)]
        fb.ftblas_kernel_timing_begin()
        e0.record()
        for s_ in range(nsteps):
            call(protect, reps[s_])
        e1.record()
        torch.cuda.synchronize(dev)
        _, kms, kn = fb.ftblas_kernel_timing_end()
        kernel_ms[(protect, inject)] = kms / kn if kn else None
        ms = e0.elapsed_time(e1) / nsteps
        corr = sum(int(fb.report_from_device(r).corrected) for r in reps) if protect else 0
        det = sum(int(fb.report_from_device(r).detected) for r in reps) if protect else 0
        fb.ftblas_set_injection(None)
        return ms, det, corr

    def timed_pair():
        """Unprotected and protected (clean) calls alternated in one region, each bracketed by
        its own CUDA events, so that both see the same clocks: a power-capped part slows
        whatever region runs later, which would otherwise tilt the overhead."""
        fb.ftblas_set_injection(None)
        for _ in range(warmup):
            call(False)
            call(True)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        call(False)
        call(True)
        e1.record()
        torch.cuda.synchronize(dev)
        # pairs covering at least 4.5 s, so that the clock sampler (every 200 ms) records
        # twenty and more samples through the region
        npairs = max(steps, min(8192, int(4500.0 / max(e0.elapsed_time(e1), 1e-3)) + 1))
        # each step: unprotected (the library's fastest form), protected, and unprotected in
        # the protected call's kernel form (the same-kernel overhead)
        # (when both calls take the same form by default, the third call is left out)
        ev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(4)) for _ in range(npairs)]
        reps = [fb.new_report(dev) for _ in range(npairs)]
        ft_form = fb.tc_cta_group(True)
        same = ft_form == fb.tc_cta_group(False)
        for i in range(npairs):
            ev[i][0].record()
            call(False)
            ev[i][1].record()
            call(True, reps[i])
            ev[i][2].record()
            if not same:
                prev = fb.ftblas_set_tc_cta_group(ft_form)
                call(False)
                fb.ftblas_set_tc_cta_group(prev)
                ev[i][3].record()
        torch.cuda.synchronize(dev)
        na = sum(a.elapsed_time(b) for a, b, _, _ in ev) / npairs
        ft = sum(b.elapsed_time(c) for _, b, c, _ in ev) / npairs
        na_same = na if same else sum(c.elapsed_time(d) for _, _, c, d in ev) / npairs
        det = sum(int(fb.report_from_device(r).detected) for r in reps)
        return na, ft, det, npairs, na_same

    def burst(protect, calls=10):
        """Mean product-kernel time of a short burst of calls after an idle second: the
        conditions of the measured burst peak (the best of 10 single GEMMs), before power
        capping sets in. The long regions above run at the power cap."""
        fb.ftblas_set_injection(None)
        torch.cuda.synchronize(dev)
        time.sleep(1.0)
        fb.ftblas_kernel_timing_begin()
        for _ in range(calls):
            call(protect)
        torch.cuda.synchronize(dev)
        _, kms, kn = fb.ftblas_kernel_timing_end()
        return kms / kn if kn else None

    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    sampler.__enter__()  # started before the first warm-up; runs through the timed regions
    ms_na, ms_ft, det_pair, npairs, ms_na_same = timed_pair()
    _, _, _ = timed(False, False)  # unprotected product-kernel time for the roofline note
    _, det0, _ = timed(True, False)  # protected product-kernel time for the roofline
    ms_inj, det_inj, corr_inj = timed(True, True)
    det0 += det_pair
    sampler.__exit__(None, None, None)
    kb_na, kb_ft = burst(False), burst(True)
    # accuracy against the FP64 product of the same operands, on a sampled 4 x 64 block
    call(True)
    torch.cuda.synchronize(dev)
    rows = np.unique(S.randint(seed, 9, 4, 0, n - 1))
    cols = np.unique(S.randint(seed, 10, 64, 0, n - 1))
    Cfull = dC.view(n, n).t()
    C = Cfull[torch.as_tensor(rows, device=dev)][:, torch.as_tensor(cols, device=dev)].double().cpu().numpy()
    A64 = deq(abits[rows, :], sa)
    B64 = deq(bbits_t[cols, :], sb).T
    ref = A64 @ B64
    scale = np.abs(A64) @ np.abs(B64)
    err_norm = float(np.max(np.abs(C - ref) / scale))
    err_rel = float(np.median(np.abs(C - ref) / np.maximum(np.abs(ref), 1e-30)))
    # detection map over p (config 3): one output error 2^p |C(i,j)| per launch at a seeded element
    det_map = {}
    for p in range(-20, 13, 2):
        hits = 0
        trials = 4
        for t in range(trials):
            fb.ftblas_set_injection(fb.make_injection(seed=seed + 1000 * p + t, site=fb.SITE_OUTPUT,
                                                      mode=fb.MODE_ADD_REL, log2_lo=p, log2_hi=p, every_n_launches=1,
                                                      errors_per_launch=1))
            rep = fb.new_report(dev)
            call(True, rep)
            torch.cuda.synchronize(dev)
            hits += int(fb.report_from_device(rep).corrected)
        det_map[str(p)] = hits / trials
    fb.ftblas_set_injection(None)
    u = "2^-22" if fp8 else "2^-23"
    pk = peaks()
    peak = pk["bf16"] * (2.0 if fp8 else 1.0)
    k_ft, k_na = kernel_ms.get((True, False)), kernel_ms.get((False, False))
    roof = None
    if k_ft and kb_ft:
        pair = fb.tc_cta_group(True) == 2
        kname = "tc_gemm_pair_kernel" if pair else "tc_gemm_kernel"
        prof = f"{kname}_{kind}_ft_{n}_dram"
        peak_sus = pk["bf16_sustained"] * (2.0 if fp8 else 1.0)
        # each kernel time against the peak measured under the same conditions: a short burst
        # against the burst peak, the long power-capped region against the sustained peak
        roof = {"bound": "tensor", "achieved": flops / kb_ft / 1e9, "peak": peak, "unit": "TFLOP/s",
                "frac": flops / kb_ft / 1e9 / peak, "kernel_ms": kb_ft,
                "timing": "mean product-kernel time of 10 protected calls after 1 s idle (burst, as the peak)",
                "achieved_sustained": flops / k_ft / 1e9, "peak_sustained": peak_sus,
                "frac_sustained": flops / k_ft / 1e9 / peak_sus, "kernel_ms_sustained": k_ft,
                "timing_sustained": "mean product-kernel time over a region of protected calls following "
                                    "seconds of back-to-back calls (power-capped)",
                "traffic": profile_traffic(prof, TC_KERNEL_SOURCES),
                "peak_source": pk["bf16_src"] + (" x 2 (nominal FP8:BF16 dense ratio 4.5/2.25)" if fp8 else ""),
                "kernel": f"{kname}<FT, {kind.upper()}> (protected product kernel, "
                          + ("CTA pairs, cta_group::2" if pair else "one CTA per tile")
                          + "; encode and resolve kernels excluded)",
                "noabft_kernel_frac": (flops / kb_na / 1e9 / peak) if kb_na else None}
    values = ("N(0,1) quantised per tensor to E4M3 (scale = amax/448)" if fp8
              else "N(0,1), A rows scaled by 2^u (u in [-8, 8])")
    return {
        "workload": f"ft_gemm_{kind}_fp32acc_{n}x{n}x{n}, {values}",
        "ft_tflops": flops / ms_ft / 1e9, "ft_tflops_injected": flops / ms_inj / 1e9,
        "noabft_tflops": flops / ms_na / 1e9,
        "abft_overhead_pct": 100.0 * (ms_ft / ms_na - 1.0),
        "noabft_tflops_same_form": flops / ms_na_same / 1e9,
        "abft_overhead_pct_same_form": 100.0 * (ms_ft / ms_na_same - 1.0),
        "kernel_forms": {"protected": "one CTA per tile" if fb.tc_cta_group(True) == 1 else "CTA pairs",
                         "unprotected": "one CTA per tile" if fb.tc_cta_group(False) == 1 else "CTA pairs",
                         "note": "abft_overhead_pct: protected call vs the fastest unprotected call; "
                                 "_same_form: vs the unprotected call of the protected call's kernel form"},
        "speedup_over_fp64_ft": (flops / ms_ft / 1e9) / fp64_tflops if fp64_tflops else None,
        "false_alarms_clean": det0, "injected": timed_steps[(True, True)], "corrected": corr_inj, "detected": det_inj,
        "undetected_below_threshold": timed_steps[(True, True)] - det_inj,
        "injected_magnitude": f"2^{18 if fp8 else 16}..2^{22 if fp8 else 20} |C(i,j)| at a seeded element per call",
        "clocks": sampler.summary(),
        "timed_steps": {"alternating_steps": npairs, "ft_injected": timed_steps[(True, True)]},
        "method": "ft_tflops, noabft_tflops and the overheads from unprotected and protected calls (and "
                  "same-form unprotected calls when the forms differ) alternated in one region (per-call CUDA "
                  "events); ft_tflops_injected from a region of injected calls; the roofline from the "
                  "product-kernel events of a short burst after an idle second (burst peak) and of a region "
                  "of protected calls (sustained peak)",
        "seed": seed,
        "l2": l2_note_tc(2 * n * n * (1 if fp8 else 2), n * n * 4),
        "error_vs_fp64": {"max_over_sum_abs_ab": err_norm, "median_rel": err_rel,
                          "sampled": f"{len(rows)} rows x {len(cols)} columns",
                          "note": f"C - (A B computed in binary64 from the same {kind.upper()} operands)"},
        "detection_map_rel_log2": det_map,
        "roofline": roof,
        "threshold": f"rigorous: gamma_K({u}) |alpha| (sum_k|A(i,k)|)(max_k sum_j|B(k,j)|) (1 + s) + 2^-23 (sum|C|)",
    }


# ------------------------------------------------------------------ emulated FP64 (NEXT-3)
def run_emulated(dev, n, steps, warmup, fp64_tflops, slices=14):
    """FP64 GEMM formed from E4M3 integer slices on the tensor cores (ftblas_dgemm_emulated)
    on config 2's workload: column-major n^3, alpha 1.5, beta 0.5, A, B, C uniform[-1,1].
    Protected and unprotected calls alternated in one region (whole calls: the split passes,
    the product kernel and the resolve pass), then a region with one seeded accumulator flip
    per call (a group value's bit 0-31, detected exactly). Reports TFLOP/s (2 n^3 per call),
    the overhead, the speedup over the native FP64 FT-DGEMM, the error against the binary64
    product on sampled rows, and the product kernel's tensor-pipe roofline (its E4M3 work is
    s (s+1) / 2 slice products of 2 n^3)."""
    import torch

    import paper_2104_00897_gb300 as fb
    import synth as S

    prev = fb.ftblas_set_emulation_slices(slices)
    A, B, Cin = gen_inputs(n, SEED)
    dA = torch.from_numpy(A).to(dev)
    dB = torch.from_numpy(B).to(dev)
    dC0 = torch.from_numpy(Cin).to(dev)
    dC = dC0.clone()
    st = torch.cuda.current_stream(dev).cuda_stream
    flops = 2.0 * n ** 3

    def call(protect, rep=None):
        a = (fb.COL_MAJOR, fb.NO_TRANS, fb.NO_TRANS, n, n, n, 1.5, dA.data_ptr(), n, dB.data_ptr(), n, 0.5,
             dC.data_ptr(), n, st)
        if protect:
            fb.check(fb.ftblas_dgemm_emulated(*a, rep.data_ptr() if rep is not None else None), "ftblas_dgemm_emulated")
        else:
            fb.check(fb.ftblas_dgemm_emulated_noabft(*a), "ftblas_dgemm_emulated_noabft")

    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    sampler.__enter__()
    fb.ftblas_set_injection(None)
    for _ in range(warmup):
        call(False)
        call(True)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    call(False)
    call(True)
    e1.record()
    torch.cuda.synchronize(dev)
    # pairs covering at least 4.5 s: twenty and more clock samples through the region
    npairs = max(steps, 4, int(4500.0 / max(e0.elapsed_time(e1), 1e-3)) + 1)
    ev = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(npairs)]
    reps = [fb.new_report(dev) for _ in range(npairs)]
    fb.ftblas_kernel_timing_begin()
    for i in range(npairs):
        ev[i][0].record()
        call(False)
        ev[i][1].record()
        call(True, reps[i])
        ev[i][2].record()
    torch.cuda.synchronize(dev)
    _, kms, kn = fb.ftblas_kernel_timing_end()  # product kernels: unprotected and protected alternate
    ms_na = sum(a.elapsed_time(b) for a, b, _ in ev) / npairs
    ms_ft = sum(b.elapsed_time(c) for _, b, c in ev) / npairs
    false_alarms = sum(int(fb.report_from_device(r).detected) for r in reps)
    # protected product-kernel time alone, for the roofline
    nreg = max(steps, 4)
    fb.ftblas_kernel_timing_begin()
    for i in range(nreg):
        call(True)
    torch.cuda.synchronize(dev)
    _, kms_ft, kn_ft = fb.ftblas_kernel_timing_end()
    # one seeded accumulator flip per call: bits 0-31 of a leading group value
    fb.ftblas_set_injection(fb.make_injection(seed=SEED + 60, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit_lo=0,
                                              bit_hi=31, every_n_launches=1, errors_per_launch=1))
    irep = [fb.new_report(dev) for _ in range(nreg)]
    e0.record()
    for i in range(nreg):
        call(True, irep[i])
    e1.record()
    torch.cuda.synchronize(dev)
    fb.ftblas_set_injection(None)
    ms_inj = e0.elapsed_time(e1) / nreg
    sampler.__exit__(None, None, None)
    ir = [fb.report_from_device(r) for r in irep]
    # accuracy: one clean call from C_in, sampled rows against the binary64 library product
    dC.copy_(dC0)
    call(True)
    torch.cuda.synchronize(dev)
    rows = np.unique(S.randint(SEED, 9, 4, 0, n - 1))
    got = dC.view(n, n).t()[torch.as_tensor(rows, device=dev)].cpu().numpy()
    Am, Bm, Cm = (X.reshape(n, n, order="F") for X in (A, B, Cin))
    ref = 1.5 * (Am[rows, :] @ Bm) + 0.5 * Cm[rows, :]
    err = float(np.abs(got - ref).max() / (np.abs(A).max() * np.abs(B).max() * n))
    fb.ftblas_set_emulation_slices(prev)
    pk = peaks()
    peak8 = 2.0 * pk["bf16"]
    k_ft = kms_ft / kn_ft if kn_ft else None
    pairs = slices * (slices + 1) // 2
    roof = None
    if k_ft:
        tensor = pairs * flops / k_ft / 1e9
        roof = {"bound": "tensor", "achieved": tensor, "peak": peak8, "unit": "TFLOP/s", "frac": tensor / peak8,
                "peak_sustained": 2.0 * pk["bf16_sustained"], "frac_sustained": tensor / (2.0 * pk["bf16_sustained"]),
                "traffic": None, "peak_source": pk["bf16_src"] + " x 2 (nominal FP8:BF16 dense ratio 4.5/2.25)",
                "kernel": f"emu_gemm_kernel<FT> ({pairs} E4M3 slice products of 2 n^3 each per call)",
                "kernel_ms": k_ft}
    return {
        "workload": f"ft_dgemm_emulated_{n}x{n}x{n}, column-major, alpha 1.5, beta 0.5, U[-1,1], {slices} slices",
        "ft_tflops": flops / ms_ft / 1e9, "ft_tflops_injected": flops / ms_inj / 1e9,
        "noabft_tflops": flops / ms_na / 1e9, "abft_overhead_pct": 100.0 * (ms_ft / ms_na - 1.0),
        "product_kernel_ms": k_ft,
        "speedup_over_native_fp64_ft": (flops / ms_ft / 1e9) / fp64_tflops if fp64_tflops else None,
        "error_vs_fp64": {"normalized_max": err, "criterion": "max|C-C_ref|/(max|A| max|B| K) <= 1e-15",
                          "bound": f"(s+3) 16^-s + 3u = {(slices + 3) * 16.0 ** -slices + 3 * 2.0 ** -53:.2e}",
                          "rows_sampled": len(rows), "reference": "binary64 product of the same operands (library matmul)"},
        "faults": {"injected": nreg, "detected": sum(int(r.detected) for r in ir),
                   "corrected": sum(int(r.corrected) for r in ir), "checksum_only": sum(int(r.checksum_only) for r in ir),
                   "uncorrectable": sum(int(r.uncorrectable) for r in ir), "false_alarms_clean": false_alarms,
                   "note": "a flip that leaves C unchanged (a fraction bit of a small group value, rounded away) "
                           "is detected and classified checksum-only"},
        "roofline": roof,
        "clocks": sampler.summary(),
        "timed_calls": {"alternating_pairs": npairs, "product_kernel_region": nreg, "injected_region": nreg},
        "method": "protected and unprotected whole calls alternated in one region of at least 4.5 s (per-call "
                  "CUDA events); the product kernel timed in a region of protected calls",
    }


SWEEP_SHAPES = ((1024, 1024, 1024), (2048, 2048, 2048), (4096, 4096, 4096), (8192, 8192, 8192),
                (16384, 16384, 16384), (8192, 8192, 256), (32768, 1024, 1024))


def run_sweep(dev, steps, warmup, shapes=SWEEP_SHAPES):
    """Config 2: the FP64 FT-DGEMM (DFMA engine, column-major, alpha 1.5, beta 0.5, U[-1,1])
    against the unprotected kernel over square sizes 1024..16384 and the skinny and tall
    shapes; the protected runs carry one accumulator flip (bits 40-62) per 10 launches,
    placed so that a timed launch is hit. TFLOP/s from the product kernels' CUDA-event
    time (ftblas_kernel_timing)."""
    import torch

    import paper_2104_00897_gb300 as fb
    import synth as S

    fb.ftblas_set_fp64_engine(fb.ENGINE_DFMA)
    peak = peaks()["alu"]
    st = torch.cuda.current_stream(dev).cuda_stream
    rows = []
    for (M, N, K) in shapes:
        seed = SEED + 7
        dA = torch.from_numpy(S.uniform(seed, 0, M * K)).to(dev)
        dB = torch.from_numpy(S.uniform(seed, 1, K * N)).to(dev)
        dC = torch.from_numpy(S.uniform(seed, 2, M * N)).to(dev)
        flops = 2.0 * M * N * K

        def measure(protect, inject):
            if protect and inject:
                fb.ftblas_set_injection(fb.make_injection(seed=seed - seed % 10 + (warmup + 1) % 10, site=fb.SITE_ACCUM,
                                                          mode=fb.MODE_BITFLIP, bit_lo=40, bit_hi=62,
                                                          every_n_launches=10, errors_per_launch=1))
            else:
                fb.ftblas_set_injection(None)
            reps = [fb.new_report(dev) for _ in range(steps)]

            def call(rep):
                a = (fb.COL_MAJOR, fb.NO_TRANS, fb.NO_TRANS, M, N, K, 1.5, dA.data_ptr(), M, dB.data_ptr(), K, 0.5,
                     dC.data_ptr(), M, st)
                if protect:
                    fb.check(fb.ftblas_dgemm(*a, rep.data_ptr() if rep is not None else None))
                else:
                    fb.check(fb.ftblas_dgemm_noabft(*a))

            for _ in range(warmup):
                call(None)
            torch.cuda.synchronize(dev)
            fb.ftblas_kernel_timing_begin()
            for s_ in range(steps):
                call(reps[s_])
            torch.cuda.synchronize(dev)
            _, kms, kn = fb.ftblas_kernel_timing_end()
            fb.ftblas_set_injection(None)
            det = cor = 0
            if protect:
                for r in reps:
                    rr = fb.report_from_device(r)
                    det += int(rr.detected)
                    cor += int(rr.corrected)
            return kms / kn, det, cor

        ms_inj, det, cor = measure(True, True)
        ms_ft, det_clean, _ = measure(True, False)
        ms_na, _, _ = measure(False, False)
        edge = fb.ftblas_verification_tile(fb.COL_MAJOR, fb.R_64F, M, N, K)[0]
        rows.append({"M": M, "N": N, "K": K, "tile": f"{edge}x{edge}", "ft_tflops_injected": flops / ms_inj / 1e9,
                     "ft_tflops_clean": flops / ms_ft / 1e9, "noabft_tflops": flops / ms_na / 1e9,
                     "pct_of_fp64_peak_ft": 100.0 * flops / ms_ft / 1e9 / peak,
                     "abft_overhead_pct_clean": 100.0 * (ms_ft / ms_na - 1.0),
                     "abft_overhead_pct_injected": 100.0 * (ms_inj / ms_na - 1.0),
                     "detected": det, "corrected": cor, "false_alarms_clean": det_clean})
        del dA, dB, dC
        torch.cuda.empty_cache()
    return {"workload": "ft_dgemm FP64 (DFMA), column-major, alpha 1.5, beta 0.5, U[-1,1]; one accumulator flip "
                        "(bits 40-62) per 10 launches in the injected runs",
            "peak_tflops": peak, "steps": steps, "warmup": warmup, "rows": rows}


def run_fp64_large(dev, n=16384):
    """Config 2's largest square point in the default line: FP64 FT-DGEMM (DFMA) n^3,
    column-major, alpha 1.5, beta 0.5, U[-1,1]; after one warm-up each, one protected call
    with one fixed accumulator flip (bit 52, middle of the matrix), one clean protected call
    and one unprotected call, timed by the product kernels' CUDA events."""
    import torch

    import paper_2104_00897_gb300 as fb
    import synth as S

    fb.ftblas_set_fp64_engine(fb.ENGINE_DFMA)
    st = torch.cuda.current_stream(dev).cuda_stream
    seed = SEED + 7
    dA = torch.from_numpy(S.uniform(seed, 0, n * n)).to(dev)
    dB = torch.from_numpy(S.uniform(seed, 1, n * n)).to(dev)
    dC = torch.from_numpy(S.uniform(seed, 2, n * n)).to(dev)
    flops = 2.0 * n ** 3
    rep = fb.new_report(dev)

    def timed(protect, pts):
        fb.ftblas_set_injection(fb.make_injection(fixed=pts) if pts else None)
        a = (fb.COL_MAJOR, fb.NO_TRANS, fb.NO_TRANS, n, n, n, 1.5, dA.data_ptr(), n, dB.data_ptr(), n, 0.5,
             dC.data_ptr(), n, st)
        fb.ftblas_kernel_timing_begin()
        fb.check(fb.ftblas_dgemm(*a, rep.data_ptr()) if protect else fb.ftblas_dgemm_noabft(*a))
        torch.cuda.synchronize(dev)
        _, kms, _ = fb.ftblas_kernel_timing_end()
        fb.ftblas_set_injection(None)
        return kms, (fb.report_from_device(rep) if protect else None)

    timed(True, None)   # warm-up
    timed(False, None)
    pt = [dict(i=n // 2 + 17, j=n // 3 + 5, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=52)]
    ms_inj, r_inj = timed(True, pt)
    ms_ft, r_ft = timed(True, None)
    ms_na, _ = timed(False, None)
    peak = peaks()["alu"]
    del dA, dB, dC
    torch.cuda.empty_cache()
    return {"workload": f"ft_dgemm FP64 (DFMA) {n}x{n}x{n}, column-major, alpha 1.5, beta 0.5, U[-1,1]",
            "ft_tflops_injected": flops / ms_inj / 1e9, "ft_tflops_clean": flops / ms_ft / 1e9,
            "noabft_tflops": flops / ms_na / 1e9, "pct_of_fp64_peak_clean": 100.0 * flops / ms_ft / 1e9 / peak,
            "abft_overhead_pct_clean": 100.0 * (ms_ft / ms_na - 1.0),
            "abft_overhead_pct_injected": 100.0 * (ms_inj / ms_na - 1.0),
            "injected": 1, "detected": int(r_inj.detected), "corrected": int(r_inj.corrected),
            "located": [(int(r.i), int(r.j)) for r in r_inj.records()], "false_alarms_clean": int(r_ft.detected),
            "method": "one timed call each (7 s per call), after one warm-up each"}


def run_level3(dev, n, steps, warmup):
    """FT-DSYMM, FT-DTRMM and FT-DTRSM (side left, upper, column-major, n x n operands,
    U[-1,1]; DTRSM on a diagonally dominant A): TFLOP/s by their own flop counts (DSYMM
    2 n^3, DTRMM and DTRSM n^3) over the whole call (copies of the symmetric / triangular
    operand and of B included), one accumulator flip in the timed DSYMM / DTRMM calls
    (inside the faulted tile's k-range for DTRMM), one flip in every internal step of the
    timed DTRSM calls."""
    import torch

    import paper_2104_00897_gb300 as fb
    import synth as S

    A = torch.from_numpy(S.uniform(SEED + 9, 0, n * n)).to(dev)
    Ad = A.clone().view(n, n)  # column-major storage: Ad[c, r] holds A(r, c)
    Ad.mul_(1.0 / (2 * n))
    Ad.diagonal().add_(1.0)
    B = torch.from_numpy(S.uniform(SEED + 9, 1, n * n)).to(dev)
    C = torch.from_numpy(S.uniform(SEED + 9, 2, n * n)).to(dev)
    st = torch.cuda.current_stream(dev).cuda_stream
    nk = -(-n // 32)
    out = {}
    for name, flops in (("dsymm", 2.0 * n ** 3), ("dtrmm", 1.0 * n ** 3), ("dtrsm", 1.0 * n ** 3)):
        def call(rep):
            if name == "dtrsm":
                fb.check(fb.ftblas_dtrsm(fb.COL_MAJOR, fb.LEFT, fb.UPPER, fb.NO_TRANS, fb.NON_UNIT, n, n, 1.0,
                                         Ad.data_ptr(), n, B.data_ptr(), n, st,
                                         rep.data_ptr() if rep is not None else None))
            elif name == "dsymm":
                fb.check(fb.ftblas_dsymm(fb.COL_MAJOR, fb.LEFT, fb.UPPER, n, n, 1.0, A.data_ptr(), n, B.data_ptr(), n,
                                         0.5, C.data_ptr(), n, st, rep.data_ptr() if rep is not None else None))
            else:
                fb.check(fb.ftblas_dtrmm(fb.COL_MAJOR, fb.LEFT, fb.UPPER, fb.NO_TRANS, fb.NON_UNIT, n, n, 1.0,
                                         A.data_ptr(), n, B.data_ptr(), n, st,
                                         rep.data_ptr() if rep is not None else None))
        for _ in range(warmup):
            call(None)
        torch.cuda.synchronize(dev)
        pts = [dict(i=n // 2 + 5, j=7, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=57, kt=(3 * nk) // 4)]
        if name == "dtrsm":  # applies to every internal step, in its own coordinates
            pts = [dict(i=5, j=7, site=fb.SITE_OUTPUT, mode=fb.MODE_BITFLIP, bit=57)]
        fb.ftblas_set_injection(fb.make_injection(fixed=pts))
        reps = [fb.new_report(dev) for _ in range(steps)]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for s_ in range(steps):
            call(reps[s_])
        e1.record()
        torch.cuda.synchronize(dev)
        fb.ftblas_set_injection(None)
        ms = e0.elapsed_time(e1) / steps
        rr = [fb.report_from_device(r) for r in reps]
        out[name] = {"tflops": flops / ms / 1e9, "ms": ms,
                     "injected": steps * ((2 * -(-n // 128) - 1) if name == "dtrsm" else 1),
                     "corrected": sum(int(r.corrected) for r in rr), "detected": sum(int(r.detected) for r in rr)}
    out["workload"] = (f"FT-DSYMM / FT-DTRMM / FT-DTRSM {n}x{n}, side left, upper, column-major, U[-1,1] "
                       "(DTRSM: A scaled by 1/(2n) plus the identity)")
    return out


def run_unfused(dev, n, steps, warmup):
    """NEXT-1 comparator: the same FP64 workload as the headline (8192^3, column-major, alpha
    1.5, beta 0.5, U[-1,1]) through ftblas_dgemm_unfused: ABFT as separate bandwidth-bound
    passes around cuBLAS's DGEMM, against cuBLAS alone. The product kernel's time comes
    from ftblas_kernel_timing (events around the library GEMM); the passes' time is the
    rest of the call."""
    import torch

    import paper_2104_00897_gb300 as fb

    A, B, Cin = gen_inputs(n, rank_seed(0))
    dA = torch.from_numpy(A).to(dev)
    dB = torch.from_numpy(B).to(dev)
    dC = torch.from_numpy(Cin).to(dev)
    st = torch.cuda.current_stream(dev).cuda_stream
    flops = 2.0 * n ** 3

    def timed(inject):
        if inject:
            fb.ftblas_set_injection(fb.make_injection(seed=SEED, site=fb.SITE_OUTPUT, mode=fb.MODE_BITFLIP, bit_lo=40,
                                                      bit_hi=62, every_n_launches=1, errors_per_launch=1))
        else:
            fb.ftblas_set_injection(None)
        reps = [fb.new_report(dev) for _ in range(steps)]

        def call(rep):
            fb.check(fb.ftblas_dgemm_unfused(fb.COL_MAJOR, fb.NO_TRANS, fb.NO_TRANS, n, n, n, 1.5, dA.data_ptr(), n,
                                             dB.data_ptr(), n, 0.5, dC.data_ptr(), n, st,
                                             rep.data_ptr() if rep is not None else None), "ftblas_dgemm_unfused")

        for _ in range(warmup):
            call(None)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fb.ftblas_kernel_timing_begin()
        e0.record()
        for s_ in range(steps):
            call(reps[s_])
        e1.record()
        torch.cuda.synchronize(dev)
        _, kms, kn = fb.ftblas_kernel_timing_end()
        fb.ftblas_set_injection(None)
        det = sum(int(fb.report_from_device(r).detected) for r in reps)
        cor = sum(int(fb.report_from_device(r).corrected) for r in reps)
        return e0.elapsed_time(e1) / steps, (kms / kn if kn else None), det, cor

    ms_clean, gemm_ms, det0, _ = timed(False)
    ms_inj, _, det, cor = timed(True)
    # cuBLAS alone (through torch): C = A B on the column-major operands (as row-major
    # transposes: C^T = B^T A^T), same sizes
    a_t = dA.view(n, n)
    b_t = dB.view(n, n)
    for _ in range(warmup):
        torch.mm(b_t, a_t)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        torch.mm(b_t, a_t)
    e1.record()
    torch.cuda.synchronize(dev)
    ms_cublas = e0.elapsed_time(e1) / steps
    pass_ms = ms_clean - gemm_ms if gemm_ms else None
    pass_bytes = (3 * n * n + 2 * n * n) * 8  # A, B, C_in and C read once each (+ prediction operands)
    return {
        "workload": f"ft_dgemm_unfused_{n}x{n}x{n}: checksum passes around cuBLAS DGEMM, alpha 1.5, beta 0.5",
        "unfused_ft_tflops": flops / ms_clean / 1e9, "unfused_ft_tflops_injected": flops / ms_inj / 1e9,
        "cublas_dgemm_tflops": flops / ms_cublas / 1e9,
        "unfused_overhead_pct_vs_cublas": 100.0 * (ms_clean / ms_cublas - 1.0),
        "checksum_passes_ms": pass_ms, "library_gemm_ms_inside_call": gemm_ms,
        "checksum_passes_gbs": (pass_bytes / (pass_ms / 1e3) / 1e9) if pass_ms and pass_ms > 0 else None,
        "false_alarms_clean": det0, "injected": steps, "detected": det, "corrected": cor,
    }


def run_linear(dev, steps, warmup, T=8192, n_in=4096, n_out=4096):
    """Config 4: Y = X W^T through FTLinearFn with X (T x n_in) BF16 N(0,1), W (n_out x n_in)
    BF16 N(0, 0.02), dY N(0,1): forward (T, n_out, n_in), dX = dY W (T, n_in, n_out) and
    dW = dY^T X (n_out, n_in, T), all three protected, one injected output fault
    (2^12..2^14 |C|) per GEMM pass. Reports the fwd+bwd step time as TFLOP/s (6 T n_in n_out
    flops per step), the faults corrected, and the gradients' error against binary64
    products of the same BF16 values on sampled rows."""
    import torch

    import paper_2104_00897_gb300 as fb
    import synth as S

    threads = max(1, min(16, os.cpu_count() or 1))
    seed = SEED + 4
    X = S.map_elementwise(S.to_bf16_bits, S.normal_matrix(seed, 0, T, n_in, threads=threads), np.uint16, threads)
    W = S.map_elementwise(S.to_bf16_bits, S.normal_matrix(seed, 1, n_out, n_in, std=0.02, threads=threads), np.uint16,
                          threads)
    dY = S.normal_matrix(seed, 2, T, n_out, threads=threads)
    x = torch.from_numpy(np.ascontiguousarray(X).view(np.int16)).to(dev).view(torch.bfloat16).requires_grad_(True)
    w = torch.from_numpy(np.ascontiguousarray(W).view(np.int16)).to(dev).view(torch.bfloat16).requires_grad_(True)
    dy = torch.from_numpy(np.ascontiguousarray(dY)).to(dev).to(torch.bfloat16)  # Y is bfloat16
    Fn = fb.FTLinearFn

    def step(mon):
        x.grad = None
        w.grad = None
        y = Fn.apply(x, w, mon)
        y.backward(dy)

    fb.ftblas_set_injection(fb.make_injection(seed=seed, site=fb.SITE_OUTPUT, mode=fb.MODE_ADD_REL, log2_lo=12,
                                              log2_hi=14, every_n_launches=1, errors_per_launch=1))
    for _ in range(warmup):
        step(None)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    step(None)
    e1.record()
    torch.cuda.synchronize(dev)
    step_ms = max(e0.elapsed_time(e1), 1e-3)
    # at least 0.3 s of further warm-up (clocks settle after the process starts), then as
    # many timed steps as cover at least 1 s (a step takes about a millisecond)
    for _ in range(int(300.0 / step_ms)):
        step(None)
    torch.cuda.synchronize(dev)
    nsteps = max(steps, min(4096, int(1000.0 / step_ms) + 1))
    mon = fb.FTMonitor(dev)
    e0.record()
    for _ in range(nsteps):
        step(mon)
    e1.record()
    torch.cuda.synchronize(dev)
    fb.ftblas_set_injection(None)
    ms = e0.elapsed_time(e1) / nsteps
    summ = mon.summary()
    # gradient error on sampled rows (the faulted elements were corrected from the checksums)
    rows = np.unique(S.randint(seed, 9, 4, 0, n_out - 1))
    Wf = S.bf16_bits_to_f64(W)
    dYq = S.bf16_bits_to_f64(S.to_bf16_bits(dy.double().cpu().numpy()))
    dX = x.grad.double().cpu().numpy()[rows]
    ref = dYq[rows] @ Wf
    err_dx = float(np.max(np.abs(dX - ref) / (np.abs(dYq[rows]) @ np.abs(Wf))))
    Xf = S.bf16_bits_to_f64(X)
    dW = w.grad.double().cpu().numpy()[rows]
    ref = dYq[:, rows].T @ Xf
    err_dw = float(np.max(np.abs(dW - ref) / (np.abs(dYq[:, rows]).T @ np.abs(Xf))))
    return {
        "workload": f"FTLinearFn Y = X W^T, X {T}x{n_in} BF16 N(0,1), W {n_out}x{n_in} BF16 N(0,0.02), dY N(0,1); "
                    "forward + backward (3 protected GEMMs with bfloat16 Y, dX, dW rounded from the verified "
                    "FP32 products; MN-major operands copied K-major by the library)",
        "step_ms": ms, "timed_steps": nsteps, "tflops": 6.0 * T * n_in * n_out / ms / 1e9, "gemm_calls": summ["calls"],
        "faults_injected": summ["calls"], "detected": summ["detected"], "corrected": summ["corrected"],
        "uncorrectable": summ["uncorrectable"],
        "grad_error_over_sum_abs": {"dX": err_dx, "dW": err_dw, "rows_sampled": int(len(rows)),
                                    "note": "bfloat16 gradients vs binary64 products of the same BF16 values"},
    }


def run_soak(dev, n, seconds, seed=SEED + 50, rate_per_s=5.0, batch=256, bit_lo=40, bit_hi=62):
    """Soak (config 5a): the FP64 FT-DGEMM (alpha = 1, beta = 0, U[-1,1] operands) launched
    back to back for `seconds`. Before each launch a Poisson(rate x launch time) number of
    accumulator bit flips (bits bit_lo..bit_hi, after BK floor(nk/2) products) is drawn on
    distinct tiles and installed as that launch's plan. Reports come back through a ring of
    `batch` report buffers read once per batch. Tally: a tile with an injection and a record
    is detected (corrected or not); a record in a tile without one is a false alarm; an
    injected tile without a record is undetected (an error at or below the threshold). The
    final C is compared with a clean run's: bitwise equal when every injected error was
    corrected, since the FP64 correction recomputes the element exactly."""
    import torch

    import paper_2104_00897_gb300 as fb

    A, B, _ = gen_inputs(n, seed)
    dA = torch.from_numpy(A).to(dev)
    dB = torch.from_numpy(B).to(dev)
    dC = torch.empty(n * n, dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream(dev).cuda_stream
    tr, tc, _ = fb.ftblas_verification_tile(fb.COL_MAJOR, fb.R_64F, n, n, n)
    ntr, ntc = -(-n // tr), -(-n // tc)
    reps = torch.zeros((batch, fb.REPORT_BYTES), dtype=torch.uint8, device=dev)

    def call(slot):
        fb.check(fb.ftblas_dgemm(fb.COL_MAJOR, fb.NO_TRANS, fb.NO_TRANS, n, n, n, 1.0, dA.data_ptr(), n,
                                 dB.data_ptr(), n, 0.0, dC.data_ptr(), n, st, reps[slot].data_ptr()), "ftblas_dgemm")

    fb.ftblas_set_injection(None)
    for _ in range(3):
        call(0)
    torch.cuda.synchronize(dev)
    clean = dC.clone()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        call(0)
    e1.record()
    torch.cuda.synchronize(dev)
    t_launch = e0.elapsed_time(e1) / 10 / 1e3
    lam = rate_per_s * t_launch
    batch = int(max(1, min(batch, seconds / t_launch / 8)))  # about 8 report read-backs over the soak
    rng = np.random.Generator(np.random.PCG64(seed))
    tally = dict(launches=0, injected=0, detected=0, corrected=0, uncorrectable=0, checksum_only=0, undetected=0,
                 false_alarms=0, status=0)
    import time
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        plans = []
        for b in range(batch):
            k = min(int(rng.poisson(lam)), fb.MAX_FIXED_INJECTIONS, ntr * ntc)
            tiles = rng.choice(ntr * ntc, size=k, replace=False) if k else []
            pts = []
            for t in tiles:
                r0, c0 = (int(t) % ntr) * tr, (int(t) // ntr) * tc
                pts.append(dict(i=r0 + int(rng.integers(0, min(tr, n - r0))), j=c0 + int(rng.integers(0, min(tc, n - c0))),
                                site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=int(rng.integers(bit_lo, bit_hi + 1))))
            fb.ftblas_set_injection(fb.make_injection(fixed=pts) if pts else None)
            call(b)
            plans.append(pts)
        host = reps.cpu().numpy()
        for b, pts in enumerate(plans):
            r = fb.FtReport.from_buffer_copy(host[b].tobytes())
            inj_tiles = {(p["i"] // tr, p["j"] // tc) for p in pts}
            rec_tiles = {}
            for rec in r.records():
                rec_tiles[(rec.tile_row, rec.tile_col)] = rec.kind
            tally["launches"] += 1
            tally["injected"] += len(pts)
            tally["status"] |= int(r.status)
            for key, kind in rec_tiles.items():
                if key in inj_tiles:
                    tally["detected"] += 1
                    tally["corrected"] += kind == fb.KIND_CORRECTED
                    tally["uncorrectable"] += kind == fb.KIND_UNCORRECTABLE
                    tally["checksum_only"] += kind == fb.KIND_CHECKSUM_ONLY
                else:
                    tally["false_alarms"] += 1
            tally["undetected"] += len(inj_tiles - set(rec_tiles))
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    fb.ftblas_set_injection(None)
    last_pts = plans[-1]
    tally.update({
        "workload": f"ft_dgemm_{n}x{n}x{n} back to back, alpha=1, beta=0, U[-1,1]",
        "seconds": wall, "launch_ms": 1e3 * t_launch, "poisson_lambda_per_launch": lam,
        "injections_per_minute": 60.0 * tally["injected"] / wall,
        "sustained_tflops": tally["launches"] * 2.0 * n ** 3 / wall / 1e12,
        "injection": f"accumulator bit flips, bits {bit_lo}..{bit_hi}, distinct tiles",
        "final_c_equals_clean": bool(torch.equal(dC, clean)),
        "last_launch_injections": len(last_pts),
    })
    return tally


# ------------------------------------------------------------------ reference arm (the oracle)
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import oracle as O
    n = args.size
    A, B, Cin = gen_inputs(n, SEED)
    threads = O.num_threads()
    per_step = max(1, min(16, threads))
    times, flops = [], 0.0
    for s in range(args.warmup + args.steps):
        f, dt, _ = oracle_sample(n, A, B, Cin, per_step, seed_tiles=1000 + s)
        if s >= args.warmup:
            times.append(dt)
            flops += f
    total = sum(times)
    value = flops / total / 1e12
    sample = f"{per_step} seeded {TILE}x{TILE} output tiles of the {n}^3 problem per step (full K, checksums included)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(n, "cpu-oracle"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, dist):
    import ctypes

    import torch

    import paper_2104_00897_gb300 as fb

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fb.load()
    n = args.size
    if args.tc_cta_group is not None:
        fb.ftblas_set_tc_cta_group(args.tc_cta_group)
    if world > 1:
        # At N > 1 the line carries the scaled headline (and its end-to-end figure) only: the
        # single-GPU sections are reported by the N = 1 run, and running them on rank 0
        # alone would hold the other GPUs idle.
        for flag in ("no_bf16", "no_fp8", "no_linear", "no_unfused", "no_level3", "no_online", "no_second_engine",
                     "no_emulated", "no_large", "no_soak_default"):
            setattr(args, flag, True)
    if args.sweep:
        if rank == 0:
            print(json.dumps({"sweep_fp64": run_sweep(dev, args.steps, args.warmup)}), flush=True)
        return 0
    if args.level3_only:
        if rank == 0:
            print(json.dumps({"level3_fp64": run_level3(dev, n, args.steps, args.warmup)}), flush=True)
        return 0
    if args.unfused_only:
        if rank == 0:
            print(json.dumps({"unfused_fp64": run_unfused(dev, n, args.steps, args.warmup)}), flush=True)
        return 0
    if args.linear_only:
        if rank == 0:
            print(json.dumps({"linear_bf16": run_linear(dev, args.steps, args.warmup)}), flush=True)
        return 0
    if args.soak > 0:
        if rank == 0:
            print(json.dumps({"soak": run_soak(dev, n, args.soak, rate_per_s=args.soak_rate)}), flush=True)
        return 0
    if args.emulated_only:
        if rank == 0:
            print(json.dumps({"fp64_emulated": run_emulated(dev, n, args.steps, args.warmup, None)}), flush=True)
        return 0
    if args.bf16_only or args.fp8_only:
        if rank == 0:
            kind = "bf16" if args.bf16_only else "fp8"
            size = n if args.bf16_only else args.fp8_size
            print(json.dumps({kind: run_tc(args, dev, kind, size, args.steps, args.warmup, None)}), flush=True)
        return 0
    flops_step = 2.0 * n * n * n
    A, B, Cin = gen_inputs(n, rank_seed(rank))
    dA = torch.from_numpy(A).to(dev)
    dB = torch.from_numpy(B).to(dev)
    dCin = torch.from_numpy(Cin).to(dev)
    dC = dCin.clone()
    stream = torch.cuda.current_stream(dev)
    st = stream.cuda_stream
    engines = {"dfma": fb.ENGINE_DFMA, "dmma": fb.ENGINE_DMMA}

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()


    def timed(protect, inject, steps, warmup, clocks=False):
        """Per-launch device times (ms) of `steps` calls after `warmup`, with reports."""
        if protect and inject:
            # one flip per 10 launches, placed so that it falls inside the timed steps
            seed = rank_seed(rank) - (rank_seed(rank) % 10) + ((warmup + 1) % 10)
            fb.ftblas_set_injection(fb.make_injection(seed=seed, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit_lo=40,
                                                      bit_hi=62, every_n_launches=10, errors_per_launch=1))
        else:
            fb.ftblas_set_injection(None)
        reps = [fb.new_report(dev) for _ in range(steps)]
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]

        def call(rep):
            args_ = (fb.COL_MAJOR, fb.NO_TRANS, fb.NO_TRANS, n, n, n, 1.5, dA.data_ptr(), n, dB.data_ptr(), n, 0.5,
                     dC.data_ptr(), n, st)
            if protect:
                fb.check(fb.ftblas_dgemm(*args_, rep.data_ptr() if rep is not None else None))
            else:
                fb.check(fb.ftblas_dgemm_noabft(*args_))

        # the clock sampler starts before the warm-up (its start-up can stall this process's
        # CUDA calls) and runs through the timed region
        sampler = ClockSampler(local) if clocks else None
        if sampler:
            sampler.__enter__()
        for _ in range(warmup):
            call(None)
        barrier()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        fb.ftblas_kernel_timing_begin()
        t0.record(stream)
        for s in range(steps):
            ev[s][0].record(stream)
            call(reps[s])
            ev[s][1].record(stream)
        t1.record(stream)
        barrier()
        _, kms, kn = fb.ftblas_kernel_timing_end()
        if sampler:
            sampler.__exit__(None, None, None)
        total_ms = max_over_ranks(t0.elapsed_time(t1), dist)
        per = [a.elapsed_time(b) for a, b in ev]
        rsum = {"detected": 0, "corrected": 0, "uncorrectable": 0, "checksum_only": 0, "tiles_checked": 0,
                "status": 0}
        if protect:
            for r in reps:
                rr = fb.report_from_device(r)
                for k in ("detected", "corrected", "uncorrectable", "checksum_only", "tiles_checked"):
                    rsum[k] += int(getattr(rr, k))
                rsum["status"] |= int(rr.status)
            status = or_over_ranks(rsum.pop("status"), dist)
            rsum = sum_over_ranks(rsum, dist)
            rsum["status"] = status
        injected = 0
        if protect and inject:
            # every rank injects in the same launches (its seed is shifted to the same residue)
            injected = world * sum(1 for L in range(warmup, warmup + steps) if L % 10 == ((warmup + 1) % 10))
        fb.ftblas_set_injection(None)
        kernel_per = [kms / kn] * kn if kn == steps else per
        return total_ms, kernel_per, rsum, injected, (sampler.summary() if sampler else None)

    results = {}
    def measure_e2e():
        """The headline metric through the host-buffer entry point, measured right after the
        device-timed runs of the headline engine (same clocks regime), clocks sampled."""
        hA = torch.from_numpy(A).pin_memory()
        hB = torch.from_numpy(B).pin_memory()
        hC = torch.from_numpy(Cin).pin_memory()
        hrep = fb.FtReport()
        fb.ftblas_set_injection(None)

        def hcall():
            fb.check(fb.ftblas_dgemm_host(fb.COL_MAJOR, fb.NO_TRANS, fb.NO_TRANS, n, n, n, 1.5, hA.data_ptr(), n,
                                          hB.data_ptr(), n, 0.5, hC.data_ptr(), n, st, ctypes.addressof(hrep)))

        # No nvidia-smi sampler here: its queries stall this process's CUDA calls, and the
        # host-buffer call synchronises every step, so they would land in the wall-clock
        # region. The device-timed runs just before carry the clock record.
        for _ in range(max(1, min(args.warmup, 2))):
            hcall()
        barrier()
        # CUDA events around each call (they bracket the copies and the kernels on the stream)
        # split the wall time into the device's share and the host's
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        fb.ftblas_kernel_timing_begin()
        t0 = time.perf_counter()
        for s_ in range(args.steps):
            evs[s_][0].record()
            hcall()
            evs[s_][1].record()
        barrier()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist)
        _, kms, kn = fb.ftblas_kernel_timing_end()
        dev_ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
        return {"value": job_tflops(world, flops_step, args.steps, 1e3 * e2e_s), "unit": UNIT,
                "h2d_bytes_per_step": 3 * n * n * 8, "d2h_bytes_per_step": n * n * 8 + fb.REPORT_BYTES,
                "wall_ms_per_call": 1e3 * e2e_s / args.steps, "stream_ms_per_call": dev_ms,
                "kernel_ms_per_call": kms / kn if kn else None}

    engine_list = [args.engine] + ([] if args.no_second_engine else [e for e in engines if e != args.engine])
    clocks = None
    e2e = None
    for eng in engine_list:
        fb.ftblas_set_fp64_engine(engines[eng])
        head = eng == args.engine
        ft_ms, ft_per, ft_rep, injected, clk = timed(True, True, args.steps, args.warmup, clocks=head)
        if head:
            clocks = clk
            if not args.no_e2e:
                e2e = measure_e2e()
        cl_ms, _, cl_rep, _, _ = timed(True, False, args.steps, args.warmup)
        na_ms, _, _, _, _ = timed(False, False, args.steps, args.warmup)
        results[eng] = dict(ft_ms=ft_ms, ft_per=ft_per, ft_rep=ft_rep, injected=injected, clean_ms=cl_ms,
                            clean_rep=cl_rep, noabft_ms=na_ms)
    fb.ftblas_set_fp64_engine(engines[args.engine])

    # Online verification (Section V.A rank-K_c steps): checks every K/4 products; timed
    # clean, then one call with two accumulator flips in the same tile, in different steps.
    # Every rank runs it: timed() synchronises the ranks around its timed region.
    online = None
    if not args.no_online:
        kc = max(1, n // 4)
        fb.ftblas_set_verification_interval(kc)
        on_ms, _, on_rep, _, _ = timed(True, False, args.steps, args.warmup)
        nk = -(-n // 32)
        pts = [dict(i=11, j=13, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=56, kt=max(1, nk // 8)),
               dict(i=99, j=77, site=fb.SITE_ACCUM, mode=fb.MODE_BITFLIP, bit=58, kt=max(2, 5 * nk // 8))]
        fb.ftblas_set_injection(fb.make_injection(fixed=pts))
        rep2 = fb.new_report(dev)
        fb.check(fb.ftblas_dgemm(fb.COL_MAJOR, fb.NO_TRANS, fb.NO_TRANS, n, n, n, 1.5, dA.data_ptr(), n,
                                 dB.data_ptr(), n, 0.5, dC.data_ptr(), n, st, rep2.data_ptr()))
        torch.cuda.synchronize(dev)
        r2 = fb.report_from_device(rep2)
        fb.ftblas_set_injection(None)
        fb.ftblas_set_verification_interval(0)
        na_ms = results[args.engine]["noabft_ms"]
        online = {"interval_products": kc, "checks_per_tile": -(-n // kc) - 1,
                  "ft_tflops_clean": flops_step * args.steps / (on_ms / 1e3) / 1e12,
                  "abft_overhead_pct_clean": 100.0 * (on_ms / na_ms - 1.0),
                  "false_alarms_clean": on_rep["detected"],
                  "two_faults_one_tile": {"injected": 2, "detected": int(r2.detected), "corrected": int(r2.corrected),
                                          "uncorrectable": int(r2.uncorrectable)}}

    # Accuracy at the stated error: one more protected call from the known C_in, checked on
    # sampled rows against the binary64 product of the same operands (a library matmul).
    err = None
    if rank == 0:
        import synth as S
        dC.copy_(dCin)
        fb.check(fb.ftblas_dgemm(fb.COL_MAJOR, fb.NO_TRANS, fb.NO_TRANS, n, n, n, 1.5, dA.data_ptr(), n,
                                 dB.data_ptr(), n, 0.5, dC.data_ptr(), n, st, None))
        torch.cuda.synchronize(dev)
        rows = np.unique(S.randint(SEED, 9, 4, 0, n - 1))
        got = dC.view(n, n).t()[torch.as_tensor(rows, device=dev)].cpu().numpy()  # column-major: C[i, :]
        Am, Bm, Cm = (X.reshape(n, n, order="F") for X in (A, B, Cin))  # column-major storage
        ref = 1.5 * (Am[rows, :] @ Bm) + 0.5 * Cm[rows, :]
        err = float(np.abs(got - ref).max() / (np.abs(A).max() * np.abs(B).max() * n))

    # End to end through the public host-buffer entry point: pinned host operands, copies
    # in, protected GEMM, copies out (C and the report), synchronised per call.
    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        f, dt, thr = oracle_sample(n, A, B, Cin, n_tiles=16)
        cpu = {"value": f / dt / 1e12, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": f"16 seeded {TILE}x{TILE} output tiles of the {n}^3 problem (full K, checksums included), "
                         f"{dt:.1f} s"}

    bf16 = fp8 = None
    fp64_ft = flops_step * args.steps / (results[args.engine]["ft_ms"] / 1e3) / 1e12
    if not args.no_bf16 and rank == 0:
        bf16 = run_tc(args, dev, "bf16", n, args.steps, args.warmup, fp64_ft)
    if not args.no_fp8 and rank == 0:
        fp8 = run_tc(args, dev, "fp8", args.fp8_size, args.steps, args.warmup, fp64_ft)
    linear = None
    if not args.no_linear and rank == 0:
        linear = run_linear(dev, args.steps, args.warmup)
    emulated = None
    if not args.no_emulated and rank == 0:
        emulated = run_emulated(dev, n, args.steps, args.warmup, fp64_ft)
    unfused = None
    if not args.no_unfused and rank == 0:
        unfused = run_unfused(dev, n, args.steps, args.warmup)
    level3 = None
    if not args.no_level3 and rank == 0:
        level3 = run_level3(dev, n, max(1, args.steps // 2), max(1, args.warmup // 2))
    large = None
    if not args.no_large and rank == 0 and n == 8192:
        large = run_fp64_large(dev, 16384)
    soak = None
    if not args.no_soak_default and rank == 0:
        soak = run_soak(dev, n, 60.0, rate_per_s=args.soak_rate)

    if rank != 0:
        return 0
    pk = peaks()
    h = results[args.engine]
    ft_ms = h["ft_ms"]
    value = job_tflops(world, flops_step, args.steps, ft_ms)
    kernel_ms = statistics.mean(h["ft_per"])
    achieved = flops_step / (kernel_ms / 1e3) / 1e12
    bound = "alu" if args.engine == "dfma" else "tensor"
    peak = pk["alu"] if bound == "alu" else pk["tensor"]

    def tf(ms):
        return flops_step * args.steps / (ms / 1e3) / 1e12

    engines_out = {}
    for eng, r in results.items():
        engines_out[eng] = {
            "ft_tflops_injected": tf(r["ft_ms"]), "ft_tflops_clean": tf(r["clean_ms"]),
            "noabft_tflops": tf(r["noabft_ms"]),
            "abft_overhead_pct_injected": 100.0 * (r["ft_ms"] / r["noabft_ms"] - 1.0),
            "abft_overhead_pct_clean": 100.0 * (r["clean_ms"] / r["noabft_ms"] - 1.0),
            "injected": r["injected"], "detected": r["ft_rep"]["detected"], "corrected": r["ft_rep"]["corrected"],
            "false_alarms_clean": r["clean_rep"]["detected"], "uncorrectable": r["ft_rep"]["uncorrectable"],
            "frac_of_fp64_alu_peak": tf(r["ft_ms"]) / pk["alu"],
            "frac_of_fp64_tensor_peak": tf(r["ft_ms"]) / pk["tensor"],
        }
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ft_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(n, args.engine, fb.ftblas_verification_tile(fb.COL_MAJOR, fb.R_64F, n, n, n)[0]),
        "pct_of_peak": 100.0 * achieved / peak,
        "abft_overhead_pct": engines_out[args.engine]["abft_overhead_pct_injected"],
        "abft_overhead_pct_clean": engines_out[args.engine]["abft_overhead_pct_clean"],
        "error_vs_fp64": {"normalized_max": err, "criterion": "max|C-C_ref|/(max|A| max|B| K) <= 1e-15",
                          "rows_sampled": 4, "reference": "binary64 product of the same operands (library matmul)"},
        "faults": {"injected": h["injected"], "detected": h["ft_rep"]["detected"],
                   "corrected": h["ft_rep"]["corrected"], "uncorrectable": h["ft_rep"]["uncorrectable"],
                   "false_alarms_clean_run": h["clean_rep"]["detected"], "status": h["ft_rep"]["status"]},
        "engines": engines_out,
        "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": (profile_traffic(f"dgemm_kernel_ft_{args.engine}_{n}_dram", FP64_KERNEL_SOURCES)
                                 if n == 8192 else None), "peak_source": pk["alu_src"] if bound == "alu" else pk["tensor_src"],
                     "kernel": "dgemm_kernel (FT, " + args.engine + ")", "kernel_ms": kernel_ms},
        "cpu_baseline": cpu,
        "bf16": bf16,
        "fp8_e4m3": fp8,
        "fp64_emulated": emulated,
        "online_verification": online,
        "linear_bf16": linear,
        "unfused_fp64": unfused,
        "level3_fp64": level3,
        "fp64_16384": large,
        "soak": soak,
        "e2e": e2e,
        "gpu_launches": world * args.steps,  # one protected product kernel per step on every rank
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist_mod.init_process_group("gloo", rank=rank, world_size=world)
        dist = dist_mod
    try:
        if args.impl == "reference":
            return run_reference(args, rank, world)
        return run_ours(args, rank, world, dist)
    finally:
        if dist is not None:
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
