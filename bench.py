#!/usr/bin/env python3
"""Throughput of the local-f_NL shell round trip (T+E realisations/s) on GB300.

One step = one full realisation of the hot path through the C ABI (fnl_generate):
Philox noise + radial filter, synthesis Legendre GEMM, ring DFTs + square, analysis
Legendre GEMM, radial quadrature for T and E.  Default workload: l_max = 1024,
N_r = 128 shells, 1537 x 3200 Gauss-Legendre grid, f_NL = 30.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec bf16x2|bf16x3|fp32|fp64]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

The default form is bf16x2 (Legendre GEMMs on tcgen05 with 2-term BF16 operands, FP32
FFT and filter, FP64 tables and quadrature).  Beside it the line carries the FP64 GPU
path on the same filters and noise: its throughput ("fp64") and the relative l2 error of
a^T, a^E, a^T_NL and a^E_NL of the mixed form against it ("rel_err").

Multi-GPU (torchrun, one rank per GPU): independent realisations per rank, no
data-path collective ("replicas only"); value = realisations of all ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "fNL T+E realisations/s at ℓmax=1024, mixed vs FP64 (rel err≤1e-5); %roofline"
UNIT = "realisations/s"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------------------------------
# algorithmic work of one realisation (per-unit figures)
# ---------------------------------------------------------------------------------------

def legendre_flops(lmax: int, ntheta: int, nr: int) -> float:
    """Useful flops of one Legendre transform direction with the equatorial symmetry:
    sum_m (lmax - m + 1) * ceil(ntheta / 2) ring pairs * 2 N_r real columns * 2."""
    npairs = (ntheta + 1) // 2
    return W.n_alm(lmax) * npairs * (2 * nr) * 2.0


def fft_bytes(lmax: int, ntheta: int, nr: int, real_bytes: int) -> float:
    """HBM bytes of the ring kernel: read F (even+odd, 2 N_r reals per (m, pair)) and write G."""
    npairs = (ntheta + 1) // 2
    return 2.0 * 2 * (lmax + 1) * npairs * (2 * nr) * real_bytes


def fft_flops(ntheta: int, nphi: int, nr: int) -> float:
    """FFT flops of the ring kernel by the usual 5 N log2 N count per complex N-point
    transform: per (ring pair, shell) one inverse and one forward transform of nphi points."""
    npairs = (ntheta + 1) // 2
    return npairs * nr * 2 * 5.0 * nphi * math.log2(nphi)


def filter_flops(lmax: int, nr: int) -> float:
    """Step (i): Phi_L = K_l n with K_l lower triangular, per (l, m) and real/imaginary part
    nr (nr + 1) / 2 multiply-adds = nr (nr + 1) flops."""
    return W.n_alm(lmax) * 2 * nr * (nr + 1.0)


def gemm_bytes(lmax: int, ntheta: int, nr: int, nterms: int) -> dict:
    """Algorithmic HBM bytes of the two Legendre GEMMs of the tensor-core forms: each lambda
    table once (nterms BF16 terms per entry), the data operand once (Phi_L as BF16 terms for
    the synthesis, G as BF16 terms for the analysis) and F written once in FP32."""
    npairs = (ntheta + 1) // 2
    cols = 2 * nr
    lam = W.n_alm(lmax) * npairs * 2.0 * nterms
    fg = 2 * (lmax + 1) * npairs * cols
    return {"synthesis_gemm": lam + W.n_alm(lmax) * cols * 2.0 * nterms + fg * 4.0,
            "analysis_gemm": lam + fg * 2.0 * nterms}


# DRAM bytes per launch from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum,
# a one-pass metric taken on the full-size command of the launch-list summary under
# profiles/), keyed by stage, workload and form, together with the SHA-256 prefix of the
# kernel's source file when it was captured: once that file changes the entry no longer
# matches and the line reports traffic as null until the kernel is captured again.
TRAFFIC = {
    ("ring_fft_square", "lmax1024_nr128", "bf16x2"): {
        "bytes": 3.180e9, "source": "paper_0909_0009_gb300/csrc/ring_square.cu", "sha16": "9baf7dba4ce68042"},
}


def traffic_of(key) -> float | None:
    """Measured DRAM bytes per launch for `key`, or None when the kernel's source has changed
    since the capture (or there is none)."""
    import hashlib
    e = TRAFFIC.get(key)
    if e is None:
        return None
    with open(os.path.join(ROOT, e["source"]), "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()[:16]
    return e["bytes"] if sha == e["sha16"] else None


# ---------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------------------

_ORACLE_SETUP = {}


def oracle_setup(wl: W.Workload):
    """Per-configuration oracle set-up (untimed, like fnl_make_shells): the Gauss-Legendre
    grid with its lambda table, filters and transfer kernels."""
    if wl.name not in _ORACLE_SETUP:
        import oracle as O
        r, w = W.radial_grid(wl.nr)
        aT, aE = W.transfer_kernels(wl.lmax, r)
        K = W.random_lower_filters(wl.lmax, wl.nr, seed=1, scale=8e-5)
        _ORACLE_SETUP[wl.name] = (r, w, aT, aE, K, O.Grid(wl.lmax, wl.ntheta, wl.nphi, store=True))
    return _ORACLE_SETUP[wl.name]


def oracle_sample(wl: W.Workload, shells: int = 1):
    """Time the FP64 oracle on a bounded sample of one realisation and scale it to a whole
    realisation: Philox noise for `shells` shells, the radial filter rows of those shells
    (all l, m), steps (ii)-(iv) for those shells, and the quadrature; every part is
    per-shell work, so the realisation costs nr / shells times the sample."""
    import oracle as O
    r, w, aT, aE, K, grid = oracle_setup(wl)
    t0 = time.perf_counter()
    n = O.philox_noise(wl.lmax, shells, 1, 0)  # first `shells` shells of the noise
    t1 = time.perf_counter()
    full_noise = np.zeros((wl.nr, n.shape[1]), dtype=np.complex128)
    full_noise[:shells] = n
    Ksub = np.ascontiguousarray(K[:, :shells, :])  # filter rows of the sampled shells only
    t2 = time.perf_counter()
    phiL = O.phi_linear(Ksub, full_noise)
    t3 = time.perf_counter()
    mu = O.mu_ensemble(K)[:shells]
    phiNL = O.phi_nonlinear(phiL, mu, grid)
    t4 = time.perf_counter()
    q = O.quadrature_weights(r[:shells], w[:shells], aT[:, :shells])
    O.radial_quadrature(phiNL, q)
    O.radial_quadrature(phiL, q)
    qE = O.quadrature_weights(r[:shells], w[:shells], aE[:, :shells])
    O.radial_quadrature(phiNL, qE)
    O.radial_quadrature(phiL, qE)
    t5 = time.perf_counter()
    sample_s = (t1 - t0) + (t3 - t2) + (t4 - t3) + (t5 - t4)
    per_real = sample_s * wl.nr / shells
    return per_real, sample_s


def blas_threads() -> int:
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        if os.environ.get(k):
            try:
                return int(os.environ[k])
            except ValueError:
                pass
    return os.cpu_count() or 1


def run_reference(args, wl: W.Workload):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    oracle_setup(wl)
    for _ in range(args.warmup):
        oracle_sample(W.Workload("warm", 32, 2, 49, 100), shells=1)
    t = 0.0
    samples = []
    for _ in range(args.steps):
        per_real, s = oracle_sample(wl, shells=1)
        t += per_real
        samples.append(s)
    value = args.steps / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(wl, "fp64-oracle"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                         "sample": f"per step: 1 of {wl.nr} shells (noise, filter rows, steps (ii)-(iv), "
                                   f"quadrature) of the l_max={wl.lmax} realisation, scaled x{wl.nr}; "
                                   f"mean sample {np.mean(samples):.1f} s"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def measure_batch(F, prec: str, device: int, reps: int = 3) -> dict:
    """Batching form: the 64 realisations of uneven l_max in {128, 256, 512, 1024} and N_r in
    {32, 64, 96, 128} (grids by the exact-square rule, f_NL uniform in [-50, 50]) as one
    captured graph (fnl_generate_batch), tile shapes from the autotuner, against the same
    realisations as single fnl_generate calls on one stream.  Filters: seeded lower-triangular
    matrices of the covariance's amplitude (the cost does not depend on their values)."""
    import torch
    insts = W.batch_instances()
    objs = {}
    for x in insts:
        key = (x.lmax, x.nr)
        if key not in objs:
            r, w = W.radial_grid(x.nr)
            aT, aE = W.transfer_kernels(x.lmax, r)
            K = W.random_lower_filters(x.lmax, x.nr, seed=x.lmax + x.nr, scale=8e-5)
            objs[key] = F.Shells(x.lmax, x.nr, x.ntheta, x.nphi, r, w, aT, aE, K=K, prec=prec, device=device)
            objs[key].autotune()
    shells = [objs[(x.lmax, x.nr)] for x in insts]
    b = F.Batch(shells)
    seeds = [x.seed for x in insts]
    reals = [x.realisation for x in insts]
    fnls = [x.fnl for x in insts]
    out = b.generate(seeds, reals, fnls)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(reps):
        b.generate([s_ + 7919 * (i + 1) for s_ in seeds], reals, fnls, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    t_graph = e0.elapsed_time(e1) / reps
    e0.record(stream)
    for s_, sd, rl, f in zip(shells, seeds, reals, fnls):
        s_.generate(sd, rl, f, parts=False)
    e1.record(stream)
    torch.cuda.synchronize()
    t_single = e0.elapsed_time(e1)
    lm = sorted({x.lmax for x in insts})
    d = {"workload": "uneven64: l_max in {128,256,512,1024}, N_r in {32,64,96,128}, 64 realisations",
         "value": len(insts) / (t_graph / 1e3), "unit": UNIT, "ms_per_graph_launch": t_graph,
         "single_calls_ms": t_single, "speedup_vs_single_calls": t_single / t_graph,
         "graph_launches_per_batch": 1, "multi_instance": b.multi, "tiles": list(b.tiles()),
         "distinct_configurations": len(objs),
         "nphi": {str(l): W.grid_for_lmax(l)[1] for l in lm}}
    b.close()
    for s_ in objs.values():
        s_.close()
    return d


def measure_sharded(F, wl, r, w, aT, aE, K, prec: str, device: int, steps: int, fnl: float, dist) -> dict:
    """Shell-sharded mode over all ranks (N > 1): each rank holds the shard of its shell range
    (fnl_make_shells_shard) and every step is ONE realisation of the workload, its partial
    outputs summed by one all-reduce (paper_0909_0009_gb300.sharded).  Strong scaling: the
    work per step is fixed as N grows.  Timed with CUDA events between barriers, max over ranks."""
    import torch

    from paper_0909_0009_gb300 import sharded
    drv = sharded.ShardedShells(wl.lmax, wl.nr, wl.ntheta, wl.nphi, r, w, aT, aE, K=K, prec=prec, device=device)
    if drv.shells is not None and prec in ("bf16x2", "bf16x3"):
        drv.shells.autotune()
    buf = torch.empty((2, drv.nalm), dtype=torch.complex128, device=f"cuda:{device}")
    for i in range(3):
        drv.generate(1, 20_000 + i, fnl, parts=False, buf=buf)
    dist.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):
        drv.generate(1, i, fnl, parts=False, buf=buf)
    e1.record(stream)
    dist.barrier()
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, f"cuda:{device}")
    out = {"value": steps / (ms / 1e3), "unit": UNIT, "scaling": "strong", "steps": steps,
           "ms_per_realisation": ms / steps, "shell_range_rank0": list(drv.range),
           "collective": "one all-reduce (sum) of a^T, a^E per realisation (2 x n_alm complex128)"}
    drv.close()
    return out


def measure_pipelined(F, sh, wl, r, w, aT, aE, K, prec: str, tiles, device: int, fnl: float, steps: int = 100) -> dict:
    """Two realisations in flight: the timed object and a second one of the same configuration
    (its own scratch) on two streams, realisations alternating between them, with and without
    the persistent GEMMs capped at half the SMs (fnl_shells_set_sm_limits).  Per-stream stage
    times from each object's stage events.  Against the serial loop of the headline."""
    import torch
    sh2 = F.Shells(wl.lmax, wl.nr, wl.ntheta, wl.nphi, r, w, aT, aE, K=K, prec=prec, device=device)
    if prec in ("bf16x2", "bf16x3"):
        sh2.set_tiles(*tiles)
    objs = [sh, sh2]
    outs = [{k: o._alm() for k in ("aT", "aE")} for o in objs]
    streams = [torch.cuda.Stream(device), torch.cuda.Stream(device)]
    res = {}
    for name, lim in (("two_streams", (0, 0)), ("two_streams_gemm_half_sms", (76, 0))):
        for o in objs:
            o.set_sm_limits(*lim)
        for k in range(2):
            objs[k].generate(1, 30_000 + k, fnl, parts=False, out=outs[k], stream=streams[k])
        torch.cuda.synchronize()
        for o in objs:
            o.profile(slots=steps)
        start = torch.cuda.Event(enable_timing=True)
        start.record(torch.cuda.current_stream())
        for st in streams:
            st.wait_event(start)
        for i in range(steps // 2):
            for k in range(2):
                objs[k].generate(1, 2 * i + k, fnl, parts=False, out=outs[k], stream=streams[k])
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for k in range(2):
            ends[k].record(streams[k])
        torch.cuda.synchronize()
        ms = max(start.elapsed_time(e) for e in ends)
        per_stream = []
        for o in objs:
            stg, calls = o.stage_ms()
            o.profile(0)
            per_stream.append({k: round(v / max(calls, 1), 4) for k, v in stg.items()})
        for o in objs:
            o.set_sm_limits(0, 0)
        res[name] = {"value": (steps // 2) * 2 / (ms / 1e3), "unit": UNIT, "sm_limits": list(lim),
                     "stage_ms_per_stream": per_stream}
    sh2.close()
    res["note"] = ("two shells objects on two streams, realisations alternating; the kernels of the two "
                   "streams overlap only where one leaves SMs idle (every stage fills all SMs and scales "
                   "with 1 / SMs), so the serial loop is as fast")
    return res


def measure_adjoint(F, device: int, reps: int = 3) -> dict:
    """Differentiation form at l_max = 512, N_r = 96 (769 x 1600): fnl_generate and
    fnl_generate_backward (dL/dn and dL/df_NL, maps recomputed) in FP64, FP32 and bf16x2 (the
    tensor-core form: both syntheses and the analysis on tcgen05)."""
    import torch
    wl = W.GRAD
    r, w = W.radial_grid(wl.nr)
    aT, aE = W.transfer_kernels(wl.lmax, r)
    K = W.random_lower_filters(wl.lmax, wl.nr, seed=2, scale=8e-5)
    stream = torch.cuda.current_stream()
    res = {"workload": wl.name, "lmax": wl.lmax, "nr": wl.nr, "ntheta": wl.ntheta, "nphi": wl.nphi}
    for prec in ("fp64", "fp32", "bf16x2"):
        sh = F.Shells(wl.lmax, wl.nr, wl.ntheta, wl.nphi, r, w, aT, aE, K=K, prec=prec, device=device)
        g = torch.randn(sh.nalm, dtype=torch.complex128, device=f"cuda:{device}")
        fw = sh.generate(2, 0, wl.fnl[0])
        sh.generate_backward(2, 0, wl.fnl[0], gT=g, gE=g, aNLT=fw["aNLT"], aNLE=fw["aNLE"])
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        for i in range(reps):
            fw = sh.generate(2, i, wl.fnl[0], out=fw)
        e1.record(stream)
        for i in range(reps):
            sh.generate_backward(2, i, wl.fnl[0], gT=g, gE=g, aNLT=fw["aNLT"], aNLE=fw["aNLE"])
        e2.record(stream)
        torch.cuda.synchronize()
        res[prec] = {"forward_ms": e0.elapsed_time(e1) / reps, "backward_ms": e1.elapsed_time(e2) / reps}
        sh.close()
    return res


def measure_maps(F, sh, out, device: int, reps: int = 5) -> dict:
    """Stokes I, Q, U maps (fnl_maps) of the timed object's last a^T, a^E (zero B modes, as
    the paper's maps): tables prepared once (untimed), then `reps` calls timed with events.
    The bound is HBM: one pass over the lambda, W and X tables (nalm x npj entries each in the
    object's real type) per call; the three ring FFTs are a few per cent of the call."""
    import torch
    t0 = time.perf_counter()
    sh.maps_prepare()
    prep = time.perf_counter() - t0
    maps = sh.maps(out["aT"], out["aE"])
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        sh.maps(out["aT"], out["aE"], out=maps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    real_bytes = 8 if sh.prec == F.FNL_FP64 else 4
    npj = ((sh.ntheta + 1) // 2 + 31) // 32 * 32
    table_bytes = 3 * sh.nalm * npj * real_bytes
    pk, pk_kind = peaks()
    return {"ms": ms, "prepare_s": prep, "table_bytes": table_bytes, "maps_per_s": 1e3 / ms,
            "roofline": {"bound": "hbm", "achieved": table_bytes / (ms / 1e3) / 1e9, "peak": pk["hbm_gbs"],
                         "unit": "GB/s", "frac": table_bytes / (ms / 1e3) / 1e9 / pk["hbm_gbs"],
                         "peak_source": f"HBM copy ({pk_kind}); whole fnl_maps call timed"}}


def measure_ksw(F, sh, out, device: int, reps: int = 5) -> dict:
    """The cubic estimator (Sect. 5) on the timed configuration: set-up (weights, FP64
    normalisation summed over l1 <= l2 <= l3), then `reps` calls of fnl_ksw_statistic on the
    last generated sky timed with events, and its f_NL estimate against the input."""
    import torch
    t0 = time.perf_counter()
    k = F.Ksw(sh)
    setup_s = time.perf_counter() - t0
    s = k.statistic(out["aT"], out["aE"])
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        k.statistic(out["aT"], out["aE"], out=s)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    res = {"ms": ms, "estimates_per_s": 1e3 / ms, "setup_s": setup_s, "norm_s": k.norm_seconds,
           "norm": k.norm, "sigma_fnl": 1.0 / math.sqrt(k.norm) if k.norm > 0 else None,
           "fnl_estimate": float(s.item()) / k.norm if k.norm > 0 else None,
           "note": "one sky: synthesis of A and B on every shell (2 N_r fields), ring cubic sums, reduction"}
    k.close()
    return res


def measure_quadrature(F, device: int, nsel: int = 64) -> dict:
    """Optimal radial quadrature (Sect. 3) for l_max 1024 on 384 fine shells over the workload's
    radial range (the 128 midpoints of the generator are fine nodes 3 i + 1): the fine covariance
    on the device (Eq. 7, FP64), the greedy choice of nsel nodes with their optimal weights, and
    the relative errors of that rule and of the generator's 128-node midpoint rule."""
    L, ntot = W.FULL.lmax, 384
    r, w = W.radial_grid(ntot)
    aT, aE = W.transfer_kernels(L, r)
    qd = F.Quadrature(L, r, w, aT, aE, device=device)
    g = qd.greedy(nsel)
    rm, wm = W.radial_grid(128)
    mT, mE = W.transfer_kernels(L, rm)
    mid = [3 * i + 1 for i in range(128)]
    rel_mid = qd.error(mid, np.stack([mT, mE]) * (wm * rm * rm)[None, None, :])
    live = qd.I2 > 0
    res = {"lmax": L, "ntot": ntot, "nsel": nsel, "covariance_s": qd.create_seconds, "greedy_s": g["seconds"],
           "rel_err_mean": float(g["rel_err"][live].mean()), "rel_err_max": float(g["rel_err"][live].max()),
           "midpoint128_rel_err_mean": float(rel_mid[live].mean()),
           "midpoint128_rel_err_max": float(rel_mid[live].max())}
    qd.close()
    return res


def measure_healpix(F, K, device: int, steps: int = 3) -> dict:
    """The paper's grid: HEALPix nside 512 at l_max 1024, N_r 128, FP32 form, against the FP32
    form on the 1537 x 3200 Gauss-Legendre grid with the same filters: realisations/s of each
    (events over `steps` calls after one warm-up) and the relative difference of a^T, a^E
    (the HEALPix rule is approximate, the Gauss-Legendre one exact)."""
    import torch
    wl = W.FULL
    r, w = W.radial_grid(wl.nr)
    aT, aE = W.transfer_kernels(wl.lmax, r)
    res = {"lmax": wl.lmax, "nr": wl.nr, "nside": 512, "precision": "fp32"}
    outs = {}
    for name, kw in (("healpix", {"nside": 512}), ("gauss_legendre", {})):
        sh = F.Shells(wl.lmax, wl.nr, wl.ntheta, wl.nphi, r, w, aT, aE, K=K, prec="fp32", device=device, **kw)
        o = sh.generate(1, 0, wl.fnl[0], parts=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(steps):
            sh.generate(1, i, wl.fnl[0], parts=False)
        e1.record()
        torch.cuda.synchronize()
        res[name + "_realisations_per_s"] = steps * 1e3 / e0.elapsed_time(e1)
        outs[name] = {k: v.cpu().numpy() for k, v in o.items()}
        sh.close()
    for X in ("aT", "aE"):
        a, b = outs["healpix"][X], outs["gauss_legendre"][X]
        res["rel_diff_" + X] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    return res


# ---------------------------------------------------------------------------------------
# replicas over realisations (one process per GPU): the only cross-rank logic of the path
# ---------------------------------------------------------------------------------------

def realisation_of(rank: int, steps: int, i: int) -> int:
    """Realisation index of step i on `rank`: ranks draw disjoint blocks of `steps`
    realisations of one seed, so N ranks generate N x steps distinct maps with no data-path
    exchange (the noise is a function of (seed, realisation) only)."""
    return rank * steps + i


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The job's time: the maximum of the ranks' times (a MAX all-reduce; identity at N = 1)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, seconds: float) -> float:
    """Whole-job realisations per second: every rank's realisations over the slowest rank's time."""
    return world * steps / seconds


def config_of(wl: W.Workload, prec: str) -> dict:
    return {"workload": wl.name, "lmax": wl.lmax, "nr": wl.nr, "ntheta": wl.ntheta, "nphi": wl.nphi,
            "fnl": wl.fnl[-1], "precision": prec,
            "l2": "inputs larger than L2 (Legendre tables and F/G scratch are several GB per step)"}


# ---------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x2", choices=["fp64", "fp32", "bf16x2", "bf16x3"])
    ap.add_argument("--workload", default=W.FULL.name, choices=sorted(W.WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="timed steps of the FP64 comparator beside a mixed run (0: skip it)")
    ap.add_argument("--no-batch", action="store_true", help="skip the uneven-batch measurement")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint measurement")
    ap.add_argument("--no-maps", action="store_true", help="skip the Stokes-maps measurement")
    ap.add_argument("--no-ksw", action="store_true", help="skip the cubic-estimator measurement")
    ap.add_argument("--no-quad", action="store_true", help="skip the optimal-quadrature measurement")
    ap.add_argument("--no-healpix", action="store_true", help="skip the HEALPix-grid measurement")
    ap.add_argument("--no-pipelined", action="store_true",
                    help="skip the two-stream measurement (two realisations in flight)")
    ap.add_argument("--no-sharded", action="store_true",
                    help="with N > 1: skip the shell-sharded measurement (one realisation over all ranks)")
    ap.add_argument("--tiles", default="auto",
                    help="tensor-core tile widths 'synthesis,analysis' (default: picked by fnl_shells_autotune)")
    args = ap.parse_args()
    wl = W.WORKLOADS[args.workload]
    if args.steps is None:
        args.steps = 5 if args.prec == "fp64" else 200
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    if args.impl == "reference":
        return run_reference(args, wl)

    import torch
    import torch.distributed as dist
    from paper_0909_0009_gb300 import fnl as F

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))

    r, w = W.radial_grid(wl.nr)
    aT, aE = W.transfer_kernels(wl.lmax, r)
    # filters K_l = chol(C_l + eps_l I) of the Eq. 7 covariance, built once on the host and
    # shared by the timed form and its FP64 comparator
    C = F.covariance(wl.lmax, r, W.COV.A, W.COV.ns, W.COV.kmin, W.COV.kmax, W.COV.nk)
    K = F.cholesky_filters(C, W.COV.jitter_rel)
    del C
    sh = F.Shells(wl.lmax, wl.nr, wl.ntheta, wl.nphi, r, w, aT, aE, K=K, prec=args.prec, device=local)
    if args.tiles == "auto":
        tiles = sh.autotune()  # tile shapes of the tensor-core GEMMs, picked by timing (set-up, untimed)
    elif args.prec in ("bf16x2", "bf16x3"):
        tiles = tuple(int(x) for x in args.tiles.split(","))
        sh.set_tiles(*tiles)
    else:
        tiles = (64, 64)
    fnl = wl.fnl[-1]
    stream = torch.cuda.current_stream()
    out = {k: sh._alm() for k in ("aT", "aE", "aLT", "aLE", "aNLT", "aNLE")}

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for i in range(args.warmup):
        sh.generate(1, 10_000 + i, fnl, out=out)
    barrier()

    # ---- timed region (device): K realisations, per-stage events on the same stream
    sh.profile(slots=min(max(args.steps, 1), 4096))
    clocks = Clocks(local)
    clocks.start()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        sh.generate(1, realisation_of(rank, args.steps, i), fnl, out=out)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    stage_sum, calls = sh.stage_ms()
    sh.profile(0)
    ms_max = max_over_ranks(ms, dist, f"cuda:{local}")
    value = job_throughput(world, args.steps, ms_max / 1e3)

    # ---- end to end: the same step through the host-output entry point (pinned buffers)
    h_aT = torch.empty(sh.nalm, dtype=torch.complex128, pin_memory=True).numpy()
    h_aE = torch.empty(sh.nalm, dtype=torch.complex128, pin_memory=True).numpy()
    e2e_steps = max(1, min(args.steps, 50 if args.prec == "fp64" else args.steps))
    barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        sh.generate_host(1, realisation_of(rank, args.steps, i), fnl, h_aT, h_aE)
    torch.cuda.synchronize()
    e2e_value = job_throughput(world, e2e_steps, max_over_ranks(time.perf_counter() - t0, dist, f"cuda:{local}"))

    # ---- measured FMA rates of this GPU (project kernels, CUDA events), the denominators of the
    # ALU-bound stages: FP32 for the filter and the ring DFTs, FP64 for the FP64 path
    fma64, fma32 = F.measure_fma_peaks(local)

    # ---- the FP64 GPU path on the same filters and noise: throughput and the error of the
    # timed form against it (the metric's "mixed vs FP64")
    fp64 = None
    if args.prec != "fp64" and args.fp64_steps > 0:
        ref = sh.generate(1, 0, fnl)
        d64 = F.Shells(wl.lmax, wl.nr, wl.ntheta, wl.nphi, r, w, aT, aE, K=K, prec="fp64", device=local)
        b = d64.generate(1, 0, fnl)
        torch.cuda.synchronize()
        rel = {}
        for k in ("aT", "aE", "aNLT", "aNLE"):
            rel[k] = float(torch.linalg.vector_norm(ref[k] - b[k]) / torch.linalg.vector_norm(b[k]))
        out64 = {k: d64._alm() for k in ("aT", "aE", "aLT", "aLE", "aNLT", "aNLE")}
        d64.generate(1, 10_000, fnl, out=out64)
        barrier()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for i in range(args.fp64_steps):
            d64.generate(1, realisation_of(rank, args.fp64_steps, i), fnl, out=out64)
        f1.record(stream)
        barrier()
        t64 = max_over_ranks(f0.elapsed_time(f1), dist, f"cuda:{local}")
        fp64 = {"value": job_throughput(world, args.fp64_steps, t64 / 1e3), "unit": UNIT,
                "steps": args.fp64_steps, "rel_err": rel, "rel_err_bound": 1e-5,
                "seed": "seed 1, realisation 0, same filters and Philox noise"}
        d64.close()
        del d64, out64, ref, b

    # shell-sharded mode (N > 1, every rank takes part): one realisation spread over the ranks
    sharded = (None if world == 1 or args.no_sharded
               else measure_sharded(F, wl, r, w, aT, aE, K, args.prec, local, min(args.steps, 50), fnl, dist))

    # the secondary measurements run once, on rank 0 (the other ranks wait at the final barrier)
    lead = rank == 0
    maps = None if args.no_maps or not lead else measure_maps(F, sh, out, local)
    ksw = None if args.no_ksw or not lead else measure_ksw(F, sh, out, local)
    quad = None if args.no_quad or not lead else measure_quadrature(F, local)
    hp = None if args.no_healpix or not lead or wl is not W.FULL else measure_healpix(F, K, local)
    batch = (None if args.no_batch or not lead or args.prec not in ("bf16x2", "bf16x3")
             else measure_batch(F, args.prec, local))
    adjoint = None if args.no_adjoint or not lead else measure_adjoint(F, local)
    pipelined = (None if args.no_pipelined or not lead or args.prec not in ("bf16x2", "bf16x3")
                 else measure_pipelined(F, sh, wl, r, w, aT, aE, K, args.prec, tiles, local, fnl))

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    # ---- rooflines of every stage from the live stage events; the dominant one is the
    # line's "roofline".  Each stage is measured against what bounds it: the tensor pipe
    # (executed MMA flops) for the Legendre GEMMs, the FP32 pipes for the filter and the
    # ring FFTs (bound by instruction issue), HBM for the quadrature.
    pk, pk_kind = peaks()
    per_stage = {k: v / max(calls, 1) for k, v in stage_sum.items()}
    mixed = args.prec in ("bf16x2", "bf16x3")
    nterm = 2 if args.prec == "bf16x2" else 3
    mult = {"bf16x2": 3, "bf16x3": 6}.get(args.prec, 1)
    flops_dir = legendre_flops(wl.lmax, wl.ntheta, wl.nr)
    gb = gemm_bytes(wl.lmax, wl.ntheta, wl.nr, nterm) if mixed else {}
    # the tensor-core GEMMs leave out the polar ring pairs of negligible lambda: their executed
    # share of the dense work (fnl_shells_gemm_work) scales the flops and the operand bytes
    share = dict(zip(("synthesis_gemm", "analysis_gemm"), sh.gemm_work())) if mixed else {}
    real_bytes = 8 if args.prec == "fp64" else 4
    stages = {}
    for st_name, ms_ in per_stage.items():
        sec = ms_ / 1e3
        if st_name in ("synthesis_gemm", "analysis_gemm"):
            if mixed:
                sh_ = share[st_name]
                e = {"bound": "tensor", "achieved": flops_dir * sh_ * mult / sec / 1e12,
                     "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s",
                     "peak_source": f"bf16 sustained ({pk_kind}); executed = {mult} x useful flops of the "
                                    f"{sh_:.3f} share of the dense Legendre work the GEMM runs (the polar ring "
                                    f"pairs where every |lambda_lm| < 2^-30 are left out)",
                     "work_share": sh_, "dense_equivalent_tflops": flops_dir * mult / sec / 1e12,
                     "hbm_frac": gb[st_name] * sh_ / sec / 1e9 / pk["hbm_gbs"]}
            elif args.prec == "fp32":
                e = {"bound": "alu", "achieved": flops_dir / sec / 1e12, "peak": fma32, "unit": "TFLOP/s",
                     "peak_source": "FP32 FFMA rate (measured, fnl_measure_fma_peaks)"}
            else:
                e = {"bound": "alu", "achieved": flops_dir / sec / 1e12, "peak": fma64, "unit": "TFLOP/s",
                     "peak_source": "FP64 DFMA rate (measured, fnl_measure_fma_peaks)"}
        elif st_name == "ring_fft_square":
            e = {"bound": "alu", "achieved": fft_flops(wl.ntheta, wl.nphi, wl.nr) / sec / 1e12,
                 "peak": fma32 if args.prec != "fp64" else fma64, "unit": "TFLOP/s",
                 "peak_source": ("FP32 FFMA" if args.prec != "fp64" else "FP64 DFMA")
                                + " rate (measured, fnl_measure_fma_peaks); flops by 5 N log2 N",
                 "hbm_frac": fft_bytes(wl.lmax, wl.ntheta, wl.nr, real_bytes) / sec / 1e9 / pk["hbm_gbs"]}
        elif st_name == "filter":
            e = {"bound": "alu", "achieved": filter_flops(wl.lmax, wl.nr) / sec / 1e12,
                 "peak": fma32 if args.prec != "fp64" else fma64, "unit": "TFLOP/s",
                 "peak_source": ("FP32 FFMA" if args.prec != "fp64" else "FP64 DFMA")
                                + " rate (measured, fnl_measure_fma_peaks); flops of K_l n (Eq. 9)"
                                + ("; the product runs on the tensor cores and the stage is bound by the "
                                   "noise draws (Philox, Box-Muller) on the ALUs" if mixed else "")}
        else:
            if mixed:  # epilogue partials (two FP64 pairs per column tile) and a^X_L in, a^X and a^X_NL out
                qb = W.n_alm(wl.lmax) * ((wl.nr * 2 + 127) // 128 * 32 + 2 * 16 + 4 * 16)
            else:      # Phi_NL rows and a^X_L in, a^X and a^X_NL out
                qb = W.n_alm(wl.lmax) * (2 * wl.nr * real_bytes + 2 * 16 + 4 * 16)
            e = {"bound": "hbm", "achieved": qb / sec / 1e9, "peak": pk["hbm_gbs"], "unit": "GB/s",
                 "peak_source": f"HBM copy ({pk_kind})"}
        e["frac"] = e["achieved"] / e["peak"]
        e["ms"] = round(ms_, 4)
        stages[st_name] = e
    dom = max(per_stage, key=per_stage.get)
    roofline = dict(stages[dom])
    roofline["kernel"] = dom
    roofline["traffic"] = traffic_of((dom, wl.name, args.prec))
    if dom == "ring_fft_square":
        roofline["algorithmic_bytes"] = fft_bytes(wl.lmax, wl.ntheta, wl.nr, real_bytes)
    roofline["stage_ms"] = {k: round(v, 4) for k, v in per_stage.items()}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32", "bf16x2": "bf16x2-split/f32", "bf16x3": "bf16x3-split/f32"}[args.prec],
        "data": "synthetic", "config": config_of(wl, args.prec), "roofline": roofline, "stages": stages,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 2 * sh.nalm * 16, "steps": e2e_steps,
                "note": "fnl_generate_host: inputs are the (seed, realisation, f_NL) scalars; a^T and a^E "
                        "land in pinned host memory every step (written by the path's last kernel "
                        "through the buffers' device mapping); the step's time includes them"},
        "gpu_launches": (6 if args.prec in ("bf16x2", "bf16x3") else 5) * args.steps,
        "tiles": {"synthesis": tiles[0], "analysis": tiles[1]},
        "clocks": clk,
        "fma_peaks": {"fp64_tflops": fma64, "fp32_tflops": fma32,
                      "how": "fnl_measure_fma_peaks: 8 independent FMA chains per thread, 8 blocks of 256 per SM, "
                             "median of 5 launches of ~10 ms, CUDA events"},
    }
    if sharded is not None:
        line["sharded"] = sharded
    if pipelined is not None:
        line["pipelined"] = pipelined
    if batch is not None:
        line["batch"] = batch
    if adjoint is not None:
        line["adjoint"] = adjoint
    if maps is not None:
        line["maps"] = maps
    if ksw is not None:
        ksw["fnl_input"] = fnl
        line["ksw"] = ksw
    if quad is not None:
        line["quadrature"] = quad
    if hp is not None:
        line["healpix"] = hp
    if fp64 is not None:
        line["fp64"] = fp64
        line["speedup_vs_fp64"] = value / fp64["value"]
    if not args.no_cpu_baseline and world == 1:
        per_real, sample_s = oracle_sample(wl, shells=2)
        line["cpu_baseline"] = {"value": 1.0 / per_real, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                                "sample": f"2 of {wl.nr} shells (Philox noise, filter rows, steps (ii)-(iv), "
                                          f"quadrature) of one l_max={wl.lmax} realisation, {sample_s:.1f} s, "
                                          f"scaled x{wl.nr // 2}"}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
