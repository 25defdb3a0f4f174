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
        sh.generate(1, rank * args.steps + i, fnl, out=out)
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    stage_sum, calls = sh.stage_ms()
    sh.profile(0)
    t = torch.tensor([ms], dtype=torch.float64, device=f"cuda:{local}")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * args.steps / (ms_max / 1e3)

    # ---- end to end: the same step through the host-output entry point (pinned buffers)
    h_aT = torch.empty(sh.nalm, dtype=torch.complex128, pin_memory=True).numpy()
    h_aE = torch.empty(sh.nalm, dtype=torch.complex128, pin_memory=True).numpy()
    e2e_steps = max(1, min(args.steps, 50 if args.prec == "fp64" else args.steps))
    barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        sh.generate_host(1, rank * args.steps + i, fnl, h_aT, h_aE)
    torch.cuda.synchronize()
    t_e2e = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device=f"cuda:{local}")
    if world > 1:
        dist.all_reduce(t_e2e, op=dist.ReduceOp.MAX)
    e2e_value = world * e2e_steps / float(t_e2e.item())

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
            d64.generate(1, rank * args.fp64_steps + i, fnl, out=out64)
        f1.record(stream)
        barrier()
        t64 = torch.tensor([f0.elapsed_time(f1)], dtype=torch.float64, device=f"cuda:{local}")
        if world > 1:
            dist.all_reduce(t64, op=dist.ReduceOp.MAX)
        fp64 = {"value": world * args.fp64_steps / (float(t64.item()) / 1e3), "unit": UNIT,
                "steps": args.fp64_steps, "rel_err": rel, "rel_err_bound": 1e-5,
                "seed": "seed 1, realisation 0, same filters and Philox noise"}
        d64.close()
        del d64, out64, ref, b

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    # ---- roofline of the dominant kernel, from the live stage events
    pk, pk_kind = peaks()
    per_stage = {k: v / max(calls, 1) for k, v in stage_sum.items()}
    dom = max(per_stage, key=per_stage.get)
    flops_dir = legendre_flops(wl.lmax, wl.ntheta, wl.nr)
    real_bytes = 8 if args.prec == "fp64" else 4
    if dom in ("synthesis_gemm", "analysis_gemm"):
        if args.prec == "fp64":
            peak, bound, unit = 1.25, "alu", "TFLOP/s"
            peak_note = "nominal GB300 FP64 rate (no measured FP64 peak); see DESIGN.md"
        elif args.prec == "fp32":
            peak, bound, unit = 2070e6 * 152 * 128 * 2 / 1e12, "alu", "TFLOP/s"
            peak_note = "FP32 FFMA: 152 SMs x 128 lanes x 2 flops x 2070 MHz"
        else:
            nterm = 3 if args.prec == "bf16x2" else 6
            peak, bound, unit = pk["bf16_tflops_sustained"], "tensor", "TFLOP/s"
            peak_note = f"bf16 sustained ({pk_kind}); executed = {nterm} x useful flops"
        mult = 1 if args.prec in ("fp64", "fp32") else (3 if args.prec == "bf16x2" else 6)
        achieved = flops_dir * mult / (per_stage[dom] / 1e3) / 1e12
    else:
        bytes_ = fft_bytes(wl.lmax, wl.ntheta, wl.nr, real_bytes)
        peak, bound, unit = pk["hbm_gbs"], "hbm", "GB/s"
        peak_note = f"HBM copy ({pk_kind})"
        achieved = bytes_ / (per_stage[dom] / 1e3) / 1e9
    roofline = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": None, "peak_source": peak_note,
                "stage_ms": {k: round(v, 4) for k, v in per_stage.items()}}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32", "bf16x2": "bf16x2-split/f32", "bf16x3": "bf16x3-split/f32"}[args.prec],
        "data": "synthetic", "config": config_of(wl, args.prec), "roofline": roofline,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 2 * sh.nalm * 16, "steps": e2e_steps,
                "note": "fnl_generate_host: inputs are the (seed, realisation, f_NL) scalars; a^T and a^E "
                        "copied to pinned host memory every step"},
        "gpu_launches": (6 if args.prec in ("bf16x2", "bf16x3") else 5) * args.steps,
        "tiles": {"synthesis": tiles[0], "analysis": tiles[1]},
        "clocks": clk,
    }
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
