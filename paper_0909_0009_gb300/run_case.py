"""Run a few realisations of one configuration through the C ABI and print the stage times.

For profilers and quick timing of a configuration that is not one of the named workloads:

  python -m paper_0909_0009_gb300.run_case --lmax 512 --nr 128 --ntheta 769 --nphi 3200 \
      --prec bf16x2 --tiles 112,128 --reps 3
  python -m paper_0909_0009_gb300.run_case --lmax 512 --nr 8 --ntheta 769 --nphi 1600 --maps --reps 3
  python -m paper_0909_0009_gb300.run_case --lmax 1024 --nr 128 --ntheta 1537 --nphi 3200 --ksw --reps 3
  python -m paper_0909_0009_gb300.run_case --lmax 1024 --nr 128 --nside 512 --prec fp32 --reps 2
  python -m paper_0909_0009_gb300.run_case --lmax 1024 --nr 128 --ntheta 1537 --nphi 3200 --quad 64 --reps 0
  python -m paper_0909_0009_gb300.run_case --batch --prec bf16x2 --reps 3

`--batch` runs the uneven 64-realisation batch of the batching form (l_max in {128, 256, 512,
1024}, N_r in {32, 64, 96, 128}): the whole batch as one graph, the batch split by band limit,
and every distinct configuration as single calls with its stage times. With `--profile-range`
one graph launch of the whole batch runs between cudaProfilerStart and cudaProfilerStop (for
`ncu --profile-from-start off`), and nothing else is timed.

Filters are seeded lower-triangular matrices of the covariance's amplitude (the cost of the
path does not depend on their values); noise is the Philox draw of (seed 1, realisation i).
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def batch_main(args) -> int:
    import collections

    import torch

    import workloads as W
    from paper_0909_0009_gb300 import fnl as F

    F.load_library()
    insts = W.batch_instances()
    objs = {}
    for x in insts:
        if (x.lmax, x.nr) not in objs:
            r, w = W.radial_grid(x.nr)
            aT, aE = W.transfer_kernels(x.lmax, r)
            K = W.random_lower_filters(x.lmax, x.nr, seed=x.lmax + x.nr, scale=8e-5)
            sh = F.Shells(x.lmax, x.nr, x.ntheta, x.nphi, r, w, aT, aE, K=K, prec=args.prec)
            sh.autotune()
            objs[(x.lmax, x.nr)] = sh
    st = torch.cuda.current_stream()
    reps = max(args.reps, 1)

    def timed(fn, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for i in range(n):
            fn(i)
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    def run_batch(sub, profile=False):
        b = F.Batch([objs[(x.lmax, x.nr)] for x in sub])
        sd, rl, fn = [x.seed for x in sub], [x.realisation for x in sub], [x.fnl for x in sub]
        out = b.generate(sd, rl, fn)
        b.generate(sd, rl, fn, out=out)
        torch.cuda.synchronize()
        if profile:
            torch.cuda.profiler.start()
            b.generate(sd, rl, fn, out=out)
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
            t = 0.0
        else:
            t = timed(lambda i: b.generate(sd, rl, fn, out=out), reps)
        tiles = b.tiles()
        b.close()
        return t, tiles

    if args.profile_range:
        run_batch(insts, profile=True)
        return 0
    t, tiles = run_batch(insts)
    print(f"whole batch: {len(insts)} realisations, {t:.3f} ms per graph launch, tiles {tiles}")
    for lm in sorted({x.lmax for x in insts}):
        sub = [x for x in insts if x.lmax == lm]
        t, tiles = run_batch(sub)
        print(f"  l_max {lm}: {len(sub)} realisations, {t:.3f} ms, tiles {tiles}")
    count = collections.Counter((x.lmax, x.nr) for x in insts)
    total = 0.0
    for (lm, nr), c in sorted(count.items()):
        sh = objs[(lm, nr)]
        for i in range(3):
            sh.generate(1, i, args.fnl, parts=False)
        n = max(5, min(200, int(2000 / ((lm / 128) ** 3 * nr / 32))))
        ms = timed(lambda i: sh.generate(1, i, args.fnl, parts=False), n)
        sh.profile(5)
        for i in range(5):
            sh.generate(1, i, args.fnl, parts=False)
        torch.cuda.synchronize()
        stg, calls = sh.stage_ms()
        sh.profile(0)
        total += c * ms
        per = {k: round(v / max(calls, 1), 4) for k, v in stg.items()}
        print(f"  single calls l_max {lm} N_r {nr} (x{c}): {ms:.4f} ms; {per}")
    print(f"sum of single calls: {total:.3f} ms")
    for sh in objs.values():
        sh.close()
    return 0


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--batch", action="store_true", help="the uneven 64-realisation batch (see above)")
    ap.add_argument("--profile-range", action="store_true",
                    help="with --batch: one graph launch inside a cudaProfilerStart/Stop range, nothing timed")
    ap.add_argument("--lmax", type=int, default=0)
    ap.add_argument("--nr", type=int, default=0)
    ap.add_argument("--ntheta", type=int, default=0)
    ap.add_argument("--nphi", type=int, default=0)
    ap.add_argument("--nside", type=int, default=0, help="HEALPix grid of this nside (FP64 / FP32 forms)")
    ap.add_argument("--quad", type=int, default=0,
                    help="also design an optimal radial rule of this many nodes on 3 N_r fine shells")
    ap.add_argument("--prec", default="bf16x2", choices=["fp64", "fp32", "bf16x2", "bf16x3"])
    ap.add_argument("--tiles", default="", help="'synthesis,analysis' tile widths of the tensor-core forms")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--fnl", type=float, default=20.0)
    ap.add_argument("--ksw", action="store_true",
                    help="also run the cubic f_NL estimator (fnl_ksw_statistic) on each realisation and time it")
    ap.add_argument("--maps", action="store_true",
                    help="also make the Stokes I, Q, U maps of each realisation (fnl_maps) and time them")
    args = ap.parse_args(argv)
    if args.batch:
        return batch_main(args)
    if args.lmax <= 0 or args.nr <= 0:
        ap.error("--lmax and --nr are required (or --batch)")

    import torch

    import workloads as W
    from paper_0909_0009_gb300 import fnl as F

    F.load_library()
    r, w = W.radial_grid(args.nr)
    aT, aE = W.transfer_kernels(args.lmax, r)
    K = W.random_lower_filters(args.lmax, args.nr, seed=1, scale=8e-5)
    if args.quad:
        rf, wf = W.radial_grid(3 * args.nr)
        fT, fE = W.transfer_kernels(args.lmax, rf)
        qd = F.Quadrature(args.lmax, rf, wf, fT, fE)
        g = qd.greedy(args.quad)
        live = qd.I2 > 0
        print(f"quadrature: covariance {qd.create_seconds:.3f} s, greedy {g['seconds']:.4f} s, "
              f"mean rel err {g['rel_err'][live].mean():.3g}")
        qd.close()
        if args.reps <= 0:
            return 0
    sh = F.Shells(args.lmax, args.nr, args.ntheta, args.nphi, r, w, aT, aE, K=K, prec=args.prec,
                  nside=args.nside or None)
    if args.tiles:
        sh.set_tiles(*(int(x) for x in args.tiles.split(",")))
    sh.profile(max(args.reps, 1))
    for i in range(args.reps):
        sh.generate(1, i, args.fnl)
    torch.cuda.synchronize()
    if args.maps:
        sh.maps_prepare()
        o = sh.generate(1, 0, args.fnl, parts=False)
        maps = sh.maps(o["aT"], o["aE"])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(max(args.reps, 1)):
            sh.maps(o["aT"], o["aE"], out=maps)
        e1.record()
        torch.cuda.synchronize()
        print(f"maps: {e0.elapsed_time(e1) / max(args.reps, 1):.4f} ms per call")
    if args.ksw:
        k = F.Ksw(sh)
        o = sh.generate(1, 0, args.fnl, parts=False)
        s = k.statistic(o["aT"], o["aE"])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(max(args.reps, 1)):
            k.statistic(o["aT"], o["aE"], out=s)
        e1.record()
        torch.cuda.synchronize()
        print(f"ksw: {e0.elapsed_time(e1) / max(args.reps, 1):.4f} ms per sky, normalisation {k.norm:.6g} "
              f"({k.norm_seconds:.3f} s), f_NL estimate {float(s.item()) / k.norm:.4g}")
        k.close()
    sh.device_status()
    ms, calls = sh.stage_ms()
    per = {k: round(v / max(calls, 1), 4) for k, v in ms.items()}
    grid = f"HEALPix nside {args.nside}" if args.nside else f"grid {args.ntheta}x{args.nphi}"
    print(f"l_max={args.lmax} N_r={args.nr} {grid} {args.prec}: "
          f"{sh.device_bytes / 1e9:.2f} GB on the device; ms per realisation {per}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
