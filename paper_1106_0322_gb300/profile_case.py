"""A short run of one workload's per-move kernels, for a profiler to capture.

One short sweep of the named workload (three scale steps, one move each, by default)
runs every per-step kernel and builds the context's workspace in the sweep's launch
configuration. Then `--reps` launches of the chosen kernels follow
on the same stream, with few launches before them:

- `loglik`: the log-likelihood GEMM (the RW sweep's per-move kernel);
- `grad`: the MALA gradient kernels, i.e. the residual likelihood pass, the adjoint GEMM
  and the gradient finish.

    python -m paper_1106_0322_gb300.profile_case --workload hit-region --mode loglik --reps 3
"""
from __future__ import annotations

import argparse


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="hit-region")
    ap.add_argument("--mode", default="loglik", choices=["loglik", "grad"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--steps", type=int, default=3, help="scale steps of the set-up sweep")
    ap.add_argument("--moves", type=int, default=1, help="moves per scale step of the set-up sweep")
    ap.add_argument("--ess-frac", type=float, default=0.75, help="1.0 resamples at every step of the set-up sweep")
    args = ap.parse_args(argv)

    import torch

    from . import Region, load, make_config, synth

    load(build_if_missing=True)
    w = synth.WORKLOADS[args.workload]
    if args.mode == "grad" and w["move"] != "mala":
        raise SystemExit(f"workload {args.workload} has no MALA moves")
    region = synth.workload_region(args.workload)
    dev = torch.device("cuda", 0)
    sched = torch.tensor(synth.workload_schedule(args.workload)[: args.steps], dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    cfg = make_config(move=w["move"], precision="split_bf16", stream=stream.cuda_stream, ess_frac=args.ess_frac)
    reg = Region(region.G, region.y, w["nu"], config=cfg)
    T, p = args.steps, w["p"]
    out = {
        "mean": torch.empty((T, p), dtype=torch.float64, device=dev),
        "quantile": torch.empty((T, p, 3), dtype=torch.float64, device=dev),
        "conc": torch.empty((T, p, 2), dtype=torch.float64, device=dev),
        "ess": torch.empty(T, dtype=torch.float64, device=dev),
        "log_z_inc": torch.empty(T, dtype=torch.float64, device=dev),
        "accept_rate": torch.empty(T, dtype=torch.float64, device=dev),
        "resampled": torch.empty(T, dtype=torch.uint8, device=dev),
    }
    reg.run_device(sched, w["N"], args.moves, 1, out)
    reg.sync()
    if args.mode == "loglik":
        reg.loglik_repeat(w["N"], args.reps, stream.cuda_stream)
    else:
        reg.grad_repeat(w["N"], args.reps, stream.cuda_stream)
    reg.sync()
    torch.cuda.synchronize()
    cfg_id, src = reg.tile_config()
    print(f"{args.workload} {args.mode}: {args.reps} launches, tile configuration {cfg_id} (source {src})")
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
