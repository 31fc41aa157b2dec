"""Write the likelihood kernel's tile table, tuning/loglik_tiles.json, on a GB300.

For a grid of shapes (n individuals, p markers, N particles) spanning the workloads -- the
hit regions' n = 1000..5000 and p = 20..500, N = 4096..16384 -- every tile configuration
valid for the shape (include/spa.h, spa_loglik_tile_config) is timed in the sweep's own launch
configuration: one short sweep packs the particle operand, then 10 warm-up and 50 timed
launches of the likelihood kernel (spa_loglik_repeat, CUDA events on the context's stream).
The fastest configuration of each shape goes into the table. The library reads the table
when it sizes a workspace and takes the nearest shape's configuration instead of timing.

  python -m paper_1106_0322_gb300.tune_tiles [--out PATH]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_OUT = os.path.join(HERE, "tuning", "loglik_tiles.json")

N_GRID = (1000, 2000, 3000, 5000)
P_GRID = (20, 50, 100, 200, 300, 500)
PARTICLES = (4096, 8192, 16384)
CONFIGS = {0: "BN 256, 3 stages, 16 epilogue warps", 1: "BN 128, 4 stages, 16 epilogue warps",
           2: "BN 256, 3 stages, 8 epilogue warps", 3: "BN 128, 6 stages, 16 epilogue warps (p <= 255)",
           4: "BN 256, 6 stages, 8 epilogue warps, particle operand in tensor memory (p <= 255)",
           5: "BN 128, 12 stages, 16 epilogue warps, particle operand in tensor memory (p <= 255)",
           6: "BN 224, 4 stages, 8 epilogue warps, compact resident particle operand (p <= 255, last k-block <= 32 wide)"}


def time_config(spa, region, cfg, N, stream, sched):
    import torch

    region.set_tile_config(cfg)
    region.run_device(sched, N, 1, 1, None)  # workspace with this configuration, packed operand
    region.sync()
    got, _ = region.tile_config()
    if got != cfg:
        return None  # not valid for this shape
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    region.loglik_repeat(N, 10, stream.cuda_stream)
    e0.record(stream)
    region.loglik_repeat(N, 50, stream.cuda_stream)
    e1.record(stream)
    e1.synchronize()
    region.sync()
    return e0.elapsed_time(e1) / 50 * 1e3


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_OUT)
    args = ap.parse_args()
    import torch

    sys.path.insert(0, os.path.dirname(HERE))
    import __graft_entry__

    __graft_entry__.build()
    import paper_1106_0322_gb300 as spa
    from paper_1106_0322_gb300 import synth

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    sched = torch.tensor(synth.geometric_schedule(2), dtype=torch.float64, device=dev)
    entries = []
    t0 = time.time()
    for n in N_GRID:
        for p in P_GRID:
            g = synth.make_region(n, p, 0.9, (0.4, -0.3), seed=n + p)
            with spa.Region(g.G, g.y, 1.0, config=spa.make_config(stream=stream.cuda_stream)) as r:
                for N in PARTICLES:
                    us = {}
                    for cfg in CONFIGS:
                        t = time_config(spa, r, cfg, N, stream, sched)
                        if t is not None:
                            us[cfg] = round(t, 3)
                    best = min(us, key=us.get)
                    entries.append({"n": n, "p": p, "N_pad": (N + 127) // 128 * 128, "config": best,
                                    "us": {str(k): v for k, v in us.items()}})
                    print(json.dumps(entries[-1]), flush=True)
    doc = {"device": torch.cuda.get_device_name(0), "generated_by": "paper_1106_0322_gb300/tune_tiles.py",
           "timing": "spa_loglik_repeat: 10 warm-up and 50 timed launches, CUDA events, microseconds per launch",
           "configs": {str(k): v for k, v in CONFIGS.items()}, "seconds": round(time.time() - t0, 1),
           "entries": entries}
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    with open(args.out, "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote", args.out, len(entries), "entries")
    return 0


if __name__ == "__main__":
    sys.exit(main())
