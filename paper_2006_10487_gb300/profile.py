"""Runs one kernel of the step on a named workload, for profilers.

python -m paper_2006_10487_gb300.profile --workload hlbm_large_fv --kernel fv
    [--precision fp32] [--warmup 2] [--reps 20] [--fv-variant N]

Creates the solver (which runs its block-shape autotuner), advances `warmup`
coarse steps, then launches `kernel` ("fv" for the Eq. 3 sub-step, "collideL"
for the lattice of level L) `reps` times back to back, twice (a warm-up graph
and a timed graph), and prints the average time per launch from CUDA events.
Under ncu, select the launches with -k and -s (the timed graph's launches
are the last `reps` of that kernel).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="hlbm_large_fv")
    ap.add_argument("--kernel", default="fv")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp16s"])
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--fv-variant", type=int, default=0, help="finite-volume kernel variant (0: autotuned)")
    args = ap.parse_args()
    import paper_2006_10487_gb300 as H
    from workloads import make_case
    case = make_case(args.workload)
    s = H.Solver(case, precision=args.precision, use_graphs=True, fv_variant=args.fv_variant)
    s.step(args.warmup)
    s.sync()
    ms = s.time_kernel(args.kernel, args.reps)
    key = "fv_bytes" if args.kernel == "fv" else "collide_bytes" + args.kernel[len("collide"):]
    nbytes = s.info(key)
    out = {"workload": args.workload, "kernel": args.kernel, "precision": args.precision,
           "launch_ms": ms, "bytes_per_launch": nbytes, "gbs": nbytes / (ms * 1e-3) / 1e9,
           "n_sub": s.info("n_sub"), "fv_variant": s.info("fv_variant"), "tile_rows": s.info("fv_tile_rows")}
    if args.kernel == "fv":
        # launches of the kernel before the timed graph: the FP32 autotuner's
        # 3 + 20 per variant timed, the warm-up steps' sub-steps, the warm-up graph
        tune = 23 * sum(1 for v in range(1, 9) if s.info(f"fv_tune_us{v}") > 0)
        out["ncu_skip"] = tune + args.warmup * 2 ** (case.n_levels - 1) * int(out["n_sub"]) + args.reps
    s.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
