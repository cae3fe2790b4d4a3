"""Run a bounded number of SVT iterations of one workload through the C-ABI (for profilers).

    python -m paper_0810_3286_gb300.profile_case --config single_1000 --iters 6 [--precision fp32]

The problem is built, configured (kick) and stepped `--iters` times; nothing is timed.  Used to
give Nsight Compute a short, representative launch sequence of the solver's kernels.
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--config", default="single_1000")
    ap.add_argument("--iters", type=int, default=6)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--lanczos-steps", type=int, default=3)
    ap.add_argument("--verbose", action="store_true", help="print every step's record")
    ap.add_argument("--no-graphs", action="store_true", help="launch kernels one by one (no CUDA graphs)")
    args = ap.parse_args()
    import torch
    from paper_0810_3286_gb300 import Solver, build
    from svt_inputs import config_problem
    build.build()
    torch.cuda.set_device(0)
    p = config_problem(args.config, args.seed)
    rows = torch.from_numpy(p.rows).cuda()
    cols = torch.from_numpy(p.cols).cuda()
    vals = torch.from_numpy(p.vals).cuda()
    s = Solver(p.n1, p.n2, rows, cols, vals, precision=args.precision, lanczos_steps=args.lanczos_steps,
               use_graphs=not args.no_graphs)
    s.configure(p.tau_default(), p.delta_default(), 1e-4, 27)
    info = None
    for _ in range(args.iters):
        info = s.step()
        if args.verbose:
            print("k=%d r=%d s=%d passes=%d cycles=%d spmm=%d res=%.3e sigma1=%.6e ms=%.3f" % (
                info["k"], info["r"], info["s"], info["passes"], info["lanczos_cycles"], info["spmm_calls"],
                info["residual"], info["sigma1"], info["ms"]))
        if info["stopped"]:
            break
    print("iterations %d rank %d residual %.3e counters %s" % (info["k"], info["r"], info["residual"], s.counters()))
    s.close()


if __name__ == "__main__":
    main()
