"""Run a few demag evaluations (and optionally RK4 steps) on one mesh, for
profilers: ``python -m paper_2008_02478_gb300.profile_demag --mesh 512,512,32
--evals 3 [--steps 1] [--tc fp16]``.  Uses random unit magnetisation, 4 nm cells."""
from __future__ import annotations

import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--mesh", default="512,512,32")
    ap.add_argument("--cell", type=float, default=4e-9)
    ap.add_argument("--evals", type=int, default=3)
    ap.add_argument("--steps", type=int, default=0)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--tc", default=None, choices=["fp16", "bf16"], help="tensor-core z stage")
    a = ap.parse_args()
    import torch

    from paper_2008_02478_gb300 import inputs
    from paper_2008_02478_gb300.binding import LLGParams, Plan
    n = tuple(int(v) for v in a.mesh.split(","))
    dt = torch.float64 if a.fp64 else torch.float32
    plan = Plan(*n, a.cell, a.cell, a.cell, fp64=a.fp64, tc=a.tc)
    m0 = inputs.random_unit(*n, seed=1)
    M = torch.tensor(8e5 * m0, dtype=dt, device="cuda")
    H = torch.empty_like(M)
    for _ in range(a.evals):
        plan.apply(M, H)
    m = torch.tensor(m0, dtype=dt, device="cuda")
    for _ in range(a.steps):
        plan.llg_step(m, LLGParams(), 1e-13)
    torch.cuda.synchronize()
    print("ok mesh=%s padded=%s" % (n, plan.padded()))


if __name__ == "__main__":
    main()
