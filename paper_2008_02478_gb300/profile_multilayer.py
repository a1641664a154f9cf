"""Run a few multi-mesh demag evaluations of the six-layer stack (for
profilers) and print the per-kernel-class CUDA-event times:
``python -m paper_2008_02478_gb300.profile_multilayer``."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import numpy as np
import torch
from paper_2008_02478_gb300 import inputs
from paper_2008_02478_gb300.binding import MultiPlan
d = inputs.MULTILAYER
cells, origins = inputs.stack_geometry(d["layers"], d["hz"], d["gaps"], d["hxy"])
mp = MultiPlan(d["layers"], cells, origins)
M = torch.tensor(np.concatenate([inputs.random_unit(*l, seed=i).reshape(-1) for i, l in enumerate(d["layers"])]) * 8e5, dtype=torch.float32, device="cuda")
H = torch.empty_like(M)
for _ in range(3): mp.apply(M, H)
mp.profile(True)
for _ in range(5): mp.apply(M, H)
k, t = mp.profile_read()
print({kk: round(v[0] / max(v[1], 1), 4) for kk, v in k.items() if v[1]})
