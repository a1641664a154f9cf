"""Checkpoint and resume of a running LLG simulation.

A checkpoint is one .npz file with the unit magnetisation m ([3][nz][ny][nx],
the plan's precision), the simulated time t (s), the current step size dt (s;
RKF45 adapts it), the number of steps taken, and the thermal field's seed and
temperature.  The step count matters beyond bookkeeping: the thermal field of
step s is drawn from a counter-based generator keyed by (seed, s, cell), so a
resumed run continues the same random sequence only once the plan's counter is
set back to the saved step (`resume` does that).  Everything else a run needs
(the plan, the LLG parameters, the field terms) is configuration that the
caller recreates.
"""
from __future__ import annotations

import numpy as np

FORMAT = 1


def save_state(path, m, t: float, dt: float, step: int, seed: int = 0, temperature: float = 0.0) -> None:
    """Write the checkpoint (m: torch tensor on any device, or numpy array)."""
    arr = m.detach().cpu().numpy() if hasattr(m, "detach") else np.asarray(m)
    if arr.ndim != 4 or arr.shape[0] != 3:
        raise ValueError("m must be [3][nz][ny][nx]")
    np.savez(path, format=np.int64(FORMAT), m=arr, t=np.float64(t), dt=np.float64(dt), step=np.int64(step),
             seed=np.uint64(seed), temperature=np.float64(temperature))


def load_state(path) -> dict:
    """Read a checkpoint: {"m": numpy array, "t", "dt", "step", "seed", "temperature"}."""
    with np.load(path) as z:
        if int(z["format"]) != FORMAT:
            raise ValueError("unknown checkpoint format %d" % int(z["format"]))
        return {"m": z["m"].copy(), "t": float(z["t"]), "dt": float(z["dt"]), "step": int(z["step"]),
                "seed": int(z["seed"]), "temperature": float(z["temperature"])}


def resume(plan, state: dict, device: str = "cuda"):
    """Put a loaded checkpoint back on a plan: returns m as a tensor on
    `device` and sets the plan's thermal step counter to the saved step.  The
    plan must have the same mesh, and the caller sets the same field terms
    (seed and temperature are in `state`) before or after this call."""
    import torch
    m = torch.tensor(state["m"], device=device)
    if tuple(m.shape) != tuple(plan.field_shape):
        raise ValueError("checkpoint mesh %s does not match the plan's %s" % (tuple(m.shape), plan.field_shape))
    plan.thermal_set_step(state["step"])
    return m
