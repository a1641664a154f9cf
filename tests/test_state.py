"""Checkpoint files (paper_2008_02478_gb300.state): the round trip keeps the
magnetisation bit for bit and the scalars exactly, and malformed input is
rejected.  The GPU side (resuming a thermal run) is in test_gpu_thermal.py."""
import numpy as np
import pytest

from paper_2008_02478_gb300 import inputs
from paper_2008_02478_gb300.state import load_state, save_state


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_round_trip(tmp_path, dtype):
    m = inputs.random_unit(7, 5, 3, seed=3).astype(dtype)
    p = tmp_path / "ck.npz"
    save_state(p, m, t=1.25e-11, dt=2.5e-14, step=500, seed=0xFEDCBA9876543210, temperature=300.0)
    s = load_state(p)
    assert s["m"].dtype == dtype and np.array_equal(s["m"], m)
    assert (s["t"], s["dt"], s["step"], s["seed"], s["temperature"]) == (1.25e-11, 2.5e-14, 500,
                                                                         0xFEDCBA9876543210, 300.0)


def test_rejects_a_field_that_is_not_three_components(tmp_path):
    with pytest.raises(ValueError):
        save_state(tmp_path / "bad.npz", np.zeros((2, 3, 4, 5)), 0.0, 1e-13, 0)


def test_rejects_an_unknown_format(tmp_path):
    p = tmp_path / "other.npz"
    np.savez(p, format=np.int64(99), m=np.zeros((3, 1, 1, 1)), t=0.0, dt=0.0, step=0, seed=np.uint64(0),
             temperature=0.0)
    with pytest.raises(ValueError):
        load_state(p)
