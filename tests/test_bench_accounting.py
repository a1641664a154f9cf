"""The byte accounting behind bench.py's roofline figures, checked against the
counts written out by hand for the 512 x 512 x 32 film (padded 1024 x 1024 x
64, FP32): the x passes move the real field and the x half spectrum, the y
passes the x half spectrum and the padded y-z spectrum, the z convolution
reads and writes the padded spectrum and reads the kernel-spectrum octant,
and an RK4 stage moves 48, 72, 72 and 60 bytes per cell."""
from types import SimpleNamespace

import pytest

import bench


def film_plan(fp64=False):
    return SimpleNamespace(shape=(512, 512, 32), padded=lambda: (1024, 1024, 64), fp64=fp64)


def test_transform_and_convolution_bytes():
    p = film_plan()
    cells = 512 * 512 * 32
    field = 3 * cells * 4                            # 100.7 MB
    x_half = 513 * 3 * 32 * 512 * 8                  # [kx][c][z][y] complex: 201.7 MB
    y_pad = 513 * 1024 * 3 * 32 * 8                  # [kx][c][z][ky] complex: 403.4 MB
    octant = 513 * 513 * 33 * 6 * 4                  # six real kernel components: 208.4 MB
    assert bench.xpass_algorithmic_bytes(p) == field + x_half
    s = bench.split_algorithmic_bytes(p)
    assert s["y_fwd"] == x_half + y_pad == s["y_inv"]
    assert s["z_conv"] == 2 * y_pad + octant
    assert s["z_conv"] == pytest.approx(1015.3e6, rel=1e-4)
    assert bench.xpass_algorithmic_bytes(p) == pytest.approx(302.4e6, rel=1e-3)


def test_rk4_stage_bytes_and_fp64():
    p = film_plan()
    cells = 512 * 512 * 32
    assert bench.llg_algorithmic_bytes(p) == (48 + 72 + 72 + 60) / 4 * cells
    assert bench.llg_algorithmic_bytes(film_plan(fp64=True)) == 2 * bench.llg_algorithmic_bytes(p)
    assert bench.split_algorithmic_bytes(film_plan(fp64=True))["z_conv"] == 2 * bench.split_algorithmic_bytes(p)["z_conv"]


def test_whole_job_rate_is_all_ranks_work_over_the_slowest():
    assert bench.whole_job_rate(4, 8388608 * 60, 0.165) == pytest.approx(4 * 8388608 * 60 / 0.165)


def test_hot_path_row_bytes():
    """Per-evaluation bytes of the rows: a3 = X^ + N^ + Y^ = 611.8 MB and the
    compulsory M + H + N^ = 409.8 MB (the figures the roofline reports)."""
    r = bench.demag_row_bytes(film_plan())
    assert r["a3"] == 2 * 513 * 3 * 32 * 512 * 8 + 513 * 513 * 33 * 6 * 4
    assert r["a3"] == pytest.approx(611.8e6, rel=1e-3)
    assert r["compulsory"] == pytest.approx(409.8e6, rel=1e-3)
    assert r["a2"] == r["a4"] == bench.xpass_algorithmic_bytes(film_plan())
    assert bench.ROW_OF["z_conv"] == "a3" and bench.ROW_OF["x_r2c"] == "a2"
