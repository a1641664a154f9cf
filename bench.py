"""Benchmark: LLG cell-steps/s (RK4, four demag evaluations per step) and demag
evals/s on a 512 x 512 x 32 film of 4 nm cells, FP32 (with the FP64 plan timed
beside it), through the C ABI of libboris.

One step = one RK4 step of the whole mesh: 4 x (x real-to-complex transform,
fused y-z spectral pass, x complex-to-real transform, fused LLG stage).
Prints one JSON line on rank 0.  Under torchrun each rank runs its own
independent replica of the film (the path does not shard): value is the sum
of all ranks' cell-steps over the slowest rank's time.

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "demag evals/s & LLG cell-steps/s at 512x512x32 FP32 vs FP64; % HBM roofline"
UNIT = "cell-steps/s"
N_MESH = (512, 512, 32)
CELL = (4e-9, 4e-9, 4e-9)
MS, A_EX, ALPHA, DT = 8e5, 1.3e-11, 0.02, 1e-13
MU0 = 4e-7 * math.pi
HEXT = (0.0, 0.0, 0.1 / MU0)  # 100 mT perpendicular applied field
GRAIN = 40e-9
SEED = 3
WORKLOAD = "512x512x32 film, 4 nm cubic cells, 2621 columnar Voronoi grains (40 nm), RK4 dt=1e-13 s"


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture on this workload, keyed by kernel (the z-convolution class names
# its variant: plain, tma1 one-stage, tma2 two-stage bulk-copy pipeline, res
# residue-split), with
# a digest of the kernel's sources at capture time; a changed source voids it.
TRAFFIC = {
    "z_conv/plain": (1035.0e6, "b51fe8b7759c3a7a", ["paper_2008_02478_gb300/csrc/demag_split.cu",
                                            "paper_2008_02478_gb300/csrc/fft_engine.cuh",
                                            "paper_2008_02478_gb300/csrc/twiddle128.h"]),
    "z_conv/res": (994.3e6, "6e0854fa9ad57272", ["paper_2008_02478_gb300/csrc/zconv_res.cu",
                                          "paper_2008_02478_gb300/csrc/bulk_async.cuh",
                                          "paper_2008_02478_gb300/csrc/fft_engine.cuh",
                                          "paper_2008_02478_gb300/csrc/twiddle128.h"]),
    "z_conv/tma2": (964.1e6, "6399403a9bae76bf", ["paper_2008_02478_gb300/csrc/zconv_tma.cu",
                                           "paper_2008_02478_gb300/csrc/bulk_async.cuh",
                                           "paper_2008_02478_gb300/csrc/fft_engine.cuh",
                                           "paper_2008_02478_gb300/csrc/twiddle128.h"]),
}


def traffic_for(kernel):
    import hashlib
    if kernel not in TRAFFIC:
        return None
    val, digest, files = TRAFFIC[kernel]
    m = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            m.update(fh.read())
    return val if m.hexdigest()[:16] == digest else None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1])]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(num(r[2]) or 0 for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def film_state():
    from paper_2008_02478_gb300 import inputs
    return inputs.voronoi_columnar(*N_MESH, CELL, GRAIN, SEED)


def yz_algorithmic_bytes(plan) -> int:
    """Compulsory bytes of one fused y-z launch: read and write every kx plane of
    the spectrum ([kx][3][nz][ny] complex) and read the kernel-spectrum octant
    (6 reals per (kx, ky', kz'))."""
    nx, ny, nz = plan.shape
    px, py, pz = plan.padded()
    es = 8 if plan.fp64 else 4
    nkx, kyh, kzh = px // 2 + 1, py // 2 + 1, pz // 2 + 1
    return nkx * (2 * 3 * nz * ny * 2 * es + kyh * kzh * 6 * es)


def xpass_algorithmic_bytes(plan) -> int:
    """x transform: read (or write) the real field, write (or read) the spectrum."""
    nx, ny, nz = plan.shape
    px = plan.padded()[0]
    es = 8 if plan.fp64 else 4
    return 3 * nx * ny * nz * es + (px // 2 + 1) * 3 * nz * ny * 2 * es


def split_algorithmic_bytes(plan):
    """y forward: read X, write the column-major padded spectrum Y; z
    convolution: read and write Y and read the kernel octant; y inverse: read
    Y, write X."""
    nx, ny, nz = plan.shape
    px, py, pz = plan.padded()
    es = 8 if plan.fp64 else 4
    nkx, kyh, kzh = px // 2 + 1, py // 2 + 1, pz // 2 + 1
    xb = nkx * 3 * nz * ny * 2 * es
    yb = nkx * py * 3 * nz * 2 * es
    kb = nkx * kyh * kzh * 6 * es
    return {"y_fwd": xb + yb, "z_conv": 2 * yb + kb, "y_inv": yb + xb}


def llg_algorithmic_bytes(plan) -> float:
    """Average bytes per RK4 stage launch (no per-cell maps): 48, 72, 72, 60
    bytes per cell for the four stages in FP32 (m_s, Hd, m0, acc, next state)."""
    nx, ny, nz = plan.shape
    es = 8 if plan.fp64 else 4
    return (48 + 72 + 72 + 60) / 4.0 * (es / 4) * nx * ny * nz


def x_c2r_rk4_algorithmic_bytes(plan) -> float:
    """Inverse x transform fused with the RK4 stage: read the x half spectrum,
    then the stage's bytes without the H_d read (36, 60, 60, 48 bytes per
    cell in FP32)."""
    nx, ny, nz = plan.shape
    px = plan.padded()[0]
    es = 8 if plan.fp64 else 4
    return (px // 2 + 1) * 3 * nz * ny * 2 * es + (36 + 60 + 60 + 48) / 4.0 * (es / 4) * nx * ny * nz


def time_steps(torch, plan, m, prm, K):
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(K):
        plan.llg_step(m, prm, DT)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def time_graph(torch, plan, m, prm, K):
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    plan.llg_run_graph(m, prm, DT, K)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def time_demag(torch, plan, M, H, K):
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(K):
        plan.apply(M, H)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def oracle_rk4_rate(nx, ny, nz, steps):
    """FP64 oracle: cell-steps/s of RK4 on an nx x ny x nz block of the same film."""
    import numpy as np

    import oracle
    from oracle import llg
    from paper_2008_02478_gb300 import inputs
    m = inputs.voronoi_columnar(nx, ny, nz, CELL, GRAIN, SEED)
    prm = llg.Params(cell=CELL, Ms=MS, A=A_EX, alpha=ALPHA, Hext=HEXT)
    dem = oracle.DemagPlan(nx, ny, nz, *CELL)
    t0 = time.perf_counter()
    for _ in range(steps):
        m = llg.rk4_step(m, DT, prm, dem.apply)
    t = time.perf_counter() - t0
    return nx * ny * nz * steps / t, t, oracle.num_threads()


def oracle_demag_rates():
    """FP64 oracle: FFT-convolution demag evaluations/s on 32x32x4 (5 nm
    cells, random unit vectors) and 256x256x8 (3 nm cells), one thread and all
    threads; each figure from at least one evaluation and about 0.5 s."""
    import oracle
    from paper_2008_02478_gb300 import inputs
    allc = oracle.num_threads()
    out = {}
    for n, h in (((32, 32, 4), 5e-9), ((256, 256, 8), 3e-9)):
        M = 8e5 * inputs.random_unit(*n, seed=1)
        plan = oracle.DemagPlan(*n, h, h, h)
        row = {}
        for th in (1, allc):
            oracle.set_threads(th)
            t0, k = time.perf_counter(), 0
            while k == 0 or time.perf_counter() - t0 < 0.5:
                plan.apply(M)
                k += 1
            row["threads_%d" % th] = k / (time.perf_counter() - t0)
        out["%dx%dx%d" % n] = row
    oracle.set_threads(allc)
    return out


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _gather_stack_cells(H, counts, cells):
    """Field values [len(cells)][3] at flat cell indices of a concatenated
    multi-layer field (each layer SoA [3][nz][ny][nx])."""
    import numpy as np
    offs = np.cumsum([0] + list(counts))
    out = []
    for g in cells:
        l = int(np.searchsorted(offs, g, side="right") - 1)
        n, loc, base = counts[l], g - offs[l], 3 * offs[l]
        out.append([H[base + c * n + loc] for c in range(3)])
    return np.array(out)


def _errs(got, ref):
    import numpy as np
    got, ref = np.asarray(got, dtype=np.float64), np.asarray(ref, dtype=np.float64)
    return {"rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
            "max_rel": float(np.abs(got - ref).max() / np.abs(ref).max())}


def multilayer_workload(torch, args, world, max_over_ranks, check_oracle):
    """Six-layer stack (Eq. 4): 500 RK4 steps of the batched plan (all layers
    in each launch, one CUDA graph per step), its demag rate against the plain
    FP32 alternatives - the six layers as separate single-mesh plans applied in
    turn (self terms only, no cross-layer field) and the same batched plan with
    the layers pulled 1 mm apart (self terms only, like-for-like cost) - and
    the H_d error of each against the oracle's direct Eq. 4 sum at sampled
    cells."""
    import numpy as np

    from oracle import multilayer as ml
    from paper_2008_02478_gb300 import inputs
    from paper_2008_02478_gb300.binding import LLGParams, MultiPlan, Plan
    d = inputs.MULTILAYER
    layers = d["layers"]
    cells, origins = inputs.stack_geometry(layers, d["hz"], d["gaps"], d["hxy"])
    counts = [l[0] * l[1] * l[2] for l in layers]
    total = sum(counts)
    t0 = time.perf_counter()
    mp = MultiPlan(layers, cells, origins)
    t_plan = time.perf_counter() - t0
    m = np.concatenate([inputs.random_unit(*l, seed=d["seed"] + i).reshape(-1) for i, l in enumerate(layers)])
    ms = np.concatenate([np.full(c, d["Ms"][i]) for i, c in enumerate(counts)])
    mg = torch.tensor(m, dtype=torch.float32, device="cuda")
    prm = LLGParams(A=A_EX, alpha=ALPHA, Ms_map=torch.tensor(ms, dtype=torch.float32, device="cuda"))
    dt_ml = 5e-14
    mp.llg_run_graph(mg, prm, dt_ml, 3)
    nsteps = 500 if not args.short else 20
    ev0, ev1 = _events(torch)
    torch.cuda.synchronize()
    ev0.record()
    mp.llg_run_graph(mg, prm, dt_ml, nsteps)
    ev1.record()
    torch.cuda.synchronize()
    t = max_over_ranks(ev0.elapsed_time(ev1) / 1e3)
    nrm = torch.sqrt((mg.view(-1)[:3 * counts[0]].view(3, -1) ** 2).sum(0))
    M = np.concatenate([(m[3 * o:3 * (o + c)].reshape(3, c) * d["Ms"][i]).reshape(-1)
                        for i, (o, c) in enumerate(zip(np.cumsum([0] + counts[:-1]), counts))])
    Md = torch.tensor(M, dtype=torch.float32, device="cuda")
    Hb = torch.empty_like(Md)
    K = 40 if not args.short else 8

    def rate(fn):
        for _ in range(2):
            fn()
        a, b = _events(torch)
        torch.cuda.synchronize()
        a.record()
        for _ in range(K):
            fn()
        b.record()
        torch.cuda.synchronize()
        return world * K / max_over_ranks(a.elapsed_time(b) / 1e3)
    batched_rate = rate(lambda: mp.apply(Md, Hb))
    z, nu, NX, NY = mp.info()
    # the six layers as separate single-mesh FP32 plans (self terms only)
    singles = [Plan(*l, *cells[i]) for i, l in enumerate(layers)]
    offs = np.cumsum([0] + counts)
    Hs = torch.empty_like(Md)
    views = [(Md[3 * offs[i]:3 * offs[i + 1]].view(3, l[2], l[1], l[0]),
              Hs[3 * offs[i]:3 * offs[i + 1]].view(3, l[2], l[1], l[0])) for i, l in enumerate(layers)]

    def per_layer():
        for p, (a, b) in zip(singles, views):
            p.apply(a, b)
    single_rate = rate(per_layer)
    # self terms only, batched: the same layers 1 mm apart (cross terms ~0)
    far = [(o[0], o[1], o[2] + 1e-3 * i) for i, o in enumerate(origins)]
    mpf = MultiPlan(layers, cells, far)
    Hf = torch.empty_like(Md)
    self_batched_rate = rate(lambda: mpf.apply(Md, Hf))
    out = {"cells": total, "z_planes": z, "inter_plane_spectra": nu, "frame": [NX, NY], "steps": nsteps,
           "cell_steps_per_s": world * total * nsteps / t, "ms_per_step": 1e3 * t / nsteps,
           "max_norm_deviation_layer0": float((nrm - 1).abs().max()),
           "plan_build_s": t_plan, "dt": dt_ml,
           "demag_evals_per_s": {"batched_eq4": batched_rate, "per_layer_single_mesh_self_only": single_rate,
                                 "batched_self_only_layers_1mm_apart": self_batched_rate},
           "batched": "all layers in each launch, one CUDA graph per RK4 step"}
    if check_oracle:
        st = ml.centred_stack(layers, d["hz"], d["gaps"], d["hxy"])
        sample = inputs.rng(9).integers(0, total, 12)
        ref = ml.direct_at(st, M, sample)
        out["h_error_vs_oracle_eq4_at_12_cells"] = {
            "batched_eq4": _errs(_gather_stack_cells(Hb.cpu().numpy(), counts, sample), ref),
            "per_layer_single_mesh_self_only": _errs(_gather_stack_cells(Hs.cpu().numpy(), counts, sample), ref),
            "batched_self_only_vs_per_layer": _errs(_gather_stack_cells(Hf.cpu().numpy(), counts, sample),
                                                    _gather_stack_cells(Hs.cpu().numpy(), counts, sample))}
    for p in singles:
        p.close()
    mpf.close()
    mp.close()
    return out


def rkf45_film_workload(torch, args):
    """256x64x1 film (the shape of muMAG standard problem 4): relaxation from
    (1,1,1)/sqrt3 at alpha = 0.5 in zero field (chunks of 200 accepted steps
    until the energy changes by less than 1e-6 relative over a chunk, or 5 ns),
    then alpha = 0.02 with 25 mT at 170 degrees in-plane and 10000 timed
    accepted RKF45 steps with the step control on the device (one host
    synchronisation for all of them)."""
    from paper_2008_02478_gb300 import inputs
    from paper_2008_02478_gb300.binding import RKF45, LLGParams, Plan
    fd = inputs.FILM_SP4_MESH
    fp = Plan(*fd["n"], *fd["cell"])
    mf = torch.tensor(inputs.uniform(*fd["n"], (1, 1, 1)), dtype=torch.float32, device="cuda")
    relax = LLGParams(Ms=8e5, A=A_EX, alpha=0.5, method=RKF45, tol=1e-5, dt_min=1e-16, dt_max=1e-12)
    h, t_sim, e_prev, chunks = 1e-14, 0.0, None, 0
    t0 = time.perf_counter()
    while t_sim < 5e-9:
        h, dts = fp.llg_run_rkf45(mf, relax, h, 200)
        t_sim += dts
        chunks += 1
        e = sum(fp.energy(mf, relax))
        if e_prev is not None and abs(e - e_prev) < 1e-6 * abs(e):
            break
        e_prev = e
        if args.short and chunks >= 3:
            break
    t_relax = time.perf_counter() - t0
    drive = LLGParams(Ms=8e5, A=A_EX, alpha=0.02, Hext=(19894.4 * math.cos(math.radians(170)),
                                                       19894.4 * math.sin(math.radians(170)), 0.0),
                      method=RKF45, tol=1e-5, dt_min=1e-16, dt_max=1e-12)
    h, _ = fp.llg_run_rkf45(mf, drive, 1e-14, 20)  # capture the drive's step graph
    n_acc = 10000 if not args.short else 500
    fp.profile_read()
    ev0, ev1 = _events(torch)
    torch.cuda.synchronize()
    ev0.record()
    h, t_drive = fp.llg_run_rkf45(mf, drive, h, n_acc)
    ev1.record()
    torch.cuda.synchronize()
    t = ev0.elapsed_time(ev1) / 1e3
    _, launches = fp.profile_read()
    out = {"relax": {"alpha": 0.5, "accepted_steps": 200 * chunks, "simulated_ns": 1e9 * t_sim,
                     "converged": t_sim < 5e-9, "wall_s": t_relax},
           "accepted_steps": n_acc, "accepted_steps_per_s": n_acc / t, "cell_steps_per_s": n_acc * 256 * 64 / t,
           "simulated_ns": 1e9 * t_drive, "last_dt": h, "kernel_launches": launches,
           "host_syncs": 1, "step_control": "on the device (graph WHILE node per step)"}
    fp.close()
    return out


def gradient_film_workload(torch, args):
    """256x256x8 film, 3 nm cells, learnable per-cell Ms and Ku: forward +
    checkpointed adjoint over 2000 RK4 steps with a checkpoint every 50."""
    from paper_2008_02478_gb300 import inputs
    from paper_2008_02478_gb300.autograd import trajectory
    from paper_2008_02478_gb300.binding import LLGParams, Plan
    gd = inputs.GRAD_FILM_MESH
    gp = Plan(*gd["n"], *gd["cell"])
    nx, ny, nz = gd["n"]
    Ms = torch.tensor(inputs.smooth_noise(nx, ny, nz, 4.0, 6e5, 1e6, 5), dtype=torch.float32, device="cuda",
                      requires_grad=True)
    Ku = torch.tensor(inputs.smooth_noise(nx, ny, nz, 4.0, 0.0, 5e5, 6), dtype=torch.float32, device="cuda",
                      requires_grad=True)
    m0 = torch.tensor(inputs.smooth_texture(nx, ny, nz, 4.0, 5), dtype=torch.float32, device="cuda")
    tgt = torch.tensor(inputs.smooth_texture(nx, ny, nz, 4.0, 3), dtype=torch.float32, device="cuda")
    base = LLGParams(A=A_EX, alpha=ALPHA, easy=(0.0, 0.0, 1.0))
    L = ((trajectory(m0, Ms, Ku, gp, base, 2, DT, 50) - tgt) ** 2).sum()
    L.backward()
    nst, ck = (2000, 50) if not args.short else (100, 50)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L = ((trajectory(m0, Ms, Ku, gp, base, nst, DT, ck) - tgt) ** 2).sum()
    L.backward()
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    out = {"steps": nst, "checkpoint_every": ck, "loss": float(L.detach()),
           "forward_plus_adjoint_steps_per_s": nst / t, "cell_steps_per_s": nst * nx * ny * nz / t,
           "grad_norms": {"Ms": float(Ms.grad.norm()), "Ku": float(Ku.grad.norm())}}
    gp.close()
    return out


def other_workloads(torch, args, world, max_over_ranks, rank):
    """Throughput of the other workloads of the build on this GPU (FP32)."""
    from paper_2008_02478_gb300.binding import LLGParams, Plan
    out = {"multilayer_6": multilayer_workload(torch, args, world, max_over_ranks, rank == 0 and not args.no_cpu)}
    # periodic 512x512x32 film: x and y periodic by 8 images each side
    t0 = time.perf_counter()
    pp = Plan(*N_MESH, *CELL, images=(8, 8, 0))
    t_pbc_plan = time.perf_counter() - t0
    mpb = torch.tensor(film_state(), dtype=torch.float32, device="cuda")
    prm_p = LLGParams(Ms=MS, A=A_EX, alpha=ALPHA, Hext=HEXT)
    pp.llg_run_graph(mpb, prm_p, DT, 3)
    K = max(4, args.steps)
    ev0, ev1 = _events(torch)
    torch.cuda.synchronize()
    ev0.record()
    pp.llg_run_graph(mpb, prm_p, DT, K)
    ev1.record()
    torch.cuda.synchronize()
    t = max_over_ranks(ev0.elapsed_time(ev1) / 1e3)
    nc = N_MESH[0] * N_MESH[1] * N_MESH[2]
    out["pbc_film_512x512x32"] = {"images": [8, 8, 0], "plan_build_s": t_pbc_plan,
                                  "cell_steps_per_s": world * nc * K / t, "ms_per_step": 1e3 * t / K}
    pp.close()
    del mpb
    # Oersted field of a current density on the 512x512x32 film
    from paper_2008_02478_gb300.binding import OerstedPlan
    t0 = time.perf_counter()
    op = OerstedPlan(*N_MESH, *CELL)
    t_oe_plan = time.perf_counter() - t0
    Jd = torch.randn((3, N_MESH[2], N_MESH[1], N_MESH[0]), dtype=torch.float32, device="cuda") * 1e11
    Hoe = torch.empty_like(Jd)
    for _ in range(3):
        op.apply(Jd, Hoe)
    K = max(4, 4 * args.steps)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(K):
        op.apply(Jd, Hoe)
    ev1.record()
    torch.cuda.synchronize()
    t = max_over_ranks(ev0.elapsed_time(ev1) / 1e3)
    out["oersted_512x512x32"] = {"evals_per_s": world * K / t, "ms_per_eval": 1e3 * t / K,
                                 "plan_build_s": t_oe_plan}
    op.close()
    del Jd, Hoe
    out["rkf45_film_256x64x1"] = rkf45_film_workload(torch, args)
    out["gradient_film_256x256x8"] = gradient_film_workload(torch, args)
    return out


class Replicas:
    """The ranks of a multi-GPU run (one independent replica per GPU under
    torchrun, no data-path collective): a barrier and a maximum over ranks for
    the timing.  backend/device: "nccl"/"cuda" for the bench, "gloo"/"cpu" for
    the host-side tests.  The process group is set up from the torchrun
    environment (MASTER_ADDR, MASTER_PORT, RANK, WORLD_SIZE)."""

    def __init__(self, world: int, backend: str = "nccl", device: str = "cuda"):
        import torch
        self.torch, self.world, self.device, self.dist = torch, world, device, None
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()
        if self.device == "cuda":
            self.torch.cuda.synchronize()

    def max(self, x: float) -> float:
        if self.dist is None:
            return x
        t = self.torch.tensor([x], dtype=self.torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.barrier()
            self.dist.destroy_process_group()
            self.dist = None


def whole_job_rate(world: int, units_per_rank: float, seconds_max: float) -> float:
    """Throughput of the whole job: every rank processes units_per_rank in the
    timed region; the job takes as long as its slowest rank."""
    return world * units_per_rank / seconds_max


def run_reference(args, rank):
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    blk = (128, 128, 32)
    oracle_rk4_rate(32, 32, 32, 1)  # warm the library
    rates, times = [], []
    for _ in range(args.warmup):
        oracle_rk4_rate(*blk, 1)
    for _ in range(args.steps):
        r, t, cores = oracle_rk4_rate(*blk, 1)
        rates.append(r)
        times.append(t)
    value = sum(blk[0] * blk[1] * blk[2] for _ in times) / sum(times)
    sample = "one RK4 step per bench step of the FP64 oracle on a %dx%dx%d block of the same film" % blk
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# FP32 FMA throughput microbenchmark: eight independent FMA chains per thread,
# scalar (fmaf) and packed (__ffma2_rn) forms; compiled with nvcc at run time.
FMA_SRC = r"""
#include <cuda_runtime.h>
extern "C" __global__ void fma_scalar(float* out, int iters, float a, float b)
{
    float x[8];
    for (int k = 0; k < 8; k++) x[k] = threadIdx.x * 1e-7f + k;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
    for (int k = 0; k < 8; k++) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
extern "C" __global__ void fma_packed(float* out, int iters, float a, float b)
{
    float2 x[8];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int k = 0; k < 8; k++) x[k] = make_float2(threadIdx.x * 1e-7f + k, k + 0.5f);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = __ffma2_rn(x[k], a2, b2);
    }
    float s = 0.f;
    for (int k = 0; k < 8; k++) s += x[k].x + x[k].y;
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
extern "C" int fma_run(int packed, int blocks, int threads, int iters, float* ms)
{
    float* out;
    if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(float)) != cudaSuccess) return 1;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int rep = 0; rep < 2; rep++) {  // the first launch warms up
        cudaEventRecord(e0);
        if (packed) fma_packed<<<blocks, threads>>>(out, iters, 0.999999f, 1e-6f);
        else fma_scalar<<<blocks, threads>>>(out, iters, 0.999999f, 1e-6f);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
    }
    cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const int rc = cudaGetLastError() != cudaSuccess;
    cudaFree(out);
    return rc;
}
"""


def fma_peak():
    """Measured FP32 FMA throughput (TFLOP/s) of the scalar and packed forms."""
    import ctypes
    import subprocess
    import tempfile

    import torch
    from paper_2008_02478_gb300 import build as bld
    d = tempfile.mkdtemp(prefix="fma_peak_")
    src, lib = os.path.join(d, "fma.cu"), os.path.join(d, "fma.so")
    with open(src, "w") as f:
        f.write(FMA_SRC)
    subprocess.run([bld.nvcc(), *bld.ARCH, "-O3", "-shared", "-Xcompiler", "-fPIC", "-o", lib, src], check=True)
    torch.cuda.init()
    so = ctypes.CDLL(lib)
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    blocks, threads, iters = nsm * 8, 256, 1 << 16
    out = {}
    for name, packed in (("scalar", 0), ("packed", 1)):
        ms = ctypes.c_float()
        if so.fma_run(packed, blocks, threads, iters, ctypes.byref(ms)):
            raise RuntimeError("FMA microbenchmark failed")
        lanes = 2 if packed else 1
        flops = 2.0 * 8 * lanes * iters * blocks * threads
        out[name] = flops / (ms.value * 1e-3) / 1e12
    return {"fp32_fma_tflops": out, "sms": nsm, "kernel": "8 independent FMA chains per thread, "
            f"{blocks} CTAs x {threads} threads x {iters} iterations"}


def fig11_sweep(torch, Plan, LLGParams, steps):
    """Fig. 11-shaped sweep: demag evaluation time and RK4 cell-steps/s for
    nz in {1, 2, 4, 8, 16, 32} and N = 2^14 .. 2^23 cells, nx = ny (ny = 2 nx
    where N / nz is not a square), 4 nm cells, perpendicular applied field."""
    import numpy as np
    from paper_2008_02478_gb300 import inputs
    rows = []
    prm = LLGParams(Ms=MS, A=A_EX, alpha=ALPHA, Hext=HEXT)
    for nz in (1, 2, 4, 8, 16, 32):
        for k in range(14, 24):
            plane = (1 << k) // nz
            lg = plane.bit_length() - 1
            nx = 1 << (lg // 2)
            ny = plane // nx
            try:
                plan = Plan(nx, ny, nz, *CELL)
            except Exception as e:  # noqa: BLE001 - reported per size
                rows.append({"nz": nz, "nx": nx, "ny": ny, "cells": nx * ny * nz, "error": str(e)[:80]})
                continue
            m0 = inputs.random_unit(nx, ny, nz, SEED)
            M = torch.tensor(MS * m0, dtype=torch.float32, device="cuda")
            H = torch.empty_like(M)
            for _ in range(3):
                plan.apply(M, H)
            K = max(4, min(200, int(2e8 // (nx * ny * nz))))
            t_eval = time_demag(torch, plan, M, H, K) / K
            m = torch.tensor(m0, dtype=torch.float32, device="cuda")
            plan.llg_run_graph(m, prm, DT, 3)
            Ks = max(2, K // 4)
            t_step = time_graph(torch, plan, m, prm, Ks) / Ks
            rows.append({"nz": nz, "nx": nx, "ny": ny, "cells": nx * ny * nz, "ms_per_eval": 1e3 * t_eval,
                         "demag_evals_per_s": 1.0 / t_eval, "ms_per_step": 1e3 * t_step,
                         "cell_steps_per_s": nx * ny * nz / t_step, "yz_schedule": list(plan.schedule())})
            plan.close()
            del M, H, m
            torch.cuda.empty_cache()
    return rows


def profile_run(args):
    """--profile demag: a few demag evaluations (and optional RK4 steps) on one
    mesh, random unit magnetisation; --profile multilayer: a few evaluations
    of the six-layer stack with the per-kernel-class CUDA-event times.  Small,
    self-contained runs for ncu captures."""
    import numpy as np
    import torch

    from paper_2008_02478_gb300 import build as bld
    from paper_2008_02478_gb300 import inputs
    from paper_2008_02478_gb300.binding import LLGParams, MultiPlan, Plan
    bld.build()
    if args.profile == "multilayer":
        d = inputs.MULTILAYER
        cells, origins = inputs.stack_geometry(d["layers"], d["hz"], d["gaps"], d["hxy"])
        mp = MultiPlan(d["layers"], cells, origins)
        M = torch.tensor(np.concatenate([inputs.random_unit(*l, seed=i).reshape(-1)
                                         for i, l in enumerate(d["layers"])]) * 8e5, dtype=torch.float32,
                         device="cuda")
        H = torch.empty_like(M)
        for _ in range(3):
            mp.apply(M, H)
        mp.profile(True)
        for _ in range(max(1, args.evals)):
            mp.apply(M, H)
        k, _ = mp.profile_read()
        print(json.dumps({kk: round(v[0] / max(v[1], 1), 4) for kk, v in k.items() if v[1]}))
        return 0
    n = tuple(int(v) for v in args.mesh.split(","))
    dt = torch.float64 if args.fp64 else torch.float32
    plan = Plan(*n, args.cell, args.cell, args.cell, fp64=args.fp64, tc=args.tc)
    m0 = inputs.random_unit(*n, seed=1)
    M = torch.tensor(8e5 * m0, dtype=dt, device="cuda")
    H = torch.empty_like(M)
    for _ in range(args.evals):
        plan.apply(M, H)
    m = torch.tensor(m0, dtype=dt, device="cuda")
    for _ in range(args.llg_steps):
        plan.llg_step(m, LLGParams(), 1e-13)
    torch.cuda.synchronize()
    print("ok mesh=%s padded=%s schedule=%s" % (n, plan.padded(), plan.schedule()))
    return 0


def demag_row_bytes(plan):
    """Algorithmic bytes of the hot-path rows per demag evaluation (FP32 or
    FP64 per the plan): X^ = the x half spectrum [kx][3][nz][ny] complex, N^ =
    the kernel-spectrum octant (6 reals per (kx, ky', kz')), M and H the real
    fields.  a2 (x R2C) = M + X^, a3 (y-z pass) = X^ + N^ + Y^ with Y^ the
    same size as X^, a4 (x C2R) = X^ + H; compulsory = M + H + N^."""
    nx, ny, nz = plan.shape
    px, py, pz = plan.padded()
    es = 8 if plan.fp64 else 4
    nkx, kyh, kzh = px // 2 + 1, py // 2 + 1, pz // 2 + 1
    field = 3 * nx * ny * nz * es
    xhat = nkx * 3 * nz * ny * 2 * es
    khat = nkx * kyh * kzh * 6 * es
    return {"a2": field + xhat, "a3": 2 * xhat + khat, "a4": xhat + field, "compulsory": 2 * field + khat,
            "field": field, "xhat": xhat, "khat": khat}


# kernel class -> the hot-path row it realises
ROW_OF = {"x_r2c": "a2", "yz_conv": "a3", "y_fwd": "a3", "z_conv": "a3", "y_inv": "a3", "x_c2r": "a4",
          "llg_stage": "a5/a6", "x_c2r_rk4": "a4+a5/a6"}
DEMAG_KERNELS = ("x_r2c", "yz_conv", "y_fwd", "z_conv", "y_inv", "x_c2r")


def film_accuracy_check(torch, plan, prm, m0, nsteps, cpu_threads):
    """The 512x512x32 film after nsteps RK4 steps (CUDA graph): energies every
    nsteps/10 steps (damped and driven by a constant field, the total must not
    rise), the largest deviation of |m| from 1, and H_d of the final state from
    the FP32 plan against the FP64 oracle's FFT convolution of the same state
    (one oracle evaluation on the host cores, timed)."""
    import numpy as np

    import oracle
    from oracle import llg
    m = torch.tensor(m0, dtype=torch.float32, device="cuda")
    energies = [sum(plan.energy(m, prm))]
    chunk = max(1, nsteps // 10)
    done = 0
    while done < nsteps:
        k = min(chunk, nsteps - done)
        plan.llg_run_graph(m, prm, DT, k)
        done += k
        energies.append(sum(plan.energy(m, prm)))
    mh = m.cpu().numpy().astype(np.float64)
    nrm_dev = float(np.abs(np.sqrt((mh * mh).sum(0)) - 1.0).max())
    M = torch.tensor(MS * mh, dtype=torch.float32, device="cuda")
    Hg = plan.apply(M).cpu().numpy().astype(np.float64)
    oracle.set_threads(cpu_threads)
    t0 = time.perf_counter()
    dem = oracle.DemagPlan(*N_MESH, *CELL)
    t_plan = time.perf_counter() - t0
    t0 = time.perf_counter()
    Ho = dem.apply(MS * mh)
    t_eval = time.perf_counter() - t0
    e_or = llg.energies(mh, llg.Params(cell=CELL, Ms=MS, A=A_EX, alpha=ALPHA, Hext=HEXT), lambda _M: Ho)
    e_gpu = plan.energy(m, prm)
    de = np.diff(np.array(energies))
    return {"steps": nsteps, "h_d_vs_oracle": _errs(Hg, Ho),
            "energies_J_gpu": list(e_gpu), "energies_J_oracle": list(e_or),
            "energy_rel_err": float(abs(sum(e_gpu) - sum(e_or)) / abs(sum(e_or))),
            "energy_trace_J": energies, "energy_never_rises": bool((de <= 1e-9 * abs(energies[0])).all()),
            "max_abs_norm_deviation": nrm_dev,
            "oracle_512x512x32_eval_s": t_eval, "oracle_plan_s": t_plan, "oracle_threads": cpu_threads}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--short", action="store_true", help="shorter extra workloads (quick checks)")
    ap.add_argument("--sweep", action="store_true",
                    help="only the Fig. 11-shaped size sweep and the FP32 FMA peak (one JSON line)")
    ap.add_argument("--profile", choices=["demag", "multilayer"], default=None,
                    help="a small run for profilers (no JSON line): see --mesh, --evals, --llg-steps")
    ap.add_argument("--mesh", default="512,512,32")
    ap.add_argument("--cell", type=float, default=4e-9)
    ap.add_argument("--evals", type=int, default=3)
    ap.add_argument("--llg-steps", type=int, default=0)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--tc", default=None, choices=["fp16", "bf16"])
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.profile:
        return profile_run(args)
    if args.warmup < 3:
        raise SystemExit("need --warmup >= 3")

    import numpy as np
    import torch

    from paper_2008_02478_gb300 import build as bld
    from paper_2008_02478_gb300.binding import LLGParams, Plan
    bld.build()
    torch.cuda.set_device(local)
    if args.sweep:
        if rank == 0:
            rows = fig11_sweep(torch, Plan, LLGParams, args.steps)
            print(json.dumps({"sweep": "Fig. 11 shape: demag evaluation time and RK4 cell-steps/s vs N and nz, FP32",
                              "data": "synthetic", "cell": CELL, "rows": rows, "fma_peak": fma_peak()}))
        return
    ranks = Replicas(world, "nccl", "cuda")
    barrier, max_over_ranks = ranks.barrier, ranks.max

    nx, ny, nz = N_MESH
    ncell = nx * ny * nz
    m0 = film_state()
    prm = LLGParams(Ms=MS, A=A_EX, alpha=ALPHA, Hext=HEXT)
    plan = Plan(nx, ny, nz, *CELL)
    m = torch.tensor(m0, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        plan.llg_step(m, prm, DT)
    plan.llg_run_graph(m, prm, DT, args.warmup)  # capture + warm the graph
    plan.profile_read()  # reset launch counters

    # ---- A: headline timing (exactly K RK4 steps), then the same K-step
    #      window repeated until at least 1 s has been timed; the clock sampler
    #      spans both
    gpu_index = int((os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",") + ["0"])[local]) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").replace(",", "").isdigit() else local
    barrier()
    with ClockSampler(gpu_index) as clk:
        t_steps = time_graph(torch, plan, m, prm, args.steps)
        barrier()
        _, launches = plan.profile_read()
        sus_t, sus_windows = 0.0, 0
        while sus_t < 1.0:
            sus_t += time_graph(torch, plan, m, prm, args.steps)
            sus_windows += 1
    barrier()
    plan.profile_read()
    t_steps = max_over_ranks(t_steps)
    sus_t = max_over_ranks(sus_t)
    clocks = clk.summary()
    value = whole_job_rate(world, ncell * args.steps, t_steps)
    sustained = {"windows": sus_windows, "steps": sus_windows * args.steps, "seconds": sus_t,
                 "ms_per_step": 1e3 * sus_t / (sus_windows * args.steps),
                 "value": whole_job_rate(world, ncell * sus_windows * args.steps, sus_t)}
    # the same steps through one boris_llg_step call each (no graph)
    t_calls = max_over_ranks(time_steps(torch, plan, m, prm, args.steps))

    # ---- demag-only timing ------------------------------------------------
    M = torch.tensor(MS * m0, dtype=torch.float32, device="cuda")
    H = torch.empty_like(M)
    for _ in range(3):
        plan.apply(M, H)
    t_dem = max_over_ranks(time_demag(torch, plan, M, H, 4 * args.steps))
    demag_rate = world * 4 * args.steps / t_dem

    # ---- B: per-kernel CUDA-event durations over at least 1 s of steps ------
    step_s = t_steps / args.steps
    n_prof = max(args.steps, int(math.ceil(1.0 / step_s)))
    plan.profile(True)
    time_steps(torch, plan, m, prm, n_prof)
    kern, _ = plan.profile_read()
    plan.profile(False)
    dominant = max(kern, key=lambda k: kern[k][0])
    # demag kernel classes are timed per evaluation (a chunked schedule
    # launches them several times per evaluation); the LLG stage per launch
    evals = max(1, kern["x_r2c"][1]) if kern.get("x_r2c") and kern["x_r2c"][1] else 1
    units = {k: (evals if k in DEMAG_KERNELS else v[1]) for k, v in kern.items()}
    per_launch_ms = {k: (v[0] / units[k] if v[1] else None) for k, v in kern.items()}
    algo = {"yz_conv": yz_algorithmic_bytes(plan), "x_r2c": xpass_algorithmic_bytes(plan),
            "x_c2r": xpass_algorithmic_bytes(plan), "llg_stage": llg_algorithmic_bytes(plan),
            "x_c2r_rk4": x_c2r_rk4_algorithmic_bytes(plan)}
    algo.update(split_algorithmic_bytes(plan))
    rows = demag_row_bytes(plan)
    peak, peak_kind = measured_peaks()
    row = ROW_OF.get(dominant)
    row_bytes = {"a2": rows["a2"], "a3": rows["a3"], "a4": rows["a4"]}.get(row, algo.get(dominant))
    achieved = row_bytes / (per_launch_ms[dominant] * 1e-3) / 1e9 if row_bytes else None
    dom_key = dominant
    if dominant == "z_conv":
        dom_key = "z_conv/" + {0: "plain", 1: "tma1", 2: "tma2", 3: "res"}.get(plan.schedule()[2], "plain")
    # per demag evaluation: the kernels that realise row a3, and all demag kernels
    a3_ms = sum(kern[k][0] for k in ("yz_conv", "y_fwd", "z_conv", "y_inv") if k in kern) / evals
    demag_ms = sum(kern[k][0] for k in DEMAG_KERNELS if k in kern) / evals
    sched_demag = sum(algo[k] * units[k] for k in DEMAG_KERNELS if k in kern and kern[k][1]) / evals
    roofline = {"bound": "hbm", "kernel": dom_key, "row": row, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": traffic_for(dom_key),
                "peak_source": peak_kind, "algorithmic_bytes_per_launch": row_bytes,
                "bytes_basis": "SURVEY 8(d) bytes of the row the kernel realises, per evaluation",
                "kernel_own_bytes_per_launch": algo.get(dominant),
                "a3_pass": {"kernels": [k for k in ("yz_conv", "y_fwd", "z_conv", "y_inv") if k in kern],
                            "bytes": rows["a3"], "ms_per_eval": a3_ms,
                            "GBps": rows["a3"] / (a3_ms * 1e-3) / 1e9 if a3_ms else None,
                            "frac": rows["a3"] / (a3_ms * 1e-3) / 1e9 / peak if a3_ms else None},
                "demag_eval": {"compulsory_bytes": rows["compulsory"], "schedule_bytes": sched_demag,
                               "ms_per_eval": demag_ms,
                               "compulsory_frac": rows["compulsory"] / (demag_ms * 1e-3) / 1e9 / peak,
                               "schedule_frac": sched_demag / (demag_ms * 1e-3) / 1e9 / peak,
                               "wasted_traffic_ratio": sched_demag / rows["compulsory"]}}
    # the whole RK4 step against the same peak: the bytes this schedule's
    # kernels move per step (algorithmic bytes per launch x launches per step)
    # and the compulsory bytes of a step (per evaluation M read, H written and
    # the kernel octant read; per stage the LLG stage's bytes)
    prof_step = n_prof
    sched_bytes = sum(algo[k] * units[k] for k in kern if k in algo and kern[k][1]) / prof_step
    compulsory = 4 * rows["compulsory"] + 4 * llg_algorithmic_bytes(plan)
    three_pass = 4 * (rows["a2"] + rows["a3"] + rows["a4"]) + 4 * llg_algorithmic_bytes(plan)
    step_roofline = {"unit": "GB/s", "peak": peak, "ms_per_step": step_s * 1e3,
                     "schedule_bytes_per_step": sched_bytes, "schedule_GBps": sched_bytes / step_s / 1e9,
                     "schedule_frac": sched_bytes / step_s / 1e9 / peak,
                     "three_pass_bytes_per_step": three_pass, "three_pass_frac": three_pass / step_s / 1e9 / peak,
                     "compulsory_bytes_per_step": compulsory, "compulsory_GBps": compulsory / step_s / 1e9,
                     "compulsory_frac": compulsory / step_s / 1e9 / peak,
                     "wasted_traffic_ratio": sched_bytes / compulsory}
    kernels = {k: {"ms_per_launch": per_launch_ms[k], "launches": kern[k][1], "row": ROW_OF.get(k),
                   "per": "evaluation" if k in DEMAG_KERNELS else "launch",
                   "share": kern[k][0] / max(1e-12, sum(v[0] for v in kern.values())),
                   "algorithmic_GBps": (algo[k] / (per_launch_ms[k] * 1e-3) / 1e9) if (k in algo and per_launch_ms[k]) else None}
               for k in kern if kern[k][1]}
    kernels_window = {"steps": n_prof, "seconds": sum(v[0] for v in kern.values()) / 1e3}

    # ---- further field terms on the same film (interfacial DMI, cubic and
    #      second-order uniaxial anisotropy): one-cell-per-thread stage kernel
    terms_line = None
    if not args.no_extra:
        from paper_2008_02478_gb300.binding import FieldTerms
        plan.set_field_terms(FieldTerms(K2=1e4, Kc1=4.5e4, cubic_e1=(1.0, 0.0, 0.0), cubic_e2=(0.0, 1.0, 0.0),
                                        dmi="interfacial", D=3e-3))
        mt = m.clone()
        plan.llg_run_graph(mt, prm, DT, 3)
        t_terms = max_over_ranks(time_graph(torch, plan, mt, prm, args.steps))
        terms_line = {"terms": "interfacial DMI D=3e-3 J/m^2 (non-homogeneous Neumann boundaries), cubic "
                               "Kc1=4.5e4 J/m^3, uniaxial K2=1e4 J/m^3",
                      "cell_steps_per_s": world * ncell * args.steps / t_terms,
                      "ms_per_step": 1e3 * t_terms / args.steps}
        # stochastic thermal field at 300 K (Philox normals regenerated in each stage)
        plan.set_field_terms(FieldTerms(temperature=300.0, seed=7))
        mt = m.clone()
        plan.llg_run_graph(mt, prm, DT, 3)
        t_th = max_over_ranks(time_graph(torch, plan, mt, prm, args.steps))
        terms_line["thermal_300K"] = {"cell_steps_per_s": world * ncell * args.steps / t_th,
                                      "ms_per_step": 1e3 * t_th / args.steps}
        plan.set_field_terms(None)
        del mt

    # ---- e2e: pinned host state, H2D + one RK4 step + D2H per step ----------
    m_host = torch.tensor(m0, dtype=torch.float32).pin_memory()
    plan.llg_run_host(m_host, prm, DT, 1)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        plan.llg_run_host(m_host, prm, DT, 1)
    t_e2e = max_over_ranks(time.perf_counter() - t0)
    e2e_bytes = 3 * ncell * 4
    e2e = {"value": world * ncell * args.steps / t_e2e, "unit": UNIT, "h2d_bytes_per_step": e2e_bytes,
           "d2h_bytes_per_step": e2e_bytes}

    # ---- FP64 plan (same kernels templated on double) ----------------------
    fp64 = None
    mixed = None
    if not args.no_fp64:
        plan64 = Plan(nx, ny, nz, *CELL, fp64=True)
        m64 = torch.tensor(m0, dtype=torch.float64, device="cuda")
        k64 = max(3, args.steps // 4)
        for _ in range(3):
            plan64.llg_step(m64, prm, DT)
        t64 = max_over_ranks(time_steps(torch, plan64, m64, prm, k64))
        M64 = torch.tensor(MS * m0, dtype=torch.float64, device="cuda")
        H64 = torch.empty_like(M64)
        plan64.apply(M64, H64)
        td64 = max_over_ranks(time_demag(torch, plan64, M64, H64, 4 * k64))
        fp64 = {"cell_steps_per_s": world * ncell * k64 / t64, "demag_evals_per_s": world * 4 * k64 / td64,
                "steps": k64}
        plan64.close()
        del m64, M64

        # H_d of the film from the FP64 plan (within 1e-9 of the FP64 oracle in
        # the parity tests) is the reference for the FP32 and mixed-precision errors
        def rel_err(Hx):
            d = (Hx.double() - H64).norm() / H64.norm()
            return float(d)

        def max_err(Hx):
            return float((Hx.double() - H64).abs().max() / H64.abs().max())
        plan.apply(M, H)
        fp64["h_rel_l2_fp32_vs_fp64"] = rel_err(H)
        fp64["h_max_rel_fp32_vs_fp64"] = max_err(H)
        mixed = {}
        for tc in ("fp16", "bf16"):
            pt = Plan(nx, ny, nz, *CELL, tc=tc)
            pt.apply(M, H)
            err, merr = rel_err(H), max_err(H)
            for _ in range(3):
                pt.apply(M, H)
            td = max_over_ranks(time_demag(torch, pt, M, H, 4 * args.steps))
            mt = torch.tensor(m0, dtype=torch.float32, device="cuda")
            pt.llg_run_graph(mt, prm, DT, 3)
            ts = max_over_ranks(time_graph(torch, pt, mt, prm, args.steps))
            pt.profile(True)
            time_steps(torch, pt, mt, prm, max(4, args.steps // 4))
            kk, _ = pt.profile_read()
            zt = kk["z_conv"][0] / max(1, kk["z_conv"][1])
            z_roof = None
            if pt.schedule()[2] == 6:
                # the 16-bit z stage's own compulsory bytes: Y16 read and written, the FP16 kernel octant
                px_, py_, pz_ = pt.padded()
                nkx_ = px_ // 2 + 1
                zbytes = 2 * nkx_ * 3 * 2 * nz * py_ * 2 + nkx_ * (pz_ // 2 + 1) * 3 * (py_ // 2 + 8) * 4
                pk, pk_src = measured_peaks()
                z_roof = {"bytes_per_launch": zbytes, "GBps": zbytes / (zt * 1e-3) / 1e9,
                          "frac": zbytes / (zt * 1e-3) / 1e9 / pk, "peak": pk, "peak_source": pk_src}
            mixed[tc] = {"demag_evals_per_s": world * 4 * args.steps / td,
                         "z_stage_roofline": z_roof,
                         "cell_steps_per_s": world * ncell * args.steps / ts,
                         "ms_per_step": 1e3 * ts / args.steps,
                         "speedup_vs_fp32_step": (ncell * args.steps / ts) / (value / world),
                         "h_rel_l2_vs_fp64": err, "h_max_rel_vs_fp64": merr,
                         "z_stage_ms_per_launch": kk["z_conv"][0] / max(1, kk["z_conv"][1]),
                         "kernels_ms_per_launch": {k: v[0] / v[1] for k, v in kk.items() if v[1]},
                         "z_stage": {6: "tcgen05, spectrum between the y and z passes stored in " +
                                        ("FP16 (power-of-two scale from max |M|)" if tc == "fp16" else "BF16"),
                                     5: "tcgen05 (tensor memory), FP32 spectrum", 4: "mma.sync"}.get(pt.schedule()[2], "?")}
            pt.close()
            del mt
        del H64

    # ---- other workloads: multi-mesh stack, RKF45 film, gradient film ------
    extra = {}
    if not args.no_extra:
        extra = other_workloads(torch, args, world, max_over_ranks, rank)

    # ---- CPU baseline: the oracle on a bounded sample -----------------------
    cpu = None
    if rank == 0 and not args.no_cpu:
        import oracle
        oracle.build()
        allc = oracle.num_threads()
        blk = (256, 256, 32)
        rate, t, cores = oracle_rk4_rate(*blk, 3)
        oracle.set_threads(1)
        blk1 = (64, 64, 8)
        rate1, t1, _ = oracle_rk4_rate(*blk1, 2)
        oracle.set_threads(allc)
        demag_rates = oracle_demag_rates()
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "three RK4 steps (12 FFT demag evaluations) of the FP64 oracle on a %dx%dx%d block of "
                         "the same film (a quarter of its cells), %.1f s" % (blk + (t,)),
               "one_thread": {"value": rate1, "unit": UNIT, "sample": "two RK4 steps on a %dx%dx%d block, %.1f s"
                              % (blk1 + (t1,))},
               "demag_evals_per_s": demag_rates}
        # the film after 1000 RK4 steps, checked by one oracle evaluation of the full mesh
        acc = film_accuracy_check(torch, plan, prm, m0, 1000 if not args.short else 50, allc)
        cpu["demag_evals_per_s"]["512x512x32"] = {"threads_%d" % allc: 1.0 / acc["oracle_512x512x32_eval_s"]}
        extra["film_512x512x32_after_steps"] = acc

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_steps / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "cells": ncell, "parallelism": "replicas" if world > 1 else "1 GPU",
                           "l2": "inputs larger than L2 (m 100.7 MB, spectrum workspace 201.7 MB, kernel "
                                 "spectrum 208.4 MB per evaluation)",
                           "padded": plan.padded(), "yz_schedule": plan.schedule()},
                "sustained": sustained,
                "demag_evals_per_s": demag_rate, "ms_per_step_without_graph": 1e3 * t_calls / args.steps,
                "fp64": fp64, "workloads": dict(extra, field_terms_512x512x32=terms_line) if terms_line else extra,
                "mixed_precision": mixed, "roofline": roofline, "step_roofline": step_roofline,
                "kernels": kernels, "kernels_window": kernels_window,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks}
        print(json.dumps(line), flush=True)
    plan.close()
    ranks.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
