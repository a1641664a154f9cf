"""GPU parity of the multi-mesh demagnetising field (Eq. 4) and the batched
multi-mesh RK4 step against the FP64 oracle (tolerance 1e-5 relative L2)."""
import numpy as np
import pytest

from oracle import llg
from oracle import multilayer as ml
from paper_2008_02478_gb300 import inputs
from tests.gpu_util import assert_close, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


def stack_case(layers, hz, gaps, hxy, seed):
    st = ml.centred_stack(layers, hz, gaps, hxy)
    Ms = [8e5, 1.4e6, 4e5, 1e6, 6e5, 1.2e6]
    m = np.concatenate([inputs.random_unit(*l, seed=seed + i).reshape(-1) for i, l in enumerate(layers)])
    ms_cells = np.concatenate([np.full(l[0] * l[1] * l[2], Ms[i % len(Ms)]) for i, l in enumerate(layers)])
    M = m.reshape(-1).copy()
    o = 0
    for i, l in enumerate(layers):
        n = l[0] * l[1] * l[2]
        M[3 * o:3 * (o + n)] *= Ms[i % len(Ms)]
        o += n
    return st, m, M, ms_cells


def make_plan(st):
    from paper_2008_02478_gb300.binding import MultiPlan
    cells = [(st.hx, st.hy, h) for h in st.hz]
    origins = [(ox * st.hx, oy * st.hy, zb) for ox, oy, zb in zip(st.ox, st.oy, st.zb)]
    return MultiPlan(st.n, cells, origins)


CASES = [
    ([(8, 8, 2), (6, 4, 3), (8, 6, 1)], [2e-9, 3e-9, 1e-9], [1e-9, 2e-9]),
    ([(12, 10, 4), (6, 6, 1), (10, 4, 2), (4, 4, 3)], [2e-9, 5e-9, 3e-9, 4e-9], [10e-9, 2e-9, 5e-9]),
    ([(9, 7, 1)], [3e-9], []),
]


@pytest.mark.parametrize("layers,hz,gaps", CASES)
def test_multilayer_demag_matches_direct_sum(layers, hz, gaps):
    torch = torch_cuda()
    st, m, M, _ = stack_case(layers, hz, gaps, 4e-9, seed=5)
    ref = ml.direct(st, M)
    plan = make_plan(st)
    H = plan.apply(torch.tensor(M, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert_close(H, ref, 1e-5)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("layers,hz,gaps", CASES[:2])
def test_every_inter_plane_sum_kernel_matches_direct_sum(layers, hz, gaps, variant, monkeypatch):
    """Each variant of the inter-plane sum (one CTA per tile, staged rows, one
    persistent launch at one or two CTAs per SM) against Eq. 4's direct sum;
    the layers have unequal z sizes, so the spectra shared by (a, b) and
    (b, a) through a N_ab = b N_ba are exercised."""
    torch = torch_cuda()
    st, m, M, _ = stack_case(layers, hz, gaps, 4e-9, seed=6)
    ref = ml.direct(st, M)
    monkeypatch.setenv("BORIS_ML_MIX", str(variant))
    plan = make_plan(st)
    assert plan.schedule()[2] == variant
    H = plan.apply(torch.tensor(M, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert_close(H, ref, 1e-5)


# frames of at least 33 cells in y (py >= 64), the paired-column sum's range
WIDE = ([(34, 33, 1), (12, 34, 2), (20, 10, 2)], [2e-9, 3e-9, 4e-9], [1e-9, 3e-9])
_wide_ref = {}


def _wide_case():
    if "ref" not in _wide_ref:
        st, m, M, _ = stack_case(*WIDE, 4e-9, seed=11)
        _wide_ref.update(st=st, M=M, ref=ml.direct(st, M))
    return _wide_ref["st"], _wide_ref["M"], _wide_ref["ref"]


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_inter_plane_sum_kernels_on_a_wide_frame(variant, monkeypatch):
    """Every inter-plane sum variant on a 34 x 34 frame (py = 128: three
    32-column tiles of folded ky, the last holding only the Nyquist column)
    against Eq. 4's direct sum over all 2338 cells."""
    torch = torch_cuda()
    st, M, ref = _wide_case()
    monkeypatch.setenv("BORIS_ML_MIX", str(variant))
    plan = make_plan(st)
    assert plan.schedule()[2] == variant
    H = plan.apply(torch.tensor(M, dtype=torch.float32, device="cuda")).cpu().numpy()
    assert_close(H, ref, 1e-5)


def test_persistent_sum_with_four_targets_per_warp(monkeypatch):
    """27 planes (four targets per warp in the persistent sum at two CTAs per
    SM): twelve cells against Eq. 4's direct sum, and the whole field against
    the one-CTA-per-tile sum."""
    torch = torch_cuda()
    layers, hz, gaps = [(34, 34, 10), (20, 36, 8), (30, 20, 9)], [2e-9, 3e-9, 4e-9], [1e-9, 3e-9]
    st, m, M, _ = stack_case(layers, hz, gaps, 4e-9, seed=12)
    Mt = torch.tensor(M, dtype=torch.float32, device="cuda")
    monkeypatch.setenv("BORIS_ML_MIX", "3")
    plan = make_plan(st)
    assert plan.info()[0] == 27 and plan.schedule()[2] == 3
    H = plan.apply(Mt).cpu().numpy()
    monkeypatch.setenv("BORIS_ML_MIX", "0")
    H0 = make_plan(st).apply(Mt).cpu().numpy()
    assert_close(H, H0, 1e-5)
    cells = inputs.rng(13).integers(0, st.total(), 12)
    ref = ml.direct_at(st, M, cells)
    offs = np.cumsum([0] + st.counts)
    got = []
    for gi in cells:
        l = int(np.searchsorted(offs, gi, side="right") - 1)
        n = st.counts[l]
        got.append([H[3 * offs[l] + c * n + gi - offs[l]] for c in range(3)])
    assert_close(np.array(got), ref, 1e-5)


def test_reciprocal_spectra_halve_the_cross_layer_set():
    """Spectra are stored once per (min(a, b), max(a, b), |dz|): two layers of
    z sizes 2 and 3 nm, one plane each, need 3 spectra (a = b = 2, a = b = 3,
    and one shared by (2, 3) and (3, 2)), not 4."""
    torch_cuda()
    st, m, M, _ = stack_case([(8, 8, 1), (8, 8, 1)], [2e-9, 3e-9], [1e-9], 4e-9, seed=1)
    plan = make_plan(st)
    assert plan.info()[1] == 3


def test_six_layer_stack_sampled():
    """The six-layer stack (512x512x8 ... 200x200x3 cells, 4 nm in-plane,
    z cells 2-5 nm, gaps 1-10 nm, Ms 4e5-1.4e6): 12 target cells against the
    oracle's direct sum over all 2.87M source cells."""
    torch = torch_cuda()
    d = inputs.MULTILAYER
    st, m, M, _ = stack_case(d["layers"], d["hz"], d["gaps"], d["hxy"], seed=d["seed"])
    plan = make_plan(st)
    assert plan.info()[0] == 34
    H = plan.apply(torch.tensor(M, dtype=torch.float32, device="cuda")).cpu().numpy()
    # H is concatenated per layer SoA; gather the sampled cells
    cells = inputs.rng(9).integers(0, st.total(), 12)
    ref = ml.direct_at(st, M, cells)
    got = []
    offs = np.cumsum([0] + st.counts)
    for g in cells:
        l = int(np.searchsorted(offs, g, side="right") - 1)
        n = st.counts[l]
        loc = g - offs[l]
        base = 3 * offs[l]
        got.append([H[base + c * n + loc] for c in range(3)])
    got = np.array(got)
    assert_close(got, ref, 1e-5)


def test_multilayer_rk4_matches_oracle():
    torch = torch_cuda()
    from paper_2008_02478_gb300.binding import LLGParams
    layers, hz, gaps = [(8, 6, 2), (6, 6, 1), (8, 4, 3)], [2e-9, 3e-9, 1e-9], [1e-9, 2e-9]
    st, m, M, ms_cells = stack_case(layers, hz, gaps, 3e-9, seed=7)
    plan = make_plan(st)
    A, alpha, Hext, dt = 1.3e-11, 0.02, (1e4, 0.0, 2e4), 1e-13
    # oracle: per-layer exchange with Neumann ends, demag by the multilayer direct sum
    def field(mm):
        Mc = mm.copy()
        o = 0
        for i, l in enumerate(layers):
            n = l[0] * l[1] * l[2]
            Mc[3 * o:3 * (o + n)] *= ms_cells[o]
            o += n
        Hd = ml.direct(st, Mc)
        H = Hd.copy()
        o = 0
        for i, l in enumerate(layers):
            n = l[0] * l[1] * l[2]
            ml_m = mm[3 * o:3 * (o + n)].reshape(3, l[2], l[1], l[0])
            prm = llg.Params(cell=(st.hx, st.hy, hz[i]), Ms=ms_cells[o], A=A)
            H[3 * o:3 * (o + n)] += llg.exchange_field(ml_m, prm, np.full(l[::-1], ms_cells[o])).reshape(-1)
            H[3 * o:3 * (o + n)] += np.repeat(np.array(Hext), n)
            o += n
        return H

    def rhs(mm):
        H = field(mm)
        out = np.zeros_like(mm)
        o = 0
        for l in layers:
            n = l[0] * l[1] * l[2]
            mv = mm[3 * o:3 * (o + n)].reshape(3, n)
            hv = H[3 * o:3 * (o + n)].reshape(3, n)
            out[3 * o:3 * (o + n)] = llg.llg_rhs(mv, hv, llg.Params(cell=(1, 1, 1), alpha=alpha)).reshape(-1)
            o += n
        return out

    ref = m.copy()
    for _ in range(3):
        k1 = rhs(ref)
        k2 = rhs(ref + 0.5 * dt * k1)
        k3 = rhs(ref + 0.5 * dt * k2)
        k4 = rhs(ref + dt * k3)
        v = ref + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        o = 0
        for l in layers:
            n = l[0] * l[1] * l[2]
            vv = v[3 * o:3 * (o + n)].reshape(3, n)
            v[3 * o:3 * (o + n)] = (vv / np.linalg.norm(vv, axis=0)).reshape(-1)
            o += n
        ref = v
    mg = torch.tensor(m, dtype=torch.float32, device="cuda")
    prm = LLGParams(A=A, alpha=alpha, Hext=Hext, Ms_map=torch.tensor(ms_cells, dtype=torch.float32, device="cuda"))
    for _ in range(3):
        plan.llg_step(mg, prm, dt)
    assert_close(mg.cpu().numpy(), ref, 1e-5)


def test_multilayer_rk4_with_surface_exchange_and_cubic_matches_oracle():
    """Eq. 5 surface exchange between consecutive layers (top plane of layer l
    with the bottom plane of layer l + 1 where they overlap in-plane, Delta =
    the receiving cell's z size) plus cubic anisotropy, against the oracle's
    RK4 with the same field built from oracle/terms.py."""
    torch = torch_cuda()
    from oracle import terms as T
    from paper_2008_02478_gb300.binding import FieldTerms, LLGParams
    layers, hz, gaps = [(8, 6, 2), (6, 6, 1), (8, 4, 3)], [2e-9, 3e-9, 1e-9], [1e-9, 2e-9]
    st, m, M, ms_cells = stack_case(layers, hz, gaps, 3e-9, seed=8)
    plan = make_plan(st)
    A, alpha, Hext, dt = 1.3e-11, 0.05, (1e4, 0.0, 2e4), 5e-14
    J1, J2, Kc1 = -1.2e-3, 2e-4, 3e4
    e1, e2 = (1.0, 0.0, 0.0), (0.0, 0.6, 0.8)
    offs = np.cumsum([0] + [a * b * c for a, b, c in layers])

    def views(v):
        return [v[3 * offs[i]:3 * offs[i + 1]].reshape(3, l[2], l[1], l[0]) for i, l in enumerate(layers)]

    def field(mm):
        Mc = mm.copy()
        for i in range(len(layers)):
            Mc[3 * offs[i]:3 * offs[i + 1]] *= ms_cells[offs[i]]
        H = ml.direct(st, Mc)
        Hv, mv = views(H), views(mm)
        for i, l in enumerate(layers):
            Ms = ms_cells[offs[i]]
            prm = llg.Params(cell=(st.hx, st.hy, hz[i]), Ms=Ms, A=A)
            Hv[i] += llg.exchange_field(mv[i], prm, np.full(l[::-1], Ms))
            Hv[i] += np.array(Hext).reshape(3, 1, 1, 1)
            Hv[i] += T.cubic_field(mv[i], e1, e2, Kc1, 0.0, Ms)
        for i in range(len(layers) - 1):
            lo, up = mv[i], mv[i + 1]
            for y in range(layers[i][1]):
                for x in range(layers[i][0]):
                    X, Y = x + st.ox[i] - st.ox[i + 1], y + st.oy[i] - st.oy[i + 1]
                    if 0 <= X < layers[i + 1][0] and 0 <= Y < layers[i + 1][1]:
                        a, b = lo[:, -1, y, x], up[:, 0, Y, X]
                        Hv[i][:, -1, y, x] += T.surface_exchange_field(a, b, J1, J2, ms_cells[offs[i]], hz[i])
                        Hv[i + 1][:, 0, Y, X] += T.surface_exchange_field(b, a, J1, J2, ms_cells[offs[i + 1]],
                                                                          hz[i + 1])
        return H

    def rhs(mm):
        H = field(mm)
        out = np.zeros_like(mm)
        for i in range(len(layers)):
            sl = slice(3 * offs[i], 3 * offs[i + 1])
            n = offs[i + 1] - offs[i]
            out[sl] = llg.llg_rhs(mm[sl].reshape(3, n), H[sl].reshape(3, n),
                                  llg.Params(cell=(1, 1, 1), alpha=alpha)).reshape(-1)
        return out

    ref = m.copy()
    for _ in range(2):
        k1 = rhs(ref)
        k2 = rhs(ref + 0.5 * dt * k1)
        k3 = rhs(ref + 0.5 * dt * k2)
        k4 = rhs(ref + dt * k3)
        v = ref + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        for i in range(len(layers)):
            sl = slice(3 * offs[i], 3 * offs[i + 1])
            n = offs[i + 1] - offs[i]
            vv = v[sl].reshape(3, n)
            v[sl] = (vv / np.linalg.norm(vv, axis=0)).reshape(-1)
        ref = v
    mg = torch.tensor(m, dtype=torch.float32, device="cuda")
    plan.set_field_terms(FieldTerms(J1=J1, J2=J2, Kc1=Kc1, cubic_e1=e1, cubic_e2=e2))
    prm = LLGParams(A=A, alpha=alpha, Hext=Hext, Ms_map=torch.tensor(ms_cells, dtype=torch.float32, device="cuda"))
    for _ in range(2):
        plan.llg_step(mg, prm, dt)
    assert np.abs(ref - m).max() > 1e-3
    assert_close(mg.cpu().numpy() - m, ref - m, 2e-4)
