"""Multi-mesh demagnetising field (Eq. 4): a stack of layers sharing the
in-plane cell (hx, hy), each with its own z cell size, in-plane offset and z
position.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The inter-mesh
tensor N(r, h_k, h_i) (Eq. 4; its formulas are in Ref. [23], not in the paper)
is the cell-averaged dipolar tensor between a target cell of z size a and a
source cell of z size b: Newell's construction with the per-axis double
integral over the two boxes, which along z becomes the four-point stencil
F(z + (a+b)/2) - F(z + (a-b)/2) - F(z - (a-b)/2) + F(z - (a+b)/2), normalised by
the target volume; it reduces to Newell's tensor for a = b.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import RS_DEFAULT, _p, lib


def pair_exact(X, Y, Z, hx, hy, a, b) -> np.ndarray:
    out = np.zeros(6)
    lib().orc_newell_pair_exact(float(X), float(Y), float(Z), float(hx), float(hy), float(a), float(b), _p(out))
    return out


def pair_asymptotic(X, Y, Z, hx, hy, a, b) -> np.ndarray:
    out = np.zeros(6)
    lib().orc_newell_pair_asymptotic(float(X), float(Y), float(Z), float(hx), float(hy), float(a), float(b), _p(out))
    return out


def pair(X, Y, Z, hx, hy, a, b, rs=RS_DEFAULT) -> np.ndarray:
    out = np.zeros(6)
    lib().orc_newell_pair(float(X), float(Y), float(Z), float(hx), float(hy), float(a), float(b), float(rs), _p(out))
    return out


@dataclass
class Stack:
    """Layers: (nx, ny, nz) cells, z size hz, in-plane offsets (cells), bottom z."""
    n: list
    hz: list
    ox: list
    oy: list
    zb: list
    hx: float
    hy: float

    @property
    def counts(self):
        return [nx * ny * nz for nx, ny, nz in self.n]

    def total(self):
        return sum(self.counts)


def centred_stack(layers, hz, gaps, hx, hy=None) -> Stack:
    """Layers laterally centred on the largest one, stacked bottom-up with the
    given gaps between consecutive layers."""
    hy = hx if hy is None else hy
    NX = max(l[0] for l in layers)
    NY = max(l[1] for l in layers)
    ox = [(NX - l[0]) // 2 for l in layers]
    oy = [(NY - l[1]) // 2 for l in layers]
    zb, z = [], 0.0
    for i, l in enumerate(layers):
        zb.append(z)
        z += l[2] * hz[i] + (gaps[i] if i < len(gaps) else 0.0)
    return Stack(list(layers), list(hz), ox, oy, zb, hx, hy)


def direct_at(stack: Stack, M: np.ndarray, cells, rs=RS_DEFAULT) -> np.ndarray:
    """Eq. 4 summed directly at the listed cells of the concatenated fields
    (each layer SoA [3][nz][ny][nx]); returns [len(cells)][3]."""
    M = np.ascontiguousarray(M, dtype=np.float64).reshape(-1)
    assert M.size == 3 * stack.total()
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    nl = len(stack.n)
    nxyz = np.ascontiguousarray(np.array(stack.n, dtype=np.int32).reshape(-1))
    hz = np.ascontiguousarray(np.array(stack.hz, dtype=np.float64))
    ox = np.ascontiguousarray(np.array(stack.ox, dtype=np.int32))
    oy = np.ascontiguousarray(np.array(stack.oy, dtype=np.int32))
    zb = np.ascontiguousarray(np.array(stack.zb, dtype=np.float64))
    H = np.zeros((len(cells), 3))
    lib().orc_multilayer_direct_at(nl, _p(nxyz), _p(hz), _p(ox), _p(oy), _p(zb), float(stack.hx), float(stack.hy),
                                   float(rs), _p(M), len(cells), _p(cells), _p(H))
    return H


def direct(stack: Stack, M: np.ndarray, rs=RS_DEFAULT) -> np.ndarray:
    """Eq. 4 at every cell; returns the concatenated SoA field."""
    H = direct_at(stack, M, np.arange(stack.total()), rs)
    out, o = [], 0
    for cnt in stack.counts:
        out.append(H[o:o + cnt].T.reshape(-1))
        o += cnt
    return np.concatenate(out)
