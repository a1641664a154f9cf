"""FP64 CPU oracle for the demagnetising field and the LLG step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline/reference legs
of ``bench.py`` may use it.  It shares no code with the CUDA library.

Paper: "Boris Computational Spintronics" (arXiv 2008.02478).
  * ``boris_oracle.c``  - Newell tensor (Table 1, Ref. [50]), far-field form,
    its sum over periodic images (multiple-images method, Section 4),
    direct-sum demag (Table 1) and convolution-theorem demag with 2x zero
    padding (Section 7), with its own mixed-radix FFT.
  * ``llg.py``          - effective field (Eq. 1 and Table 1), LLG right-hand
    side, RK4 / RKF45 steps (Section 2), energies, and the discrete adjoint of
    an RK4 step.
  * ``multilayer.py``   - the multi-mesh convolution sum (Eq. 4).
  * ``boris_oracle.c`` also holds the Oersted kernel (Table 1, its Ref. [63]
    not in the paper): H = J x g with g = -(1/(4 pi V)) grad of the two-box
    Coulomb integral, obtained as the antiderivative of Newell's N_kk along
    axis k, and the direct-sum Oersted field.
  * ``thermal.py``      - the stochastic thermal field (Philox4x32-10 counter
    generator, Box-Muller normals, Brown's fluctuation magnitude).
  * ``terms.py``        - further Table 1 field terms (second-order uniaxial
    and cubic anisotropy, bulk and interfacial DMI with their boundary
    conditions) and the surface exchange of Eq. 5.

The cross-layer tensor for cells of unequal thickness (``multilayer.py``) is
pinned by its equal-thickness reduction, reciprocity, source splitting and
Gauss-Legendre quadrature of the dipole kernel over the two boxes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "boris_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

#: far-field switch radius, in units of the largest cell dimension
RS_DEFAULT = 40.0


def build(force: bool = False) -> str:
    """Compile ``boris_oracle.c`` into ``liboracle.so`` beside it (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            d, i, vp = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            L.orc_newell_f.restype = d
            L.orc_newell_f.argtypes = [d, d, d]
            L.orc_newell_g.restype = d
            L.orc_newell_g.argtypes = [d, d, d]
            L.orc_newell_exact.argtypes = [d, d, d, d, d, d, vp]
            L.orc_newell_asymptotic.argtypes = [d, d, d, d, d, d, vp]
            L.orc_tensor_table.argtypes = [i, i, i, d, d, d, d, vp]
            L.orc_tensor_table_pbc.argtypes = [i, i, i, d, d, d, d, i, i, i, vp]
            L.orc_oersted_g.argtypes = [d, d, d, d, d, d, d, vp]
            L.orc_oersted_table.argtypes = [i, i, i, d, d, d, d, vp]
            L.orc_oersted_direct.argtypes = [i, i, i, vp, vp, vp]
            L.orc_demag_direct.argtypes = [i, i, i, vp, vp, vp]
            L.orc_demag_direct_at.argtypes = [i, i, i, vp, vp, i, vp, vp]
            L.orc_fft1d.argtypes = [vp, i, i]
            L.orc_fft3d.argtypes = [vp, i, i, i, i]
            L.orc_demag_plan.restype = vp
            L.orc_demag_plan.argtypes = [i, i, i, vp]
            L.orc_demag_plan_free.argtypes = [vp]
            L.orc_demag_plan_spectrum.argtypes = [vp, vp]
            L.orc_demag_plan_dims.argtypes = [vp, vp]
            L.orc_demag_fft.restype = i
            L.orc_demag_fft.argtypes = [vp, vp, vp]
            L.orc_num_threads.restype = i
            L.orc_set_threads.argtypes = [i]
            L.orc_newell_pair_exact.argtypes = [d, d, d, d, d, d, d, vp]
            L.orc_newell_pair_asymptotic.argtypes = [d, d, d, d, d, d, d, vp]
            L.orc_newell_pair.argtypes = [d, d, d, d, d, d, d, d, vp]
            L.orc_multilayer_direct_at.argtypes = [i, vp, vp, vp, vp, vp, d, d, d, vp, i, vp, vp]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on (timing runs)."""
    lib().orc_set_threads(int(n))


# --------------------------------------------------------------------------
# Newell tensor
# --------------------------------------------------------------------------
def newell_f(x, y, z) -> float:
    return lib().orc_newell_f(float(x), float(y), float(z))


def newell_g(x, y, z) -> float:
    return lib().orc_newell_g(float(x), float(y), float(z))


def newell_exact(X, Y, Z, dx, dy, dz) -> np.ndarray:
    """Exact cell-averaged tensor (xx, yy, zz, xy, xz, yz) at separation (X,Y,Z)."""
    out = np.zeros(6)
    lib().orc_newell_exact(float(X), float(Y), float(Z), float(dx), float(dy), float(dz), _p(out))
    return out


def newell_asymptotic(X, Y, Z, dx, dy, dz) -> np.ndarray:
    out = np.zeros(6)
    lib().orc_newell_asymptotic(float(X), float(Y), float(Z), float(dx), float(dy), float(dz), _p(out))
    return out


def tensor_table(nx, ny, nz, dx, dy, dz, rs: float = RS_DEFAULT) -> np.ndarray:
    """Tensor on the displacement octant, shape [6][nz][ny][nx]."""
    out = np.zeros((6, nz, ny, nx))
    lib().orc_tensor_table(nx, ny, nz, float(dx), float(dy), float(dz), float(rs), _p(out))
    return out


def tensor_table_pbc(nx, ny, nz, dx, dy, dz, images, rs: float = RS_DEFAULT) -> np.ndarray:
    """Tensor summed over the periodic images (multiple-images method; images =
    (kx, ky, kz) images on each side along x, y, z, 0 for a non-periodic axis),
    shape [6][nz][ny][nx]."""
    out = np.zeros((6, nz, ny, nx))
    kx, ky, kz = (int(v) for v in images)
    lib().orc_tensor_table_pbc(nx, ny, nz, float(dx), float(dy), float(dz), float(rs), kx, ky, kz, _p(out))
    return out


def oersted_g(X, Y, Z, dx, dy, dz, rs: float = RS_DEFAULT) -> np.ndarray:
    """Cell-averaged Oersted vector g at displacement (X, Y, Z) (target - source):
    the field of a uniform current density J in the source cell, averaged over
    the target cell, is J x g."""
    out = np.zeros(3)
    lib().orc_oersted_g(float(X), float(Y), float(Z), float(dx), float(dy), float(dz), float(rs), _p(out))
    return out


def oersted_table(nx, ny, nz, dx, dy, dz, rs: float = RS_DEFAULT) -> np.ndarray:
    out = np.zeros((3, nz, ny, nx))
    lib().orc_oersted_table(nx, ny, nz, float(dx), float(dy), float(dz), float(rs), _p(out))
    return out


def oersted_direct(J: np.ndarray, G: np.ndarray) -> np.ndarray:
    """H = sum_r J(r) x g(r0 - r) (A/m) for a current density J [3][nz][ny][nx] (A/m^2)."""
    J = np.ascontiguousarray(J, dtype=np.float64)
    _, nz, ny, nx = J.shape
    H = np.zeros_like(J)
    lib().orc_oersted_direct(nx, ny, nz, _p(np.ascontiguousarray(G)), _p(J), _p(H))
    return H


# --------------------------------------------------------------------------
# Demag
# --------------------------------------------------------------------------
def demag_direct(M: np.ndarray, T: np.ndarray) -> np.ndarray:
    """O(N^2) direct sum H = -sum N(r - r0) M(r); M is [3][nz][ny][nx] FP64."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    _, nz, ny, nx = M.shape
    H = np.zeros_like(M)
    lib().orc_demag_direct(nx, ny, nz, _p(np.ascontiguousarray(T)), _p(M), _p(H))
    return H


def demag_direct_at(M: np.ndarray, T: np.ndarray, cells) -> np.ndarray:
    """Direct sum at the flat cell indices ``cells``; returns [len(cells)][3]."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    _, nz, ny, nx = M.shape
    cells = np.ascontiguousarray(cells, dtype=np.int64)
    H = np.zeros((len(cells), 3))
    lib().orc_demag_direct_at(nx, ny, nz, _p(np.ascontiguousarray(T)), _p(M), len(cells), _p(cells), _p(H))
    return H


class DemagPlan:
    """Convolution-theorem demag with the padded-tensor spectrum precomputed."""

    def __init__(self, nx, ny, nz, dx, dy, dz, rs: float = RS_DEFAULT, table: np.ndarray | None = None):
        self.shape = (nx, ny, nz)
        self.cell = (dx, dy, dz)
        self.table = tensor_table(nx, ny, nz, dx, dy, dz, rs) if table is None else np.ascontiguousarray(table)
        self._h = lib().orc_demag_plan(nx, ny, nz, _p(self.table))
        if not self._h:
            raise MemoryError("oracle plan allocation failed")

    def padded_dims(self):
        d = np.zeros(3, dtype=np.int32)
        lib().orc_demag_plan_dims(self._h, _p(d))
        return tuple(int(v) for v in d)

    def spectrum(self) -> np.ndarray:
        """Complex kernel spectrum, shape [6][pz][py][px]."""
        px, py, pz = self.padded_dims()
        out = np.zeros((6, pz, py, px), dtype=np.complex128)
        lib().orc_demag_plan_spectrum(self._h, _p(out))
        return out

    def apply(self, M: np.ndarray) -> np.ndarray:
        M = np.ascontiguousarray(M, dtype=np.float64)
        assert M.shape == (3, self.shape[2], self.shape[1], self.shape[0])
        H = np.zeros_like(M)
        if lib().orc_demag_fft(self._h, _p(M), _p(H)) != 0:
            raise MemoryError("oracle demag allocation failed")
        return H

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_demag_plan_free(h)
            self._h = None


def fft1d(a: np.ndarray, sign: int = -1) -> np.ndarray:
    a = np.array(a, dtype=np.complex128)
    lib().orc_fft1d(_p(a), a.size, int(sign))
    return a


def fft3d(a: np.ndarray, sign: int = -1) -> np.ndarray:
    """In-place-style 3D transform of a [n2][n1][n0] complex array."""
    a = np.array(a, dtype=np.complex128, order="C")
    n2, n1, n0 = a.shape
    lib().orc_fft3d(_p(a), n0, n1, n2, int(sign))
    return a
