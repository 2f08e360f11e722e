"""Python front end of the FP64 oracle (test infrastructure only).

Loads ``idg_oracle.c`` compiled by :func:`build` (gcc, OpenMP, -ffp-contract=off)
and exposes each step of Algorithms 1 and 2 of the paper on numpy arrays.  Only
the tests, the smoke check and the CPU-baseline leg of the benchmark use this
module; the GPU library never imports it.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "idg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libidg_oracle.so")
_lib = None

D_FIELDS = 10
D_BL, D_SLOT, D_T0, D_NT, D_C0, D_NC, D_Q0, D_R0, D_LAYER, D_KP = range(10)


def build(force: bool = False) -> str:
    """Compile the oracle shared library in-tree; returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    i32, i64, f64 = ctypes.c_int, ctypes.c_long, ctypes.c_double
    lib.oracle_plan.restype = i64
    lib.oracle_plan.argtypes = [P, P, P, i32, i32, i32, i32, i32, i32, f64, f64, f64, i32,
                                P, i64, P, P, P]
    lib.oracle_subgrid_images.restype = None
    lib.oracle_subgrid_images.argtypes = [P, P, P, P, P, P, P, i32, i32, i32, i32, i32, f64, f64, i32,
                                          P, P, i64, P]
    lib.oracle_dft2.restype = None
    lib.oracle_dft2.argtypes = [P, i64, i32, i32]
    lib.oracle_add.restype = None
    lib.oracle_add.argtypes = [P, P, i64, P, i32, i32, P]
    lib.oracle_split.restype = None
    lib.oracle_split.argtypes = [P, P, i64, P, i32, i32, P]
    lib.oracle_degrid_images.restype = None
    lib.oracle_degrid_images.argtypes = [P, P, P, P, P, P, i32, i32, i32, i32, i32, f64, f64, i32,
                                         P, P, i64, P, P]
    _lib = lib
    return lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


@dataclasses.dataclass
class OraclePlan:
    desc: np.ndarray          # int32 [n_sub][10]
    n_dropped: int
    n_w: int
    k_min: int

    @property
    def n_sub(self):
        return self.desc.shape[0]


def plan(wl) -> OraclePlan:
    """Partition of the workload's visibilities into subgrids (Sect. 3.2)."""
    lib = _load()
    uvw = _c(wl.uvw_m, np.float64)
    fr = _c(wl.freqs_hz, np.float64)
    offs = _c(wl.aterm_offsets, np.int32)
    nd, nw, km = ctypes.c_long(), ctypes.c_int(), ctypes.c_int()
    args = (_ptr(uvw), _ptr(fr), _ptr(offs), wl.n_bl, wl.n_t, wl.n_chan, wl.n_slots,
            wl.subgrid_size, wl.grid_size, wl.cell_size, wl.w_step, float(wl.kernel_size), wl.max_timesteps)
    n = lib.oracle_plan(*args, None, 0, ctypes.byref(nd), ctypes.byref(nw), ctypes.byref(km))
    desc = np.zeros((n, D_FIELDS), dtype=np.int32)
    n2 = lib.oracle_plan(*args, _ptr(desc), n, ctypes.byref(nd), ctypes.byref(nw), ctypes.byref(km))
    assert n2 == n
    return OraclePlan(desc, int(nd.value), int(nw.value), int(km.value))


def _ids(p: OraclePlan, ids):
    if ids is None:
        return np.arange(p.n_sub, dtype=np.int32)
    return np.ascontiguousarray(ids, dtype=np.int32)


def _common(wl, vis=None, flags=None, aterms="wl", taper=None):
    A = wl.aterms if isinstance(aterms, str) else aterms
    return dict(
        uvw=_c(wl.uvw_m, np.float64), fr=_c(wl.freqs_hz, np.float64), bl=_c(wl.baselines, np.int32),
        vis=_c(wl.vis if vis is None else vis, np.complex64),
        flags=_c(wl.flags if flags is None else flags, np.uint8),
        aterms=_c(A, np.complex64), taper=_c(wl.taper if taper is None else taper, np.float32))


def subgrid_images(wl, p: OraclePlan, ids=None, vis=None, flags=None, aterms="wl", taper=None) -> np.ndarray:
    """Tapered, A-term corrected subgrid images [n][L][L][4] complex128 (Alg. 1 before the FFT)."""
    lib = _load()
    ids = _ids(p, ids)
    c = _common(wl, vis, flags, aterms, taper)
    L = wl.subgrid_size
    out = np.zeros((ids.shape[0], L, L, 4), dtype=np.complex128)
    lib.oracle_subgrid_images(_ptr(c["uvw"]), _ptr(c["fr"]), _ptr(c["bl"]), _ptr(c["vis"]), _ptr(c["flags"]),
                              _ptr(c["aterms"]), _ptr(c["taper"]), wl.n_t, wl.n_chan, wl.n_stations, L,
                              wl.grid_size, wl.cell_size, wl.w_step, p.k_min, _ptr(p.desc), _ptr(ids),
                              ids.shape[0], _ptr(out))
    return out


def dft2(sub: np.ndarray, sign: int) -> np.ndarray:
    """Centred 2D DFT with 1/L^2 of [n][L][L][4] subgrids; sign -1 to uv, +1 to image."""
    lib = _load()
    out = np.array(sub, dtype=np.complex128, order="C", copy=True)
    lib.oracle_dft2(_ptr(out), out.shape[0], out.shape[1], int(sign))
    return out


def add(wl, p: OraclePlan, sub: np.ndarray, ids=None, grid: Optional[np.ndarray] = None) -> np.ndarray:
    lib = _load()
    ids = _ids(p, ids)
    N = wl.grid_size
    if grid is None:
        grid = np.zeros((p.n_w, N, N, 4), dtype=np.complex128)
    sub = np.ascontiguousarray(sub, dtype=np.complex128)
    lib.oracle_add(_ptr(p.desc), _ptr(ids), ids.shape[0], _ptr(sub), wl.subgrid_size, N, _ptr(grid))
    return grid


def split(wl, p: OraclePlan, grid: np.ndarray, ids=None) -> np.ndarray:
    lib = _load()
    ids = _ids(p, ids)
    L = wl.subgrid_size
    g = np.ascontiguousarray(grid, dtype=np.complex128)
    out = np.zeros((ids.shape[0], L, L, 4), dtype=np.complex128)
    lib.oracle_split(_ptr(p.desc), _ptr(ids), ids.shape[0], _ptr(g), L, wl.grid_size, _ptr(out))
    return out


def degrid_images(wl, p: OraclePlan, img: np.ndarray, ids=None, flags=None, aterms="wl", taper=None,
                  out: Optional[np.ndarray] = None) -> np.ndarray:
    """Visibilities from image-domain subgrids (Alg. 2 after the IFFT); others stay 0."""
    lib = _load()
    ids = _ids(p, ids)
    c = _common(wl, None if wl.vis is not None else np.zeros(1, np.complex64), flags, aterms, taper)
    if out is None:
        out = np.zeros((wl.n_bl, wl.n_t, wl.n_chan, 4), dtype=np.complex128)
    img = np.ascontiguousarray(img, dtype=np.complex128)
    lib.oracle_degrid_images(_ptr(c["uvw"]), _ptr(c["fr"]), _ptr(c["bl"]), _ptr(c["flags"]), _ptr(c["aterms"]),
                             _ptr(c["taper"]), wl.n_t, wl.n_chan, wl.n_stations, wl.subgrid_size, wl.grid_size,
                             wl.cell_size, wl.w_step, p.k_min, _ptr(p.desc), _ptr(ids), ids.shape[0],
                             _ptr(img), _ptr(out))
    return out


def grid(wl, p: OraclePlan, vis=None, flags=None, aterms="wl", taper=None, ids=None) -> np.ndarray:
    """Algorithm 1 without the final full-grid FFT: the master uv grid [n_w][N][N][4]."""
    img = subgrid_images(wl, p, ids, vis, flags, aterms, taper)
    uv = dft2(img, -1)
    return add(wl, p, uv, ids)


def degrid(wl, p: OraclePlan, g: np.ndarray, flags=None, aterms="wl", taper=None, ids=None) -> np.ndarray:
    """Algorithm 2 without the initial full-image steps: visibilities [n_bl][n_t][n_chan][4]."""
    sub = split(wl, p, g, ids)
    img = dft2(sub, +1)
    return degrid_images(wl, p, img, ids, flags, aterms, taper)
