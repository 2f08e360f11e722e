"""Thin Python binding of the C ABI in ``include/idg.h`` (ctypes).

Argument marshalling only: every step of gridding and degridding runs in the
library's CUDA kernels.  Device buffers are torch CUDA tensors (torch supplies
device memory and streams); host buffers are numpy arrays.  The functions
carry the C names without the ``idg_`` prefix.  Importing works without a GPU;
calling anything that needs the library raises if it has not been built.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libidg_gb300.so")

IDG_OK = 0
STATUS_NAMES = {0: "IDG_OK", 1: "IDG_ERR_INVALID_ARG", 2: "IDG_ERR_NO_MEMORY", 3: "IDG_ERR_CUDA",
                4: "IDG_ERR_TIMEOUT", 5: "IDG_ERR_DEVICE_CHECK", 6: "IDG_ERR_UNSUPPORTED"}
DESC_FIELDS = 10
PHASOR_SINCOS, PHASOR_RECURRENCE = 0, 1
FFT_FP32, FFT_TC_SPLIT = 0, 1
ADDER_ATOMIC, ADDER_COMPENSATED, ADDER_SORTED = 0, 1, 2

# Every symbol the header declares (checked by the CPU test-suite).
EXPORTED = [
    "idg_plan_options_default", "idg_plan_create", "idg_plan_info", "idg_plan_export", "idg_plan_destroy",
    "idg_grid", "idg_degrid", "idg_grid_host", "idg_degrid_host",
    "idg_grid_subgrids", "idg_fft_subgrids", "idg_add_subgrids", "idg_split_subgrids", "idg_degrid_subgrids",
    "idg_status_string", "idg_last_error", "idg_supported_subgrid_sizes",
    "idg_profile_enable", "idg_profile_read", "idg_grid_no_alloc",
    "idg_kernel_variant_count", "idg_kernel_variant_name", "idg_set_kernel_variant", "idg_get_kernel_variant",
    "idg_autotune", "idg_batch_create", "idg_batch_grid", "idg_batch_degrid", "idg_batch_info",
    "idg_batch_destroy", "idg_device_errors", "idg_taper_window", "idg_taper_aliasing",
    "idg_image_from_grid", "idg_grid_from_image", "idg_plan_set_kernel_variant", "idg_plan_get_kernel_variant",
    "idg_grid_range", "idg_degrid_range", "idg_selftest_wait_timeout", "idg_aterm_gradient",
    "idg_classical_grid", "idg_batch_autotune", "idg_grid_degrid_host",
]
BATCH_GRAPH = 1
KERNELS = ["gridder", "fft", "adder", "splitter", "degridder", "batch_grid", "batch_degrid", "calib_residual",
           "calib_gradient", "classical_kernels", "classical_grid"]


class IDGError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class PlanOptions(ctypes.Structure):
    _fields_ = [("kernel_size", ctypes.c_double), ("max_timesteps_per_subgrid", ctypes.c_int),
                ("precision_mode", ctypes.c_int), ("fft_mode", ctypes.c_int), ("adder_mode", ctypes.c_int),
                ("n_host_threads", ctypes.c_int)]


class PlanStats(ctypes.Structure):
    _fields_ = [("n_subgrids", ctypes.c_int64), ("n_vis_planned", ctypes.c_int64),
                ("n_vis_dropped", ctypes.c_int64), ("max_kp", ctypes.c_int64),
                ("n_w_layers", ctypes.c_int32), ("w_layer_min", ctypes.c_int32),
                ("subgrid_size", ctypes.c_int32), ("grid_size", ctypes.c_int32),
                ("n_bl", ctypes.c_int32), ("n_t", ctypes.c_int32), ("n_chan", ctypes.c_int32),
                ("n_stations", ctypes.c_int32), ("n_slots", ctypes.c_int32), ("device", ctypes.c_int32),
                ("separable", ctypes.c_int32), ("sep_phase", ctypes.c_double),
                ("n_sep_subgrids", ctypes.c_int64), ("n_vis_sep", ctypes.c_int64),
                ("n_split_subgrids", ctypes.c_int64), ("n_pieces", ctypes.c_int64), ("n_vis_split", ctypes.c_int64)]


_lib = None


def load(path: str = LIB_PATH):
    """Load the library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"the CUDA library {path} is not built: run paper_1909_07226_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "idg_plan_options_default": (None, [P]),
        "idg_plan_create": (I32, [P, P, P, P, I32, I32, I32, I32, I32, I32, I32, D, D, P, P]),
        "idg_plan_info": (I32, [P, P]),
        "idg_plan_export": (I32, [P, P, I64]),
        "idg_plan_destroy": (None, [P]),
        "idg_grid": (I32, [P, P, P, P, P, P, P]),
        "idg_degrid": (I32, [P, P, P, P, P, P, P]),
        "idg_grid_host": (I32, [P, P, P, P, P, P, P]),
        "idg_grid_range": (I32, [P, I64, I64, P, P, P, P, P, P]),
        "idg_aterm_gradient": (I32, [P, P, P, P, P, P, P, P, P, P]),
        "idg_classical_grid": (I32, [P, I32, I32, D, P, P, P, P, P, P]),
        "idg_degrid_range": (I32, [P, I64, I64, P, P, P, P, P, P]),
        "idg_degrid_host": (I32, [P, P, P, P, P, P, P]),
        "idg_grid_degrid_host": (I32, [P, P, P, P, P, P, P, P, P]),
        "idg_grid_subgrids": (I32, [P, I64, I64, P, P, P, P, P, P]),
        "idg_fft_subgrids": (I32, [P, I64, I32, P, P]),
        "idg_add_subgrids": (I32, [P, I64, I64, P, P, P]),
        "idg_split_subgrids": (I32, [P, I64, I64, P, P, P]),
        "idg_degrid_subgrids": (I32, [P, I64, I64, P, P, P, P, P, P]),
        "idg_status_string": (ctypes.c_char_p, [I32]),
        "idg_last_error": (ctypes.c_char_p, []),
        "idg_supported_subgrid_sizes": (I32, [P, I32]),
        "idg_profile_enable": (None, [I32]),
        "idg_profile_read": (I32, [P, P, P, I32]),
        "idg_grid_no_alloc": (I32, [P, P, P, P, P, P, P]),
        "idg_kernel_variant_count": (I32, [I32, I32]),
        "idg_kernel_variant_name": (ctypes.c_char_p, [I32, I32, I32]),
        "idg_set_kernel_variant": (I32, [I32, I32, I32]),
        "idg_get_kernel_variant": (I32, [I32, I32]),
        "idg_plan_set_kernel_variant": (I32, [P, I32, I32]),
        "idg_plan_get_kernel_variant": (I32, [P, I32]),
        "idg_autotune": (I32, [P, P, P, P, P, P, I64, P, P, I32, P]),
        "idg_batch_create": (I32, [P, P, I32, I32, P]),
        "idg_batch_grid": (I32, [P, P]),
        "idg_batch_degrid": (I32, [P, P]),
        "idg_batch_info": (I32, [P, P, P, P]),
        "idg_batch_autotune": (I32, [P, P, I32, P]),
        "idg_batch_destroy": (None, [P]),
        "idg_device_errors": (I32, [P]),
        "idg_selftest_wait_timeout": (I32, [I64, P]),
        "idg_taper_window": (I32, [I32, D, I32, P, P]),
        "idg_taper_aliasing": (I32, [I32, D, P, P]),
        "idg_image_from_grid": (I32, [P, P, P, P, P]),
        "idg_grid_from_image": (I32, [P, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != IDG_OK:
        msg = load().idg_last_error()
        raise IDGError(status, where, msg.decode() if msg else "")


def plan_options_default() -> PlanOptions:
    o = PlanOptions()
    load().idg_plan_options_default(ctypes.byref(o))
    return o


def supported_subgrid_sizes():
    lib = load()
    buf = (ctypes.c_int32 * 16)()
    n = lib.idg_supported_subgrid_sizes(buf, 16)
    return [int(buf[i]) for i in range(min(n, 16))]


TAPER_PSWF, TAPER_IDG_OPTIMAL = 0, 1


def taper_window(subgrid_size: int, beta: float, kind: int = TAPER_IDG_OPTIMAL):
    """1D anti-aliasing window a[L] (a[L/2] = 1) and its aliasing level eps
    (idg_taper_window, host FP64): kind TAPER_PSWF is psi_0(pi beta / 2, .) with
    eps = sqrt(1 - lambda_0) (Sect. 4.1); TAPER_IDG_OPTIMAL is the optimal window of
    image domain gridding with eps = sqrt(smallest eigenvalue of Rbar) (Sect. 4.3)."""
    a = np.zeros(subgrid_size, dtype=np.float64)
    eps = ctypes.c_double(0.0)
    _check(load().idg_taper_window(int(subgrid_size), float(beta), int(kind), a.ctypes.data, ctypes.byref(eps)),
           "idg_taper_window")
    return a, eps.value


def taper_aliasing(subgrid_size: int, beta: float, a) -> float:
    """Side-lobe level of window a[L] in image domain gridding (idg_taper_aliasing)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != (subgrid_size,):
        raise ValueError(f"a must have shape ({subgrid_size},)")
    eps = ctypes.c_double(0.0)
    _check(load().idg_taper_aliasing(int(subgrid_size), float(beta), a.ctypes.data, ctypes.byref(eps)),
           "idg_taper_aliasing")
    return eps.value


def _window_ptr(window, L):
    if window is None:
        return None, None
    w = np.ascontiguousarray(window, dtype=np.float64)
    if w.shape != (L,):
        raise ValueError(f"the window must have shape ({L},)")
    return w, w.ctypes.data


def image_from_grid(plan: Plan, grid, window, image_out, stream=None):
    """idg_image_from_grid: grid [n_w][N][N][4] -> image [N][N][4] (CUDA complex64 tensors);
    window: the taper's 1D window a[L] (numpy, host) or None."""
    import torch
    sh = _shapes(plan)
    N = plan.stats.grid_size
    w, wp = _window_ptr(window, plan.stats.subgrid_size)
    _check(load().idg_image_from_grid(plan.handle, _dptr(grid, "grid", torch.complex64, sh["grid"]), wp,
                                      _dptr(image_out, "image", torch.complex64, (N, N, 4)), _stream(stream)),
           "idg_image_from_grid")


def grid_from_image(plan: Plan, image, window, grid_out, stream=None):
    """idg_grid_from_image: image [N][N][4] -> grid [n_w][N][N][4], the adjoint."""
    import torch
    sh = _shapes(plan)
    N = plan.stats.grid_size
    w, wp = _window_ptr(window, plan.stats.subgrid_size)
    _check(load().idg_grid_from_image(plan.handle, _dptr(image, "image", torch.complex64, (N, N, 4)), wp,
                                      _dptr(grid_out, "grid", torch.complex64, sh["grid"]), _stream(stream)),
           "idg_grid_from_image")


def profile_enable(on: bool = True):
    load().idg_profile_enable(1 if on else 0)


def profile_read(reset: bool = True) -> dict:
    """Per-kernel {launches, ms, work} since the last reset (see idg_profile_read)."""
    n = len(KERNELS)
    la = (ctypes.c_int64 * n)()
    ms = (ctypes.c_double * n)()
    wk = (ctypes.c_double * n)()
    _check(load().idg_profile_read(la, ms, wk, 1 if reset else 0), "idg_profile_read")
    return {k: dict(launches=int(la[i]), ms=float(ms[i]), work=float(wk[i])) for i, k in enumerate(KERNELS)}


# ---------------------------------------------------------------------------
# kernel variants and the autotuner

KERNEL_ID = {k: i for i, k in enumerate(KERNELS)}


def kernel_variants(kernel: str, L: int):
    lib = load()
    k = KERNEL_ID[kernel]
    n = lib.idg_kernel_variant_count(k, L)
    return [lib.idg_kernel_variant_name(k, L, v).decode() for v in range(n)]


def set_kernel_variant(kernel: str, L: int, variant: int):
    _check(load().idg_set_kernel_variant(KERNEL_ID[kernel], L, variant), "idg_set_kernel_variant")


def get_kernel_variant(kernel: str, L: int) -> int:
    return int(load().idg_get_kernel_variant(KERNEL_ID[kernel], L))


def plan_set_kernel_variant(plan, kernel: str, variant: int):
    """The plan's own kernel choice (-1: follow the process-wide choice for its L)."""
    _check(load().idg_plan_set_kernel_variant(plan.handle, KERNEL_ID[kernel], int(variant)),
           "idg_plan_set_kernel_variant")


def plan_get_kernel_variant(plan, kernel: str) -> int:
    """The variant the plan's calls use for `kernel`."""
    return int(load().idg_plan_get_kernel_variant(plan.handle, KERNEL_ID[kernel]))


def device_errors(stream=None):
    """idg_device_errors: synchronise the stream and raise IDGError if a bounded
    device wait (tensor-core gridder) gave up since the last call."""
    _check(load().idg_device_errors(_stream(stream)), "idg_device_errors")


def selftest_wait_timeout(max_polls: int = 4096, stream=None):
    """idg_selftest_wait_timeout: enqueue a kernel whose bounded wait runs out on purpose."""
    _check(load().idg_selftest_wait_timeout(int(max_polls), _stream(stream)), "idg_selftest_wait_timeout")


def autotune(plan, vis, flags, aterms, taper, vis_scratch=None, max_subgrids: int = 4096, stream=None) -> dict:
    """idg_autotune: time every gridder (and degridder) variant on a sample of the
    plan's subgrids and select the fastest for this plan.  Returns the timings."""
    import torch
    L = plan.stats.subgrid_size
    sh = _shapes(plan)
    cap = 32
    gms = (ctypes.c_double * cap)(*([-1.0] * cap))
    dms = (ctypes.c_double * cap)(*([-1.0] * cap))
    _check(load().idg_autotune(plan.handle, _dptr(vis, "vis", torch.complex64, sh["vis"]),
                               _dptr(flags, "flags", torch.uint8, sh["flags"], True),
                               _dptr(aterms, "aterms", torch.complex64, sh["aterms"], True),
                               _dptr(taper, "taper", torch.float32, sh["taper"], True),
                               _dptr(vis_scratch, "vis_scratch", torch.complex64, sh["vis"], True),
                               int(max_subgrids), gms, dms, cap, _stream(stream)), "idg_autotune")
    g_names, d_names = kernel_variants("gridder", L), kernel_variants("degridder", L)
    return {"L": L,
            "gridder": {"ms": {n: gms[i] for i, n in enumerate(g_names)},
                        "chosen": plan_get_kernel_variant(plan, "gridder")},
            "degridder": {"ms": {n: dms[i] for i, n in enumerate(d_names) if dms[i] >= 0},
                          "chosen": plan_get_kernel_variant(plan, "degridder")}}


def _device_key() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def save_tuning(path: str):
    """Persist the current per-L variant choices for this GPU model (JSON)."""
    import json
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    entry = {}
    for L in supported_subgrid_sizes():
        entry[str(L)] = {"gridder": get_kernel_variant("gridder", L), "degridder": get_kernel_variant("degridder", L)}
    data[_device_key()] = entry
    with open(path, "w") as f:
        json.dump(data, f, indent=1)


def load_tuning(path: str) -> bool:
    """Restore choices saved by save_tuning for this GPU model; False if none."""
    import json
    if not os.path.exists(path):
        return False
    with open(path) as f:
        data = json.load(f)
    entry = data.get(_device_key())
    if not entry:
        return False
    for L, ch in entry.items():
        for k, v in ch.items():
            if v < len(kernel_variants(k, int(L))):
                set_kernel_variant(k, int(L), int(v))
    return True


@dataclasses.dataclass
class Plan:
    handle: ctypes.c_void_p
    stats: PlanStats

    @property
    def n_subgrids(self):
        return int(self.stats.n_subgrids)

    @property
    def n_w_layers(self):
        return int(self.stats.n_w_layers)

    def export(self) -> np.ndarray:
        desc = np.zeros((self.n_subgrids, DESC_FIELDS), dtype=np.int32)
        _check(load().idg_plan_export(self.handle, desc.ctypes.data_as(ctypes.c_void_p), self.n_subgrids),
               "idg_plan_export")
        return desc

    def destroy(self):
        if self.handle:
            load().idg_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def _np(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def plan_create(uvw_m, freqs_hz, baselines, aterm_offsets, n_stations: int, subgrid_size: int, grid_size: int,
                cell_size: float, w_step: float = 0.0, options: Optional[PlanOptions] = None, **opt) -> Plan:
    """idg_plan_create from host numpy arrays; keyword options override fields of `options`."""
    lib = load()
    uvw = _np(uvw_m, np.float64)
    fr = _np(freqs_hz, np.float64)
    bl = _np(baselines, np.int32)
    offs = _np(aterm_offsets, np.int32)
    o = options if options is not None else plan_options_default()
    for k, v in opt.items():
        setattr(o, k, v)
    h = ctypes.c_void_p()
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(lib.idg_plan_create(vp(uvw), vp(fr), vp(bl), vp(offs), uvw.shape[0], uvw.shape[1], fr.shape[0],
                               int(n_stations), offs.shape[0] - 1, int(subgrid_size), int(grid_size),
                               float(cell_size), float(w_step), ctypes.byref(o), ctypes.byref(h)),
           "idg_plan_create")
    st = PlanStats()
    _check(lib.idg_plan_info(h, ctypes.byref(st)), "idg_plan_info")
    return Plan(h, st)


def plan_from_workload(wl, **opt) -> Plan:
    return plan_create(wl.uvw_m, wl.freqs_hz, wl.baselines, wl.aterm_offsets, wl.n_stations, wl.subgrid_size,
                       wl.grid_size, wl.cell_size, wl.w_step, kernel_size=float(wl.kernel_size),
                       max_timesteps_per_subgrid=int(wl.max_timesteps), **opt)


# ---------------------------------------------------------------------------
# device-buffer calls (torch CUDA tensors)

def _dptr(t, name, dtype=None, shape=None, optional=False):
    if t is None:
        if optional:
            return None
        raise ValueError(f"{name} is required")
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _shapes(plan: Plan):
    s = plan.stats
    L, N = s.subgrid_size, s.grid_size
    return dict(vis=(s.n_bl, s.n_t, s.n_chan, 4), flags=(s.n_bl, s.n_t, s.n_chan),
                aterms=(s.n_slots, s.n_stations, L, L, 4), taper=(L, L), grid=(s.n_w_layers, N, N, 4))


def grid(plan: Plan, vis, flags, aterms, taper, grid_out, stream=None):
    import torch
    sh = _shapes(plan)
    _check(load().idg_grid(plan.handle, _dptr(vis, "vis", torch.complex64, sh["vis"]),
                           _dptr(flags, "flags", torch.uint8, sh["flags"], True),
                           _dptr(aterms, "aterms", torch.complex64, sh["aterms"], True),
                           _dptr(taper, "taper", torch.float32, sh["taper"], True),
                           _dptr(grid_out, "grid", torch.complex64, sh["grid"]), _stream(stream)), "idg_grid")


def degrid(plan: Plan, grid_in, flags, aterms, taper, vis_out, stream=None):
    import torch
    sh = _shapes(plan)
    _check(load().idg_degrid(plan.handle, _dptr(grid_in, "grid", torch.complex64, sh["grid"]),
                             _dptr(flags, "flags", torch.uint8, sh["flags"], True),
                             _dptr(aterms, "aterms", torch.complex64, sh["aterms"], True),
                             _dptr(taper, "taper", torch.float32, sh["taper"], True),
                             _dptr(vis_out, "vis_out", torch.complex64, sh["vis"]), _stream(stream)), "idg_degrid")


def aterm_gradient(plan: Plan, grid_in, vis, flags, aterms, taper, residual_out, gradient, cost=None, stream=None):
    """idg_aterm_gradient: residuals (overwritten), the A-term gradient (added into
    `gradient`, shaped like the A-terms) and, if `cost` (a one-element float64 CUDA
    tensor) is given, the cost added into it."""
    import torch
    sh = _shapes(plan)
    _check(load().idg_aterm_gradient(plan.handle, _dptr(grid_in, "grid", torch.complex64, sh["grid"]),
                                     _dptr(vis, "vis", torch.complex64, sh["vis"]),
                                     _dptr(flags, "flags", torch.uint8, sh["flags"], True),
                                     _dptr(aterms, "aterms", torch.complex64, sh["aterms"], True),
                                     _dptr(taper, "taper", torch.float32, sh["taper"], True),
                                     _dptr(residual_out, "residual", torch.complex64, sh["vis"]),
                                     _dptr(gradient, "gradient", torch.complex64, sh["aterms"]),
                                     _dptr(cost, "cost", torch.float64, (1,), True), _stream(stream)),
           "idg_aterm_gradient")


def classical_grid(plan: Plan, support: int, oversample: int, w_plane_step: float, vis, flags, aterms, taper,
                   grid_out, stream=None):
    """idg_classical_grid: classical gridding with oversampled A/W-projection kernels
    rebuilt per subgrid.  aterms: [n_slots][n_stations][M][M][4] on the kernel lattice
    (or None); taper: [M][M] (or None for the PSWF window of width M)."""
    import torch
    sh = _shapes(plan)
    M = int(support)
    _check(load().idg_classical_grid(plan.handle, M, int(oversample), float(w_plane_step),
                                     _dptr(vis, "vis", torch.complex64, sh["vis"]),
                                     _dptr(flags, "flags", torch.uint8, sh["flags"], True),
                                     _dptr(aterms, "aterms", torch.complex64, sh["aterms"][:2] + (M, M, 4), True),
                                     _dptr(taper, "taper", torch.float32, (M, M), True),
                                     _dptr(grid_out, "grid", torch.complex64, sh["grid"]), _stream(stream)),
           "idg_classical_grid")


def grid_range(plan: Plan, first: int, count: int, vis, flags, aterms, taper, grid_out, stream=None):
    """idg_grid_range: the subgrids [first, first + count) (plan order) added into grid_out."""
    import torch
    sh = _shapes(plan)
    _check(load().idg_grid_range(plan.handle, int(first), int(count), _dptr(vis, "vis", torch.complex64, sh["vis"]),
                                 _dptr(flags, "flags", torch.uint8, sh["flags"], True),
                                 _dptr(aterms, "aterms", torch.complex64, sh["aterms"], True),
                                 _dptr(taper, "taper", torch.float32, sh["taper"], True),
                                 _dptr(grid_out, "grid", torch.complex64, sh["grid"]), _stream(stream)),
           "idg_grid_range")


def degrid_range(plan: Plan, first: int, count: int, grid_in, flags, aterms, taper, vis_out, stream=None):
    """idg_degrid_range: the visibilities of subgrids [first, first + count) written to vis_out."""
    import torch
    sh = _shapes(plan)
    _check(load().idg_degrid_range(plan.handle, int(first), int(count),
                                   _dptr(grid_in, "grid", torch.complex64, sh["grid"]),
                                   _dptr(flags, "flags", torch.uint8, sh["flags"], True),
                                   _dptr(aterms, "aterms", torch.complex64, sh["aterms"], True),
                                   _dptr(taper, "taper", torch.float32, sh["taper"], True),
                                   _dptr(vis_out, "vis_out", torch.complex64, sh["vis"]), _stream(stream)),
           "idg_degrid_range")


def grid_no_alloc(plan: Plan, vis, flags, aterms, taper, grid_out, stream=None):
    """idg_grid without device allocation: the subgrid scratch is the library's
    built-in 64 MiB array (for callers that cannot allocate device memory)."""
    import torch
    sh = _shapes(plan)
    _check(load().idg_grid_no_alloc(plan.handle, _dptr(vis, "vis", torch.complex64, sh["vis"]),
                                    _dptr(flags, "flags", torch.uint8, sh["flags"], True),
                                    _dptr(aterms, "aterms", torch.complex64, sh["aterms"], True),
                                    _dptr(taper, "taper", torch.float32, sh["taper"], True),
                                    _dptr(grid_out, "grid", torch.complex64, sh["grid"]), _stream(stream)),
           "idg_grid_no_alloc")


def grid_subgrids(plan: Plan, first: int, count: int, vis, flags, aterms, taper, subgrids, stream=None):
    import torch
    sh = _shapes(plan)
    L = plan.stats.subgrid_size
    _check(load().idg_grid_subgrids(plan.handle, first, count, _dptr(vis, "vis", torch.complex64, sh["vis"]),
                                    _dptr(flags, "flags", torch.uint8, sh["flags"], True),
                                    _dptr(aterms, "aterms", torch.complex64, sh["aterms"], True),
                                    _dptr(taper, "taper", torch.float32, sh["taper"], True),
                                    _dptr(subgrids, "subgrids", torch.complex64, (count, L, L, 4)),
                                    _stream(stream)), "idg_grid_subgrids")


def fft_subgrids(plan: Plan, count: int, direction: int, subgrids, stream=None):
    import torch
    L = plan.stats.subgrid_size
    _check(load().idg_fft_subgrids(plan.handle, count, direction,
                                   _dptr(subgrids, "subgrids", torch.complex64, (count, L, L, 4)),
                                   _stream(stream)), "idg_fft_subgrids")


def add_subgrids(plan: Plan, first: int, count: int, subgrids, grid_out, stream=None):
    import torch
    L = plan.stats.subgrid_size
    _check(load().idg_add_subgrids(plan.handle, first, count,
                                   _dptr(subgrids, "subgrids", torch.complex64, (count, L, L, 4)),
                                   _dptr(grid_out, "grid", torch.complex64, _shapes(plan)["grid"]),
                                   _stream(stream)), "idg_add_subgrids")


def split_subgrids(plan: Plan, first: int, count: int, grid_in, subgrids, stream=None):
    import torch
    L = plan.stats.subgrid_size
    _check(load().idg_split_subgrids(plan.handle, first, count,
                                     _dptr(grid_in, "grid", torch.complex64, _shapes(plan)["grid"]),
                                     _dptr(subgrids, "subgrids", torch.complex64, (count, L, L, 4)),
                                     _stream(stream)), "idg_split_subgrids")


def degrid_subgrids(plan: Plan, first: int, count: int, subgrids, flags, aterms, taper, vis_out, stream=None):
    import torch
    sh = _shapes(plan)
    L = plan.stats.subgrid_size
    _check(load().idg_degrid_subgrids(plan.handle, first, count,
                                      _dptr(subgrids, "subgrids", torch.complex64, (count, L, L, 4)),
                                      _dptr(flags, "flags", torch.uint8, sh["flags"], True),
                                      _dptr(aterms, "aterms", torch.complex64, sh["aterms"], True),
                                      _dptr(taper, "taper", torch.float32, sh["taper"], True),
                                      _dptr(vis_out, "vis_out", torch.complex64, sh["vis"]), _stream(stream)),
           "idg_degrid_subgrids")


# ---------------------------------------------------------------------------
# host-buffer calls (numpy arrays; page-locked memory gives full copy speed)

def _hptr(a, name, dtype, shape, optional=False):
    if a is None:
        if optional:
            return None
        raise ValueError(f"{name} is required")
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags.c_contiguous or tuple(a.shape) != tuple(shape):
            raise ValueError(f"{name} must be a C-contiguous {dtype} array of shape {shape}")
        return a.ctypes.data_as(ctypes.c_void_p)
    import torch
    if isinstance(a, torch.Tensor) and not a.is_cuda and a.is_contiguous() and tuple(a.shape) == tuple(shape):
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError(f"{name} must be a host array")


def grid_host(plan: Plan, vis, flags, aterms, taper, grid_out, stream=None):
    sh = _shapes(plan)
    _check(load().idg_grid_host(plan.handle, _hptr(vis, "vis", np.complex64, sh["vis"]),
                                _hptr(flags, "flags", np.uint8, sh["flags"], True),
                                _hptr(aterms, "aterms", np.complex64, sh["aterms"], True),
                                _hptr(taper, "taper", np.float32, sh["taper"], True),
                                _hptr(grid_out, "grid", np.complex64, sh["grid"]), _stream(stream)),
           "idg_grid_host")


def degrid_host(plan: Plan, grid_in, flags, aterms, taper, vis_out, stream=None):
    sh = _shapes(plan)
    _check(load().idg_degrid_host(plan.handle, _hptr(grid_in, "grid", np.complex64, sh["grid"]),
                                  _hptr(flags, "flags", np.uint8, sh["flags"], True),
                                  _hptr(aterms, "aterms", np.complex64, sh["aterms"], True),
                                  _hptr(taper, "taper", np.float32, sh["taper"], True),
                                  _hptr(vis_out, "vis_out", np.complex64, sh["vis"]), _stream(stream)),
           "idg_degrid_host")


def grid_degrid_host(plan: Plan, vis, model, flags, aterms, taper, grid_out, vis_out, stream=None):
    """idg_grid_degrid_host: vis gridded into grid_out and the model grid degridded into
    vis_out in one pipelined call (host arrays)."""
    sh = _shapes(plan)
    _check(load().idg_grid_degrid_host(plan.handle, _hptr(vis, "vis", np.complex64, sh["vis"]),
                                       _hptr(model, "model", np.complex64, sh["grid"]),
                                       _hptr(flags, "flags", np.uint8, sh["flags"], True),
                                       _hptr(aterms, "aterms", np.complex64, sh["aterms"], True),
                                       _hptr(taper, "taper", np.float32, sh["taper"], True),
                                       _hptr(grid_out, "grid", np.complex64, sh["grid"]),
                                       _hptr(vis_out, "vis_out", np.complex64, sh["vis"]), _stream(stream)),
           "idg_grid_degrid_host")


# ---------------------------------------------------------------------------
# batched form

class JobBuffers(ctypes.Structure):
    _fields_ = [("vis", ctypes.c_void_p), ("vis_out", ctypes.c_void_p), ("flags", ctypes.c_void_p),
                ("aterms", ctypes.c_void_p), ("taper", ctypes.c_void_p), ("grid", ctypes.c_void_p)]


class Batch:
    """idg_batch: jobs (plan + device tensors) gridded/degridded together in work
    classes per subgrid size (one persistent launch, or tensor-core launches per
    job).  Keeps references to the plans and tensors so they outlive the batch."""

    def __init__(self, plans, jobs, graph: bool = False):
        import torch
        self._keep = (list(plans), [dict(j) for j in jobs])
        n = len(plans)
        bufs = (JobBuffers * n)()
        for i, (p, j) in enumerate(zip(plans, jobs)):
            sh = _shapes(p)
            bufs[i].vis = _dptr(j.get("vis"), "vis", torch.complex64, sh["vis"], True)
            bufs[i].vis_out = _dptr(j.get("vis_out"), "vis_out", torch.complex64, sh["vis"], True)
            bufs[i].flags = _dptr(j.get("flags"), "flags", torch.uint8, sh["flags"], True)
            bufs[i].aterms = _dptr(j.get("aterms"), "aterms", torch.complex64, sh["aterms"], True)
            bufs[i].taper = _dptr(j.get("taper"), "taper", torch.float32, sh["taper"], True)
            bufs[i].grid = _dptr(j.get("grid"), "grid", torch.complex64, sh["grid"], True)
        arr = (ctypes.c_void_p * n)(*[p.handle for p in plans])
        h = ctypes.c_void_p()
        _check(load().idg_batch_create(arr, bufs, n, BATCH_GRAPH if graph else 0, ctypes.byref(h)),
               "idg_batch_create")
        self.handle = h

    def grid(self, stream=None):
        _check(load().idg_batch_grid(self.handle, _stream(stream)), "idg_batch_grid")

    def degrid(self, stream=None):
        _check(load().idg_batch_degrid(self.handle, _stream(stream)), "idg_batch_degrid")

    def autotune(self, stream=None):
        """idg_batch_autotune: keep the fastest persistent shape per class and direction
        (the trial launches add into the grids: zero them afterwards).  Returns the
        trial times in milliseconds."""
        cap = 256
        ms = (ctypes.c_double * cap)(*([-1.0] * cap))
        _check(load().idg_batch_autotune(self.handle, ms, cap, _stream(stream)), "idg_batch_autotune")
        return [ms[i] for i in range(cap) if ms[i] >= 0]

    def info(self):
        nv, ni, nl = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        _check(load().idg_batch_info(self.handle, ctypes.byref(nv), ctypes.byref(ni), ctypes.byref(nl)),
               "idg_batch_info")
        return {"n_vis": nv.value, "n_items": ni.value, "n_launches": nl.value}

    def destroy(self):
        if getattr(self, "handle", None):
            load().idg_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
