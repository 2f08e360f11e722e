"""Helpers shared by the GPU tests (device upload and the parity measure)."""
import numpy as np

REL_RMS_TOL = 1e-5     # grid and visibilities vs the FP64 oracle (relative RMS)
MAX_ERR_TOL = 1e-3     # max |gpu - ref| / max |ref|, reported and loosely bounded


def dev(a, torch_dtype=None):
    import torch
    if a is None:
        return None
    t = torch.from_numpy(np.ascontiguousarray(a))
    if torch_dtype is not None:
        t = t.to(torch_dtype)
    return t.cuda()


def workload_to_device(wl):
    import torch
    return dict(vis=dev(wl.vis), flags=dev(wl.flags), aterms=dev(wl.aterms),
                taper=dev(wl.taper.astype(np.float32)))


def parity(gpu, ref, name="", tol=REL_RMS_TOL, max_tol=MAX_ERR_TOL):
    gpu = np.asarray(gpu).astype(np.complex128)
    ref = np.asarray(ref).astype(np.complex128)
    assert gpu.shape == ref.shape, (gpu.shape, ref.shape)
    nref = np.linalg.norm(ref.ravel())
    err = np.linalg.norm((gpu - ref).ravel())
    rel = err / nref if nref > 0 else err
    mref = np.max(np.abs(ref)) if ref.size else 0.0
    mx = np.max(np.abs(gpu - ref)) / mref if mref > 0 else (np.max(np.abs(gpu)) if gpu.size else 0.0)
    print(f"parity {name}: rel_rms={rel:.3e} max_err/max_ref={mx:.3e}")
    assert rel <= tol, f"{name}: relative RMS error {rel:.3e} > {tol:.1e}"
    assert mx <= max_tol, f"{name}: max error {mx:.3e} > {max_tol:.1e}"
    return rel, mx
