"""Helpers shared by the GPU tests (device upload and the parity measure)."""
import numpy as np

REL_RMS_TOL = 1e-5     # grid and visibilities vs the FP64 oracle (relative RMS)
# max |gpu - ref| / max |ref|: the largest single error against the largest value.
# FP32 sums of up to a few thousand terms with FP32 phasors stay near 1e-6 of the
# largest term (the largest seen over every GPU test is 5.9e-6); 2e-5 leaves room
# for the longest sums and the split-FP16 forms.
MAX_ERR_TOL = 2e-5
# per-element relative error |gpu - ref| / |ref|, over the elements within two
# decades of the largest (smaller ones carry the absolute error of the big terms
# of their sums and are covered by MAX_ERR_TOL); reported and bounded
ELEM_FLOOR = 1e-2
ELEM_REL_TOL = 1e-3     # largest seen: 2.0e-4 (grid + image chain)


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


def parity(gpu, ref, name="", tol=REL_RMS_TOL, max_tol=MAX_ERR_TOL, elem_tol=ELEM_REL_TOL):
    """Relative RMS error (bounded by tol), the largest error against the largest
    reference value (bounded by max_tol), and the largest per-element relative
    error over elements within two decades of the largest (bounded by elem_tol)."""
    gpu = np.asarray(gpu).astype(np.complex128)
    ref = np.asarray(ref).astype(np.complex128)
    assert gpu.shape == ref.shape, (gpu.shape, ref.shape)
    nref = np.linalg.norm(ref.ravel())
    diff = np.abs(gpu - ref)
    err = np.linalg.norm(diff.ravel())
    rel = err / nref if nref > 0 else err
    aref = np.abs(ref)
    mref = np.max(aref) if ref.size else 0.0
    mx = np.max(diff) / mref if mref > 0 else (np.max(np.abs(gpu)) if gpu.size else 0.0)
    big = aref >= ELEM_FLOOR * mref if mref > 0 else np.zeros(ref.shape, dtype=bool)
    elem = float(np.max(diff[big] / aref[big])) if big.any() else 0.0
    print(f"parity {name}: rel_rms={rel:.3e} max_err/max_ref={mx:.3e} "
          f"max_elem_rel(|ref|>={ELEM_FLOOR:g} max)={elem:.3e} n={ref.size}")
    assert rel <= tol, f"{name}: relative RMS error {rel:.3e} > {tol:.1e}"
    assert mx <= max_tol, f"{name}: max error {mx:.3e} > {max_tol:.1e}"
    assert elem <= elem_tol, f"{name}: per-element relative error {elem:.3e} > {elem_tol:.1e}"
    return rel, mx
