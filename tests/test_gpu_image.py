"""Image-side steps on the GPU (idg_image_from_grid / idg_grid_from_image) against the
oracle (``oracle/image.py``): relative RMS <= 1e-5, over the whole image and with several
w-layers; and the GPU chain (grid, then image) against direct imaging of the same
visibilities within the aliasing level of the taper on the inner image."""
import numpy as np
import pytest

from tests.gpu_util import dev, parity, workload_to_device
from oracle import image as OI
from oracle import oracle as O
from paper_1909_07226_gb300 import idg, synthetic as syn

pytestmark = pytest.mark.gpu
C = 299792458.0


@pytest.fixture(scope="module", autouse=True)
def _lib():
    idg.load()


def _w0s(p, wl):
    s = p.stats
    return [(k + s.w_layer_min) * wl.w_step for k in range(s.n_w_layers)] if wl.w_step > 0 else [0.0]


def _wl(w_step, N=256, L=32, beta=7.0, seed=5):
    wl = syn.make_small(seed=seed, n_st=5, n_t=24, n_chan=4, L=L, N=N, aterms="identity", max_t=8, flag_p=0.0,
                        diameter_m=3000.0 if w_step == 0 else 20000.0, w_step=w_step, beta=beta)
    a, _ = idg.taper_window(L, beta, idg.TAPER_PSWF)
    wl.taper = np.outer(a, a)
    return wl, a


@pytest.mark.parametrize("w_step,with_window", [(0.0, True), (40.0, True), (40.0, False)])
def test_image_from_grid_and_back(w_step, with_window):
    import torch
    wl, a = _wl(w_step)
    p = idg.plan_from_workload(wl)
    N, S, L = wl.grid_size, wl.grid_size * wl.cell_size, wl.subgrid_size
    w0s = _w0s(p, wl)
    assert len(w0s) == p.n_w_layers and (w_step == 0 or p.n_w_layers > 1)
    window = a if with_window else None
    rng = np.random.default_rng(11)
    G = (rng.standard_normal((p.n_w_layers, N, N, 4)) + 1j * rng.standard_normal((p.n_w_layers, N, N, 4))).astype(np.complex64)
    img = torch.empty((N, N, 4), dtype=torch.complex64, device="cuda")
    idg.image_from_grid(p, dev(G), window, img)
    parity(img.cpu().numpy(), OI.image_from_grid(G, S, w0s, window, L), f"image_from_grid w_step={w_step}")
    I = (rng.standard_normal((N, N, 4)) + 1j * rng.standard_normal((N, N, 4))).astype(np.complex64)
    g = torch.empty((p.n_w_layers, N, N, 4), dtype=torch.complex64, device="cuda")
    idg.grid_from_image(p, dev(I), window, g)
    parity(g.cpu().numpy(), OI.grid_from_image(I, S, w0s, window, L), f"grid_from_image w_step={w_step}")
    idg.device_errors()


@pytest.mark.parametrize("w_step", [0.0, 40.0])
def test_gpu_chain_matches_oracle_and_direct_imaging(w_step):
    import torch
    wl, a = _wl(w_step)
    p = idg.plan_from_workload(wl)
    op = O.plan(wl)
    N, S, L = wl.grid_size, wl.grid_size * wl.cell_size, wl.subgrid_size
    d = workload_to_device(wl)
    g = torch.zeros((p.n_w_layers, N, N, 4), dtype=torch.complex64, device="cuda")
    idg.grid(p, d["vis"], d["flags"], d["aterms"], d["taper"], g)
    img = torch.empty((N, N, 4), dtype=torch.complex64, device="cuda")
    idg.image_from_grid(p, g, a, img)
    got = img.cpu().numpy()
    ref = OI.image_from_grid(O.grid(wl, op), S, _w0s(p, wl), a, L)
    lx = (np.arange(N) - N / 2) * S / N
    inner = (np.abs(lx)[None, :] < 0.35 * S) & (np.abs(lx)[:, None] < 0.35 * S)
    parity(got[inner], ref[inner], f"grid + image chain w_step={w_step}")
    # physics: direct imaging of the same visibilities, within the taper's aliasing level
    npr = OI.nprime(N, S)
    sc = wl.freqs_hz / C
    D = np.zeros((N, N), complex)
    for dd in op.desc:
        b = dd[0]
        for t in range(dd[2], dd[2] + dd[3]):
            for c in range(dd[4], dd[4] + dd[5]):
                u, v, w = wl.uvw_m[b, t] * sc[c]
                D += wl.vis[b, t, c, 0] * np.exp(2j * np.pi * (u * lx[None, :] + v * lx[:, None] + w * npr))
    rel = np.sqrt(np.mean(np.abs(got[:, :, 0] - D)[inner] ** 2) / np.mean(np.abs(D[inner]) ** 2))
    assert rel < 2e-4, rel
    idg.device_errors()


def test_image_steps_reject_unsupported_sizes_and_bad_windows():
    import torch
    wl = syn.make_small(seed=3, n_st=4, n_t=8, n_chan=2, L=16, N=192, aterms="identity", max_t=8)
    p = idg.plan_from_workload(wl)
    g = torch.zeros((p.n_w_layers, 192, 192, 4), dtype=torch.complex64, device="cuda")
    img = torch.empty((192, 192, 4), dtype=torch.complex64, device="cuda")
    with pytest.raises(idg.IDGError):
        idg.image_from_grid(p, g, None, img)
    wl2, a = _wl(0.0, N=64, L=16)
    p2 = idg.plan_from_workload(wl2)
    g2 = torch.zeros((p2.n_w_layers, 64, 64, 4), dtype=torch.complex64, device="cuda")
    img2 = torch.empty((64, 64, 4), dtype=torch.complex64, device="cuda")
    with pytest.raises(ValueError):
        idg.image_from_grid(p2, g2, a[:-1], img2)
    with pytest.raises(idg.IDGError):
        idg.image_from_grid(p2, g2, np.full(16, np.nan), img2)


@pytest.mark.parametrize("N", [32, 64, 128, 512, 1024, 2048, 4096])
def test_transform_sizes(N):
    # every transform size the image steps support (radix-16 line transforms with a
    # smaller last radix, four-step columns N = N1 N2), both directions, against the
    # oracle (without the window division: the transform is what is tested here)
    import torch
    L = 16 if N < 64 else 32
    # (an image of width S = 0.5 in direction cosines keeps every pixel inside the unit circle)
    wl = syn.make_small(seed=7, n_st=4, n_t=4, n_chan=2, L=L, N=N, aterms="identity", max_t=4, with_vis=False,
                        cell=0.5 / N)
    a = None
    p = idg.plan_from_workload(wl)
    S = N * wl.cell_size
    rng = np.random.default_rng(N)
    G = (rng.standard_normal((1, N, N, 4)) + 1j * rng.standard_normal((1, N, N, 4))).astype(np.complex64)
    img = torch.empty((N, N, 4), dtype=torch.complex64, device="cuda")
    idg.image_from_grid(p, dev(G), a, img)
    parity(img.cpu().numpy(), OI.image_from_grid(G, S, [0.0], a, L), f"image_from_grid N={N}")
    g = torch.empty((1, N, N, 4), dtype=torch.complex64, device="cuda")
    idg.grid_from_image(p, dev(G[0]), a, g)
    parity(g.cpu().numpy(), OI.grid_from_image(G[0], S, [0.0], a, L), f"grid_from_image N={N}")
