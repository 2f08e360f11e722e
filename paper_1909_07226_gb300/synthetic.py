"""Seeded synthetic inputs shaped like the interferometric workloads of the paper.

This module is the one place that makes inputs.  It holds none of the image
domain gridding arithmetic: it only produces station layouts, earth-rotation
uvw coordinates, frequencies, point-source visibilities (the scalar/polarised
measurement equation, Eq. 1-2 of the paper, used purely as a data model),
smooth direction-dependent 2x2 Jones screens sampled on the subgrid pixel
lattice, flags and the anti-aliasing taper.  Both the FP64 oracle and the CUDA
path receive the arrays made here, so a test always compares the two sides on
identical inputs.

The paper measures on a LOFAR observation (the "Toothbrush" field, Sect. 5.1)
that is not available; the workloads below stand in for it with the same
instrument class: 4 polarisations, 1-10 s integrations, ~1 MHz channels around
140 MHz, a compact core plus remote stations.

Conventions shared with the rest of the library (they define the *inputs*):
  * visibilities  complex64 [n_bl][n_t][n_chan][4], pol order XX, XY, YX, YY,
    read as the 2x2 matrix [[XX, XY], [YX, YY]];
  * uvw           float64   [n_bl][n_t][3], metres, uvw = x_q - x_p for the
    baseline (p, q);
  * frequencies   float64   [n_chan], Hz, channel centres;
  * A-terms       complex64 [n_slots][n_stations][L][L][4], the Jones matrix of
    each station sampled at subgrid pixel (y, x), i.e. at direction cosines
    l = (x - L/2) S/L, m = (y - L/2) S/L with S = N * cell;
  * taper         float32   [L][L], separable c[y][x] = a_y a_x (Sect. 4.2).
"""
from __future__ import annotations

import concurrent.futures
import dataclasses
import math
import os
from typing import Optional

import numpy as np

C_LIGHT = 299792458.0          # m/s
OMEGA_EARTH = 7.2921150e-5     # rad/s, sidereal rotation rate
LOFAR_LATITUDE_DEG = 52.91     # array latitude (the paper's instrument; not stated there)
SOURCE_DEC_DEG = 52.0          # phase centre declination

# ---------------------------------------------------------------------------
# station layouts, baselines, uvw


def stations_uniform_disc(rng: np.random.Generator, n: int, diameter_m: float) -> np.ndarray:
    """n stations uniform in a disc; returns ENU positions [n][3] (metres, U=0)."""
    r = 0.5 * diameter_m * np.sqrt(rng.random(n))
    th = 2.0 * np.pi * rng.random(n)
    return np.stack([r * np.cos(th), r * np.sin(th), np.zeros(n)], axis=1)


def stations_core_remote(rng: np.random.Generator, n_core: int, sigma_m: float,
                         n_remote: int, r_min_m: float, r_max_m: float) -> np.ndarray:
    """Gaussian core (sigma per axis) plus remote stations at log-uniform radius."""
    core = rng.normal(0.0, sigma_m, size=(n_core, 2))
    lr = rng.uniform(math.log(r_min_m), math.log(r_max_m), size=n_remote)
    th = rng.uniform(0.0, 2.0 * np.pi, size=n_remote)
    remote = np.stack([np.exp(lr) * np.cos(th), np.exp(lr) * np.sin(th)], axis=1)
    en = np.concatenate([core, remote], axis=0)
    return np.concatenate([en, np.zeros((en.shape[0], 1))], axis=1)


def all_baselines(n_stations: int) -> np.ndarray:
    """Cross-correlation station pairs (p, q), p < q, in row-major order."""
    p, q = np.triu_indices(n_stations, k=1)
    return np.stack([p, q], axis=1).astype(np.int32)


def earth_rotation_uvw(enu: np.ndarray, baselines: np.ndarray, hour_angle: np.ndarray,
                       dec_rad: float, lat_rad: float) -> np.ndarray:
    """uvw in metres, [n_bl][n_t][3], for a phase centre at declination dec.

    Textbook transform (Thompson, Moran & Swenson, Eq. 4.1): ENU -> equatorial
    (X, Y, Z), then the rotation by hour angle H and declination.
    """
    e, n, u = enu[:, 0], enu[:, 1], enu[:, 2]
    X = -math.sin(lat_rad) * n + math.cos(lat_rad) * u
    Y = e
    Z = math.cos(lat_rad) * n + math.sin(lat_rad) * u
    p, q = baselines[:, 0], baselines[:, 1]
    bx = (X[q] - X[p])[:, None]
    by = (Y[q] - Y[p])[:, None]
    bz = (Z[q] - Z[p])[:, None]
    sH, cH = np.sin(hour_angle)[None, :], np.cos(hour_angle)[None, :]
    sd, cd = math.sin(dec_rad), math.cos(dec_rad)
    uu = sH * bx + cH * by
    vv = -sd * cH * bx + sd * sH * by + cd * bz
    ww = cd * cH * bx - cd * sH * by + sd * bz
    return np.ascontiguousarray(np.stack([uu, vv, ww], axis=2), dtype=np.float64)


def hour_angles(n_t: int, dt_s: float, start_rad: float = None) -> np.ndarray:
    """Hour angles of n_t integrations; symmetric about transit unless a start is given."""
    t = np.arange(n_t, dtype=np.float64)
    if start_rad is None:
        return (t - 0.5 * (n_t - 1)) * dt_s * OMEGA_EARTH
    return start_rad + t * dt_s * OMEGA_EARTH


def channel_centres(f_lo_hz: float, df_hz: float, n_chan: int) -> np.ndarray:
    return f_lo_hz + (np.arange(n_chan, dtype=np.float64) + 0.5) * df_hz


# ---------------------------------------------------------------------------
# anti-aliasing taper (an input of the gridder; Sect. 4.1-4.2)


def _pswf0_legendre_coeffs(c: float, n_terms: int = 64) -> np.ndarray:
    """Coefficients of the zeroth prolate spheroidal wave function psi_0(c, .)
    in normalised even Legendre polynomials.

    Legendre-expansion method (Bouwkamp 1947; Xiao, Rokhlin & Yarvin 2001): psi_0
    is the eigenvector of the symmetric tridiagonal matrix of the prolate
    differential operator in the basis sqrt(k + 1/2) P_k, restricted to even k,
    belonging to the smallest eigenvalue.
    """
    ks = np.arange(0, 2 * n_terms, 2, dtype=np.float64)
    diag = ks * (ks + 1) + c * c * (2 * ks * (ks + 1) - 1) / ((2 * ks + 3) * (2 * ks - 1))
    k = ks[:-1]
    off = c * c * (k + 2) * (k + 1) / ((2 * k + 3) * np.sqrt((2 * k + 1) * (2 * k + 5)))
    mat = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    w, v = np.linalg.eigh(mat)
    d = v[:, np.argmin(w)]
    return d if d[0] > 0 else -d


def _eval_even_legendre_series(d: np.ndarray, x: np.ndarray) -> np.ndarray:
    """sum_j d_j sqrt(2j + 1/2) P_{2j}(x), P_n from the three-term Legendre recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p_prev = np.ones_like(x)          # P_{n-1}, n = 1
    p_cur = x.copy()                  # P_n
    n = 1
    out = d[0] * math.sqrt(0.5) * np.ones_like(x)
    for j in range(1, d.shape[0]):
        while n < 2 * j:
            p_next = ((2 * n + 1) * x * p_cur - n * p_prev) / (n + 1)
            p_prev, p_cur = p_cur, p_next
            n += 1
        out = out + d[j] * math.sqrt(2 * j + 0.5) * p_cur
    return out


def pswf_1d(L: int, beta: float) -> np.ndarray:
    """1D taper a_x = psi_0(c = pi*beta/2, eta = 2(x - L/2)/L), normalised a_{L/2} = 1."""
    c = math.pi * beta / 2.0
    d = _pswf0_legendre_coeffs(c)
    eta = 2.0 * (np.arange(L, dtype=np.float64) - L / 2) / L
    a = _eval_even_legendre_series(d, eta)
    a0 = _eval_even_legendre_series(d, np.zeros(1))[0]
    return a / a0


def kaiser_bessel_1d(L: int, beta: float) -> np.ndarray:
    """1D Kaiser-Bessel taper I0(pi*alpha*sqrt(1-eta^2))/I0(pi*alpha), alpha = beta/2."""
    eta = 2.0 * (np.arange(L, dtype=np.float64) - L / 2) / L
    alpha = beta / 2.0
    return np.i0(math.pi * alpha * np.sqrt(np.clip(1.0 - eta * eta, 0.0, None))) / np.i0(math.pi * alpha)


def separable_taper(a: np.ndarray) -> np.ndarray:
    """c[y][x] = a_y a_x as float32 (Sect. 4.2)."""
    return np.ascontiguousarray(np.outer(a, a).astype(np.float32))


# ---------------------------------------------------------------------------
# direction-dependent Jones screens


@dataclasses.dataclass
class JonesScreens:
    """Per (slot, station): g_x, g_y = (1 + 0.1 a(l,m)) exp(i phi(l,m)) with a, phi
    quadratic polynomials in normalised (l, m), |a| <= 1, |phi| <= 1 rad over the
    field; leakage d, d' constant complex.  Jones = [[g_x, d], [d', g_y]]."""
    amp: np.ndarray      # [n_slots][n_st][2][6]
    phase: np.ndarray    # [n_slots][n_st][2][6]
    leak: np.ndarray     # [n_slots][n_st][2] complex
    half_extent: float   # S/2, the normalisation of (l, m)

    def evaluate(self, l: np.ndarray, m: np.ndarray) -> np.ndarray:
        """Jones at direction cosines (broadcast l, m) -> [n_slots][n_st][...][4] complex128."""
        x = np.asarray(l, dtype=np.float64) / self.half_extent
        y = np.asarray(m, dtype=np.float64) / self.half_extent
        basis = np.stack([np.ones_like(x), x, y, x * x, x * y, y * y], axis=0)   # [6][...]
        a = np.tensordot(self.amp, basis, axes=([3], [0]))      # [s][st][2][...]
        ph = np.tensordot(self.phase, basis, axes=([3], [0]))
        g = (1.0 + 0.1 * a) * np.exp(1j * ph)
        shape = g.shape[:2] + g.shape[3:]
        d0 = np.broadcast_to(self.leak[:, :, 0].reshape(self.leak.shape[:2] + (1,) * (g.ndim - 3)), shape)
        d1 = np.broadcast_to(self.leak[:, :, 1].reshape(self.leak.shape[:2] + (1,) * (g.ndim - 3)), shape)
        return np.stack([g[:, :, 0], d0, d1, g[:, :, 1]], axis=-1)


def random_jones_screens(rng: np.random.Generator, n_slots: int, n_st: int, half_extent: float,
                         leakage: float = 0.05) -> JonesScreens:
    amp = rng.normal(size=(n_slots, n_st, 2, 6))
    amp /= np.sum(np.abs(amp), axis=-1, keepdims=True)          # |a| <= 1 on |x|,|y| <= 1
    ph = rng.normal(size=(n_slots, n_st, 2, 6))
    ph /= np.sum(np.abs(ph), axis=-1, keepdims=True)             # |phi| <= 1 rad
    leak = leakage * (rng.normal(size=(n_slots, n_st, 2)) + 1j * rng.normal(size=(n_slots, n_st, 2))) / math.sqrt(2.0)
    return JonesScreens(amp, ph, leak, half_extent)


def subgrid_pixel_lm(L: int, S: float):
    """Direction cosines of the subgrid pixel lattice, l_x = (x - L/2) S / L."""
    c = (np.arange(L, dtype=np.float64) - L / 2) * S / L
    return c[None, :], c[:, None]        # l varies along x (columns), m along y (rows)


def aterms_on_subgrid(screens: JonesScreens, L: int, S: float) -> np.ndarray:
    """A-term array [n_slots][n_st][L][L][4] complex64 sampled at subgrid pixels."""
    l, m = subgrid_pixel_lm(L, S)
    l2 = np.broadcast_to(l, (L, L))
    m2 = np.broadcast_to(m, (L, L))
    return np.ascontiguousarray(screens.evaluate(l2, m2).astype(np.complex64))


def identity_aterms(n_slots: int, n_st: int, L: int) -> np.ndarray:
    a = np.zeros((n_slots, n_st, L, L, 4), dtype=np.complex64)
    a[..., 0] = 1.0
    a[..., 3] = 1.0
    return a


# ---------------------------------------------------------------------------
# visibilities from point sources (measurement equation as a data model)


def point_source_visibilities(uvw_m: np.ndarray, freqs_hz: np.ndarray, baselines: np.ndarray,
                              src_l: np.ndarray, src_m: np.ndarray, src_flux: np.ndarray,
                              screens: Optional[JonesScreens] = None,
                              aterm_offsets: Optional[np.ndarray] = None) -> np.ndarray:
    """V_pq = sum_s I_s J_p(l_s) J_q(l_s)^H exp(-2 pi i (u l_s + v m_s + w n'_s)).

    Unpolarised sources (brightness I_s times the 2x2 identity).  Returns
    complex64 [n_bl][n_t][n_chan][4].  For uniformly spaced channels the phase
    is advanced over channels by a complex recurrence from an FP64 anchor,
    which is plenty for synthetic input data.
    """
    n_bl, n_t, _ = uvw_m.shape
    n_chan = freqs_hz.shape[0]
    n_src = src_l.shape[0]
    src_n1 = np.sqrt(1.0 - src_l ** 2 - src_m ** 2) - 1.0
    out = np.empty((n_bl, n_t, n_chan, 4), dtype=np.complex64)
    if aterm_offsets is None:
        aterm_offsets = np.array([0, n_t])
    n_slots = len(aterm_offsets) - 1
    if screens is not None:
        jones = screens.evaluate(src_l, src_m)                 # [slots][st][src][4]
    uniform = n_chan > 1 and np.allclose(np.diff(freqs_hz), freqs_hz[1] - freqs_hz[0], rtol=0, atol=1e-6)
    coh0 = np.zeros((n_src, 4), dtype=np.complex128)
    coh0[:, 0] = src_flux
    coh0[:, 3] = src_flux

    def one_baseline(b, phs):
        p, q = baselines[b]
        # geometric path difference in metres per (t, src)
        geo = uvw_m[b, :, 0:1] * src_l[None, :] + uvw_m[b, :, 1:2] * src_m[None, :] + uvw_m[b, :, 2:3] * src_n1[None, :]
        if uniform:
            ph = np.exp(-2j * np.pi * geo * (freqs_hz[0] / C_LIGHT))
            step = np.exp(-2j * np.pi * geo * ((freqs_hz[1] - freqs_hz[0]) / C_LIGHT))
            for c in range(n_chan):
                phs[:, c, :] = ph
                ph = ph * step
        else:
            phs[:] = np.exp(-2j * np.pi * geo[:, None, :] * (freqs_hz[None, :, None] / C_LIGHT))
        for a in range(n_slots):
            t0, t1 = int(aterm_offsets[a]), int(aterm_offsets[a + 1])
            if screens is None:
                coh = coh0
            else:
                jp, jq = jones[a, p], jones[a, q]                 # [src][4]
                coh = np.stack([jp[:, 0] * np.conj(jq[:, 0]) + jp[:, 1] * np.conj(jq[:, 1]),
                                jp[:, 0] * np.conj(jq[:, 2]) + jp[:, 1] * np.conj(jq[:, 3]),
                                jp[:, 2] * np.conj(jq[:, 0]) + jp[:, 3] * np.conj(jq[:, 1]),
                                jp[:, 2] * np.conj(jq[:, 2]) + jp[:, 3] * np.conj(jq[:, 3])], axis=-1)
                coh = coh * src_flux[:, None]
            blk = phs[t0:t1].reshape(-1, n_src) @ coh
            out[b, t0:t1] = blk.reshape(t1 - t0, n_chan, 4)

    def worker(bs):
        phs = np.empty((n_t, n_chan, n_src), dtype=np.complex128)
        for b in bs:
            one_baseline(b, phs)

    n_workers = max(1, min(os.cpu_count() or 1, 16, n_bl // 8 + 1))
    if n_workers == 1:
        worker(range(n_bl))
    else:
        with concurrent.futures.ThreadPoolExecutor(n_workers) as ex:
            list(ex.map(worker, [range(i, n_bl, n_workers) for i in range(n_workers)]))
    return out


def gaussian_noise(rng: np.random.Generator, shape, sigma: float) -> np.ndarray:
    """Complex Gaussian noise, sigma per real and imaginary part, complex64."""
    re = rng.standard_normal(size=tuple(shape) + (2,), dtype=np.float32)
    re *= np.float32(sigma)
    return re.view(np.complex64)[..., 0]


def random_flags(rng: np.random.Generator, shape, p: float) -> np.ndarray:
    return (rng.random(shape) < p).astype(np.uint8)


# ---------------------------------------------------------------------------
# named workloads


@dataclasses.dataclass
class Workload:
    name: str
    uvw_m: np.ndarray
    freqs_hz: np.ndarray
    baselines: np.ndarray
    aterm_offsets: np.ndarray
    n_stations: int
    subgrid_size: int
    grid_size: int
    cell_size: float
    w_step: float
    kernel_size: float
    max_timesteps: int
    taper: np.ndarray
    aterms: Optional[np.ndarray] = None
    vis: Optional[np.ndarray] = None
    flags: Optional[np.ndarray] = None
    screens: Optional[JonesScreens] = None
    sources: Optional[tuple] = None

    @property
    def n_bl(self):
        return self.uvw_m.shape[0]

    @property
    def n_t(self):
        return self.uvw_m.shape[1]

    @property
    def n_chan(self):
        return self.freqs_hz.shape[0]

    @property
    def n_slots(self):
        return self.aterm_offsets.shape[0] - 1

    @property
    def n_vis(self):
        return self.n_bl * self.n_t * self.n_chan

    @property
    def image_size(self):
        return self.grid_size * self.cell_size


SEED_BASE = 1909
CONFIG_INDEX = {"tiny": 0, "lofar": 1, "precision": 2, "batched": 3, "serving": 4}


def make_tiny(seed: Optional[int] = None, with_vis: bool = True) -> Workload:
    """8 stations uniform in a 2 km disc, 64 x 10 s, 8 x 1 MHz at 140-148 MHz,
    10 point sources U(0.1,1) Jy in a 4x4 degree field + N(0, 0.01) noise,
    identity A-terms, L=24, beta=7, 16 timesteps per subgrid, 512^2 grid."""
    rng = np.random.default_rng(SEED_BASE + CONFIG_INDEX["tiny"] if seed is None else seed)
    enu = stations_uniform_disc(rng, 8, 2000.0)
    bl = all_baselines(8)
    ha = hour_angles(64, 10.0)
    uvw = earth_rotation_uvw(enu, bl, ha, math.radians(SOURCE_DEC_DEG), math.radians(LOFAR_LATITUDE_DEG))
    freqs = channel_centres(140e6, 1e6, 8)
    L, N, cell, beta = 24, 512, 2.0e-4, 7.0
    wl = Workload("tiny", uvw, freqs, bl, np.array([0, 64], dtype=np.int32), 8, L, N, cell, 0.0, beta, 16,
                  separable_taper(pswf_1d(L, beta)))
    half = math.radians(2.0)
    sl = rng.uniform(-half, half, 10)
    sm = rng.uniform(-half, half, 10)
    sf = rng.uniform(0.1, 1.0, 10)
    wl.sources = (sl, sm, sf)
    wl.aterms = identity_aterms(1, 8, L)
    if with_vis:
        vis = point_source_visibilities(uvw, freqs, bl, sl, sm, sf)
        vis += gaussian_noise(rng, vis.shape, 0.01)
        wl.vis = vis
    return wl


def make_lofar(seed: Optional[int] = None, with_vis: bool = True, n_t: int = 4096,
               slot_len: int = 128, name: str = "lofar") -> Workload:
    """48 stations (40 Gaussian core sigma=3 km + 8 remote to 50 km), 4096 x 1 s,
    16 x 1 MHz at 130-146 MHz, 20 sources in the central 80% of the field,
    smooth random 2x2 A-terms per station refreshed every slot_len timesteps,
    L=32, beta=7, 128 timesteps per subgrid, 4096^2 grid, cell 1e-5 rad."""
    idx = CONFIG_INDEX["precision" if name == "precision" else "lofar"]
    rng = np.random.default_rng(SEED_BASE + idx if seed is None else seed)
    enu = stations_core_remote(rng, 40, 3000.0, 8, 5000.0, 50000.0)
    bl = all_baselines(48)
    ha = hour_angles(n_t, 1.0)
    uvw = earth_rotation_uvw(enu, bl, ha, math.radians(SOURCE_DEC_DEG), math.radians(LOFAR_LATITUDE_DEG))
    freqs = channel_centres(130e6, 1e6, 16)
    L, N, cell, beta = 32, 4096, 1.0e-5, 7.0
    offs = np.arange(0, n_t + 1, slot_len, dtype=np.int32)
    if offs[-1] != n_t:
        offs = np.append(offs, np.int32(n_t))
    S = N * cell
    wl = Workload(name, uvw, freqs, bl, offs, 48, L, N, cell, 0.0, beta, 128,
                  separable_taper(pswf_1d(L, beta)))
    screens = random_jones_screens(rng, offs.shape[0] - 1, 48, S / 2)
    wl.screens = screens
    wl.aterms = aterms_on_subgrid(screens, L, S)
    sl = rng.uniform(-0.4 * S, 0.4 * S, 20)
    sm = rng.uniform(-0.4 * S, 0.4 * S, 20)
    sf = rng.uniform(0.1, 1.0, 20)
    wl.sources = (sl, sm, sf)
    if with_vis:
        vis = point_source_visibilities(uvw, freqs, bl, sl, sm, sf, screens, offs)
        vis += gaussian_noise(rng, vis.shape, 0.01)
        wl.vis = vis
    return wl


def make_small(seed: int, n_st: int = 6, n_t: int = 24, n_chan: int = 4, L: int = 16, N: int = 128,
               cell: float = None, beta: float = 7.0, max_t: int = 8, n_slots: int = 2,
               w_step: float = 0.0, flag_p: float = 0.0, diameter_m: float = 3000.0,
               f_lo: float = 140e6, df: float = 1e6, dt: float = 30.0, aterms: str = "random",
               n_src: int = 4, with_vis: bool = True, taper: str = "pswf") -> Workload:
    """A small randomised workload for unit tests (all knobs exposed)."""
    rng = np.random.default_rng(seed)
    enu = stations_uniform_disc(rng, n_st, diameter_m)
    bl = all_baselines(n_st)
    ha = hour_angles(n_t, dt)
    uvw = earth_rotation_uvw(enu, bl, ha, math.radians(SOURCE_DEC_DEG), math.radians(LOFAR_LATITUDE_DEG))
    freqs = channel_centres(f_lo, df, n_chan)
    if cell is None:
        # longest baseline at the top frequency reaches ~80% of the grid half-width
        bmax = np.max(np.abs(uvw[:, :, :2])) * freqs[-1] / C_LIGHT
        cell = 0.8 * (N / 2) / (bmax * N)
    offs = np.linspace(0, n_t, n_slots + 1).round().astype(np.int32)
    S = N * cell
    a = pswf_1d(L, beta) if taper == "pswf" else (kaiser_bessel_1d(L, beta) if taper == "kb" else np.ones(L))
    wl = Workload("small", uvw, freqs, bl, offs, n_st, L, N, cell, w_step, beta, max_t, separable_taper(a))
    if aterms == "random":
        wl.screens = random_jones_screens(rng, n_slots, n_st, S / 2)
        wl.aterms = aterms_on_subgrid(wl.screens, L, S)
    elif aterms == "identity":
        wl.aterms = identity_aterms(n_slots, n_st, L)
    sl = rng.uniform(-0.3 * S, 0.3 * S, n_src)
    sm = rng.uniform(-0.3 * S, 0.3 * S, n_src)
    sf = rng.uniform(0.1, 1.0, n_src)
    wl.sources = (sl, sm, sf)
    if with_vis:
        vis = point_source_visibilities(uvw, freqs, bl, sl, sm, sf, wl.screens if aterms == "random" else None, offs)
        vis += gaussian_noise(rng, vis.shape, 0.01)
        wl.vis = vis
    if flag_p > 0:
        wl.flags = random_flags(rng, (bl.shape[0], n_t, n_chan), flag_p)
    return wl


def random_grid(rng: np.random.Generator, n_w: int, N: int) -> np.ndarray:
    """A random complex64 uv grid [n_w][N][N][4] (input of degridding tests)."""
    g = rng.normal(size=(n_w, N, N, 4, 2)).astype(np.float32)
    return np.ascontiguousarray(g.view(np.complex64)[..., 0])


def make_batched_jobs(n_jobs: int = 256, seed: Optional[int] = None, scale_t: float = 1.0):
    """The uneven batch: n_jobs snapshot jobs, each with U{12..64} stations in a
    Gaussian layout (sigma 3 km), U{64..1024} timesteps of 1 s from a random
    start hour angle, U{4..32} channels of 0.2 MHz placed uniformly so the band
    lies in 100-200 MHz, flag probability U[0, 0.2], subgrid size from
    {16, 24, 32}, grid size from {1024, 2048, 4096}, image pixel
    cell = 1/(2.2 max|uv|) (so the longest baseline lands N/2.2 pixels from the
    centre), 128 timesteps per subgrid, beta = 7, identity A-terms.  Visibility
    values are not made here.  scale_t shrinks the timestep counts for tests."""
    rng = np.random.default_rng(SEED_BASE + CONFIG_INDEX["batched"] if seed is None else seed)
    jobs = []
    for j in range(n_jobs):
        n_st = int(rng.integers(12, 65))
        n_t = max(2, int(int(rng.integers(64, 1025)) * scale_t))
        n_ch = int(rng.integers(4, 33))
        p_flag = float(rng.uniform(0.0, 0.2))
        L = int(rng.choice([16, 24, 32]))
        N = int(rng.choice([1024, 2048, 4096]))
        enu = np.concatenate([rng.normal(0.0, 3000.0, size=(n_st, 2)), np.zeros((n_st, 1))], axis=1)
        bl = all_baselines(n_st)
        ha0 = float(rng.uniform(-3.0, 3.0)) * np.pi / 12.0
        uvw = earth_rotation_uvw(enu, bl, hour_angles(n_t, 1.0, start_rad=ha0), math.radians(SOURCE_DEC_DEG),
                                 math.radians(LOFAR_LATITUDE_DEG))
        df = 0.2e6
        f_lo = float(rng.uniform(100e6, 200e6 - n_ch * df))
        freqs = channel_centres(f_lo, df, n_ch)
        uv_max = float(np.max(np.hypot(uvw[:, :, 0], uvw[:, :, 1]))) * freqs[-1] / C_LIGHT
        cell = 1.0 / (2.2 * uv_max)
        wl = Workload(f"batch{j}", uvw, freqs, bl, np.array([0, n_t], dtype=np.int32), n_st, L, N, cell, 0.0, 7.0,
                      128, separable_taper(pswf_1d(L, 7.0)))
        wl.flag_p = p_flag
        jobs.append(wl)
    return jobs
