"""Seeded synthetic LWA-like inputs for the EPIC imaging path.

This module only *creates inputs*: antenna layouts, channel frequencies, the
illumination kernel, per-antenna gains and packed 4+4-bit voltages.  It holds
none of the imaging arithmetic (no cell mapping, gridding, transform, products
or autocorrelation handling), so the CUDA path and the FP64 oracle can both be
fed from it without sharing any of the method.

Shapes follow the LWA-SV station described in Sec. 2.1 of the paper (256
dual-polarisation dipoles in a 110 m x 100 m pseudo-random ellipse, 25 kHz
channels, 40 us spectra, 4+4-bit complex samples).  The paper's observatory data
is not public, so these seeded draws stand in for it.

Voltage model (per channel c, polarisation p, time t, antenna a):
    e = sum_s z_s(t) * exp(-2 pi i (u_a l_s + v_a m_s)) + n
with z_s complex Gaussian of variance flux_s (independent per c, p, t),
n complex Gaussian with sigma per component, (u_a, v_a) = (x_a, y_a) f_c / c0
relative to the layout centroid.  This is the sign convention of Eq. 1: a
source at (l, m) has visibility phase exp(-2 pi i (u l + v m)).  The complex
value is quantised by rounding half away from zero and clipping to [-7, 7],
then packed as one byte: real part in the high nibble, imaginary part in the
low nibble, both two's complement.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

C0 = 299_792_458.0
SEED_BASE = 20230120
CI4_CLIP = 7
LWA_MIN_SPACING_M = 4.0


def seeds(cfg: int) -> dict:
    base = SEED_BASE + 100 * cfg
    return {"layout": base + 0, "sky": base + 1, "voltages": base + 2, "gains": base + 3}


# ---------------------------------------------------------------- layouts

def layout_disc(n: int, radius_m: float, rng: np.random.Generator,
                min_spacing_m: float = 0.0) -> np.ndarray:
    """n positions uniform in a disc, optional minimum spacing (sequential rejection)."""
    return _rejection(n, lambda k: _disc_draw(k, radius_m, rng), min_spacing_m)


def layout_ellipse(n: int, semi_x_m: float, semi_y_m: float, rng: np.random.Generator,
                   min_spacing_m: float = 0.0) -> np.ndarray:
    """n positions uniform in an axis-aligned ellipse with a minimum spacing."""
    def draw(k):
        pts = _disc_draw(k, 1.0, rng)
        pts[:, 0] *= semi_x_m
        pts[:, 1] *= semi_y_m
        return pts
    return _rejection(n, draw, min_spacing_m)


def _disc_draw(k: int, radius: float, rng: np.random.Generator) -> np.ndarray:
    r = radius * np.sqrt(rng.random(k))
    th = 2.0 * np.pi * rng.random(k)
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)


def _rejection(n, draw, min_spacing):
    out = np.empty((0, 2))
    tries = 0
    while len(out) < n:
        tries += 1
        if tries > 10000:
            raise RuntimeError("layout rejection sampling did not converge")
        cand = draw(256)
        for p in cand:
            if len(out) == n:
                break
            if min_spacing > 0 and len(out):
                d2 = np.sum((out - p) ** 2, axis=1)
                if np.min(d2) < min_spacing ** 2:
                    continue
            out = np.vstack([out, p[None, :]])
    return np.ascontiguousarray(out, dtype=np.float64)


# ---------------------------------------------------------------- kernel / gains

def gaussian_kernel(K: int) -> np.ndarray:
    """K x K real Gaussian illumination kernel, sigma = (K-1)/4 cells, sum = 1.

    Returned as complex64 [K][K]; index [dy + (K-1)/2][dx + (K-1)/2].
    K = 1 gives the single-cell kernel W = 1.
    """
    if K % 2 != 1:
        raise ValueError("K must be odd")
    h = (K - 1) // 2
    if K == 1:
        return np.ones((1, 1), np.complex64)
    sigma = (K - 1) / 4.0
    d = np.arange(-h, h + 1, dtype=np.float64)
    w = np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / (2 * sigma ** 2))
    w /= w.sum()
    return w.astype(np.complex64)


def antenna_kernels(A: int, K: int, rng: np.random.Generator) -> np.ndarray:
    """Per-antenna kernels complex64 [A][K][K]: Gaussians whose width varies by
    +-20 % between antennas, with a small random phase gradient (heterogeneous
    beams / A-projection), each normalised to sum 1 in amplitude."""
    h = (K - 1) // 2
    d = np.arange(-h, h + 1, dtype=np.float64)
    out = np.empty((A, K, K), np.complex64)
    for a in range(A):
        sigma = max((K - 1) / 4.0, 0.5) * rng.uniform(0.8, 1.2)
        w = np.exp(-(d[:, None] ** 2 + d[None, :] ** 2) / (2 * sigma ** 2))
        w /= w.sum()
        gx, gy = rng.uniform(-0.3, 0.3, 2)
        out[a] = w * np.exp(1j * (gx * d[None, :] + gy * d[:, None]))
    return out


def random_gains(C: int, A: int, P: int, rng: np.random.Generator) -> np.ndarray:
    """complex64 [C][A][P] with |g| ~ U[0.8, 1.2] and arg g ~ U[0, 2 pi)."""
    amp = rng.uniform(0.8, 1.2, size=(C, A, P))
    ph = rng.uniform(0.0, 2 * np.pi, size=(C, A, P))
    return (amp * np.exp(1j * ph)).astype(np.complex64)


# ---------------------------------------------------------------- voltages

def pack_ci4(re: np.ndarray, im: np.ndarray) -> np.ndarray:
    """Pack integer parts in [-8, 7] into bytes: high nibble = re, low = im."""
    re = np.asarray(re, np.int64)
    im = np.asarray(im, np.int64)
    if re.min(initial=0) < -8 or re.max(initial=0) > 7 or im.min(initial=0) < -8 or im.max(initial=0) > 7:
        raise ValueError("ci4 parts must lie in [-8, 7]")
    return (((re & 0xF) << 4) | (im & 0xF)).astype(np.uint8)


def quantise(x: np.ndarray) -> np.ndarray:
    """Round half away from zero and clip to [-7, 7]."""
    q = np.sign(x) * np.floor(np.abs(x) + 0.5)
    return np.clip(q, -CI4_CLIP, CI4_CLIP).astype(np.int64)


def sky_voltages(ant_xy: np.ndarray, freq_hz: np.ndarray, T: int, P: int,
                 src_lm: np.ndarray, src_flux: np.ndarray, noise_sigma: float,
                 rng: np.random.Generator) -> np.ndarray:
    """Packed ci4 voltages uint8 [T][C][A][P] from point sources plus noise."""
    A = ant_xy.shape[0]
    C = len(freq_hz)
    xy = ant_xy - ant_xy.mean(axis=0)
    out = np.empty((T, C, A, P), np.uint8)
    S = len(src_flux)
    amp = np.sqrt(np.asarray(src_flux, np.float64) / 2.0)
    for c in range(C):
        uv = xy * (freq_hz[c] / C0)                        # wavelengths
        phase = np.exp(-2j * np.pi * (np.outer(src_lm[:, 0], uv[:, 0])
                                      + np.outer(src_lm[:, 1], uv[:, 1])))  # [S][A]
        for p in range(P):
            z = (rng.standard_normal((T, S)) + 1j * rng.standard_normal((T, S))) * amp
            sig = z @ phase if S else np.zeros((T, A), np.complex128)
            nre = rng.standard_normal((T, A), dtype=np.float32) * noise_sigma
            nim = rng.standard_normal((T, A), dtype=np.float32) * noise_sigma
            out[:, c, :, p] = pack_ci4(quantise(sig.real + nre), quantise(sig.imag + nim))
    return out


def geometric_delays(ant_xy: np.ndarray, T: int, l0: float = 0.3, m0: float = -0.2,
                     dl: float = 1e-4, dm: float = 5e-5) -> np.ndarray:
    """[T][A] float64 geometric delays (s) towards a phase centre that drifts
    as the sky turns: (l, m)(t) = (l0 + t dl, m0 + t dm).  Positions are taken
    relative to the layout centroid; an antenna further along the direction
    sees the wavefront earlier, tau_a(t) = -(x_a l(t) + y_a m(t)) / c0."""
    xy = np.asarray(ant_xy, np.float64)
    xy = xy - xy.mean(axis=0)
    t = np.arange(T, dtype=np.float64)
    l = l0 + dl * t
    m = m0 + dm * t
    return -(np.outer(l, xy[:, 0]) + np.outer(m, xy[:, 1])) / C0


def random_ci4(shape, rng: np.random.Generator, lo: int = -7, hi: int = 7) -> np.ndarray:
    """Uniform random packed ci4 bytes with parts in [lo, hi]."""
    re = rng.integers(lo, hi + 1, size=shape)
    im = rng.integers(lo, hi + 1, size=shape)
    return pack_ci4(re, im)


# ---------------------------------------------------------------- workloads

@dataclass
class Workload:
    name: str
    ant_xy: np.ndarray            # float64 [A][2] metres
    n_pol: int
    kernel: np.ndarray            # complex64 [K][K]
    grid_n: np.ndarray            # int32 [C]
    freq_hz: np.ndarray           # float64 [C]
    du: float                     # cell size in wavelengths
    T: int
    v: np.ndarray                 # uint8 [T][C][A][P]
    gains: np.ndarray | None      # complex64 [C][A][P] or None (unit)
    meta: dict = field(default_factory=dict)

    @property
    def A(self):
        return self.ant_xy.shape[0]

    @property
    def C(self):
        return len(self.freq_hz)

    @property
    def K(self):
        return self.kernel.shape[0]

    @property
    def spectra(self):
        return self.T * self.C * self.n_pol


def select_channels(wl: Workload, channels) -> Workload:
    """The same workload restricted to the given channels (in that order):
    voltages, gains, grid sides and frequencies are sliced, nothing is redrawn."""
    ch = np.asarray(list(channels), np.int64)
    if ch.size == 0:
        raise ValueError("select_channels needs at least one channel")
    return Workload(f"{wl.name}[ch {ch[0]}..{ch[-1]}]", wl.ant_xy, wl.n_pol, wl.kernel,
                    np.ascontiguousarray(wl.grid_n[ch]), np.ascontiguousarray(wl.freq_hz[ch]), wl.du, wl.T,
                    np.ascontiguousarray(wl.v[:, ch]),
                    None if wl.gains is None else np.ascontiguousarray(wl.gains[ch]), dict(wl.meta))


def _lm_uniform_disc(n, rmax, rng):
    r = rmax * np.sqrt(rng.random(n))
    th = 2 * np.pi * rng.random(n)
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)


def tiny(T: int = 64, seed_cfg: int = 1) -> Workload:
    """16 single-pol antennas in a 20 m-radius disc, 4 channels at 40-40.75 MHz,
    3x3 Gaussian kernel, 32x32 grid, one point source in noise, unit gains."""
    s = seeds(seed_cfg)
    ant = layout_disc(16, 20.0, np.random.default_rng(s["layout"]))
    freq = 40.0e6 + 0.25e6 * np.arange(4)
    rs = np.random.default_rng(s["sky"])
    lm = _lm_uniform_disc(1, 0.7, rs)
    v = sky_voltages(ant, freq, T, 1, lm, np.array([1.0]), 2.0,
                     np.random.default_rng(s["voltages"]))
    return Workload("tiny-16ant-32grid", ant, 1, gaussian_kernel(3),
                    np.full(4, 32, np.int32), freq, 0.5, T, v, None,
                    {"src_lm": lm, "src_flux": [1.0]})


def lwa(T: int = 1000, C: int = 64, seed_cfg: int = 2, with_gains: bool = True,
        first_channel: int = 0) -> Workload:
    """LWA-station-like: 256 dual-pol antennas in a 110x100 m ellipse (min spacing
    4 m; random sequential packing jams below 256 dipoles at 5 m), C channels of 25 kHz from 60 MHz, 5x5 kernel, 128x128 grid, three point
    sources (1.0/0.3/0.1) plus a diffuse Gaussian sky (256 components, sigma 0.3,
    total flux 0.5), noise sigma 2, random per-(c,a,p) gains."""
    s = seeds(seed_cfg)
    ant = layout_ellipse(256, 55.0, 50.0, np.random.default_rng(s["layout"]), LWA_MIN_SPACING_M)
    freq = 60.0e6 + 25.0e3 * (first_channel + np.arange(C))
    rs = np.random.default_rng(s["sky"])
    lm_pts = _lm_uniform_disc(3, 0.7, rs)
    lm_diff = rs.normal(0.0, 0.3, size=(256, 2))
    lm_diff = lm_diff[np.hypot(lm_diff[:, 0], lm_diff[:, 1]) < 0.95][:256]
    lm = np.vstack([lm_pts, lm_diff])
    flux = np.concatenate([[1.0, 0.3, 0.1], np.full(len(lm_diff), 0.5 / len(lm_diff))])
    v = sky_voltages(ant, freq, T, 2, lm, flux, 2.0, np.random.default_rng(s["voltages"] + 7919 * first_channel))
    g = random_gains(C, 256, 2, np.random.default_rng(s["gains"] + 7919 * first_channel)) if with_gains else None
    return Workload(f"lwa-256ant-{C}ch-128grid-{T}t", ant, 2, gaussian_kernel(5),
                    np.full(C, 128, np.int32), freq, 0.5, T, v, g,
                    {"src_lm": lm_pts, "src_flux": [1.0, 0.3, 0.1]})


def uneven(T: int = 1000, C: int = 192, seed_cfg: int = 4) -> Workload:
    """192 channels evenly spaced over 30-80 MHz in three groups of 64 whose grid
    side follows frequency (64, 96, 128); the LWA layout and sky of `lwa`."""
    s = seeds(seed_cfg)
    ant = layout_ellipse(256, 55.0, 50.0, np.random.default_rng(seeds(2)["layout"]), LWA_MIN_SPACING_M)
    freq = np.linspace(30.0e6, 80.0e6, C)
    grid = np.where(freq < 30e6 + 50e6 / 3, 64, np.where(freq < 30e6 + 100e6 / 3, 96, 128)).astype(np.int32)
    rs = np.random.default_rng(s["sky"])
    lm_pts = _lm_uniform_disc(3, 0.7, rs)
    lm_diff = rs.normal(0.0, 0.3, size=(256, 2))
    lm_diff = lm_diff[np.hypot(lm_diff[:, 0], lm_diff[:, 1]) < 0.95][:256]
    lm = np.vstack([lm_pts, lm_diff])
    flux = np.concatenate([[1.0, 0.3, 0.1], np.full(len(lm_diff), 0.5 / len(lm_diff))])
    v = sky_voltages(ant, freq, T, 2, lm, flux, 2.0, np.random.default_rng(s["voltages"]))
    g = random_gains(C, 256, 2, np.random.default_rng(s["gains"]))
    return Workload(f"uneven-256ant-{C}ch-64/96/128grid-{T}t", ant, 2, gaussian_kernel(5),
                    grid, freq, 0.5, T, v, g, {"src_lm": lm_pts})


def dense(T: int = 500, C: int = 256, seed_cfg: int = 5) -> Workload:
    """2048 dual-pol antennas in a 350 m-diameter disc (min spacing 3 m), C
    channels of 25 kHz centred on 50 MHz, 7x7 kernel, 512x512 grid, ten point
    sources with log-uniform flux in [0.01, 1]."""
    s = seeds(seed_cfg)
    ant = layout_disc(2048, 175.0, np.random.default_rng(s["layout"]), 3.0)
    freq = 50.0e6 + 25.0e3 * (np.arange(C) - C // 2)
    rs = np.random.default_rng(s["sky"])
    lm = _lm_uniform_disc(10, 0.7, rs)
    flux = np.exp(rs.uniform(np.log(0.01), np.log(1.0), 10))
    v = sky_voltages(ant, freq, T, 2, lm, flux, 2.0, np.random.default_rng(s["voltages"]))
    g = random_gains(C, 2048, 2, np.random.default_rng(s["gains"]))
    return Workload(f"dense-2048ant-{C}ch-512grid-{T}t", ant, 2, gaussian_kernel(7),
                    np.full(C, 512, np.int32), freq, 0.5, T, v, g, {"src_lm": lm})


def random_small(A: int, P: int, C: int, T: int, N: int, K: int, seed: int,
                 spread_cells: float | None = None, gains: bool = True,
                 du: float = 0.5, f0: float = 50e6, full_range: bool = False) -> Workload:
    """Small random case for parity/property tests: A antennas uniform in a disc
    sized to spread over about `spread_cells` cells at f0, uniform random ci4
    (parts in [-7, 7]; with full_range every byte value 0..255 is equally
    likely, -8 included, and the first 256 bytes of the voltage array are the
    256 values in order, so each one occurs)."""
    rng = np.random.default_rng(seed)
    lam = C0 / f0
    spread = spread_cells if spread_cells is not None else N / 2 - K
    radius = 0.5 * spread * du * lam
    ant = layout_disc(A, radius, rng)
    freq = f0 + 25e3 * np.arange(C)
    v = random_ci4((T, C, A, P), rng, lo=-8 if full_range else -7)
    if full_range:
        flat = v.reshape(-1)
        n = min(256, flat.size)
        flat[:n] = np.arange(n, dtype=np.uint8)
    g = random_gains(C, A, P, rng) if gains else None
    kern = gaussian_kernel(K)
    if K > 1:
        # a non-symmetric complex kernel exercises conjugation / orientation
        kern = (kern * np.exp(1j * 0.3 * np.arange(K)[None, :] - 1j * 0.2 * np.arange(K)[:, None])).astype(np.complex64)
    return Workload(f"random-A{A}-P{P}-C{C}-T{T}-N{N}-K{K}", ant, P, kern,
                    np.full(C, N, np.int32), freq, du, T, v, g, {})
