"""FP64 oracle for the downstream transient search on the image cube.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only callers; the CUDA library never imports it and
shares no code with it.

What it computes (Sec. 4: light curves extracted per channel from the images,
the dispersive delay corrected across the band before integrating, and a
single-pulse search of the de-dispersed light curves; Sec. 5 names real-time
de-dispersion and transient detection as the next modules):

  dm_shifts     integer delay, in samples, of channel c at trial DM d relative to
                the highest frequency:  s = floor(k_DM DM (f_c^-2 - f_max^-2) / dt + 1/2),
                f in MHz, k_DM = 4.148808e3 s MHz^2 pc^-1 cm^3 (the cold-plasma
                dispersion constant; the paper does not print it)
  dedisperse    D[d][t][p] = sum_c I[t + s[d][c]][c][p],  t < T - max s
  single_pulse  per (d, p): mu, sigma = mean and population standard deviation
                of D[d][:, p]; boxcar S/N(t, w) = (sum_{k<w} D[t+k] - w mu) /
                (sigma sqrt(w)) for t <= T_out - w; the best (S/N, t, w), first
                in (w ascending, t ascending) order on ties; sigma = 0 gives
                S/N 0 at (t 0, the first width)
  candidates    the (d, p) whose best S/N reaches the threshold
"""
from __future__ import annotations

import numpy as np

K_DM = 4.148808e3


def dm_shifts(freq_hz, dt_s: float, dms) -> np.ndarray:
    """[n_dm][C] int64 delays in samples (>= 0) relative to the top channel."""
    f = np.asarray(freq_hz, np.float64) / 1e6
    fmax = np.max(f)
    out = np.zeros((len(dms), len(f)), np.int64)
    for i, dm in enumerate(np.asarray(dms, np.float64)):
        for c in range(len(f)):
            x = K_DM * dm * (1.0 / (f[c] * f[c]) - 1.0 / (fmax * fmax)) / dt_s
            out[i, c] = int(np.floor(x + 0.5))
    return out


def dedisperse(cube, shifts) -> np.ndarray:
    """cube [T][C][P] intensities -> [n_dm][T_out][P] FP64 sums along the dispersion sweeps."""
    x = np.asarray(cube, np.float64)
    T, C, P = x.shape
    smax = int(np.max(shifts)) if shifts.size else 0
    T_out = T - smax
    if T_out <= 0:
        raise ValueError("the largest delay leaves no complete sweep")
    out = np.zeros((shifts.shape[0], T_out, P), np.float64)
    for d in range(shifts.shape[0]):
        for c in range(C):
            s = int(shifts[d, c])
            out[d] += x[s:s + T_out, c, :]
    return out


def boxcar_snr(series, w: int) -> np.ndarray:
    """S/N of every width-w window of one series (FP64), by the definition above."""
    x = np.asarray(series, np.float64)
    mu = np.mean(x)
    sigma = np.sqrt(np.mean((x - mu) ** 2))
    L = len(x)
    sums = np.array([np.sum(x[t:t + w]) for t in range(L - w + 1)])
    if sigma == 0:
        return np.zeros(L - w + 1)
    return (sums - w * mu) / (sigma * np.sqrt(w))


def single_pulse(dd, widths):
    """dd [n_dm][T_out][P] -> best_snr [n_dm][P], best_t, best_w (first best in
    (w ascending, t ascending) order)."""
    x = np.asarray(dd, np.float64)
    n_dm, T_out, P = x.shape
    ws = sorted(int(w) for w in widths if int(w) <= T_out)
    if not ws:
        raise ValueError("no boxcar width fits the light curve")
    snr = np.zeros((n_dm, P))
    bt = np.zeros((n_dm, P), np.int64)
    bw = np.full((n_dm, P), ws[0], np.int64)
    for d in range(n_dm):
        for p in range(P):
            best, arg = -np.inf, (0, ws[0])
            for w in ws:
                s = boxcar_snr(x[d, :, p], w)
                t = int(np.argmax(s))
                if s[t] > best:
                    best, arg = s[t], (t, w)
            snr[d, p] = best if np.isfinite(best) else 0.0
            bt[d, p], bw[d, p] = arg
    return snr, bt, bw


def candidates(best_snr, threshold: float):
    """Sorted list of (dm index, pixel) whose best S/N reaches the threshold."""
    d, p = np.nonzero(np.asarray(best_snr) >= threshold)
    return sorted(zip(d.tolist(), p.tolist()))
