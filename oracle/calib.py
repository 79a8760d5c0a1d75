"""FP64 oracle for the E-field-domain gain solver.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only callers; the CUDA library never imports it and
shares no code with it.

Sec. 1 cites a feedback calibration scheme for EPIC that works on the antenna
E-fields (EPICal) and Sec. 5 lists real-time calibration as future work; the
paper gives no algorithm, so this restates a single-calibrator solver in that
spirit (the readings are in the design notes):

  phi_a       = exp(-2 pi i (kx_a lx + ky_a ly) / N), the calibrator's geometric
                phase at antenna a's cell k_a for a source at image offset
                (lx, ly) = (l N du, m N du) pixels (same sign convention as the
                imaging oracle: such a source appears at +(lx, ly))
  per (channel, polarisation), starting from g = 1 and for each iteration:
  E(t)        = (1/A) sum_a g_a e_a(t) conj(phi_a)      beamformed calibrator field
  g_a        <- sum_t E(t) phi_a conj(e_a(t)) / sum_t |e_a(t)|^2
                (least squares g_a e_a(t) ~ E(t) phi_a; 0 when e_a is all zero)
  normalise   antenna 0's phase to 0 (when g_0 != 0), then the RMS |g| to 1

The iteration needs the unit-gain beam to see the calibrator: when the
instrumental gains sum to zero, E vanishes and the exact update is g = 0 (in
floating point the phases' rounding leaves a residue that the normalisation
would blow up, so callers avoid that degenerate case).
"""
from __future__ import annotations

import numpy as np


def ci4_complex(v):
    """uint8 ci4 bytes -> complex128 (high nibble real, low nibble imaginary, two's complement)."""
    b = np.asarray(v, np.uint8).astype(np.int16)
    re = ((b >> 4) & 0xF)
    im = b & 0xF
    re = np.where(re >= 8, re - 16, re)
    im = np.where(im >= 8, im - 16, im)
    return re + 1j * im


def cal_phases(cells, grid_n, l, m, du):
    """[C][A] complex phases phi_a of the calibrator direction (l, m) per channel."""
    cells = np.asarray(cells, np.float64)
    C, A, _ = cells.shape
    out = np.zeros((C, A), np.complex128)
    for c in range(C):
        N = float(grid_n[c])
        lx, ly = l * N * du, m * N * du
        out[c] = np.exp(-2j * np.pi * (cells[c, :, 0] * lx + cells[c, :, 1] * ly) / N)
    return out


def solve_gains(v, cells, grid_n, l, m, du, n_iter):
    """v [T][C][A][P] ci4 -> gains [C][A][P] complex128 by the iteration above."""
    e = ci4_complex(v)                       # [T][C][A][P]
    T, C, A, P = e.shape
    phi = cal_phases(cells, grid_n, l, m, du)
    g = np.ones((C, A, P), np.complex128)
    for c in range(C):
        for p in range(P):
            ec = e[:, c, :, p]                    # [T][A]
            den = np.sum(np.abs(ec) ** 2, axis=0)
            gp = np.ones(A, np.complex128)
            for _ in range(n_iter):
                E = (ec * (gp * np.conj(phi[c]))[None, :]).sum(axis=1) / A          # [T]
                num = phi[c] * np.sum(E[:, None] * np.conj(ec), axis=0)
                gp = np.where(den > 0, num / np.where(den > 0, den, 1.0), 0.0)
                if gp[0] != 0:
                    gp = gp * np.conj(gp[0]) / abs(gp[0])
                rms = np.sqrt(np.mean(np.abs(gp) ** 2))
                if rms > 0:
                    gp = gp / rms
            g[c, :, p] = gp
    return g
