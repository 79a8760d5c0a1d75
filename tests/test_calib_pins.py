"""Pins of the gain-solver oracle (E-field-domain single-calibrator solver in the
spirit of the EPICal scheme Sec. 1 cites): exact recovery from an integer
construction, the calibrated fixed point, invariances, and the calibrated image."""
import numpy as np
import pytest

import oracle
from oracle import calib
from paper_2301_09662_gb300 import synth


def _exact_case(n_sources_noise=False, seed=3):
    """Quarter-field calibrator (phi_a = (-i)^(kx+ky), integer-valued), Gaussian-integer
    instrumental gains G_a and signal s(t): e_a(t) = G_a s(t) phi_a is exact ci4."""
    N, A, T, C, P = 32, 14, 9, 2, 2
    wl = synth.random_small(A=A, P=P, C=C, T=T, N=N, K=1, seed=seed, gains=False)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    rng = np.random.default_rng(seed)
    # instrumental gains with non-negative real parts: their sum, the unit-gain beam's
    # response to the calibrator, can never vanish (the solver's one degenerate case)
    units = np.array([1, 1j, 1 + 1j, 1 - 1j])
    G = units[rng.integers(0, 4, (C, A, P))]
    s = rng.integers(-2, 3, (T, C, P)) + 1j * rng.integers(-2, 3, (T, C, P))
    s[0] = 2 + 1j                                     # the calibrator is never silent
    phi = (-1j) ** ((cells[:, :, 0] + cells[:, :, 1]) % 4)      # [C][A]
    e = s[:, :, None, :] * G[None] * phi[None, :, :, None]
    v = synth.pack_ci4(np.rint(e.real).astype(int), np.rint(e.imag).astype(int))
    l = m = 1.0 / (4.0 * wl.du)                       # (lx, ly) = (N/4, N/4) pixels
    return wl, cells, v, G, l, m


def _normalised(g):
    """antenna 0 phase 0, RMS amplitude 1, per (channel, polarisation)."""
    g = g * np.conj(g[:, :1, :]) / np.abs(g[:, :1, :])
    return g / np.sqrt(np.mean(np.abs(g) ** 2, axis=1, keepdims=True))


def test_phases_of_the_quarter_field_are_the_lattice_units():
    wl, cells, v, G, l, m = _exact_case()
    phi = calib.cal_phases(cells, wl.grid_n, l, m, wl.du)
    assert np.allclose(phi, (-1j) ** ((cells[:, :, 0] + cells[:, :, 1]) % 4), atol=1e-12)


@pytest.mark.parametrize("n_iter", [1, 3])
def test_exact_recovery_of_inverse_gains(n_iter):
    wl, cells, v, G, l, m = _exact_case()
    g = calib.solve_gains(v, cells, wl.grid_n, l, m, wl.du, n_iter)
    assert np.allclose(g, _normalised(1.0 / G), rtol=0, atol=1e-12)


def test_calibrated_input_is_a_fixed_point():
    wl, cells, v, G, l, m = _exact_case()
    e = calib.ci4_complex(v) / G[None]               # remove the instrument: exact Gaussian integers
    v0 = synth.pack_ci4(np.rint(e.real).astype(int), np.rint(e.imag).astype(int))
    g = calib.solve_gains(v0, cells, wl.grid_n, l, m, wl.du, 2)
    assert np.allclose(g, 1.0, atol=1e-12)


def test_antenna_permutation_equivariance():
    wl, cells, v, G, l, m = _exact_case(seed=5)
    g = calib.solve_gains(v, cells, wl.grid_n, l, m, wl.du, 2)
    perm = np.r_[0, np.random.default_rng(1).permutation(np.arange(1, wl.A))]   # keep the reference
    gp = calib.solve_gains(v[:, :, perm], cells[:, perm], wl.grid_n, l, m, wl.du, 2)
    assert np.allclose(gp, g[:, perm], atol=1e-12)


def test_solved_gains_focus_the_calibrator():
    """With the solved gains every antenna's corrected voltage is kappa s(t) phi_a (kappa
    = g_a G_a, common), so the O1 image of the calibrator through a point kernel
    (W = 1) is the closed form |kappa|^2 (A^2 - A) sum_t |s_t|^2 at its pixel."""
    wl, cells, v, G, l, m = _exact_case(seed=7)
    g = calib.solve_gains(v, cells, wl.grid_n, l, m, wl.du, 2)
    kappa = g * G                                     # [C][A][P], constant over a
    assert np.allclose(kappa, kappa[:, :1, :], atol=1e-12)
    e = calib.ci4_complex(v)
    s2 = np.sum(np.abs(e[:, :, 0, :] / (G[None, :, 0, :] * 1.0)) ** 2, axis=0)   # sum_t |s_t|^2 per (c, p)
    img = oracle.split_channels(oracle.epic_direct(v, g, cells, wl.grid_n, np.ones((1, 1), np.complex64)),
                                wl.grid_n, 2)
    N = wl.grid_n[0]
    i = j = N // 2 + N // 4
    A = wl.A
    for c in range(wl.C):
        XX = img[c][0].real
        expect = abs(kappa[c, 0, 0]) ** 2 * (A * A - A) * s2[c, 0]
        assert abs(XX[i, j] - expect) < 1e-10 * expect
        assert np.unravel_index(np.argmax(XX), XX.shape) == (i, j)


def test_degenerate_unit_gain_beam_gives_zero_gains():
    """When the instrumental gains sum to zero the calibrator's field beamformed with
    unit gains vanishes: the first update is exactly zero (checked on lattice phases
    built without rounding), and the solver must not invent gains from noise."""
    N, A, T, C, P = 32, 4, 5, 1, 1
    wl = synth.random_small(A=A, P=P, C=C, T=T, N=N, K=1, seed=9, gains=False)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    G = np.array([1, -1, 1j, -1j]).reshape(1, A, 1)
    s = np.array([1 + 1j, 2, -1, 1j, 2 - 1j]).reshape(T, 1, 1)
    phi = (-1j) ** ((cells[:, :, 0] + cells[:, :, 1]) % 4)
    e = s[:, :, None, :] * G[None] * phi[None, :, :, None]
    ec = e[:, 0, :, 0]
    E = (ec * np.conj(phi[0])[None, :]).sum(axis=1) / A         # exact lattice phases
    assert np.all(E == 0)
