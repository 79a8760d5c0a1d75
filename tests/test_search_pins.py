"""Pins of the transient-search oracle (de-dispersion and single-pulse search
on the image cube; Sec. 4 pulsar and giant-pulse observations, Sec. 5) against
closed forms and brute force."""
import numpy as np
import pytest

from oracle import search


def test_dispersion_delay_textbook_value():
    # DM = 1 pc cm^-3 delays 500 MHz by 4.148808 ms x (1/0.25 - 1) = 12.446 ms behind 1 GHz
    s = search.dm_shifts([500e6, 1000e6], 1e-3, [1.0, 0.0, 2.0])
    assert s.tolist() == [[12, 0], [0, 0], [25, 0]]
    s = search.dm_shifts([500e6, 1000e6], 1e-4, [1.0])
    assert s.tolist() == [[124, 0]]            # 124.46 samples of 0.1 ms, rounded


def test_shifts_monotone_and_zero_at_top():
    f = 42.1e6 + 25e3 * np.arange(72)
    s = search.dm_shifts(f, 0.04, np.arange(0, 25.6, 0.2))
    assert np.all(s[:, -1] == 0)
    assert np.all(np.diff(s, axis=1) <= 0)     # lower frequency, later arrival
    assert np.all(np.diff(s, axis=0) >= 0)     # larger DM, later arrival
    assert s[0].max() == 0


def test_zero_dm_is_channel_sum():
    rng = np.random.default_rng(1)
    cube = rng.normal(size=(40, 7, 11))
    dd = search.dedisperse(cube, np.zeros((1, 7), np.int64))
    assert np.allclose(dd[0], cube.sum(axis=1), rtol=0, atol=1e-12)


def test_dispersed_impulse_is_collected_at_its_dm():
    f = 42.1e6 + 25e3 * np.arange(24)
    dms = np.arange(0, 20, 0.5)
    sh = search.dm_shifts(f, 0.04, dms)
    true = 27
    T, P, t0, pix = 400, 5, 60, 3
    cube = np.zeros((T, len(f), P))
    for c in range(len(f)):
        cube[t0 + sh[true, c], c, pix] = 2.0
    dd = search.dedisperse(cube, sh)
    assert dd[true, t0, pix] == 2.0 * len(f)
    # every other trial with a different sweep collects less at its best time
    for d in range(len(dms)):
        if not np.array_equal(sh[d], sh[true]):
            assert dd[d, :, pix].max() < 2.0 * len(f)
    snr, bt, bw = search.single_pulse(dd, [1, 2, 4])
    assert np.unravel_index(np.argmax(snr[:, pix]), snr[:, pix].shape)[0] in \
        [d for d in range(len(dms)) if np.array_equal(sh[d], sh[true])]
    assert bt[true, pix] == t0 and bw[true, pix] == 1


@pytest.mark.parametrize("L,w0,t0", [(50, 4, 10), (128, 1, 0), (77, 8, 69), (64, 16, 20)])
def test_boxcar_closed_form(L, w0, t0):
    # one boxcar of height a, width w0 on zero: mu = a w0/L, sigma^2 = a^2 (w0/L)(1 - w0/L),
    # so the matched window scores (a w0 (1 - w0/L)) / (sigma sqrt(w0)) = sqrt(L - w0)
    x = np.zeros((1, L, 1))
    x[0, t0:t0 + w0, 0] = 3.7
    snr, bt, bw = search.single_pulse(x, [1, 2, 4, 8, 16, 32])
    assert abs(snr[0, 0] - np.sqrt(L - w0)) < 1e-12
    assert (bt[0, 0], bw[0, 0]) == (t0, w0)


def test_snr_affine_invariance_and_flat_series():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(3, 90, 4))
    a = search.single_pulse(x, [1, 2, 4, 8])
    b = search.single_pulse(5.5 * x - 17.0, [1, 2, 4, 8])
    assert np.allclose(a[0], b[0], rtol=1e-12, atol=1e-12)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    flat = np.full((1, 30, 2), 4.0)
    s, t, w = search.single_pulse(flat, [2, 4])
    assert np.all(s == 0) and np.all(t == 0) and np.all(w == 2)


def test_candidates_threshold():
    snr = np.array([[1.0, 7.0], [6.5, 2.0]])
    assert search.candidates(snr, 6.5) == [(0, 1), (1, 0)]
