"""Pins for the FP64 oracle: each test ties it to something other than itself.

P1  the paper's equivalence (Eq. 2-4): EPIC direct image == FX-correlator image
P2  one antenna: nothing but the autocorrelation, which subtraction removes
P3  two antennas: a single fringe with a closed form
P4  zenith point source: closed-form peak at the centre pixel
P5  quarter-field point source: closed-form peak at l = (N/4, N/4)
P6  Parseval: image power without subtraction == N^2 x grid power
P7  brute-force DFT beamformer (sum over antennas, no grid, no FFT)
P8  invariances (antenna / time permutation, one-cell translation, XX/YY real,
    YX = conj(XY), gain scaling, MEAN flag, empty integration)
P9  the oracle's FFT vs a direct DFT and numpy.fft
P10 ci4 unpacking vs a table built from the definition
P11 antenna -> cell map (Sec. 3.1 nearest neighbour, reading 7) vs cell
    indices worked out by hand from the definition
"""
import os

import numpy as np
import pytest

import oracle
from paper_2301_09662_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def ci4_table():
    rows = np.loadtxt(os.path.join(GOLDEN, "ci4_table.txt"), dtype=int, comments="#")
    return rows[:, 1], rows[:, 2]


def unpack_np(v):
    re, im = ci4_table()
    return re[v] + 1j * im[v]


def what(W, N):
    """W^(l) = sum_d W(d) exp(+2 pi i d.l/N) on the shifted pixel layout (numpy)."""
    K = W.shape[0]
    h = (K - 1) // 2
    l = np.arange(N) - N // 2
    d = np.arange(-h, h + 1)
    ex = np.exp(2j * np.pi * np.outer(d, l) / N)          # [dx][lx]
    # out[i][j] = sum_{dy,dx} W[dy][dx] e^{2 pi i (dx lx_j + dy ly_i)/N}
    return np.einsum("yx,yi,xj->ij", W.astype(np.complex128), ex, ex)


def beamformer_image(v, g, cells, N, W, autosub=True):
    """Brute-force Eq. 4 for one channel: F(l) = W^(l) sum_a e~_a exp(2 pi i k_a.l/N)."""
    T, A, P = v.shape
    e = unpack_np(v)
    if g is not None:
        e = e * g[None]
    l = np.arange(N) - N // 2
    ph_x = np.exp(2j * np.pi * np.outer(cells[:, 0], l) / N)  # [a][lx]
    ph_y = np.exp(2j * np.pi * np.outer(cells[:, 1], l) / N)  # [a][ly]
    Wh = what(W, N)
    F = np.einsum("tap,ai,aj->tpij", e, ph_y, ph_x) * Wh[None, None]
    pq = [(0, 0), (1, 1), (0, 1), (1, 0)] if P == 2 else [(0, 0)]
    out = []
    for p, q in pq:
        s = np.sum(F[:, p] * np.conj(F[:, q]), axis=0)
        if autosub:
            auto = np.sum(e[:, :, p] * np.conj(e[:, :, q]))
            s = s - auto * np.abs(Wh) ** 2
        out.append(s)
    return np.array(out)


def rel_err(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# ------------------------------------------------------------------ P10

def test_p10_ci4_all_bytes():
    re, im = ci4_table()
    for b in range(256):
        assert oracle.ci4_unpack(b) == (re[b], im[b]), b


def test_p10_synth_pack_roundtrip():
    re, im = ci4_table()
    parts = np.arange(-8, 8)
    R, I = np.meshgrid(parts, parts, indexing="ij")
    b = synth.pack_ci4(R.ravel(), I.ravel())
    assert np.array_equal(re[b], R.ravel()) and np.array_equal(im[b], I.ravel())


# ------------------------------------------------------------------ P9

@pytest.mark.parametrize("n", [2, 3, 8, 12, 16, 32, 48, 96, 128])
@pytest.mark.parametrize("sign", [+1, -1])
def test_p9_fft_vs_direct_dft(n, sign):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    k = np.arange(n)
    D = np.exp(sign * 2j * np.pi * np.outer(k, k) / n)
    ref = D @ x
    assert rel_err(oracle.fft1d(x, sign), ref) < 1e-13
    np_ref = np.fft.ifft(x) * n if sign > 0 else np.fft.fft(x)
    assert rel_err(oracle.fft1d(x, sign), np_ref) < 1e-13


@pytest.mark.parametrize("N", [8, 32, 96])
def test_p9_ifft2_vs_numpy(N):
    rng = np.random.default_rng(N)
    g = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    assert rel_err(oracle.ifft2(g), np.fft.ifft2(g) * N * N) < 1e-13


# ------------------------------------------------------------------ P1

P1_CASES = [(A, N, K, P) for A in (2, 3, 5) for N in (8, 16) for K in (1, 3) for P in (1, 2)]


@pytest.mark.parametrize("A,N,K,P", P1_CASES)
def test_p1_direct_equals_fx(A, N, K, P):
    wl = synth.random_small(A=A, P=P, C=2, T=5, N=N, K=K, seed=100 * A + N + K + P)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    o1 = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, wl.kernel)
    o2 = oracle.epic_fx(wl.v, wl.gains, cells, wl.grid_n, wl.kernel)
    assert rel_err(o1, o2) < 1e-12


def test_p1_tiny_workload_direct_equals_fx():
    wl = synth.tiny()
    o1 = oracle.workload_image(wl, form="direct")
    o2 = oracle.workload_image(wl, form="fx")
    assert rel_err(o1, o2) < 1e-12


def test_p1_wraparound_footprint():
    """Footprints that cross the grid edge: both forms use the circular grid."""
    wl = synth.random_small(A=4, P=2, C=1, T=4, N=8, K=3, seed=7)
    cells = np.array([[[0, 0], [7, 3], [4, 7], [2, 5]]], np.int32)
    o1 = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, wl.kernel)
    o2 = oracle.epic_fx(wl.v, wl.gains, cells, wl.grid_n, wl.kernel)
    assert rel_err(o1, o2) < 1e-12


# ------------------------------------------------------------------ P2

@pytest.mark.parametrize("P", [1, 2])
def test_p2_single_antenna(P):
    wl = synth.random_small(A=1, P=P, C=2, T=9, N=16, K=3, seed=3)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    o = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, wl.kernel)
    raw = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, wl.kernel, oracle.NO_AUTOSUB)
    assert np.max(np.abs(o)) <= 1e-12 * np.max(np.abs(raw))
    # without subtraction: XX = sum_t |e~|^2 |W^(l)|^2
    for c, (img, rimg) in enumerate(zip(oracle.split_channels(o, wl.grid_n, P),
                                        oracle.split_channels(raw, wl.grid_n, P))):
        e = unpack_np(wl.v[:, c, 0, 0]) * wl.gains[c, 0, 0]
        ref = np.sum(np.abs(e) ** 2) * np.abs(what(wl.kernel, 16)) ** 2
        assert rel_err(rimg[0], ref) < 1e-13


# ------------------------------------------------------------------ P3

@pytest.mark.parametrize("K", [1, 3, 5])
def test_p3_two_antenna_fringe(K):
    N = 16
    wl = synth.random_small(A=2, P=2, C=1, T=11, N=N, K=K, seed=30 + K)
    cells = np.array([[[5, 6], [9, 8]]], np.int32)
    o = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, wl.kernel).reshape(4, N, N)
    e = unpack_np(wl.v[:, 0]) * wl.gains[0][None]           # [t][a][p]
    d = cells[0, 0] - cells[0, 1]
    l = np.arange(N) - N // 2
    ph = np.exp(2j * np.pi * (d[0] * l[None, :] + d[1] * l[:, None]) / N)   # [i][j]
    W2 = np.abs(what(wl.kernel, N)) ** 2
    for ix, (p, q) in enumerate([(0, 0), (1, 1), (0, 1), (1, 0)]):
        V12 = np.sum(e[:, 0, p] * np.conj(e[:, 1, q]))
        V21 = np.sum(e[:, 1, p] * np.conj(e[:, 0, q]))
        ref = W2 * (V12 * ph + V21 * np.conj(ph))
        assert np.max(np.abs(o[ix] - ref)) < 1e-13 * np.max(np.abs(ref))


# ------------------------------------------------------------------ P4 / P5

def _point_source_case(quarter):
    N, K, A, T = 32, 3, 12, 6
    wl = synth.random_small(A=A, P=1, C=1, T=T, N=N, K=K, seed=44, gains=False)
    wl.kernel = synth.gaussian_kernel(K)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    rng = np.random.default_rng(5)
    s_re = rng.integers(-7, 8, T)
    s_im = rng.integers(-7, 8, T)
    s = s_re + 1j * s_im
    n = (cells[0, :, 0] + cells[0, :, 1]) if quarter else np.zeros(A, int)
    rot = (-1j) ** n                                         # exact unit phases
    e = s[:, None] * rot[None, :]                            # [t][a]
    v = synth.pack_ci4(np.rint(e.real).astype(int), np.rint(e.imag).astype(int))
    wl.v = v.reshape(T, 1, A, 1)
    img = oracle.epic_direct(wl.v, None, cells, wl.grid_n, wl.kernel).reshape(N, N)
    return wl, img, s, N, A


def test_p4_zenith_point_source():
    wl, img, s, N, A = _point_source_case(quarter=False)
    expect = abs(np.sum(wl.kernel.astype(np.complex128))) ** 2 * (A * A - A) * np.sum(np.abs(s) ** 2)
    assert abs(img[N // 2, N // 2] - expect) < 1e-13 * expect
    assert np.unravel_index(np.argmax(img.real), img.shape) == (N // 2, N // 2)


def test_p5_quarter_field_point_source():
    wl, img, s, N, A = _point_source_case(quarter=True)
    i = j = N // 2 + N // 4
    W2 = np.abs(what(wl.kernel, N)) ** 2
    expect = W2[i, j] * (A * A - A) * np.sum(np.abs(s) ** 2)
    assert abs(img[i, j] - expect) < 1e-13 * expect
    # the normalised image (divide by the kernel taper) peaks at the source
    assert np.unravel_index(np.argmax(img.real / W2), img.shape) == (i, j)


# ------------------------------------------------------------------ P6

@pytest.mark.parametrize("P,K", [(1, 3), (2, 5)])
def test_p6_parseval(P, K):
    N = 16
    wl = synth.random_small(A=6, P=P, C=2, T=4, N=N, K=K, seed=60 + P)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    raw = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, wl.kernel, oracle.NO_AUTOSUB)
    energy = oracle.grid_energy(wl.v, wl.gains, cells, wl.grid_n, wl.kernel)
    for c, img in enumerate(oracle.split_channels(raw, wl.grid_n, P)):
        for p in range(P):
            tot = np.sum(img[p].real)
            assert abs(tot - N * N * energy[c, p]) < 1e-12 * abs(tot)


# ------------------------------------------------------------------ P7

@pytest.mark.parametrize("A,P,K,N", [(3, 1, 1, 8), (7, 2, 1, 16), (6, 2, 3, 16), (9, 2, 5, 32)])
def test_p7_brute_force_beamformer(A, P, K, N):
    wl = synth.random_small(A=A, P=P, C=2, T=5, N=N, K=K, seed=70 + A)
    if K == 1:
        wl.kernel = np.ones((1, 1), np.complex64)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    o = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, wl.kernel)
    for c, img in enumerate(oracle.split_channels(o, wl.grid_n, P)):
        ref = beamformer_image(wl.v[:, c], wl.gains[c], cells[c], N, wl.kernel)
        assert rel_err(img, ref) < 1e-12


# ------------------------------------------------------------------ P8

@pytest.fixture(scope="module")
def base_case():
    wl = synth.random_small(A=7, P=2, C=2, T=6, N=16, K=3, seed=80)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    o = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, wl.kernel)
    return wl, cells, o


def test_p8_antenna_permutation(base_case):
    wl, cells, o = base_case
    perm = np.random.default_rng(1).permutation(wl.A)
    o2 = oracle.epic_direct(wl.v[:, :, perm], wl.gains[:, perm], cells[:, perm], wl.grid_n, wl.kernel)
    assert rel_err(o2, o) < 1e-13


def test_p8_time_permutation(base_case):
    wl, cells, o = base_case
    perm = np.random.default_rng(2).permutation(wl.T)
    o2 = oracle.epic_direct(wl.v[perm], wl.gains, cells, wl.grid_n, wl.kernel)
    assert rel_err(o2, o) < 1e-13


def test_p8_translation_by_one_cell(base_case):
    wl, cells, o = base_case
    o2 = oracle.epic_direct(wl.v, wl.gains, cells + np.array([1, -1], np.int32), wl.grid_n, wl.kernel)
    assert rel_err(o2, o) < 1e-12


def test_p8_product_symmetries(base_case):
    wl, cells, o = base_case
    for img in oracle.split_channels(o, wl.grid_n, 2):
        assert np.all(img[0].imag == 0) and np.all(img[1].imag == 0)
        assert np.array_equal(img[3], np.conj(img[2]))


def test_p8_gain_scaling(base_case):
    wl, cells, o = base_case
    c = 1.7 - 0.4j
    o2 = oracle.epic_direct(wl.v, wl.gains.astype(np.complex128) * c, cells, wl.grid_n, wl.kernel)
    assert rel_err(o2, o * abs(c) ** 2) < 1e-13


def test_p8_mean_flag_and_empty(base_case):
    wl, cells, o = base_case
    om = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, wl.kernel, oracle.MEAN)
    assert rel_err(om * wl.T, o) < 1e-14
    oe = oracle.epic_direct(wl.v[:0], wl.gains, cells, wl.grid_n, wl.kernel)
    assert np.all(oe == 0)


# ------------------------------------------------------------------ per-antenna kernels (Eq. 3, W_a)

def beamformer_image_ak(v, g, cells, N, Wa):
    """Brute-force Eq. 4 with one kernel per antenna:
    F(l) = sum_a e~_a W^_a(l) exp(2 pi i k_a.l/N); autos = sum_a |e~_a|^2 |W^_a|^2."""
    T, A, P = v.shape
    e = unpack_np(v) * g[None]
    l = np.arange(N) - N // 2
    ph_x = np.exp(2j * np.pi * np.outer(cells[:, 0], l) / N)
    ph_y = np.exp(2j * np.pi * np.outer(cells[:, 1], l) / N)
    Wh = np.array([what(Wa[a], N) for a in range(A)])                 # [a][i][j]
    F = np.einsum("tap,ai,aj,aij->tpij", e, ph_y, ph_x, Wh)
    out = []
    for p, q in [(0, 0), (1, 1), (0, 1), (1, 0)]:
        s = np.sum(F[:, p] * np.conj(F[:, q]), axis=0)
        auto = np.einsum("ta,aij->ij", e[:, :, p] * np.conj(e[:, :, q]), np.abs(Wh) ** 2)
        out.append(s - auto)
    return np.array(out)


@pytest.mark.parametrize("A,K,N", [(3, 3, 16), (5, 5, 16), (7, 3, 32)])
def test_antenna_kernels_direct_equals_fx(A, K, N):
    wl = synth.random_small(A=A, P=2, C=2, T=5, N=N, K=K, seed=900 + A)
    Wa = synth.antenna_kernels(A, K, np.random.default_rng(A))
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    o1 = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, Wa)
    o2 = oracle.epic_fx(wl.v, wl.gains, cells, wl.grid_n, Wa)
    assert rel_err(o1, o2) < 1e-12
    raw1 = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, Wa, oracle.NO_AUTOSUB)
    raw2 = oracle.epic_fx(wl.v, wl.gains, cells, wl.grid_n, Wa, oracle.NO_AUTOSUB)
    assert rel_err(raw1, raw2) < 1e-12


def test_antenna_kernels_brute_force_beamformer():
    A, K, N = 6, 5, 32
    wl = synth.random_small(A=A, P=2, C=1, T=4, N=N, K=K, seed=910)
    Wa = synth.antenna_kernels(A, K, np.random.default_rng(1))
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    o = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, Wa).reshape(4, N, N)
    ref = beamformer_image_ak(wl.v[:, 0], wl.gains[0], cells[0], N, Wa)
    assert rel_err(o, ref) < 1e-12


def test_antenna_kernels_identical_reduce_to_shared_kernel():
    wl = synth.random_small(A=8, P=2, C=2, T=5, N=16, K=3, seed=920)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    Wa = np.repeat(wl.kernel[None], wl.A, axis=0)
    o_shared = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, wl.kernel)
    o_each = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, Wa)
    assert rel_err(o_each, o_shared) < 1e-13


def test_antenna_kernels_single_antenna_is_zero():
    wl = synth.random_small(A=1, P=2, C=1, T=6, N=16, K=5, seed=930)
    Wa = synth.antenna_kernels(1, 5, np.random.default_rng(2))
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    o = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, Wa)
    raw = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, Wa, oracle.NO_AUTOSUB)
    assert np.max(np.abs(o)) <= 1e-12 * np.max(np.abs(raw))


# ------------------------------------------------------------------ delay correction
# Sec. 2.2: a per-(t, antenna) geometric-delay phase exp(+2 pi i f_c tau_a(t))
# multiplies each voltage before gridding.

def _steered_case(time_varying):
    """Quarter-field source whose phase pattern (-i)^{(kx+ky) m_t} is undone by
    delays with f tau_a(t) = ((kx+ky) m_t mod 4) / 4: the corrected voltages are
    all s_t, so the image is the zenith closed form of P4."""
    N, K, A, T = 32, 3, 12, 6
    wl = synth.random_small(A=A, P=1, C=1, T=T, N=N, K=K, seed=44, gains=False)
    wl.kernel = synth.gaussian_kernel(K)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    rng = np.random.default_rng(6)
    s = rng.integers(-7, 8, T) + 1j * rng.integers(-7, 8, T)
    m = rng.integers(0, 4, T) if time_varying else np.ones(T, int)
    n = cells[0, :, 0] + cells[0, :, 1]
    e = s[:, None] * (-1j) ** (np.outer(m, n) % 4)
    v = synth.pack_ci4(np.rint(e.real).astype(int), np.rint(e.imag).astype(int)).reshape(T, 1, A, 1)
    f = wl.freq_hz[0]
    tau = (np.outer(m, n) % 4) / (4.0 * f)
    return wl, cells, v, tau, s, N, A


@pytest.mark.parametrize("time_varying", [False, True])
def test_delays_steer_source_to_phase_centre(time_varying):
    wl, cells, v, tau, s, N, A = _steered_case(time_varying)
    img = oracle.epic_direct(v, None, cells, wl.grid_n, wl.kernel, freq=wl.freq_hz, delays=tau).reshape(N, N)
    expect = abs(np.sum(wl.kernel.astype(np.complex128))) ** 2 * (A * A - A) * np.sum(np.abs(s) ** 2)
    assert abs(img[N // 2, N // 2] - expect) < 1e-12 * expect
    assert np.unravel_index(np.argmax(img.real), img.shape) == (N // 2, N // 2)
    # without the correction the source stays off centre
    raw = oracle.epic_direct(v, None, cells, wl.grid_n, wl.kernel).reshape(N, N)
    assert raw[N // 2, N // 2].real < 0.5 * expect


def test_delays_integer_turns_are_identity():
    wl = synth.random_small(A=7, P=2, C=1, T=5, N=16, K=3, seed=950)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    n = np.random.default_rng(3).integers(-5, 6, (wl.T, wl.A))
    tau = n / wl.freq_hz[0]
    o = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, wl.kernel, freq=wl.freq_hz, delays=tau)
    ref = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, wl.kernel)
    assert rel_err(o, ref) < 1e-12


def test_delays_constant_in_time_equal_gains():
    wl = synth.random_small(A=6, P=2, C=3, T=4, N=16, K=3, seed=960)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    tau_a = np.random.default_rng(4).uniform(-80e-9, 80e-9, wl.A)
    tau = np.repeat(tau_a[None], wl.T, axis=0)
    o = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, wl.kernel, freq=wl.freq_hz, delays=tau)
    g2 = wl.gains * np.exp(2j * np.pi * np.outer(wl.freq_hz, tau_a))[:, :, None]
    ref = oracle.epic_direct(wl.v, g2, cells, wl.grid_n, wl.kernel)
    assert rel_err(o, ref) < 1e-11


@pytest.mark.parametrize("A,N,K,P", [(5, 16, 3, 2), (8, 16, 1, 1)])
def test_delays_direct_equals_fx(A, N, K, P):
    wl = synth.random_small(A=A, P=P, C=2, T=5, N=N, K=K, seed=970 + A)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    tau = synth.geometric_delays(wl.ant_xy, wl.T, dl=3e-3, dm=-2e-3)
    o1 = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, wl.kernel, freq=wl.freq_hz, delays=tau)
    o2 = oracle.epic_fx(wl.v, wl.gains, cells, wl.grid_n, wl.kernel, freq=wl.freq_hz, delays=tau)
    assert rel_err(o1, o2) < 1e-12


def test_delays_leave_the_auto_term_unchanged():
    wl = synth.random_small(A=6, P=2, C=2, T=5, N=16, K=3, seed=980)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    tau = synth.geometric_delays(wl.ant_xy, wl.T, dl=2e-3)
    kw = dict(freq=wl.freq_hz, delays=tau)
    auto_d = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, wl.kernel, oracle.NO_AUTOSUB, **kw) - \
        oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, wl.kernel, **kw)
    auto = oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, wl.kernel, oracle.NO_AUTOSUB) - \
        oracle.epic_direct(wl.v, wl.gains, cells, wl.grid_n, wl.kernel)
    assert rel_err(auto_d, auto) < 1e-11


def test_geometric_delays_recipe():
    ant = np.array([[10.0, 0.0], [-10.0, 0.0], [0.0, 5.0], [0.0, -5.0]])
    tau = synth.geometric_delays(ant, 3, l0=0.5, m0=0.0, dl=0.0, dm=0.0)
    # the antenna at +x along l = 0.5 sees the wavefront 10 m * 0.5 / c0 earlier
    assert np.allclose(tau[:, 0], -5.0 / synth.C0, rtol=0, atol=1e-20)
    assert np.allclose(tau[:, 1], 5.0 / synth.C0, rtol=0, atol=1e-20)
    assert np.all(tau[:, 2:] == 0)


# ---------------------------------------------------------------- P11 cell map

C0 = 299_792_458.0

# Three antennas around the centroid (10, -4) m, at offsets that are exact in
# binary: in cells of 0.5 m (du = 0.5 at f = c0) they sit at (+1.5, +2.5),
# (-2.5, -1.5) and (+1, -1).  The x and y offsets differ (a swapped axis moves
# them), the half-cell offsets are ties (rounding must go away from zero), and
# the centroid is far from the origin (it must be subtracted).  Every quotient
# x f / (c0 du) below is exactly representable, so the expected cells are
# integers worked out by hand:
#   k = llround((x - x_c) f / (c0 du)) + N / 2, per axis.
P11_ANT = np.array([[10.75, -2.75], [8.75, -4.75], [10.5, -4.5]])
P11_CASES = [
    # (du, f (Hz), N, expected [A][2])
    (0.5, C0, 32, [[18, 19], [13, 14], [17, 15]]),            # ties at +-1.5, +-2.5
    (0.5, 2 * C0, 64, [[35, 37], [27, 29], [34, 30]]),        # offsets x2
    (0.5, C0 / 2, 16, [[9, 9], [7, 7], [9, 7]]),              # +-0.75, +-1.25, ties at +-0.5
    (0.25, C0, 32, [[19, 21], [11, 13], [18, 14]]),           # finer cells: offsets x2
    (0.25, 2 * C0, 64, [[38, 42], [22, 26], [36, 28]]),       # offsets x4
]


@pytest.mark.parametrize("du,f,N,expect", P11_CASES)
def test_p11_cell_map_by_hand(du, f, N, expect):
    cells = oracle.cell_map(P11_ANT, np.array([f]), np.array([N], np.int32), du)
    assert cells.shape == (1, 3, 2)
    assert cells[0].tolist() == expect


def test_p11_cell_map_channels_are_independent():
    # all five channel set-ups of one du in one call give the same cells as one at a time
    for du in (0.5, 0.25):
        sel = [c for c in P11_CASES if c[0] == du]
        f = np.array([c[1] for c in sel])
        n = np.array([c[2] for c in sel], np.int32)
        cells = oracle.cell_map(P11_ANT, f, n, du)
        for i, c in enumerate(sel):
            assert cells[i].tolist() == c[3]


def test_p11_cell_map_plausible_mistakes_fail():
    # what a dropped centroid, swapped axes, floor or ties-to-even rounding would give
    # on the first case: none of them equals the hand-worked cells the oracle matches
    du, f, N, expect = P11_CASES[0]
    off = (P11_ANT - P11_ANT.mean(axis=0)) * f / (C0 * du)
    rnd_away = np.sign(off) * np.floor(np.abs(off) + 0.5)
    assert (rnd_away + N // 2).astype(int).tolist() == expect
    wrong = {
        "no centroid": np.sign(P11_ANT * f / (C0 * du)) * np.floor(np.abs(P11_ANT * f / (C0 * du)) + 0.5) + N // 2,
        "swapped axes": rnd_away[:, ::-1] + N // 2,
        "floor": np.floor(off) + N // 2,
        "ties to even": np.rint(off) + N // 2,
        "du ignored": np.sign(off * du) * np.floor(np.abs(off * du) + 0.5) + N // 2,
    }
    for name, w in wrong.items():
        assert w.astype(int).tolist() != expect, name


# ---------------------------------------------------------------- E-field images

def beamformer_field(v, g, cells, N, W):
    """Brute-force F_p(l, t) = W^(l) sum_a e~_a exp(2 pi i k_a.l / N) for one
    channel, [T][P][N][N] on the shifted layout (no grid, no FFT)."""
    e = unpack_np(v)                                  # [T][A][P]
    if g is not None:
        e = e * g[None]
    l = np.arange(N) - N // 2
    ph_x = np.exp(2j * np.pi * np.outer(cells[:, 0], l) / N)
    ph_y = np.exp(2j * np.pi * np.outer(cells[:, 1], l) / N)
    return np.einsum("tap,ai,aj->tpij", e, ph_y, ph_x) * what(W, N)[None, None]


@pytest.mark.parametrize("A,P,K,N", [(5, 1, 1, 8), (9, 2, 3, 16), (12, 2, 5, 32)])
def test_efield_brute_force_beamformer(A, P, K, N):
    wl = synth.random_small(A=A, P=P, C=2, T=3, N=N, K=K, seed=1200 + A)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    F = oracle.epic_efield(wl.v, wl.gains, cells, wl.grid_n, wl.kernel)
    per = P * N * N
    for c in range(2):
        ref = beamformer_field(wl.v[:, c], wl.gains[c], cells[c], N, wl.kernel)
        got = F[:, c * per:(c + 1) * per].reshape(wl.T, P, N, N)
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_efield_parseval_per_sample():
    # sum_l |F_p(l, t)|^2 = N^2 sum_k |G_p(k, t)|^2 for every sample (one sample per call)
    wl = synth.random_small(A=20, P=2, C=2, T=4, N=32, K=3, seed=1210)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    F = oracle.epic_efield(wl.v, wl.gains, cells, wl.grid_n, wl.kernel).reshape(wl.T, 2, 2, 32 * 32)
    for t in range(wl.T):
        en = oracle.grid_energy(wl.v[t:t + 1], wl.gains, cells, wl.grid_n, wl.kernel)   # [C][P]
        got = np.sum(np.abs(F[t]) ** 2, axis=-1)
        assert np.allclose(got, 32 * 32 * en, rtol=1e-12)


def test_efield_quarter_field_closed_form():
    # e_a = s_t (-i)^{kx + ky}: F(l = (N/4, N/4), t) = s_t A W^(l), the peak of |F|
    wl, _, s, N, A = _point_source_case(True)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    F = oracle.epic_efield(wl.v, None, cells, wl.grid_n, wl.kernel).reshape(len(s), N, N)
    Wh = what(wl.kernel, N)
    i = j = N // 2 + N // 4
    assert np.allclose(F[:, i, j], s * A * Wh[i, j], rtol=1e-13, atol=1e-12)
    for t in range(len(s)):
        assert np.argmax(np.abs(F[t])) == i * N + j


def test_efield_products_give_the_unsubtracted_image():
    # sum_t F_p F_q^* over the E-field images is the integration before autocorrelation removal
    wl = synth.random_small(A=15, P=2, C=2, T=5, N=16, K=3, seed=1220)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    F = oracle.epic_efield(wl.v, wl.gains, cells, wl.grid_n, wl.kernel).reshape(wl.T, 2, 2, 16 * 16)
    ref = beamformer_image(wl.v[:, 0], wl.gains[0], cells[0], 16, wl.kernel, autosub=False)
    X, Y = F[:, 0, 0], F[:, 0, 1]
    S = [np.sum(X * X.conj(), 0), np.sum(Y * Y.conj(), 0), np.sum(X * Y.conj(), 0), np.sum(Y * X.conj(), 0)]
    assert np.max(np.abs(np.array(S).reshape(ref.shape) - ref)) < 1e-11 * np.max(np.abs(ref))
