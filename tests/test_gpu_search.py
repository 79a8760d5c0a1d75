"""Transient search on the GPU (epic_search_*, Sec. 4 de-dispersion and
single-pulse search of per-pixel light curves): parity with the FP64 search
oracle on ragged shapes, strided Stokes-series input, candidate compaction,
and the whole chain from voltages -- a dispersed pulse imaged by
epic_image_series and found again at its pixel and DM."""
import numpy as np
import pytest

import oracle
from oracle import search as osearch
from paper_2301_09662_gb300 import epic, synth

pytestmark = pytest.mark.gpu


def _cube(T, C, P, seed, pulses=()):
    rng = np.random.default_rng(seed)
    cube = rng.normal(10.0, 1.0, (T, C, P))
    for (t0, pix, amp, sh) in pulses:
        for c in range(C):
            cube[t0 + sh[c], c, pix] += amp
    return cube.astype(np.float32)


def _diag(cap, pix2, tma):
    """Search plan diagnostics for one kernel form: DM block ("32", "16" or "0" =
    the direct form), two-pixel staged form ("1"/"0"), TMA form ("1"/"0")."""
    d = {"32": epic.EPIC_SEARCH_DIAG_DM32, "16": 0, "0": epic.EPIC_SEARCH_DIAG_DIRECT}[cap]
    if pix2 == "0":
        d |= epic.EPIC_SEARCH_DIAG_NO_PIX2
    if tma == "0":
        d |= epic.EPIC_SEARCH_DIAG_NO_TMA
    return d


def _setup(T=150, C=20, P=300, n_dm=13, seed=1):
    f = 42.1e6 + 25e3 * np.arange(C)
    dms = np.linspace(0, 12, n_dm)
    dt = 0.04
    sh = osearch.dm_shifts(f, dt, dms)
    return f, dms, dt, sh


def test_dedisperse_parity_ragged():
    import torch
    T, C, P = 150, 20, 300
    f, dms, dt, sh = _setup(T, C, P)
    cube = _cube(T, C, P, 3)
    s = epic.Search(f, dt, dms, P, T)
    assert s.t_out == T - sh.max() and s.max_shift == sh.max()
    dd = s.dedisperse(torch.from_numpy(cube).cuda()).cpu().numpy()
    ref = osearch.dedisperse(cube, sh)
    assert np.max(np.abs(dd - ref)) <= 1e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("grid", ["fine", "coarse", "unsorted"])
def test_dedisperse_forms_agree_bitwise(grid):
    """The 32- and 16-trial staged blocks (TMA producer warp or cp.async
    staging; two pixels per lane with packed adds, or one) and the direct form
    sum every sweep in channel order, so they agree bit for bit; all match the
    oracle.  'fine'
    trials differ by 0 or 1 sample per step (the register-shared second
    window), 'coarse' by 1 to 3 (its own window), 'unsorted' by either sign."""
    import torch
    T, C, P = 300, 20, 71                           # 71 pixels: ragged pixel blocks, an odd last pixel
    f = 42.1e6 + 25e3 * np.arange(C)
    dt = 0.04
    dms = {"fine": np.arange(45) * 0.25, "coarse": np.arange(37) * 1.7,
           "unsorted": np.random.default_rng(2).permutation(np.arange(45) * 0.25)}[grid]
    sh = osearch.dm_shifts(f, dt, dms)
    cube = _cube(T, C, P, 9)
    ref = osearch.dedisperse(cube, sh)
    x = torch.from_numpy(cube).cuda()                  # odd pitch: one pixel per lane
    pad4 = np.full((T, C, P + 1), np.nan, np.float32)  # 72-float pitch: the TMA form applies
    pad4[:, :, :P] = cube
    x_pad4 = torch.from_numpy(pad4.reshape(-1)).cuda()
    outs = []
    for cap, pix2, tma in (("32", "1", "1"), ("16", "1", "1"), ("32", "1", "0"), ("16", "1", "0"),
                           ("32", "0", "1"), ("16", "0", "1"), ("0", "1", "1")):
        s = epic.Search(f, dt, dms, P, T, diag=_diag(cap, pix2, tma))
        outs.append(s.dedisperse(x_pad4, strides=(C * (P + 1), P + 1, 1)).cpu().numpy())
        outs.append(s.dedisperse(x).cpu().numpy())
        assert s.status() == epic.EPIC_OK
        s.close()
    assert np.max(np.abs(outs[0] - ref)) <= 1e-5 * np.max(np.abs(ref))
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)


@pytest.mark.parametrize("T,C,P,n_dm,layout", [
    (40, 1, 8, 1, "tcp"),        # one channel, one trial, eight pixels: the 64-pixel box overhangs
    (12, 6, 4, 3, "tcp"),        # t_out below one 16-sample tile
    (90, 9, 132, 37, "tcp"),     # ragged in every axis (TMA form: pitch a multiple of 4)
    (90, 9, 130, 37, "tcp"),     # the same with an even pitch (two-pixel cp.async form)
    (80, 7, 64, 20, "ctp"),      # channel-major cube: the time stride is the smaller one
])
def test_dedisperse_edge_shapes_all_forms(T, C, P, n_dm, layout):
    import torch
    f = 42.1e6 + 25e3 * np.arange(C)
    dms = np.linspace(0, 3, n_dm)
    sh = osearch.dm_shifts(f, 0.04, dms)
    cube = _cube(T, C, P, T + C + P)
    ref = osearch.dedisperse(cube, sh)
    if layout == "tcp":
        x, strides = torch.from_numpy(cube).cuda(), None
    else:
        x = torch.from_numpy(np.ascontiguousarray(cube.transpose(1, 0, 2))).cuda()
        strides = (P, T * P, 1)
    outs = []
    for cap, pix2, tma in (("16", "1", "1"), ("16", "1", "0"), ("16", "0", "1"), ("32", "1", "1"), ("0", "1", "1")):
        s = epic.Search(f, 0.04, dms, P, T, widths=(1,), diag=_diag(cap, pix2, tma))
        outs.append(s.dedisperse(x, strides=strides).cpu().numpy())
        assert s.status() == epic.EPIC_OK
        s.close()
    assert np.max(np.abs(outs[0] - ref)) <= 1e-5 * np.max(np.abs(ref))
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)


def test_dedisperse_wait_timeout_sets_status():
    """Failure detection without a fault: the TMA form's producer withholds
    channel 0, the consumers' bounded wait runs out, the plan's status word
    reads EPIC_ERR_TIMEOUT, and a fresh plan on the same context is correct."""
    import torch
    T, C, P = 120, 12, 128
    f, dms, dt, sh = _setup(T, C, P, n_dm=8)
    cube = _cube(T, C, P, 12)
    x = torch.from_numpy(cube).cuda()
    s = epic.Search(f, dt, dms, P, T, diag=epic.EPIC_SEARCH_DIAG_WITHHOLD_TMA)
    s.dedisperse(x)
    assert s.status() == epic.EPIC_ERR_TIMEOUT
    assert s.status() == epic.EPIC_OK               # reading clears it
    s.close()
    s = epic.Search(f, dt, dms, P, T)
    dd = s.dedisperse(x).cpu().numpy()
    assert s.status() == epic.EPIC_OK
    ref = osearch.dedisperse(cube, sh)
    assert np.max(np.abs(dd - ref)) <= 1e-5 * np.max(np.abs(ref))
    s.close()


@pytest.mark.parametrize("T,widths", [(20, (1, 2, 4, 8, 16, 32)), (64, (2, 8)), (97, (1, 32)), (33, (32,))])
def test_single_pulse_lengths_and_width_sets(T, widths):
    """Light curves shorter than one 32-sample chunk, an exact number of chunks,
    a ragged tail, widths longer than the curve (never scored) and width subsets."""
    import torch
    n_dm, P = 3, 45
    f = 42.1e6 + 25e3 * np.arange(4)
    s = epic.Search(f, 0.04, [0.0] * n_dm, P, T, widths=widths)
    rng = np.random.default_rng(T)
    dd = rng.normal(50.0, 3.0, (n_dm, T, P)).astype(np.float32)
    dd[1, T // 3:T // 3 + 3, 7] += 25.0
    snr, bt, bw, cand, n = s.single_pulse(torch.from_numpy(dd).cuda(), threshold=4.0)
    snr, bt, bw = snr.cpu().numpy(), bt.cpu().numpy(), bw.cpu().numpy()
    rs, rt, rw = osearch.single_pulse(dd, widths)
    assert np.max(np.abs(snr - rs)) < 1e-3
    for d, p in zip(*np.nonzero((bt != rt) | (bw != rw))):
        assert int(bw[d, p]) in widths and int(bt[d, p]) + int(bw[d, p]) <= T
        alt = osearch.boxcar_snr(dd[d, :, p], int(bw[d, p]))[int(bt[d, p])]
        assert abs(alt - rs[d, p]) < 1e-3
    nc = int(n.item())
    got = [tuple(x) for x in cand[:nc].cpu().numpy().tolist()]
    assert got == sorted(got)
    sure = {(int(d), int(p)) for d, p in zip(*np.nonzero(rs >= 4.0 + 1e-3))}
    maybe = {(int(d), int(p)) for d, p in zip(*np.nonzero(rs >= 4.0 - 1e-3))}
    assert sure <= set(got) <= maybe
    s.close()


def test_dedisperse_strided_stokes_series_layout():
    """I in the real part of slot 0 of a complex64 [T][C][4][P] series is searched in place."""
    import torch
    T, C, P = 96, 12, 200
    f, dms, dt, sh = _setup(T, C, P, n_dm=9)
    cube = _cube(T, C, P, 4)
    series = np.zeros((T, C, 4, P), np.complex64)
    series[:, :, 0, :] = cube
    series[:, :, 1, :] = 99.0 + 7j             # other Stokes images must not leak in
    s = epic.Search(f, dt, dms, P, T)
    flat = torch.from_numpy(series.view(np.float32).reshape(-1)).cuda()
    dd_s = s.dedisperse(flat, strides=(C * 4 * P * 2, 4 * P * 2, 2)).cpu().numpy()
    dd_c = s.dedisperse(torch.from_numpy(cube).cuda()).cpu().numpy()
    assert np.array_equal(dd_s, dd_c)


def test_single_pulse_parity_and_candidates():
    import torch
    T, C, P = 150, 20, 300
    f, dms, dt, sh = _setup(T, C, P)
    pulses = [(30, 17, 6.0, sh[5]), (80, 250, 4.0, sh[11]), (5, 299, 8.0, sh[0])]
    cube = _cube(T, C, P, 5, pulses)
    widths = (1, 2, 4, 8, 16, 32)
    s = epic.Search(f, dt, dms, P, T, widths=widths)
    dd = s.dedisperse(torch.from_numpy(cube).cuda())
    snr, bt, bw, cand, n = s.single_pulse(dd, threshold=6.0, cand_cap=8192)
    snr, bt, bw = snr.cpu().numpy(), bt.cpu().numpy(), bw.cpu().numpy()
    ref = osearch.dedisperse(cube, sh)
    rs, rt, rw = osearch.single_pulse(ref, widths)
    assert np.max(np.abs(snr - rs)) < 1e-3
    # where the arg-max differs (near ties in FP32), the GPU's window scores the oracle's best
    for d, p in zip(*np.nonzero((bt != rt) | (bw != rw))):
        alt = osearch.boxcar_snr(ref[d, :, p], int(bw[d, p]))[int(bt[d, p])]
        assert abs(alt - rs[d, p]) < 1e-3
    # the injected pulses are the strongest detections of their pixels
    for (t0, pix, amp, shp) in pulses:
        d = int(np.argmax(snr[:, pix]))
        assert np.array_equal(sh[d], shp)
        assert abs(int(bt[d, pix]) - t0) <= 1
    # candidates: every pair clearly above threshold, in index order, none clearly below
    nc = int(n.item())
    got = [tuple(x) for x in cand[:nc].cpu().numpy().tolist()]
    assert got == sorted(got)
    sure = {(int(d), int(p)) for d, p in zip(*np.nonzero(rs >= 6.0 + 1e-3))}
    maybe = {(int(d), int(p)) for d, p in zip(*np.nonzero(rs >= 6.0 - 1e-3))}
    assert sure <= set(got) <= maybe


def test_candidate_capacity_reports_the_full_count():
    import torch
    T, C, P = 64, 8, 100
    f, dms, dt, sh = _setup(T, C, P, n_dm=4)
    cube = _cube(T, C, P, 6)
    s = epic.Search(f, dt, dms, P, T, widths=(1,))
    dd = s.dedisperse(torch.from_numpy(cube).cuda())
    snr, _, _, cand, n = s.single_pulse(dd, threshold=-1e30, cand_cap=10)
    assert int(n.item()) == 4 * P
    assert cand.cpu().numpy().tolist() == [[0, i] for i in range(10)]


def test_flat_light_curves_score_zero():
    import torch
    T, C, P = 40, 4, 33
    f = 42.1e6 + 25e3 * np.arange(C)
    s = epic.Search(f, 0.04, [0.0], P, T, widths=(2, 4))
    cube = torch.full((T, C, P), 3.0, dtype=torch.float32, device="cuda")
    snr, bt, bw, _, n = s.single_pulse(s.dedisperse(cube), threshold=0.5)
    assert torch.all(snr == 0) and torch.all(bt == 0) and torch.all(bw == 2) and int(n.item()) == 0


def test_dispersed_pulse_from_voltages_is_found():
    """A quarter-field point source pulses once; each channel sees it at its own
    delay (DM sweep).  epic_image_series (Stokes) images the voltages, the
    search recovers the source pixel and the trial whose delays match."""
    import torch
    N, K, A, C, spi, n_img = 32, 3, 24, 12, 2, 64
    f0, df, dt_img = 42.1e6, 25e3, 0.04
    wl = synth.random_small(A=A, P=2, C=C, T=spi * n_img, N=N, K=K, seed=77, gains=False, f0=f0)
    wl.freq_hz = f0 + df * np.arange(C)
    wl.kernel = synth.gaussian_kernel(K)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    dms = np.arange(0, 30, 1.0)
    sh = osearch.dm_shifts(wl.freq_hz, dt_img, dms)
    true = 21
    rng = np.random.default_rng(8)
    T = spi * n_img
    re = rng.integers(-2, 3, (T, C, A, 2))
    im = rng.integers(-2, 3, (T, C, A, 2))
    img0 = 10
    for c in range(C):
        n_a = cells[c, :, 0] + cells[c, :, 1]
        rot = (-1j) ** (n_a % 4)
        for t in range(spi * (img0 + sh[true, c]), spi * (img0 + sh[true, c] + 1)):
            for p in range(2):
                e = 4 * rot
                re[t, c, :, p] = np.clip(re[t, c, :, p] + np.rint(e.real).astype(int), -7, 7)
                im[t, c, :, p] = np.clip(im[t, c, :, p] + np.rint(e.imag).astype(int), -7, 7)
    wl.v = synth.pack_ci4(re, im)
    plan = epic.Plan.from_workload(wl, flags=epic.EPIC_STOKES)
    v = torch.from_numpy(wl.v).cuda()
    series = plan.image_series(v, spi)
    torch.cuda.synchronize()
    assert plan.status() == epic.EPIC_OK
    flat = series.view(torch.float32).reshape(-1).contiguous()
    s = epic.Search(wl.freq_hz, dt_img, dms, N * N, n_img, widths=(1, 2, 4))
    dd = s.dedisperse(flat, strides=(plan.out_floats, 4 * N * N * 2, 2))
    snr, bt, bw, cand, n = s.single_pulse(dd, threshold=8.0)
    snr = snr.cpu().numpy()
    d, pix = np.unravel_index(np.argmax(snr), snr.shape)
    src = (N // 2 + N // 4) * N + (N // 2 + N // 4)
    assert pix == src
    assert np.array_equal(sh[d], sh[true])
    assert int(bt[d, pix].item()) == img0 and int(bw[d, pix].item()) == 1
