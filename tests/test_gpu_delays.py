"""Geometric-delay correction on the GPU (epic_image_ex, the delay-correction
block of Sec. 2.2): parity with the FP64 oracle for every kernel form, the
phase-centre steering closed form, and the plain path left unchanged."""
import numpy as np
import pytest

import oracle
from paper_2301_09662_gb300 import epic, synth
from gpu_helpers import peak_rel_err, torch_inputs

pytestmark = pytest.mark.gpu


def _run(wl, tau, precision=epic.EPIC_FP32, flags=0):
    import torch
    p = epic.Plan.from_workload(wl, precision=precision, flags=flags)
    v, g = torch_inputs(wl)
    d = torch.from_numpy(np.ascontiguousarray(tau)).cuda()
    out = p.image(v, g, delays=d)
    torch.cuda.synchronize()
    assert p.status() == epic.EPIC_OK
    return out.cpu().numpy().astype(np.complex128), p, v, g, d


@pytest.mark.parametrize("N,P", [(128, 2), (64, 2), (96, 2), (32, 1)])
def test_delays_fp32_parity(N, P):
    wl = synth.random_small(A=40, P=P, C=3, T=37, N=N, K=5 if N > 32 else 3, seed=1100 + N + P)
    tau = synth.geometric_delays(wl.ant_xy, wl.T, dl=2e-3, dm=-1e-3)
    gpu, *_ = _run(wl, tau)
    ref = oracle.workload_image(wl, delays=tau)
    assert np.max(peak_rel_err(gpu, ref, wl.grid_n, P)) < 1e-5


@pytest.mark.parametrize("precision,tol", [(epic.EPIC_TC_SPLIT_FP16, 1e-5), (epic.EPIC_TC_SPLIT_BF16, 1e-4)])
def test_delays_tensor_parity(precision, tol):
    wl = synth.random_small(A=48, P=2, C=2, T=29, N=128, K=5, seed=1150)
    tau = synth.geometric_delays(wl.ant_xy, wl.T, dl=1e-3)
    gpu, *_ = _run(wl, tau, precision=precision)
    ref = oracle.workload_image(wl, delays=tau)
    assert np.max(peak_rel_err(gpu, ref, wl.grid_n, 2)) < tol


def test_delays_taper_parity():
    wl = synth.random_small(A=40, P=2, C=2, T=21, N=128, K=5, seed=1160)
    tau = synth.geometric_delays(wl.ant_xy, wl.T, dl=-2e-3)
    gpu, *_ = _run(wl, tau, flags=epic.EPIC_KERNEL_TAPER)
    ref = oracle.workload_image(wl, delays=tau)
    assert np.max(peak_rel_err(gpu, ref, wl.grid_n, 2)) < 1e-5


def test_delays_steer_source_to_phase_centre():
    """Quarter-field source, delays that undo its per-antenna phases: the GPU
    image is the zenith closed form |sum W|^2 (A^2 - A) sum_t |s_t|^2."""
    N, K, A, T = 32, 3, 12, 6
    wl = synth.random_small(A=A, P=1, C=1, T=T, N=N, K=K, seed=44, gains=False)
    wl.kernel = synth.gaussian_kernel(K)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    rng = np.random.default_rng(6)
    s = rng.integers(-7, 8, T) + 1j * rng.integers(-7, 8, T)
    m = rng.integers(0, 4, T)
    n = cells[0, :, 0] + cells[0, :, 1]
    e = s[:, None] * (-1j) ** (np.outer(m, n) % 4)
    wl.v = synth.pack_ci4(np.rint(e.real).astype(int), np.rint(e.imag).astype(int)).reshape(T, 1, A, 1)
    tau = (np.outer(m, n) % 4) / (4.0 * wl.freq_hz[0])
    gpu, *_ = _run(wl, tau)
    img = gpu.reshape(N, N)
    expect = abs(np.sum(wl.kernel.astype(np.complex128))) ** 2 * (A * A - A) * np.sum(np.abs(s) ** 2)
    assert abs(img[N // 2, N // 2] - expect) < 1e-5 * expect
    assert np.unravel_index(np.argmax(img.real), img.shape) == (N // 2, N // 2)


def test_lwa_channels_with_delays():
    """Full LWA geometry (256 dual-pol antennas, 1000 spectra) on two channels."""
    wl = synth.lwa(T=1000, C=2, first_channel=17)
    tau = synth.geometric_delays(wl.ant_xy, wl.T)
    gpu, *_ = _run(wl, tau)
    ref = oracle.workload_image(wl, delays=tau)
    assert np.max(peak_rel_err(gpu, ref, wl.grid_n, 2)) < 1e-5


def test_no_delays_matches_plain_path_and_graph_key():
    """delays = None is epic_image bit for bit; switching between delay arrays
    and back re-keys the captured graph each time."""
    import torch
    wl = synth.random_small(A=32, P=2, C=2, T=16, N=128, K=5, seed=1170)
    p = epic.Plan.from_workload(wl)
    v, g = torch_inputs(wl)
    plain = p.image(v, g).cpu().numpy()
    t1 = torch.from_numpy(synth.geometric_delays(wl.ant_xy, wl.T, dl=2e-3)).cuda()
    t2 = torch.zeros_like(t1)
    with_d = p.image(v, g, delays=t1).cpu().numpy()
    zero_d = p.image(v, g, delays=t2).cpu().numpy()
    again = p.image(v, g).cpu().numpy()
    assert np.array_equal(plain, again)
    assert np.array_equal(plain, zero_d)          # exp(0) = 1 exactly
    assert not np.allclose(with_d, plain)
    assert p.status() == epic.EPIC_OK


def test_delays_shape_checked_on_host():
    import torch
    wl = synth.random_small(A=8, P=2, C=1, T=4, N=128, K=5, seed=1180)
    p = epic.Plan.from_workload(wl)
    v, g = torch_inputs(wl)
    with pytest.raises(ValueError):
        p.image(v, g, delays=torch.zeros(4, 7, dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        p.image(v, g, delays=torch.zeros(4, 8, dtype=torch.float32, device="cuda"))


def test_series_with_delays_equals_blockwise_delay_images():
    """epic_image_series_ex: each image equals epic_image_ex of its own block of
    spectra with that block's delays (delays indexed like the voltages, across
    series batches)."""
    import torch
    wl = synth.random_small(A=32, P=2, C=2, T=4 * 70, N=128, K=5, seed=1190)
    tau = synth.geometric_delays(wl.ant_xy, wl.T, dl=2e-3, dm=-1e-3)
    p = epic.Plan.from_workload(wl)
    v, g = torch_inputs(wl)
    d = torch.from_numpy(tau).cuda()
    series = p.image_series(v, 4, g, delays=d).cpu().numpy()
    torch.cuda.synchronize()
    assert p.status() == epic.EPIC_OK
    for k in (0, 33, 69):
        blk = p.image(v[4 * k:4 * k + 4].contiguous(), g, delays=d[4 * k:4 * k + 4].contiguous()).cpu().numpy()
        ref = np.max(np.abs(blk))
        assert np.max(np.abs(series[k] - blk)) < 1e-5 * ref
