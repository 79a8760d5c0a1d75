"""Time-resolved imaging (epic_image_series) and Stokes output, against the
FP64 oracle: every image of a series must equal the oracle's integration of
its own block of spectra, and Stokes images the fixed combinations of the
oracle's polarisation products."""
import numpy as np
import pytest

import oracle
from paper_2301_09662_gb300 import epic, synth

from gpu_helpers import peak_rel_err, run_gpu, torch_inputs

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def _block(wl, t0, t1):
    sub = synth.Workload(wl.name, wl.ant_xy, wl.n_pol, wl.kernel, wl.grid_n, wl.freq_hz, wl.du, t1 - t0,
                         wl.v[t0:t1], wl.gains, {})
    return sub


@pytest.mark.parametrize("flags,precision", [(0, epic.EPIC_FP32), (epic.EPIC_MEAN, epic.EPIC_FP32),
                                             (epic.EPIC_KERNEL_TAPER, epic.EPIC_FP32),
                                             (0, epic.EPIC_TC_SPLIT_FP16)])
def test_series_images_equal_block_integrations(flags, precision):
    import torch
    spi = 4
    wl = synth.random_small(A=60, P=2, C=2, T=12, N=128, K=5, seed=401)
    p = epic.Plan.from_workload(wl, flags=flags, precision=precision)
    v, g = torch_inputs(wl)
    out = p.image_series(v, spi, g)
    torch.cuda.synchronize()
    assert p.status() == epic.EPIC_OK
    got = out.cpu().numpy().astype(np.complex128)
    for i in range(wl.T // spi):
        ref = oracle.workload_image(_block(wl, i * spi, (i + 1) * spi), flags=flags & ~epic.EPIC_KERNEL_TAPER)
        assert peak_rel_err(got[i], ref, wl.grid_n, 2).max() < FP32_TOL


@pytest.mark.parametrize("precision", [epic.EPIC_FP32, epic.EPIC_TC_SPLIT_FP16])
def test_series_on_a_large_grid_side(precision):
    """At N = 512 a plain integration takes the fold path; a series needs one
    time chunk per image, so it runs the per-class gridding of the same plan."""
    import torch
    spi = 3
    wl = synth.random_small(A=64, P=2, C=1, T=6, N=512, K=3, seed=405)
    p = epic.Plan.from_workload(wl, precision=precision)
    v, g = torch_inputs(wl)
    out = p.image_series(v, spi, g)
    whole = p.image(v, g)
    torch.cuda.synchronize()
    assert p.status() == epic.EPIC_OK
    got = out.cpu().numpy().astype(np.complex128)
    for i in range(wl.T // spi):
        ref = oracle.workload_image(_block(wl, i * spi, (i + 1) * spi))
        assert peak_rel_err(got[i], ref, wl.grid_n, 2).max() < FP32_TOL
    ref = oracle.workload_image(wl)
    assert peak_rel_err(whole.cpu().numpy().astype(np.complex128), ref, wl.grid_n, 2).max() < FP32_TOL


def test_series_mixed_grid_sides_and_single_pol():
    import torch
    wl = synth.random_small(A=30, P=1, C=3, T=9, N=64, K=3, seed=402)
    wl.grid_n = np.array([32, 64, 96], np.int32)
    p = epic.Plan.from_workload(wl)
    v, g = torch_inputs(wl)
    got = p.image_series(v, 3, g).cpu().numpy().astype(np.complex128)
    for i in range(3):
        ref = oracle.workload_image(_block(wl, 3 * i, 3 * i + 3))
        assert peak_rel_err(got[i], ref, wl.grid_n, 1).max() < FP32_TOL


def test_series_longer_than_one_batch_lwa():
    """20 images of 50 spectra from the full LWA workload (more images than one
    batch holds); two channels of two images against the oracle."""
    import torch
    wl = synth.lwa()
    p = epic.Plan.from_workload(wl)
    v, g = torch_inputs(wl)
    out = p.image_series(v, 50, g)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.complex128)
    for i in (0, 17):
        ref = oracle.workload_image(_block(wl, 50 * i, 50 * i + 50), channels=[7, 50])
        sel = np.concatenate([p.split(got[i])[c].ravel() for c in (7, 50)])
        assert peak_rel_err(sel, ref, wl.grid_n[[7, 50]], 2).max() < FP32_TOL


def test_series_rejects_ragged_length():
    import torch
    wl = synth.random_small(A=10, P=2, C=1, T=10, N=64, K=3, seed=403)
    p = epic.Plan.from_workload(wl)
    v, g = torch_inputs(wl)
    with pytest.raises(ValueError):
        p.image_series(v, 3, g)
    rc = epic.load().epic_image_series(p._h, v.data_ptr(), None, 10, 3, v.data_ptr(), None)
    assert rc == epic.EPIC_ERR_ARG


def test_stokes_output():
    wl = synth.random_small(A=80, P=2, C=2, T=7, N=128, K=5, seed=404)
    got, _ = run_gpu(wl, flags=epic.EPIC_STOKES)
    ref = oracle.workload_image(wl)
    for c, (a, b) in enumerate(zip(oracle.split_channels(got, wl.grid_n, 2), oracle.split_channels(ref, wl.grid_n, 2))):
        xx, yy, xy = b[0].real, b[1].real, b[2]
        stokes = np.array([xx + yy, xx - yy, 2 * xy.real, 2 * xy.imag])
        peak = max(np.abs(xx).max(), np.abs(yy).max())
        assert np.max(np.abs(a.real - stokes)) / peak < 2 * FP32_TOL
        assert np.all(a.imag == 0)
