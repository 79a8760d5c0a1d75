"""Per-antenna illumination kernels W_a (Eq. 3; A-projection, Sec. 3.1) on the
GPU against the FP64 oracle: gridding through each antenna's own kernel and
the autocorrelation term sum_a A_a |W^_a|^2 from the auto-correlation grid."""
import numpy as np
import pytest

import oracle
from paper_2301_09662_gb300 import epic, synth

from gpu_helpers import peak_rel_err, run_gpu

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def _with_antenna_kernels(wl, seed):
    wl.kernel = synth.antenna_kernels(wl.A, wl.K, np.random.default_rng(seed))
    return wl


@pytest.mark.parametrize("A,P,C,T,N,K", [(20, 1, 2, 7, 32, 3), (40, 2, 2, 6, 64, 5), (70, 2, 1, 5, 96, 3),
                                         (150, 2, 2, 5, 128, 5), (60, 2, 1, 3, 256, 5)])
def test_antenna_kernels_match_oracle(A, P, C, T, N, K):
    wl = _with_antenna_kernels(synth.random_small(A=A, P=P, C=C, T=T, N=N, K=K, seed=600 + A), A)
    gpu, _ = run_gpu(wl, flags=epic.EPIC_ANTENNA_KERNELS)
    ref = oracle.workload_image(wl)
    assert peak_rel_err(gpu, ref, wl.grid_n, P).max() < FP32_TOL


@pytest.mark.parametrize("flags", [epic.EPIC_NO_AUTOSUB, epic.EPIC_MEAN, epic.EPIC_STOKES])
def test_antenna_kernels_flags(flags):
    wl = _with_antenna_kernels(synth.random_small(A=50, P=2, C=2, T=6, N=128, K=5, seed=610), 3)
    gpu, _ = run_gpu(wl, flags=flags | epic.EPIC_ANTENNA_KERNELS)
    ref = oracle.workload_image(wl, flags=flags & ~epic.EPIC_STOKES)
    if flags & epic.EPIC_STOKES:
        conv = []
        for b in oracle.split_channels(ref, wl.grid_n, 2):
            xx, yy, xy = b[0].real, b[1].real, b[2]
            conv.append(np.array([xx + yy, xx - yy, 2 * xy.real, 2 * xy.imag]).astype(np.complex128))
        peaks = [max(np.abs(b[0]).max(), np.abs(b[1]).max()) for b in oracle.split_channels(ref, wl.grid_n, 2)]
        for a, r, pk in zip(oracle.split_channels(gpu, wl.grid_n, 2), conv, peaks):
            assert np.max(np.abs(a - r)) / pk < 2 * FP32_TOL
    else:
        assert peak_rel_err(gpu, ref, wl.grid_n, 2).max() < FP32_TOL


def test_identical_antenna_kernels_equal_shared_kernel():
    wl = synth.random_small(A=64, P=2, C=2, T=5, N=128, K=5, seed=620)
    shared, _ = run_gpu(wl)
    wl.kernel = np.repeat(wl.kernel[None], wl.A, axis=0)
    each, _ = run_gpu(wl, flags=epic.EPIC_ANTENNA_KERNELS)
    assert peak_rel_err(each, shared, wl.grid_n, 2).max() < 1e-6


def test_antenna_kernels_lwa_full_size_sampled_channels():
    wl = _with_antenna_kernels(synth.lwa(), 7)
    gpu, p = run_gpu(wl, flags=epic.EPIC_ANTENNA_KERNELS)
    chans = [11, 52]
    ref = oracle.workload_image(wl, channels=chans)
    got = np.concatenate([p.split(gpu)[c].ravel() for c in chans])
    assert peak_rel_err(got, ref, wl.grid_n[chans], 2).max() < FP32_TOL
