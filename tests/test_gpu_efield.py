"""The electric-field images (epic_image_efield) against the oracle's E-field
images: F_p(l, t) for every sample, channel and polarisation, fft-shifted, no
products.  Error metric: per channel, max |F_gpu - F_oracle| over samples,
polarisations and pixels divided by the largest |F_oracle| of the channel;
bound 1e-5 (the FP32 transform's)."""
import numpy as np
import pytest

import oracle
from paper_2301_09662_gb300 import epic, synth

from gpu_helpers import peak_rel_err, torch_inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5


def _efield(wl, **kw):
    import torch
    p = epic.Plan.from_workload(wl, **kw)
    v, g = torch_inputs(wl)
    out = p.image_efield(v, g)
    torch.cuda.synchronize()
    assert p.status() == epic.EPIC_OK
    res = out.cpu().numpy().astype(np.complex128)
    return res, p


def _channel_err(got, ref, grid_n, P):
    errs, off = [], 0
    for N in grid_n:
        sz = P * int(N) * int(N)
        a, b = got[:, off:off + sz], ref[:, off:off + sz]
        errs.append(np.max(np.abs(a - b)) / np.max(np.abs(b)))
        off += sz
    return np.array(errs)


CASES = [
    # A,  P, C, T, N,   K
    (64, 2, 2, 5, 64, 5),
    (100, 2, 2, 3, 96, 5),
    (256, 2, 2, 4, 128, 5),
    (48, 1, 2, 5, 128, 3),
    (80, 2, 1, 3, 256, 7),
    (120, 2, 1, 2, 512, 7),
    (40, 2, 2, 7, 128, 1),
]


@pytest.mark.parametrize("A,P,C,T,N,K", CASES)
def test_efield_matches_oracle(A, P, C, T, N, K):
    wl = synth.random_small(A=A, P=P, C=C, T=T, N=N, K=K, seed=1300 + A + N)
    got, p = _efield(wl)
    p.close()
    ref = oracle.workload_efield(wl)
    assert got.shape == ref.shape
    assert _channel_err(got, ref, wl.grid_n, P).max() < TOL


def test_efield_products_equal_the_unsubtracted_image():
    """sum_t F_p F_q^* of the E-field images is epic_image without the autocorrelation removal."""
    import torch
    wl = synth.random_small(A=96, P=2, C=2, T=6, N=128, K=5, seed=1310)
    F, p = _efield(wl, flags=epic.EPIC_NO_AUTOSUB)
    v, g = torch_inputs(wl)
    img = p.image(v, g).cpu().numpy().astype(np.complex128)
    p.close()
    N = 128
    F = F.reshape(wl.T, wl.C, 2, N * N)
    prod = np.stack([np.sum(F[:, :, 0] * F[:, :, 0].conj(), 0), np.sum(F[:, :, 1] * F[:, :, 1].conj(), 0),
                     np.sum(F[:, :, 0] * F[:, :, 1].conj(), 0), np.sum(F[:, :, 1] * F[:, :, 0].conj(), 0)], 1)
    assert peak_rel_err(prod.reshape(-1), img, wl.grid_n, 2).max() < TOL


def test_efield_mixed_sides_and_time_chunks():
    wl = synth.random_small(A=60, P=2, C=3, T=40, N=64, K=3, seed=1320)
    wl.grid_n = np.array([64, 96, 128], np.int32)
    got, p = _efield(wl)
    p.close()
    assert _channel_err(got, oracle.workload_efield(wl), wl.grid_n, 2).max() < TOL


def test_efield_lwa_shape_sampled_channels():
    """The LWA-like array (256 dual-pol antennas, 64 channels, 5 x 5 kernel, side 128)
    over 16 samples; two channels checked against the oracle."""
    wl = synth.lwa(T=16)
    got, p = _efield(wl)
    p.close()
    per = 2 * 128 * 128
    for c in (5, 50):
        ref = oracle.workload_efield(wl, channels=[c])
        a = got[:, c * per:(c + 1) * per]
        assert np.max(np.abs(a - ref)) / np.max(np.abs(ref)) < TOL


def test_efield_unsupported_forms_are_rejected():
    import torch
    wl = synth.random_small(A=16, P=2, C=1, T=2, N=32, K=3, seed=1330)
    p = epic.Plan.from_workload(wl)            # side 32: shared-memory kernel, no E-field form
    v, g = torch_inputs(wl)
    with pytest.raises(epic.EpicError):
        p.image_efield(v, g)
    p.close()
    wl = synth.random_small(A=32, P=2, C=1, T=2, N=64, K=3, seed=1331)
    p = epic.Plan.from_workload(wl, precision=epic.EPIC_TC_SPLIT_FP16)
    v, g = torch_inputs(wl)
    with pytest.raises(epic.EpicError):
        p.image_efield(v, g)
    p.close()
