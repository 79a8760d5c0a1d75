"""Parity of the tensor-core form (tcgen05 DFT-as-GEMM, both 64-point transform
stages) with the FP64 oracle, per operand precision: split FP16 within 1e-5 of
the channel peak, single FP16 within 2e-3, and the two-part BF16 split within
1e-4 (BF16 keeps 8 significant bits, so hi + lo carry about 16: a product
error near 2^-16 ~ 1.5e-5 relative per operand element, summed over the
transform; the bound is the one derived for that split, not the FP16 one)."""
import numpy as np
import pytest

import oracle
from paper_2301_09662_gb300 import epic, synth

from gpu_helpers import peak_rel_err, run_gpu

pytestmark = pytest.mark.gpu

SPLIT_TOL = 1e-5
FP16_TOL = 2e-3
BF16_TOL = 1e-4


def _cmp(wl, precision, flags=0, channels=None):
    gpu, p = run_gpu(wl, precision=precision, flags=flags)
    ref = oracle.workload_image(wl, flags=flags, channels=channels)
    if channels is not None:
        gpu = np.concatenate([p.split(gpu)[c].ravel() for c in channels])
        return peak_rel_err(gpu, ref, wl.grid_n[channels], 2)
    return peak_rel_err(gpu, ref, wl.grid_n, 2)


def test_tensor_split_fp16_smallest_case():
    wl = synth.random_small(A=24, P=2, C=1, T=2, N=64, K=3, seed=301)
    assert _cmp(wl, epic.EPIC_TC_SPLIT_FP16).max() < SPLIT_TOL


@pytest.mark.parametrize("A,C,T,N,K", [(64, 2, 7, 64, 5), (256, 2, 6, 128, 5), (300, 1, 5, 128, 7),
                                       (80, 1, 4, 256, 5)])
def test_tensor_split_fp16(A, C, T, N, K):
    wl = synth.random_small(A=A, P=2, C=C, T=T, N=N, K=K, seed=302 + A + N)
    assert _cmp(wl, epic.EPIC_TC_SPLIT_FP16).max() < SPLIT_TOL


@pytest.mark.parametrize("precision,tol", [(epic.EPIC_TC_SPLIT_FP16, SPLIT_TOL), (epic.EPIC_TC_SPLIT_BF16, BF16_TOL)])
def test_tensor_large_grid_fold_path(precision, tol):
    """At N = 512 the tensor plan takes the fold path: every class grid is formed
    once per (channel, sample) by alias_fold_kernel and the two-stage tensor
    kernel loads it instead of gridding."""
    wl = synth.random_small(A=150, P=2, C=2, T=7, N=512, K=5, seed=331)
    assert _cmp(wl, precision).max() < tol


def test_tensor_single_fp16():
    wl = synth.random_small(A=256, P=2, C=2, T=6, N=128, K=5, seed=310)
    err = _cmp(wl, epic.EPIC_TC_FP16).max()
    assert err < FP16_TOL
    assert err > SPLIT_TOL        # the split is what buys the accuracy


def test_tensor_split_bf16():
    wl = synth.random_small(A=256, P=2, C=2, T=6, N=128, K=5, seed=311)
    assert _cmp(wl, epic.EPIC_TC_SPLIT_BF16).max() < BF16_TOL


def test_tensor_split_fp16_with_taper_and_flags():
    wl = synth.random_small(A=120, P=2, C=2, T=9, N=128, K=5, seed=312)
    for flags in (epic.EPIC_KERNEL_TAPER, epic.EPIC_MEAN, epic.EPIC_NO_AUTOSUB):
        assert _cmp(wl, epic.EPIC_TC_SPLIT_FP16, flags=flags).max() < SPLIT_TOL


@pytest.mark.parametrize("precision,tol", [(epic.EPIC_TC_SPLIT_FP16, SPLIT_TOL), (epic.EPIC_TC_FP16, FP16_TOL),
                                           (epic.EPIC_TC_SPLIT_BF16, BF16_TOL)])
def test_tensor_lwa_full_size_sampled_channels(precision, tol):
    """The full LWA-like integration (256 dual-pol antennas, 64 channels, 1000
    spectra, grid 128) in each tensor precision, two channels against the oracle."""
    wl = synth.lwa()
    assert _cmp(wl, precision, channels=[3, 60]).max() < tol


@pytest.mark.parametrize("precision,tol", [(epic.EPIC_TC_SPLIT_FP16, SPLIT_TOL), (epic.EPIC_TC_SPLIT_BF16, BF16_TOL)])
def test_tensor_uneven_workload_full_size_sampled_channels(precision, tol):
    """The full uneven band (192 channels over 30-80 MHz, grid sides 64/96/128,
    1000 spectra) in one tensor plan: side 64 on the pair kernel's one-class form,
    96 and 128 on its two-class forms; one channel of each group against the
    oracle."""
    wl = synth.uneven()
    chans = [0, 100, 191]
    assert sorted(set(int(wl.grid_n[c]) for c in chans)) == [64, 96, 128]
    assert _cmp(wl, precision, channels=chans).max() < tol


def test_bounded_wait_reports_timeout_and_context_survives():
    """Failure detection without a fault: the tensor kernel withholds its MMA,
    so the mbarrier it waits on never completes; the bounded wait gives up,
    the plan's status word reads EPIC_ERR_TIMEOUT, and the next plan on the
    same context images correctly."""
    import torch
    from gpu_helpers import torch_inputs
    wl = synth.random_small(A=40, P=2, C=1, T=3, N=64, K=3, seed=320)
    p = epic.Plan.from_workload(wl, precision=epic.EPIC_TC_SPLIT_FP16, flags=epic.EPIC_DIAG_WITHHOLD_MMA)
    v, g = torch_inputs(wl)
    p.image(v, g)
    torch.cuda.synchronize()
    assert p.status() == epic.EPIC_ERR_TIMEOUT
    assert p.status() == epic.EPIC_OK          # reading clears it
    p.close()
    assert _cmp(wl, epic.EPIC_TC_SPLIT_FP16).max() < SPLIT_TOL


@pytest.mark.parametrize("T", [1, 2, 65])
def test_two_stage_form_sample_counts(T):
    """One sample (no overlap), two (one hand-off each way) and an odd count over
    several time chunks: the row/column stage pipeline drains every sample."""
    wl = synth.random_small(A=40, P=2, C=1, T=T, N=64, K=3, seed=340 + T)
    assert _cmp(wl, epic.EPIC_TC_SPLIT_FP16).max() < SPLIT_TOL


@pytest.mark.parametrize("precision,tol", [(epic.EPIC_TC_SPLIT_FP16, SPLIT_TOL), (epic.EPIC_TC_SPLIT_BF16, BF16_TOL)])
def test_mixed_grid_sides_in_a_tensor_plan(precision, tol):
    """Channel groups of sides 64, 96 and 128 in one tensor plan, every one on the
    tensor cores (side 96 through 48-point DFTs); every channel meets the form's
    bound."""
    wl = synth.random_small(A=40, P=2, C=3, T=17, N=64, K=5, seed=350)
    wl.grid_n = np.array([64, 96, 128], np.int32)
    assert _cmp(wl, precision).max() < tol


# ---- grid side 128: two pixel classes per CTA from one gridding (the pair kernel)

PAIR_CASES = [
    # A,  C, T,  K,  N
    (64, 2, 9, 5, 128),
    (256, 2, 6, 5, 128),
    (100, 3, 13, 3, 128),    # A * P not a multiple of 32: partial bank groups
    (256, 1, 7, 7, 128),
    (120, 2, 5, 1, 128),     # point kernel
    (480, 1, 4, 5, 128),     # lists and voltages too large for the pair kernel: the two-stage kernel
    (64, 2, 9, 5, 64),       # side 64: the pair kernel's one-class form
    (100, 3, 13, 3, 64),
    (60, 2, 5, 7, 64),
    (96, 2, 9, 5, 96),       # side 96: 48-point DFTs in the 64-point operands
    (100, 2, 7, 3, 96),
    (200, 1, 5, 7, 96),
]


@pytest.mark.parametrize("A,C,T,K,N", PAIR_CASES)
@pytest.mark.parametrize("precision,tol", [(epic.EPIC_TC_SPLIT_FP16, SPLIT_TOL), (epic.EPIC_TC_FP16, FP16_TOL),
                                           (epic.EPIC_TC_SPLIT_BF16, BF16_TOL)])
def test_pair_kernel_matches_oracle(A, C, T, K, N, precision, tol):
    wl = synth.random_small(A=A, P=2, C=C, T=T, N=N, K=K, seed=600 + A + K + T + N)
    assert _cmp(wl, precision).max() < tol


@pytest.mark.parametrize("N", [128, 96, 64])
def test_pair_kernel_agrees_with_single_class_kernel(N):
    """The gather-gridding pair kernel (two classes per CTA at sides 128 and 96,
    its one-class form at side 64) and the form EPIC_DIAG_NO_PAIR selects (the
    two-stage kernel; at side 96, which has no other tensor kernel, the FP32 form)
    compute the same images up to rounding of different summation orders."""
    wl = synth.random_small(A=200 if N == 128 else 90, P=2, C=2, T=11, N=N, K=5, seed=610 + N)
    a, pa = run_gpu(wl, precision=epic.EPIC_TC_SPLIT_FP16)
    if N == 96:   # a tensor plan of side 96 alone has no other tensor kernel: the FP32 form
        b, pb = run_gpu(wl, precision=epic.EPIC_FP32)
    else:
        b, pb = run_gpu(wl, precision=epic.EPIC_TC_SPLIT_FP16, flags=epic.EPIC_DIAG_NO_PAIR)
    pa.close()
    pb.close()
    assert peak_rel_err(a, b, wl.grid_n, 2).max() < 5e-6
    assert peak_rel_err(a, oracle.workload_image(wl), wl.grid_n, 2).max() < SPLIT_TOL


@pytest.mark.parametrize("N", [128, 96, 64])
@pytest.mark.parametrize("T", [1, 2, 3, 64])
def test_pair_kernel_sample_counts(T, N):
    """One sample (prologue only), two, three, and many over several time chunks:
    the gather / row stage / column stages pipeline drains every sample."""
    wl = synth.random_small(A=48, P=2, C=1, T=T, N=N, K=3, seed=620 + T + N)
    assert _cmp(wl, epic.EPIC_TC_SPLIT_FP16).max() < SPLIT_TOL


def test_pair_kernel_with_taper_and_flags():
    wl = synth.random_small(A=96, P=2, C=2, T=8, N=128, K=5, seed=630)
    for flags in (epic.EPIC_KERNEL_TAPER, epic.EPIC_MEAN, epic.EPIC_NO_AUTOSUB):
        assert _cmp(wl, epic.EPIC_TC_SPLIT_FP16, flags=flags).max() < SPLIT_TOL
    # Stokes: I = XX + YY, Q = XX - YY, U = 2 Re XY, V = 2 Im XY from the oracle's products
    st, p = run_gpu(wl, precision=epic.EPIC_TC_SPLIT_FP16, flags=epic.EPIC_STOKES)
    p.close()
    ref = oracle.workload_image(wl)
    for a, b in zip(oracle.split_channels(st, wl.grid_n, 2), oracle.split_channels(ref, wl.grid_n, 2)):
        xx, yy, xy = b[0].real, b[1].real, b[2]
        stokes = np.stack([xx + yy, xx - yy, 2 * xy.real, 2 * xy.imag])
        peak = max(np.max(np.abs(xx)), np.max(np.abs(yy)))
        assert np.max(np.abs(a.real - stokes)) / peak < 2 * SPLIT_TOL


def test_wide_aperture_at_side_128_keeps_parity():
    """An aperture spanning more than 64 rows at side 128 folds rows onto each
    other; the plan then images that side with one class per CTA, still exact."""
    wl = synth.random_small(A=90, P=2, C=2, T=5, N=128, K=3, seed=640, spread_cells=100)
    assert _cmp(wl, epic.EPIC_TC_SPLIT_FP16).max() < SPLIT_TOL


def test_pair_kernel_bounded_wait_reports_timeout():
    """Failure detection in the pair kernel without a fault: no MMA is issued,
    the bounded waits give up, the status reads EPIC_ERR_TIMEOUT, and a fresh
    plan images correctly afterwards."""
    import torch
    from gpu_helpers import torch_inputs
    wl = synth.random_small(A=40, P=2, C=1, T=3, N=128, K=3, seed=650)
    p = epic.Plan.from_workload(wl, precision=epic.EPIC_TC_SPLIT_FP16, flags=epic.EPIC_DIAG_WITHHOLD_MMA)
    v, g = torch_inputs(wl)
    p.image(v, g)
    torch.cuda.synchronize()
    assert p.status() == epic.EPIC_ERR_TIMEOUT
    p.close()
    assert _cmp(wl, epic.EPIC_TC_SPLIT_FP16).max() < SPLIT_TOL


def test_pair_kernel_series_and_delays():
    """Image series (one time chunk per image) and delay correction through the pair kernel."""
    import torch
    from gpu_helpers import torch_inputs
    wl = synth.random_small(A=64, P=2, C=2, T=12, N=128, K=5, seed=660)
    p = epic.Plan.from_workload(wl, precision=epic.EPIC_TC_SPLIT_FP16)
    v, g = torch_inputs(wl)
    imgs = p.image_series(v, 4, g).cpu().numpy().astype(np.complex128)
    tau = synth.geometric_delays(wl.ant_xy, wl.T, dl=1e-3)
    d = torch.from_numpy(tau).cuda()
    withd = p.image(v, g, delays=d).cpu().numpy().astype(np.complex128)
    torch.cuda.synchronize()
    assert p.status() == epic.EPIC_OK
    p.close()
    for i in range(3):
        sub = synth.Workload(wl.name, wl.ant_xy, 2, wl.kernel, wl.grid_n, wl.freq_hz, wl.du, 4,
                             wl.v[4 * i:4 * i + 4], wl.gains, {})
        assert peak_rel_err(imgs[i], oracle.workload_image(sub), wl.grid_n, 2).max() < SPLIT_TOL
    assert peak_rel_err(withd, oracle.workload_image(wl, delays=tau), wl.grid_n, 2).max() < SPLIT_TOL


# ---- the precision form on the tiny configuration's shapes: single polarisation and grid side 32
# (side 32 is transformed zero-padded to 64 points; its even frequencies are the 32-point image)

def _cmp_p(wl, precision, flags=0):
    gpu, p = run_gpu(wl, precision=precision, flags=flags)
    p.close()
    return peak_rel_err(gpu, oracle.workload_image(wl, flags=flags), wl.grid_n, wl.n_pol)


@pytest.mark.parametrize("precision,tol", [(epic.EPIC_TC_SPLIT_FP16, SPLIT_TOL), (epic.EPIC_TC_FP16, FP16_TOL),
                                           (epic.EPIC_TC_SPLIT_BF16, BF16_TOL)])
def test_tensor_form_on_the_tiny_workload(precision, tol):
    """16 single-pol antennas, 4 channels at 40-41 MHz, 3 x 3 kernel, 32 x 32 grid,
    64 spectra: the tensor form against both oracles (O1 direct, O2 FX)."""
    wl = synth.tiny()
    gpu, p = run_gpu(wl, precision=precision)
    p.close()
    assert peak_rel_err(gpu, oracle.workload_image(wl), wl.grid_n, 1).max() < tol
    assert peak_rel_err(gpu, oracle.workload_image(wl, form="fx"), wl.grid_n, 1).max() < tol


@pytest.mark.parametrize("A,P,C,T,N,K", [(64, 1, 2, 9, 128, 5), (100, 1, 2, 7, 64, 3), (40, 2, 2, 6, 32, 3),
                                         (24, 1, 3, 5, 32, 1), (64, 1, 1, 4, 256, 5)])
def test_tensor_single_polarisation_and_side_32(A, P, C, T, N, K):
    wl = synth.random_small(A=A, P=P, C=C, T=T, N=N, K=K, seed=700 + A + N)
    assert _cmp_p(wl, epic.EPIC_TC_SPLIT_FP16).max() < SPLIT_TOL


def test_tensor_side_32_with_flags_and_taper():
    wl = synth.random_small(A=40, P=2, C=2, T=6, N=32, K=3, seed=720)
    for flags in (epic.EPIC_MEAN, epic.EPIC_NO_AUTOSUB, epic.EPIC_KERNEL_TAPER):
        assert _cmp_p(wl, epic.EPIC_TC_SPLIT_FP16, flags=flags).max() < SPLIT_TOL


def test_autotuned_tensor_plan_keeps_parity():
    """epic_autotune on a tensor plan with pair-kernel groups (sides 64 and 128)
    measures time-chunk counts and then re-deals the pair kernel's lists under a
    few schedules, keeping the fastest: the images stay within the split-FP16
    bound."""
    import torch
    wl = synth.random_small(A=120, P=2, C=4, T=40, N=128, K=5, seed=1210)
    wl.grid_n = np.array([64, 128, 128, 64], np.int32)
    p = epic.Plan.from_workload(wl, precision=epic.EPIC_TC_SPLIT_FP16)
    p.autotune(wl.T)
    v, g = torch.from_numpy(wl.v).cuda(), torch.from_numpy(wl.gains).cuda()
    out = p.image(v, g)
    torch.cuda.synchronize()
    assert p.status() == epic.EPIC_OK
    ref = oracle.workload_image(wl)
    assert peak_rel_err(out.cpu().numpy().astype(np.complex128), ref, wl.grid_n, 2).max() < SPLIT_TOL
    p.close()


@pytest.mark.parametrize("N", [128, 64])
def test_pair_kernel_empty_integration_is_zero(N):
    """n_spectra = 0 through a pair-kernel plan: an all-zero image, status OK."""
    import torch
    wl = synth.random_small(A=48, P=2, C=2, T=4, N=N, K=5, seed=1300 + N)
    p = epic.Plan.from_workload(wl, precision=epic.EPIC_TC_SPLIT_FP16)
    v = torch.from_numpy(wl.v[:0].copy()).cuda()
    g = torch.from_numpy(wl.gains).cuda()
    out = p.image(v, g)
    torch.cuda.synchronize()
    assert p.status() == epic.EPIC_OK
    assert torch.count_nonzero(out) == 0
    p.close()
