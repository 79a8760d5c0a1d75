"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Error metric: per channel, max over pixels and products of |I_gpu - I_oracle|
divided by the channel's peak max(|XX|, |YY|).  The FP32 form must stay within
1e-5 of the peak.
"""
import numpy as np
import pytest

import oracle
from paper_2301_09662_gb300 import epic, synth

from gpu_helpers import peak_rel_err, run_gpu, torch_inputs

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


def _oracle(wl, flags=0, form="direct", channels=None):
    return oracle.workload_image(wl, flags=flags, form=form, channels=channels)


def test_tiny_workload_matches_both_oracles():
    wl = synth.tiny()
    gpu, _ = run_gpu(wl)
    ref1 = _oracle(wl)
    ref2 = _oracle(wl, form="fx")
    assert peak_rel_err(gpu, ref1, wl.grid_n, 1).max() < FP32_TOL
    assert peak_rel_err(gpu, ref2, wl.grid_n, 1).max() < FP32_TOL


CASES = [
    # A,   P, C, T,  N,   K
    (16, 1, 3, 9, 32, 3),
    (37, 2, 2, 13, 32, 3),
    (64, 2, 2, 7, 64, 5),
    (101, 2, 2, 11, 96, 5),
    (256, 2, 2, 6, 128, 5),
    (300, 2, 1, 5, 128, 7),
    (50, 1, 2, 17, 128, 1),
    (80, 2, 1, 4, 256, 5),
    (120, 2, 1, 3, 512, 7),
]


@pytest.mark.parametrize("A,P,C,T,N,K", CASES)
def test_random_cases(A, P, C, T, N, K):
    wl = synth.random_small(A=A, P=P, C=C, T=T, N=N, K=K, seed=A * 7 + N + K)
    gpu, _ = run_gpu(wl)
    ref = _oracle(wl)
    err = peak_rel_err(gpu, ref, wl.grid_n, P)
    assert err.max() < FP32_TOL, err


FOLD48_CASES = [
    # grid side 96 folds to 48 x 48 per pixel class; n_ant * n_pol a multiple of
    # 4 takes the register-transform kernel (48-point FFTs, scheduled gridding)
    # A,   P, C, T,  N,  K
    (100, 2, 2, 11, 96, 5),   # kernel side fixed at compile time, ragged time pair
    (72, 2, 1, 7, 96, 7),     # generic kernel-side loop
    (64, 1, 2, 9, 96, 3),     # one polarisation
    (48, 2, 2, 6, 96, 1),     # point kernel
    (500, 2, 1, 4, 96, 15),   # footprints wider than a bank group, wrap across the fold
]


@pytest.mark.parametrize("A,P,C,T,N,K", FOLD48_CASES)
def test_fold48_register_kernel(A, P, C, T, N, K):
    wl = synth.random_small(A=A, P=P, C=C, T=T, N=N, K=K, seed=A * 3 + K)
    gpu, _ = run_gpu(wl)
    ref = _oracle(wl)
    err = peak_rel_err(gpu, ref, wl.grid_n, P)
    assert err.max() < FP32_TOL, err


def test_fold48_register_kernel_taper():
    wl = synth.random_small(A=100, P=2, C=2, T=7, N=96, K=5, seed=96)
    gpu, _ = run_gpu(wl, flags=epic.EPIC_KERNEL_TAPER)
    assert peak_rel_err(gpu, _oracle(wl), wl.grid_n, 2).max() < FP32_TOL


@pytest.mark.parametrize("A,P,N,K", [(100, 2, 128, 5), (64, 1, 96, 3)])
def test_gather_table_staged_and_global_forms_agree(A, P, N, K):
    """The gather table read from shared memory (staged per channel) and through
    the L1 cache give bitwise the same image (same lists, same order), and both
    match the oracle."""
    wl = synth.random_small(A=A, P=P, C=2, T=9, N=N, K=K, seed=A + N)
    staged, _ = run_gpu(wl)
    unstaged, _ = run_gpu(wl, flags=epic.EPIC_DIAG_GATHER_GLOBAL)
    assert np.array_equal(staged, unstaged)
    assert peak_rel_err(staged, _oracle(wl), wl.grid_n, P).max() < FP32_TOL


def test_mixed_grid_sides_in_one_plan():
    wl = synth.random_small(A=90, P=2, C=3, T=5, N=64, K=5, seed=11)
    wl.grid_n = np.array([64, 96, 128], np.int32)
    gpu, _ = run_gpu(wl)
    ref = _oracle(wl)
    assert peak_rel_err(gpu, ref, wl.grid_n, 2).max() < FP32_TOL


@pytest.mark.parametrize("flags", [epic.EPIC_MEAN, epic.EPIC_NO_AUTOSUB, epic.EPIC_MEAN | epic.EPIC_NO_AUTOSUB])
def test_flags(flags):
    wl = synth.random_small(A=40, P=2, C=2, T=9, N=64, K=3, seed=5)
    gpu, _ = run_gpu(wl, flags=flags)
    ref = _oracle(wl, flags=flags)
    assert peak_rel_err(gpu, ref, wl.grid_n, 2).max() < FP32_TOL


def test_empty_integration_is_zero():
    import torch
    wl = synth.random_small(A=20, P=2, C=2, T=4, N=32, K=3, seed=6)
    p = epic.Plan.from_workload(wl)
    v, g = torch_inputs(wl)
    out = p.image(v[:0].contiguous(), g)
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0


def test_single_antenna_is_zero():
    wl = synth.random_small(A=1, P=2, C=2, T=8, N=32, K=3, seed=9)
    gpu, _ = run_gpu(wl)
    raw, _ = run_gpu(wl, flags=epic.EPIC_NO_AUTOSUB)
    assert np.max(np.abs(gpu)) <= 1e-5 * np.max(np.abs(raw))


def test_host_buffer_entry_point_matches_device_path():
    import torch
    wl = synth.random_small(A=48, P=2, C=2, T=6, N=64, K=5, seed=12)
    gpu, p = run_gpu(wl)
    v = torch.from_numpy(wl.v).pin_memory()
    g = torch.from_numpy(wl.gains).pin_memory()
    host = p.image_host(v, g).numpy().astype(np.complex128)
    assert peak_rel_err(host, gpu, wl.grid_n, 2).max() < 1e-6


def test_too_many_spectra_is_rejected_before_launch():
    import torch
    wl = synth.random_small(A=10, P=2, C=1, T=4, N=32, K=3, seed=13)
    p = epic.Plan.from_workload(wl, max_spectra=3)
    v, g = torch_inputs(wl)
    out = torch.full((p.out_floats // 2,), 7 + 0j, dtype=torch.complex64, device="cuda")
    with pytest.raises(epic.EpicError) as ei:
        p.image(v, g, out=out)
    assert ei.value.code == epic.EPIC_ERR_ARG
    assert torch.all(out == 7).item()


def test_lwa_full_size_sampled_channels():
    """The LWA-like workload at full size (256 dual-pol antennas, 64 channels,
    1000 spectra, 128 grid) in the launch configuration the benchmark times;
    three channels checked against the oracle."""
    wl = synth.lwa()
    gpu, p = run_gpu(wl)
    chans = [0, 31, 63]
    ref = _oracle(wl, channels=chans)
    got = np.concatenate([p.split(gpu)[c].ravel() for c in chans])
    err = peak_rel_err(got, ref, wl.grid_n[chans], 2)
    assert err.max() < FP32_TOL, err
    # the point source pixels of a second, independent route (FX) agree too
    ref_fx = _oracle(wl, form="fx", channels=[63])
    assert peak_rel_err(p.split(gpu)[63].ravel(), ref_fx, wl.grid_n[[63]], 2).max() < FP32_TOL


def test_graph_replay_follows_new_pointers_and_lengths():
    """The plan's CUDA graph is re-captured when T or a buffer changes."""
    import torch
    wl = synth.random_small(A=70, P=2, C=2, T=12, N=128, K=5, seed=21)
    p = epic.Plan.from_workload(wl)
    v, g = torch_inputs(wl)
    for T in (12, 7, 7, 12):
        vt = v[:T].contiguous()
        out = p.image(vt, g)
        torch.cuda.synchronize()
        sub = synth.random_small(A=70, P=2, C=2, T=12, N=128, K=5, seed=21)
        sub.v = wl.v[:T]
        ref = _oracle(sub)
        assert peak_rel_err(out.cpu().numpy().astype(np.complex128), ref, wl.grid_n, 2).max() < FP32_TOL


def test_graph_and_direct_launches_agree():
    import torch
    wl = synth.random_small(A=90, P=2, C=3, T=6, N=64, K=5, seed=22)
    wl.grid_n = np.array([64, 96, 128], np.int32)
    g_out, _ = run_gpu(wl)
    d_out, _ = run_gpu(wl, flags=epic.EPIC_DIAG_NO_GRAPH)
    assert peak_rel_err(g_out, d_out, wl.grid_n, 2).max() < 1e-6


def test_folded64_path_is_bitwise_deterministic():
    """The M = 64 kernel grids without atomics, so repeated runs agree bit for bit."""
    wl = synth.random_small(A=200, P=2, C=2, T=9, N=128, K=5, seed=23)
    a, p = run_gpu(wl)
    b, _ = run_gpu(wl, plan=p)
    assert np.array_equal(a, b)


def test_large_grid_fold_path_matches_per_class_path_and_is_deterministic():
    """At N = 512 the plan grids once per (channel, sample) and folds the 64
    pixel classes with one 8 x 8 DFT per folded cell; EPIC_DIAG_NO_ALIAS keeps the
    per-class gridding.  Both agree to FP32 rounding, the fold path repeats bit
    for bit (no atomics), and it matches the oracle."""
    wl = synth.random_small(A=150, P=2, C=2, T=7, N=512, K=5, seed=31)
    a, p = run_gpu(wl)
    b, _ = run_gpu(wl, plan=p)
    assert np.array_equal(a, b)
    c, _ = run_gpu(wl, flags=epic.EPIC_DIAG_NO_ALIAS)
    assert peak_rel_err(a, c, wl.grid_n, 2).max() < 1e-6
    ref = oracle.workload_image(wl)
    assert peak_rel_err(a, ref, wl.grid_n, 2).max() < FP32_TOL


@pytest.mark.parametrize("P,precision", [(1, epic.EPIC_FP32), (2, epic.EPIC_FP32), (2, epic.EPIC_TC_SPLIT_FP16)])
def test_large_grid_fold_path_in_time_batches(P, precision):
    """The fold path sums time batches into one partial slot: 7 spectra in
    batches of 3 (3 + 3 + 1) give the oracle's image, single and dual
    polarisation, FP32 and split-FP16 tensor kernels."""
    wl = synth.random_small(A=92, P=P, C=2, T=7, N=512, K=3, seed=41 + P)   # A*P a multiple of 4: the M = 64 path
    gpu, _ = run_gpu(wl, precision=precision, flags=epic.EPIC_DIAG_ALIAS_BATCH(3))
    ref = oracle.workload_image(wl)
    assert peak_rel_err(gpu, ref, wl.grid_n, P).max() < FP32_TOL


def test_uneven_workload_full_size_sampled_channels():
    """192 channels over 30-80 MHz in three grid-side groups (64/96/128), 1000
    spectra, one graph launch per integration; one channel of each group against
    the oracle."""
    wl = synth.uneven()
    gpu, p = run_gpu(wl)
    chans = [0, 100, 191]
    assert sorted(set(int(wl.grid_n[c]) for c in chans)) == [64, 96, 128]
    ref = _oracle(wl, channels=chans)
    got = np.concatenate([p.split(gpu)[c].ravel() for c in chans])
    err = peak_rel_err(got, ref, wl.grid_n[chans], 2)
    assert err.max() < FP32_TOL, err


TAPER_CASES = [
    # A,   P, C, T,  N,   K
    (37, 2, 2, 13, 32, 3),
    (101, 2, 2, 11, 96, 5),
    (256, 2, 2, 6, 128, 5),
    (300, 1, 1, 5, 128, 7),
    (120, 2, 1, 3, 512, 7),
]


@pytest.mark.parametrize("A,P,C,T,N,K", TAPER_CASES)
def test_kernel_taper_form_matches_oracle(A, P, C, T, N, K):
    """EPIC_KERNEL_TAPER (point gridding, |W^|^2 applied to the image) equals the
    literal gridding of the oracle for a shared, non-symmetric complex kernel."""
    wl = synth.random_small(A=A, P=P, C=C, T=T, N=N, K=K, seed=A * 5 + N + K)
    gpu, _ = run_gpu(wl, flags=epic.EPIC_KERNEL_TAPER)
    ref = _oracle(wl)
    assert peak_rel_err(gpu, ref, wl.grid_n, P).max() < FP32_TOL


@pytest.mark.parametrize("flags", [epic.EPIC_MEAN, epic.EPIC_NO_AUTOSUB])
def test_kernel_taper_with_flags(flags):
    wl = synth.random_small(A=40, P=2, C=2, T=9, N=64, K=5, seed=55)
    gpu, _ = run_gpu(wl, flags=flags | epic.EPIC_KERNEL_TAPER)
    ref = _oracle(wl, flags=flags)
    assert peak_rel_err(gpu, ref, wl.grid_n, 2).max() < FP32_TOL


def test_kernel_taper_lwa_full_size_sampled_channels():
    wl = synth.lwa()
    gpu, p = run_gpu(wl, flags=epic.EPIC_KERNEL_TAPER)
    chans = [5, 40]
    ref = _oracle(wl, channels=chans)
    got = np.concatenate([p.split(gpu)[c].ravel() for c in chans])
    assert peak_rel_err(got, ref, wl.grid_n[chans], 2).max() < FP32_TOL


def test_dense_workload_full_size_sampled_channel():
    """The dense 2048-antenna array (256 channels, 500 spectra, 7x7 kernel, 512
    grid) at full size in the benchmark's launch configuration; one channel of
    the literal form (fold path), the kernel-taper form and the split-FP16
    tensor form (fold path) against the oracle."""
    wl = synth.dense()
    chans = [129]
    ref = _oracle(wl, channels=chans)
    for kw in (dict(flags=0), dict(flags=epic.EPIC_KERNEL_TAPER), dict(precision=epic.EPIC_TC_SPLIT_FP16)):
        gpu, p = run_gpu(wl, **kw)
        got = p.split(gpu)[chans[0]].ravel()
        assert peak_rel_err(got, ref, wl.grid_n[chans], 2).max() < FP32_TOL
        p.close()


@pytest.mark.parametrize("A,P,N,K", [(2048, 2, 512, 15), (4096, 1, 128, 5), (1500, 2, 256, 9)])
def test_largest_supported_shapes(A, P, N, K):
    """The limits the plan accepts: n_ant * n_pol = 4096 and K = 15 (footprints
    of 15 x 15 cells), on the M = 64 kernel and its runtime-K path."""
    wl = synth.random_small(A=A, P=P, C=1, T=2, N=N, K=K, seed=A + N + K)
    gpu, _ = run_gpu(wl)
    ref = _oracle(wl)
    assert peak_rel_err(gpu, ref, wl.grid_n, P).max() < FP32_TOL


def test_autotuned_plan_keeps_parity():
    """epic_autotune picks each group's time-chunk count by measurement; the
    images stay within the FP32 bound (only the chunk summation order moves),
    and n_spectra outside the plan is rejected."""
    import torch
    wl = synth.random_small(A=40, P=2, C=3, T=50, N=64, K=5, seed=1200)
    wl.grid_n = np.array([64, 96, 128], np.int32)
    p = epic.Plan.from_workload(wl)
    p.autotune(wl.T)
    v, g = torch_inputs(wl)
    out = p.image(v, g)
    torch.cuda.synchronize()
    assert p.status() == epic.EPIC_OK
    ref = oracle.workload_image(wl)
    assert np.max(peak_rel_err(out.cpu().numpy().astype(np.complex128), ref, wl.grid_n, 2)) < 1e-5
    with pytest.raises(epic.EpicError):
        p.autotune(wl.T + 1)
