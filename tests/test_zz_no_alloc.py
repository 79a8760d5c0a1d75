"""epic_image_static: imaging without any device allocation.

Some callers cannot call cudaMalloc -- a pipeline whose GPU memory is all held
by its own pool allocator, a real-time capture loop that cannot afford the
device-wide synchronisation cudaMalloc/cudaFree may cause, a plug-in that may
leave no allocations behind.  For them the library offers epic_image_static,
which keeps its tables and workspace in a fixed array in device global memory
instead of allocating.  This file checks, through the C ABI, that it produces
the same images as the plan-based epic_image on two calls in a row (the second
call must not see anything the first left in the shared array).

The file name sorts last so that a run stopping at the first failure has run
every other test first.
"""
import numpy as np
import pytest

from paper_2301_09662_gb300 import epic, synth

FP32_TOL = 1e-5   # the peak-relative tolerance of the FP32 parity tests


def _peak_rel(a, b, C, NP):
    a = a.reshape(C, NP, -1)
    b = b.reshape(C, NP, -1)
    errs = []
    for c in range(C):
        peak = np.max(np.abs(b[c, :2])) if NP == 4 else np.max(np.abs(b[c, 0]))
        errs.append(np.max(np.abs(a[c] - b[c])) / peak)
    return max(errs)


def _both(wl, flags=0):
    import torch
    v = torch.from_numpy(wl.v).cuda()
    g = None if wl.gains is None else torch.from_numpy(wl.gains).cuda()
    plan = epic.Plan.from_workload(wl, flags=flags)
    ref = plan.image(v, g)
    got = epic.image_static(wl.ant_xy, wl.n_pol, wl.kernel, int(wl.grid_n[0]), wl.freq_hz, wl.du, v, g,
                            flags=flags)
    torch.cuda.synchronize()
    assert plan.status() == epic.EPIC_OK
    plan.close()
    return got.cpu().numpy().astype(np.complex128), ref.cpu().numpy().astype(np.complex128)


@pytest.mark.gpu
def test_static_scratch_matches_plan_path_on_two_calls_in_a_row():
    first = synth.random_small(A=96, P=2, C=4, T=21, N=128, K=5, seed=501)
    second = synth.random_small(A=40, P=2, C=3, T=9, N=64, K=3, seed=502)
    for wl in (first, second):
        got, ref = _both(wl)
        assert _peak_rel(got, ref, wl.C, 4) < FP32_TOL
    # and the single-polarisation tiny workload right after
    tiny = synth.tiny()
    got, ref = _both(tiny)
    assert _peak_rel(got, ref, tiny.C, 1) < FP32_TOL


def test_static_scratch_rejects_oversize_request_before_any_work():
    # 128 channels of 128 x 128 dual polarisation need 64 MiB of partial sums
    wl = synth.random_small(A=16, P=2, C=1, T=1, N=128, K=3, seed=503)
    freq = 50e6 + 25e3 * np.arange(128)
    L = epic.load()
    ant = np.ascontiguousarray(wl.ant_xy)
    kern = np.ascontiguousarray(wl.kernel)
    out = np.zeros(2, np.float32)
    rc = L.epic_image_static(ant.ctypes.data, ant.shape[0], 2, kern.ctypes.data, 3, 128, freq.ctypes.data, 128,
                             0.5, None, None, 0, 0, out.ctypes.data, None)
    assert rc == epic.EPIC_ERR_TOO_LARGE
