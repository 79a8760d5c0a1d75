"""epic_image_static: imaging without any device allocation.

Some callers cannot call cudaMalloc -- a pipeline whose GPU memory is all held
by its own pool allocator, a real-time capture loop that cannot afford the
device-wide synchronisation cudaMalloc/cudaFree may cause, a plug-in that may
leave no allocations behind.  For them the library offers epic_image_static,
which keeps its tables and workspace in a fixed array in device global memory
instead of allocating.  These tests check, through the C ABI, that it

* matches the FP64 oracle and the plan-based epic_image within the FP32
  tolerance, on two calls in a row (the second must not see anything the first
  left in the shared array), for grid sides 32, 64, 96 and 128;
* leaves the device's free memory unchanged across a call (nothing allocated);
* works as the very first imaging call of a fresh process, before any plan
  exists, and keeps working plans working when it runs between them (the
  kernels' shared-memory limits are process-wide).

The file name sorts last so that a run stopping at the first failure has run
every other test first.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_2301_09662_gb300 import epic, synth

FP32_TOL = 1e-5   # the peak-relative tolerance of the FP32 parity tests
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _peak_rel(a, b, C, NP):
    a = a.reshape(C, NP, -1)
    b = b.reshape(C, NP, -1)
    errs = []
    for c in range(C):
        peak = np.max(np.abs(b[c, :2])) if NP == 4 else np.max(np.abs(b[c, 0]))
        errs.append(np.max(np.abs(a[c] - b[c])) / peak)
    return max(errs)


def _static(wl, v, g, out=None, flags=0):
    return epic.image_static(wl.ant_xy, wl.n_pol, wl.kernel, int(wl.grid_n[0]), wl.freq_hz, wl.du, v, g,
                             flags=flags, out=out)


def _inputs(wl):
    import torch
    v = torch.from_numpy(wl.v).cuda()
    g = None if wl.gains is None else torch.from_numpy(wl.gains).cuda()
    return v, g


def _check_against_oracle_and_plan(wl, got):
    import torch
    v, g = _inputs(wl)
    plan = epic.Plan.from_workload(wl)
    ref = plan.image(v, g)
    torch.cuda.synchronize()
    assert plan.status() == epic.EPIC_OK
    plan.close()
    NP = 4 if wl.n_pol == 2 else 1
    o = oracle.workload_image(wl)
    assert _peak_rel(got, o, wl.C, NP) < FP32_TOL
    assert _peak_rel(got, ref.cpu().numpy().astype(np.complex128), wl.C, NP) < FP32_TOL


@pytest.mark.gpu
def test_static_scratch_matches_oracle_and_plan_path_on_two_calls_in_a_row():
    import torch
    cases = [
        synth.random_small(A=96, P=2, C=4, T=21, N=128, K=5, seed=501),
        synth.random_small(A=40, P=2, C=3, T=9, N=64, K=3, seed=502),
        synth.random_small(A=50, P=2, C=2, T=7, N=96, K=5, seed=504),
        synth.tiny(),
    ]
    # back to back on one stream, the later call reusing the array the earlier one left
    outs = []
    for wl in cases:
        v, g = _inputs(wl)
        outs.append(_static(wl, v, g))
    torch.cuda.synchronize()
    for wl, got in zip(cases, outs):
        _check_against_oracle_and_plan(wl, got.cpu().numpy().astype(np.complex128))


@pytest.mark.gpu
def test_static_call_allocates_no_device_memory():
    import torch
    wl = synth.random_small(A=64, P=2, C=3, T=11, N=128, K=5, seed=505)
    v, g = _inputs(wl)
    out = torch.empty(wl.C * 4 * 128 * 128, dtype=torch.complex64, device="cuda")
    _static(wl, v, g, out=out)            # the first call on the device looks up the array's address
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        _static(wl, v, g, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    _check_against_oracle_and_plan(wl, out.cpu().numpy().astype(np.complex128))


@pytest.mark.gpu
def test_static_call_between_plans_keeps_larger_plans_working():
    import torch
    big = synth.random_small(A=300, P=2, C=2, T=5, N=32, K=5, seed=506)    # side 32: shared-memory kernel
    small = synth.random_small(A=20, P=2, C=2, T=5, N=32, K=3, seed=507)
    vb, gb = _inputs(big)
    plan = epic.Plan.from_workload(big)
    first = plan.image(vb, gb).cpu().numpy().astype(np.complex128)
    vs, gs = _inputs(small)
    got = _static(small, vs, gs)
    again = plan.image(vb, gb)
    torch.cuda.synchronize()
    assert plan.status() == epic.EPIC_OK
    plan.close()
    ref = oracle.workload_image(big)
    # the side-32 kernel grids with shared-memory atomics, so repeats agree to rounding, not bit for bit
    assert _peak_rel(again.cpu().numpy().astype(np.complex128), ref, big.C, 4) < FP32_TOL
    assert _peak_rel(first, ref, big.C, 4) < FP32_TOL
    assert _peak_rel(got.cpu().numpy().astype(np.complex128), oracle.workload_image(small), small.C, 4) < FP32_TOL


_FRESH = r"""
import sys
sys.path.insert(0, {root!r})
import numpy as np, torch
import oracle
from paper_2301_09662_gb300 import epic, synth
torch.cuda.set_device(0)
wl = synth.random_small(A=48, P=2, C=2, T=9, N=96, K=5, seed=508)
v = torch.from_numpy(wl.v).cuda(); g = torch.from_numpy(wl.gains).cuda()
out = epic.image_static(wl.ant_xy, 2, wl.kernel, 96, wl.freq_hz, wl.du, v, g)   # before any plan
got = out.cpu().numpy().astype(np.complex128)
plan = epic.Plan.from_workload(wl)
ref = plan.image(v, g).cpu().numpy().astype(np.complex128)
assert plan.status() == epic.EPIC_OK
o = oracle.workload_image(wl)
for c in range(wl.C):
    sl = slice(c * 4 * 96 * 96, (c + 1) * 4 * 96 * 96)
    peak = np.max(np.abs(o[sl][: 2 * 96 * 96]))
    assert np.max(np.abs(got[sl] - o[sl])) / peak < {tol}, "oracle"
    assert np.max(np.abs(got[sl] - ref[sl])) / peak < {tol}, "plan"
print("fresh ok")
"""


@pytest.mark.gpu
def test_static_call_first_in_a_fresh_process():
    code = _FRESH.format(root=ROOT, tol=FP32_TOL)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "fresh ok" in r.stdout, r.stdout + r.stderr


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
