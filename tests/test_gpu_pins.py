"""GPU-side pins: the CUDA path against values fixed by the definitions, not
only against the oracle.

* The antenna -> cell map (Sec. 3.1, nearest neighbour on a lambda/2 grid):
  antennas at metre positions whose cells are worked out by hand (ties at half
  cells, x and y offsets that differ, a centroid far from the origin) carry a
  quarter-field source phased with those hand cells, e_a = s_t (-i)^{kx_a}.
  The image then peaks at l = (N/4, 0) with the closed-form value
  (A^2 - A) sum_t |s_t|^2 (K = 1) only if the library maps every antenna to
  the hand cell: a cell off by one turns that antenna's phase by a quarter
  turn, swapped axes move the peak.
* Every ci4 byte value, -8 included (Sec. 2.1 "4+4 complex integers"):
  voltages uniform over all 256 bytes, at the full gain range, against the
  oracle in the FP32, kernel-taper and split-FP16 tensor forms.
"""
import numpy as np
import pytest

import oracle
from paper_2301_09662_gb300 import epic, synth

from gpu_helpers import peak_rel_err, run_gpu

pytestmark = pytest.mark.gpu

C0 = 299_792_458.0
TOL = 1e-5

# four antennas around the centroid (10, -4) m; at du = 0.5 and f = c0 (cells of
# 0.5 m) their offsets are (+1.5, +2.5), (-2.5, -1.5), (+1, -1), (0, 0) cells
ANT = np.array([[10.75, -2.75], [8.75, -4.75], [10.5, -4.5], [10.0, -4.0]])
# (f, N, hand cells [A][2]) at du = 0.5: k = llround(offset f / (c0 du)) + N/2
# (the half-cell offsets are ties: llround goes away from zero)
HAND = [
    (C0, 32, [[18, 19], [13, 14], [17, 15], [16, 16]]),
    (C0, 64, [[34, 35], [29, 30], [33, 31], [32, 32]]),
    (C0, 128, [[66, 67], [61, 62], [65, 63], [64, 64]]),
    (2 * C0, 128, [[67, 69], [59, 61], [66, 62], [64, 64]]),   # offsets x2: no ties
]


def _fringe_workload(f, N, cells, P):
    cells = np.array(cells)
    s = np.array([2, 1 + 1j, -1, 2j, 1 - 2j, -2])            # per-sample amplitudes
    ph = (-1j) ** (cells[:, 0] % 4)                           # source at l = (N/4, 0)
    e = s[:, None] * ph[None, :]                              # [T][A], Gaussian integers
    re = np.rint(e.real).astype(int)
    im = np.rint(e.imag).astype(int)
    v = synth.pack_ci4(re, im)[:, None, :, None].repeat(P, axis=3)   # [T][1][A][P]
    wl = synth.Workload("cell-map-pin", ANT.copy(), P, synth.gaussian_kernel(1), np.array([N], np.int32),
                        np.array([f]), 0.5, len(s), np.ascontiguousarray(v), None, {})
    return wl, float(np.sum(np.abs(s) ** 2))


@pytest.mark.parametrize("f,N,cells", HAND)
@pytest.mark.parametrize("P,precision", [(1, epic.EPIC_FP32), (2, epic.EPIC_FP32), (1, epic.EPIC_TC_SPLIT_FP16),
                                         (2, epic.EPIC_TC_SPLIT_FP16)])
def test_cell_map_hand_worked_quarter_field_peak(f, N, cells, P, precision):
    wl, s2 = _fringe_workload(f, N, cells, P)
    A = ANT.shape[0]
    gpu, plan = run_gpu(wl, precision=precision)
    plan.close()
    img = oracle.split_channels(gpu, wl.grid_n, P)[0]
    expect = (A * A - A) * s2
    i, j = N // 2, N // 2 + N // 4                             # pixel of l = (N/4, 0)
    for k in range(2 if P == 2 else 1):                       # XX (and YY)
        assert abs(img[k, i, j] - expect) < 1e-5 * expect
        assert np.abs(img[k]).max() < expect * (1 + 1e-5)     # nothing above it (grating lobes may equal it)
    if P == 2:
        assert abs(img[2, i, j] - expect) < 1e-5 * expect    # XY: identical polarisations


FULL_RANGE_CASES = [
    # A,  P, C, T,  N,   K, precision, flags
    (256, 2, 2, 9, 128, 5, epic.EPIC_FP32, 0),
    (256, 2, 2, 9, 128, 5, epic.EPIC_FP32, epic.EPIC_KERNEL_TAPER),
    (256, 2, 2, 9, 128, 5, epic.EPIC_TC_SPLIT_FP16, 0),
    (256, 2, 2, 9, 128, 5, epic.EPIC_TC_SPLIT_FP16, epic.EPIC_KERNEL_TAPER),
    (64, 1, 2, 9, 32, 3, epic.EPIC_FP32, 0),
    (64, 1, 2, 9, 32, 3, epic.EPIC_TC_SPLIT_FP16, 0),
    (100, 2, 2, 9, 96, 5, epic.EPIC_FP32, 0),
]


@pytest.mark.parametrize("A,P,C,T,N,K,precision,flags", FULL_RANGE_CASES)
def test_every_ci4_byte_value_matches_oracle(A, P, C, T, N, K, precision, flags):
    wl = synth.random_small(A=A, P=P, C=C, T=T, N=N, K=K, seed=808 + A + N, full_range=True)
    assert np.array_equal(np.unique(wl.v), np.arange(256))
    assert ((wl.v >> 4) == 8).any() and ((wl.v & 15) == 8).any()   # -8 in both parts
    gpu, plan = run_gpu(wl, precision=precision, flags=flags)
    plan.close()
    err = peak_rel_err(gpu, oracle.workload_image(wl), wl.grid_n, P)
    assert err.max() < TOL, err
