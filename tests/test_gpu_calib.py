"""E-field-domain gain solver on the GPU (epic_solve_gains): exact recovery on the
integer construction, parity with the FP64 oracle on a noisy calibrator scene
with instrumental gains, and the solved gains focusing epic_image on the
calibrator."""
import numpy as np
import pytest

import oracle
from oracle import calib
from paper_2301_09662_gb300 import epic, synth

from gpu_helpers import torch_inputs

pytestmark = pytest.mark.gpu


def _solve_gpu(wl, l, m, n_iter):
    import torch
    p = epic.Plan.from_workload(wl)
    v, _ = torch_inputs(wl)
    g = p.solve_gains(v, l, m, n_iter)
    torch.cuda.synchronize()
    return g.cpu().numpy().astype(np.complex128), p


def test_exact_recovery_of_inverse_gains():
    N, A, T, C, P = 32, 14, 9, 2, 2
    wl = synth.random_small(A=A, P=P, C=C, T=T, N=N, K=1, seed=3, gains=False)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    rng = np.random.default_rng(3)
    # instrumental gains with non-negative real parts: their sum, the unit-gain beam's
    # response to the calibrator, can never vanish (the solver's one degenerate case)
    units = np.array([1, 1j, 1 + 1j, 1 - 1j])
    G = units[rng.integers(0, 4, (C, A, P))]
    s = rng.integers(-2, 3, (T, C, P)) + 1j * rng.integers(-2, 3, (T, C, P))
    s[0] = 2 + 1j
    phi = (-1j) ** ((cells[:, :, 0] + cells[:, :, 1]) % 4)
    e = s[:, :, None, :] * G[None] * phi[None, :, :, None]
    wl.v = synth.pack_ci4(np.rint(e.real).astype(int), np.rint(e.imag).astype(int))
    l = m = 1.0 / (4.0 * wl.du)
    g, _ = _solve_gpu(wl, l, m, 2)
    ref = 1.0 / G
    ref = ref * np.conj(ref[:, :1]) / np.abs(ref[:, :1])
    ref = ref / np.sqrt(np.mean(np.abs(ref) ** 2, axis=1, keepdims=True))
    assert np.max(np.abs(g - ref)) < 1e-5


def _calibrator_scene(seed, A=64, C=3, T=200, N=64, flux=9.0, noise=1.0):
    """A strong calibrator at (l, m) = (1/4, -1/8) (lattice pixel (8, -4) at N = 64,
    du = 1/2) plus noise; instrumental gains |G| in [0.7, 1.3], any phase, applied
    before quantisation."""
    wl = synth.random_small(A=A, P=2, C=C, T=T, N=N, K=5, seed=seed, gains=False)
    rng = np.random.default_rng(seed)
    l0, m0 = 0.25, -0.125
    xy = wl.ant_xy - wl.ant_xy.mean(axis=0)
    G = rng.uniform(0.7, 1.3, (C, A, 2)) * np.exp(2j * np.pi * rng.uniform(0, 1, (C, A, 2)))
    re = np.empty((T, C, A, 2), np.int64)
    im = np.empty_like(re)
    for c in range(C):
        uv = xy * (wl.freq_hz[c] / synth.C0)
        ph = np.exp(-2j * np.pi * (uv[:, 0] * l0 + uv[:, 1] * m0))
        for p in range(2):
            sig = np.sqrt(flux / 2) * (rng.standard_normal(T) + 1j * rng.standard_normal(T))
            x = (sig[:, None] * ph[None, :] + noise * (rng.standard_normal((T, A)) + 1j * rng.standard_normal((T, A))))
            x = x * G[c, :, p][None, :]
            re[:, c, :, p] = synth.quantise(x.real)
            im[:, c, :, p] = synth.quantise(x.imag)
    wl.v = synth.pack_ci4(re, im)
    return wl, l0, m0, G


@pytest.mark.parametrize("n_iter", [1, 3])
def test_parity_on_a_noisy_calibrator_scene(n_iter):
    wl, l0, m0, G = _calibrator_scene(seed=11)
    g, _ = _solve_gpu(wl, l0, m0, n_iter)
    cells = oracle.cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    ref = calib.solve_gains(wl.v, cells, wl.grid_n, l0, m0, wl.du, n_iter)
    assert np.max(np.abs(g - ref)) < 5e-5


def test_solved_gains_focus_the_image_on_the_calibrator():
    import torch
    wl, l0, m0, G = _calibrator_scene(seed=12, A=96, T=300)
    g, p = _solve_gpu(wl, l0, m0, 2)
    v, _ = torch_inputs(wl)
    N = int(wl.grid_n[0])
    i, j = int(round(m0 * N * wl.du)) + N // 2, int(round(l0 * N * wl.du)) + N // 2
    raw = p.split(p.image(v, None).cpu().numpy())
    cal = p.split(p.image(v, torch.from_numpy(g.astype(np.complex64)).cuda()).cpu().numpy())
    for c in range(wl.C):
        before, after = raw[c][0].real, cal[c][0].real      # XX
        assert np.unravel_index(np.argmax(after), after.shape) == (i, j)
        # in units of the image's own spread the calibrator stands ~30 sigma high once
        # calibrated, and is lost (|peak| ~ 1 sigma) under the random instrumental phases
        assert after[i, j] / np.std(after) > 20.0
        assert abs(before[i, j]) / np.std(before) < 5.0


def test_solver_rejects_bad_arguments():
    import torch
    wl = synth.random_small(A=8, P=2, C=1, T=4, N=64, K=3, seed=1)
    p = epic.Plan.from_workload(wl)
    v, _ = torch_inputs(wl)
    with pytest.raises(epic.EpicError):
        p.solve_gains(v, 0.1, 0.1, 0)
    big = torch.zeros((5, 1, 8, 2), dtype=torch.uint8, device="cuda")
    with pytest.raises(epic.EpicError):
        p.solve_gains(big, 0.1, 0.1, 1)
