"""CPU-side checks of the C ABI: the library loads, exports every symbol that
include/epic.h declares, and rejects bad plans on the host before any CUDA
call.  No compute runs here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2301_09662_gb300 import build_lib, epic, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_lib.build()
    return epic.load()


def header_symbols():
    src = open(os.path.join(ROOT, "include", "epic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(epic_[a-z_]+)\s*\(", src)))


def test_header_declares_the_binding_exports():
    assert header_symbols() == sorted(epic.EXPORTS)


def test_library_exports_every_header_symbol(lib):
    for name in header_symbols():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_strerror_texts(lib):
    for code in range(0, -9, -1):
        assert epic.strerror(code) not in ("", "unknown error")
    assert epic.strerror(-99) == "unknown error"


def _geom(**kw):
    wl = synth.random_small(A=8, P=2, C=2, T=4, N=32, K=3, seed=1)
    args = dict(ant_xy=wl.ant_xy, n_pol=2, kernel=wl.kernel, grid_n=wl.grid_n, freq_hz=wl.freq_hz, du=0.5,
                max_spectra=4, precision=epic.EPIC_FP32, flags=0)
    args.update(kw)
    return args


@pytest.mark.parametrize("bad,code", [
    (dict(n_pol=3), epic.EPIC_ERR_ARG),
    (dict(kernel=np.ones((2, 2), np.complex64)), epic.EPIC_ERR_ARG),
    (dict(du=0.0), epic.EPIC_ERR_ARG),
    (dict(du=0.75), epic.EPIC_ERR_ARG),
    (dict(max_spectra=-1), epic.EPIC_ERR_ARG),
    (dict(flags=64), epic.EPIC_ERR_ARG),
    (dict(flags=epic.EPIC_STOKES, n_pol=1), epic.EPIC_ERR_ARG),
    (dict(precision=9), epic.EPIC_ERR_ARG),
    (dict(grid_n=np.array([32, 40], np.int32)), epic.EPIC_ERR_UNSUPPORTED),
    (dict(freq_hz=np.array([50e6, -1.0])), epic.EPIC_ERR_ARG),
])
def test_plan_rejects_bad_arguments_on_host(lib, bad, code):
    rc, h = epic.make_plan_raw(**_geom(**bad))
    assert rc == code and not h.value


def test_plan_rejects_footprint_outside_grid(lib):
    # 60 m baselines at 80 MHz are ~32 cells at lambda/2: too wide for N = 32
    ant = np.array([[-60.0, 0.0], [60.0, 0.0], [0.0, 5.0]])
    rc, h = epic.make_plan_raw(**_geom(ant_xy=ant, grid_n=np.array([32], np.int32),
                                       freq_hz=np.array([80e6])))
    assert rc == epic.EPIC_ERR_OUT_OF_GRID and not h.value


def test_null_handles_are_rejected(lib):
    assert lib.epic_image(None, None, None, 0, None, None) == epic.EPIC_ERR_ARG
    assert lib.epic_image_host(None, None, None, 0, None, None) == epic.EPIC_ERR_ARG
    assert lib.epic_image_ex(None, None, None, None, 0, None, None) == epic.EPIC_ERR_ARG
    assert lib.epic_autotune(None, 1, None) == epic.EPIC_ERR_ARG
    assert lib.epic_image_series_ex(None, None, None, None, 0, 1, None, None) == epic.EPIC_ERR_ARG
    assert lib.epic_solve_gains(None, None, 1, 0.0, 0.0, 1, None, None) == epic.EPIC_ERR_ARG
    assert lib.epic_status(None) == epic.EPIC_ERR_ARG
    assert lib.epic_out_floats(None) == 0
    lib.epic_destroy(None)
    h = ctypes.c_void_p()
    assert lib.epic_plan(ctypes.byref(h), None, 1, 1, None, 1, None, None, 1, 0.5, 1, 0, 0) == epic.EPIC_ERR_ARG


def _seven_antennas():
    return synth.random_small(A=8, P=2, C=2, T=4, N=32, K=3, seed=1).ant_xy[:7]


@pytest.mark.parametrize("bad", [dict(grid_n=np.array([96, 96], np.int32), n_pol=1),
                                 dict(n_pol=1, ant_xy=_seven_antennas())])
def test_tensor_form_rejects_unsupported_shapes_on_host(lib, bad):
    # every channel on side 96 with single polarisation (side 96 is on the tensor cores only
    # through the dual-polarisation pair kernel), or n_ant * n_pol not a multiple of 4
    rc, h = epic.make_plan_raw(**_geom(precision=epic.EPIC_TC_SPLIT_FP16, **bad))
    assert rc == epic.EPIC_ERR_UNSUPPORTED and not h.value


def test_antenna_kernel_flag_combinations_rejected_on_host(lib):
    wl = synth.random_small(A=8, P=2, C=2, T=4, N=32, K=3, seed=1)
    Wa = synth.antenna_kernels(8, 3, np.random.default_rng(0))
    rc, h = epic.make_plan_raw(**_geom(kernel=Wa.reshape(8 * 3, 3)[:3],
                                       flags=epic.EPIC_ANTENNA_KERNELS | epic.EPIC_KERNEL_TAPER))
    assert rc == epic.EPIC_ERR_ARG and not h.value
    rc, h = epic.make_plan_raw(**_geom(flags=epic.EPIC_ANTENNA_KERNELS, precision=epic.EPIC_TC_SPLIT_FP16,
                                       grid_n=np.array([64, 64], np.int32)))
    assert rc == epic.EPIC_ERR_UNSUPPORTED and not h.value


def test_search_plan_rejects_bad_arguments_on_host(lib):
    f = np.array([42.1e6, 42.125e6, 42.15e6])
    dm = np.array([0.0, 5.0])
    h = ctypes.c_void_p()
    P = lambda a: a.ctypes.data if a is not None else None
    assert lib.epic_search_plan(ctypes.byref(h), P(f), 3, 0.04, P(dm), 2, 64, 100, 0) == epic.EPIC_ERR_ARG
    assert lib.epic_search_plan(ctypes.byref(h), P(f), 3, 0.04, P(dm), 2, 64, 100, 64) == epic.EPIC_ERR_ARG
    assert lib.epic_search_plan(ctypes.byref(h), P(f), 3, -1.0, P(dm), 2, 64, 100, 1) == epic.EPIC_ERR_ARG
    assert lib.epic_search_plan(ctypes.byref(h), None, 3, 0.04, P(dm), 2, 64, 100, 1) == epic.EPIC_ERR_ARG
    neg = np.array([-1.0])
    assert lib.epic_search_plan(ctypes.byref(h), P(f), 3, 0.04, P(neg), 1, 64, 100, 1) == epic.EPIC_ERR_ARG
    # DM 5000 delays the lowest channel by far more than 100 samples of 40 ms
    big = np.array([5000.0])
    assert lib.epic_search_plan(ctypes.byref(h), P(f), 3, 0.04, P(big), 1, 64, 100, 1) == epic.EPIC_ERR_TOO_LARGE
    assert lib.epic_search_plan(ctypes.byref(h), P(f), 3, 0.04, P(dm), 2, 64, 20, 32) == epic.EPIC_ERR_TOO_LARGE
    assert h.value is None
    assert lib.epic_search_info(None, None, None) == epic.EPIC_ERR_ARG
    assert lib.epic_search_status(None) == epic.EPIC_ERR_ARG
    assert lib.epic_dedisperse(None, None, 1, 1, 1, None, None) == epic.EPIC_ERR_ARG
    assert lib.epic_single_pulse(None, None, 0.0, None, None, None, None, 0, None, None) == epic.EPIC_ERR_ARG
    lib.epic_search_destroy(None)
