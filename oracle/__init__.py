"""FP64 CPU oracle for the EPIC imaging path (ctypes wrapper over epic_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The CUDA library never imports this
package, and the C source shares no code with it.

Functions (each cites the passage it follows; see epic_oracle.c for the
readings of points the paper leaves open):
  ci4_unpack      Sec. 2.1, 4+4-bit complex samples
  cell_map        Sec. 3.1, nearest-neighbour antenna -> grid-cell map
  kernel_power    |W^(l)|^2, the image of one antenna's footprint (Eq. 4)
  fft1d / ifft2   the oracle's own mixed-radix FFT (Eq. 4's FT^-1)
  epic_direct     O1, Eq. 4 with the block chain of Sec. 2.2 (optionally with
                  the delay-correction block's per-(t, a) phases)
  epic_fx         O2, Eq. 1-3 (FX correlator + gridding with W (x) W^*)
                  (both take one [K][K] kernel or per-antenna [A][K][K] kernels, Eq. 3)
  grid_energy     sum_t sum_k |G_p(k, t)|^2 with O1's gridding (Parseval pin)
  epic_efield     O1's steps a1-a4 alone: the electric-field image F_p(l, t) of
                  every sample (the abstract and Sec. 1, "electric field or
                  intensity images"), fft-shifted, no products
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "epic_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MEAN = 1
NO_AUTOSUB = 2


def build(force: bool = False) -> str:
    """Compile epic_oracle.c with gcc (OpenMP) into liboracle.so next to it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=gnu11", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i = ctypes.c_int
            L.oracle_ci4_unpack.argtypes = [ctypes.c_uint8, ctypes.POINTER(i), ctypes.POINTER(i)]
            L.oracle_cell_map.argtypes = [P, i, P, i, P, ctypes.c_double, P]
            L.oracle_cell_map.restype = i
            L.oracle_kernel_power.argtypes = [P, i, i, P]
            L.oracle_fft1d.argtypes = [P, i, i]
            L.oracle_ifft2.argtypes = [P, i]
            for name in ("oracle_epic_direct", "oracle_epic_fx"):
                f = getattr(L, name)
                f.argtypes = [P, P, i, i, i, i, P, P, P, i, i, P, P, ctypes.c_uint, P]
                f.restype = i
            L.oracle_epic_efield.argtypes = [P, P, i, i, i, i, P, P, P, i, i, P, P, P]
            L.oracle_epic_efield.restype = i
            L.oracle_grid_energy.argtypes = [P, P, i, i, i, i, P, P, P, i, i, P]
            L.oracle_grid_energy.restype = i
            L.oracle_threads.restype = i
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def threads() -> int:
    return lib().oracle_threads()


def ci4_unpack(b: int) -> tuple[int, int]:
    re, im = ctypes.c_int(), ctypes.c_int()
    lib().oracle_ci4_unpack(int(b), ctypes.byref(re), ctypes.byref(im))
    return re.value, im.value


def cell_map(ant_xy, freq_hz, grid_n, du) -> np.ndarray:
    ant = np.ascontiguousarray(ant_xy, np.float64)
    f = np.ascontiguousarray(freq_hz, np.float64)
    n = np.ascontiguousarray(grid_n, np.int32)
    out = np.zeros((len(f), ant.shape[0], 2), np.int32)
    rc = lib().oracle_cell_map(_ptr(ant), ant.shape[0], _ptr(f), len(f), _ptr(n), float(du), _ptr(out))
    if rc:
        raise ValueError("oracle_cell_map: bad arguments")
    return out


def kernel_power(W, N: int) -> np.ndarray:
    w = np.ascontiguousarray(W, np.complex128)
    out = np.zeros((N, N), np.float64)
    lib().oracle_kernel_power(_ptr(w), w.shape[0], N, _ptr(out))
    return out


def fft1d(x, sign: int = +1) -> np.ndarray:
    y = np.ascontiguousarray(x, np.complex128).copy()
    lib().oracle_fft1d(_ptr(y), len(y), sign)
    return y


def ifft2(g) -> np.ndarray:
    y = np.ascontiguousarray(g, np.complex128).copy()
    lib().oracle_ifft2(_ptr(y), y.shape[0])
    return y


def _common(v, gains, cells, grid_n, W):
    """W is [K][K] (one kernel) or [A][K][K] (one kernel per antenna)."""
    v = np.ascontiguousarray(v, np.uint8)
    T, C, A, P = v.shape
    g = None if gains is None else np.ascontiguousarray(gains, np.complex128)
    cells = np.ascontiguousarray(cells, np.int32)
    n = np.ascontiguousarray(grid_n, np.int32)
    w = np.ascontiguousarray(W, np.complex128)
    if w.ndim == 3 and w.shape[0] != A:
        raise ValueError("per-antenna kernels must be [A][K][K]")
    return v, g, cells, n, w, T, C, A, P


def out_size(grid_n, P) -> int:
    NP = 4 if P == 2 else 1
    return int(sum(NP * int(N) * int(N) for N in grid_n))


def split_channels(flat, grid_n, P):
    """Split the packed output into a list of [NP][N][N] complex arrays."""
    NP = 4 if P == 2 else 1
    out, off = [], 0
    for N in grid_n:
        sz = NP * int(N) * int(N)
        out.append(flat[off:off + sz].reshape(NP, N, N))
        off += sz
    return out


def _run(name, v, gains, cells, grid_n, W, flags, freq=None, delays=None):
    v, g, cells, n, w, T, C, A, P = _common(v, gains, cells, grid_n, W)
    f = d = None
    if delays is not None:
        if freq is None:
            raise ValueError("delays need the channel frequencies")
        f = np.ascontiguousarray(freq, np.float64)
        d = np.ascontiguousarray(delays, np.float64)
        if f.shape != (C,) or d.shape != (T, A):
            raise ValueError("freq must be [C] and delays [T][A]")
    out = np.zeros(out_size(n, P), np.complex128)
    rc = getattr(lib(), name)(_ptr(v), _ptr(g), T, C, A, P, _ptr(cells), _ptr(n), _ptr(w),
                              w.shape[-1], int(w.ndim == 3), _ptr(f), _ptr(d), int(flags), _ptr(out))
    if rc:
        raise ValueError(f"{name}: bad arguments")
    return out


def epic_direct(v, gains, cells, grid_n, W, flags: int = 0, freq=None, delays=None) -> np.ndarray:
    """O1: packed complex128 output, per channel [NP][N][N] (XX, YY, XY, YX).
    delays ([T][A] seconds, with freq [C] Hz) apply the Sec. 2.2 delay correction."""
    return _run("oracle_epic_direct", v, gains, cells, grid_n, W, flags, freq, delays)


def epic_fx(v, gains, cells, grid_n, W, flags: int = 0, freq=None, delays=None) -> np.ndarray:
    """O2: same output as epic_direct, by the FX-correlator route."""
    return _run("oracle_epic_fx", v, gains, cells, grid_n, W, flags, freq, delays)


def epic_efield(v, gains, cells, grid_n, W, freq=None, delays=None) -> np.ndarray:
    """E-field images F_p(l, t): complex128 [T][sum_c P N_c^2], per sample the
    channels packed in order, each [P][N][N] on the fft-shifted layout."""
    v, g, cells, n, w, T, C, A, P = _common(v, gains, cells, grid_n, W)
    f = d = None
    if delays is not None:
        f = np.ascontiguousarray(freq, np.float64)
        d = np.ascontiguousarray(delays, np.float64)
        if f.shape != (C,) or d.shape != (T, A):
            raise ValueError("freq must be [C] and delays [T][A]")
    per = int(sum(P * int(N) * int(N) for N in n))
    out = np.zeros((T, per), np.complex128)
    rc = lib().oracle_epic_efield(_ptr(v), _ptr(g), T, C, A, P, _ptr(cells), _ptr(n), _ptr(w), w.shape[-1],
                                  int(w.ndim == 3), _ptr(f), _ptr(d), _ptr(out))
    if rc:
        raise ValueError("oracle_epic_efield: bad arguments")
    return out


def workload_efield(wl, channels=None) -> np.ndarray:
    """epic_efield on a synth.Workload (optionally a subset of channels)."""
    cells = cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    v, g, grid_n = wl.v, wl.gains, wl.grid_n
    if channels is not None:
        ch = np.asarray(channels)
        v, g, cells, grid_n = v[:, ch], (None if g is None else g[ch]), cells[ch], grid_n[ch]
    return epic_efield(v, g, cells, grid_n, wl.kernel)


def grid_energy(v, gains, cells, grid_n, W) -> np.ndarray:
    v, g, cells, n, w, T, C, A, P = _common(v, gains, cells, grid_n, W)
    out = np.zeros((C, P), np.float64)
    rc = lib().oracle_grid_energy(_ptr(v), _ptr(g), T, C, A, P, _ptr(cells), _ptr(n), _ptr(w),
                                  w.shape[-1], int(w.ndim == 3), _ptr(out))
    if rc:
        raise ValueError("oracle_grid_energy: bad arguments")
    return out


def workload_image(wl, flags: int = 0, channels=None, form: str = "direct", delays=None) -> np.ndarray:
    """Run O1 (or O2) on a synth.Workload, optionally on a subset of channels
    and with [T][A] geometric delays.

    Returns the packed output for the selected channels in channel order."""
    cells = cell_map(wl.ant_xy, wl.freq_hz, wl.grid_n, wl.du)
    v, g, grid_n, freq = wl.v, wl.gains, wl.grid_n, wl.freq_hz
    if channels is not None:
        ch = np.asarray(channels)
        v = v[:, ch]
        g = None if g is None else g[ch]
        cells = cells[ch]
        grid_n = grid_n[ch]
        freq = freq[ch]
    fn = epic_direct if form == "direct" else epic_fx
    return fn(v, g, cells, grid_n, wl.kernel, flags, freq=freq, delays=delays)
