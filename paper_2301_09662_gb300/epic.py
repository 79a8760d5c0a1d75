"""Thin Python binding of libepic (include/epic.h) over ctypes.

Argument marshalling only: every step of the imaging path runs in the CUDA
library.  PyTorch provides device memory and the current stream.  If the
library has not been built, every entry point raises (there is no CPU path).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libepic.so")

EPIC_OK = 0
EPIC_ERR_ARG = -1
EPIC_ERR_OUT_OF_GRID = -2
EPIC_ERR_UNSUPPORTED = -3
EPIC_ERR_CUDA = -4
EPIC_ERR_TIMEOUT = -5
EPIC_ERR_NOMEM = -6
EPIC_ERR_DEVICE = -7
EPIC_ERR_TOO_LARGE = -8

EPIC_FP32 = 0
EPIC_TC_SPLIT_FP16 = 1
EPIC_TC_FP16 = 2
EPIC_TC_SPLIT_BF16 = 3

EPIC_MEAN = 1
EPIC_NO_AUTOSUB = 2
EPIC_KERNEL_TAPER = 4
EPIC_STOKES = 8
EPIC_ANTENNA_KERNELS = 16
STOKES = ("I", "Q", "U", "V")

# diagnostic plan options (tests and measurements only; include/epic.h)
EPIC_DIAG_NO_GRAPH = 1 << 8
EPIC_DIAG_GATHER_GLOBAL = 1 << 9
EPIC_DIAG_NO_ALIAS = 1 << 10
EPIC_DIAG_WITHHOLD_MMA = 1 << 11
EPIC_DIAG_NO_PAIR = 1 << 12


def EPIC_DIAG_ALIAS_BATCH(n: int) -> int:
    return (int(n) & 255) << 16


EPIC_SEARCH_DIAG_DM32 = 1 << 8
EPIC_SEARCH_DIAG_DIRECT = 1 << 9
EPIC_SEARCH_DIAG_NO_PIX2 = 1 << 10
EPIC_SEARCH_DIAG_NO_TMA = 1 << 11
EPIC_SEARCH_DIAG_WITHHOLD_TMA = 1 << 12

PRODUCTS = ("XX", "YY", "XY", "YX")

#: every symbol include/epic.h declares
EXPORTS = ("epic_plan", "epic_image", "epic_image_ex", "epic_image_efield", "epic_efield_floats", "epic_measure_peak", "epic_autotune", "epic_solve_gains", "epic_image_series_ex", "epic_image_host", "epic_image_host_async", "epic_host_wait", "epic_out_floats", "epic_status",
           "epic_set_profiling", "epic_stage_times", "epic_image_static", "epic_image_series", "epic_destroy",
           "epic_strerror", "epic_search_plan", "epic_search_info", "epic_dedisperse", "epic_single_pulse",
           "epic_search_status", "epic_search_destroy")

_lib = None


class EpicError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = load().epic_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")


def load():
    """Load libepic.so (built by build_lib.build()); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i, u = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint
    L.epic_plan.argtypes = [ctypes.POINTER(vp), vp, i, i, vp, i, vp, vp, i, ctypes.c_double, i, i, u]
    L.epic_plan.restype = i
    L.epic_image.argtypes = [vp, vp, vp, i, vp, vp]
    L.epic_image.restype = i
    L.epic_image_host.argtypes = [vp, vp, vp, i, vp, vp]
    L.epic_image_series.argtypes = [vp, vp, vp, i, i, vp, vp]
    L.epic_image_series.restype = i
    L.epic_image_host.restype = i
    L.epic_image_host_async.argtypes = [vp, vp, vp, i, vp, vp]
    L.epic_image_host_async.restype = i
    L.epic_host_wait.argtypes = [vp]
    L.epic_host_wait.restype = i
    L.epic_image_ex.argtypes = [vp, vp, vp, vp, i, vp, vp]
    L.epic_image_ex.restype = i
    L.epic_autotune.argtypes = [vp, i, vp]
    L.epic_autotune.restype = i
    L.epic_solve_gains.argtypes = [vp, vp, i, ctypes.c_double, ctypes.c_double, i, vp, vp]
    L.epic_solve_gains.restype = i
    L.epic_image_series_ex.argtypes = [vp, vp, vp, vp, i, i, vp, vp]
    L.epic_image_series_ex.restype = i
    L.epic_image_efield.argtypes = [vp, vp, vp, i, vp, vp]
    L.epic_image_efield.restype = i
    L.epic_efield_floats.argtypes = [vp]
    L.epic_efield_floats.restype = ctypes.c_size_t
    L.epic_measure_peak.argtypes = [i, i, ctypes.POINTER(ctypes.c_double), vp]
    L.epic_measure_peak.restype = i
    L.epic_out_floats.argtypes = [vp]
    L.epic_out_floats.restype = ctypes.c_size_t
    L.epic_status.argtypes = [vp]
    L.epic_status.restype = i
    L.epic_set_profiling.argtypes = [vp, i]
    L.epic_set_profiling.restype = i
    L.epic_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_float), i]
    L.epic_stage_times.restype = i
    L.epic_image_static.argtypes = [vp, i, i, vp, i, i, vp, i, ctypes.c_double, vp, vp, i, u, vp, vp]
    L.epic_image_static.restype = i
    L.epic_destroy.argtypes = [vp]
    L.epic_destroy.restype = None
    L.epic_strerror.argtypes = [i]
    L.epic_strerror.restype = ctypes.c_char_p
    ll = ctypes.c_longlong
    L.epic_search_plan.argtypes = [ctypes.POINTER(vp), vp, i, ctypes.c_double, vp, i, i, i, u]
    L.epic_search_plan.restype = i
    L.epic_search_info.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i)]
    L.epic_search_info.restype = i
    L.epic_dedisperse.argtypes = [vp, vp, ll, ll, ll, vp, vp]
    L.epic_dedisperse.restype = i
    L.epic_single_pulse.argtypes = [vp, vp, ctypes.c_float, vp, vp, vp, vp, i, vp, vp]
    L.epic_single_pulse.restype = i
    L.epic_search_status.argtypes = [vp]
    L.epic_search_status.restype = i
    L.epic_search_destroy.argtypes = [vp]
    L.epic_search_destroy.restype = None
    _lib = L
    return L


def _stream_handle(stream):
    """cudaStream_t of a torch stream, a raw handle, or torch's current stream (None)."""
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def strerror(code: int) -> str:
    return load().epic_strerror(code).decode()


def _check(rc: int, what: str):
    if rc != EPIC_OK:
        raise EpicError(rc, what)


class Plan:
    """An imaging plan: array geometry, kernel, channel grid sides (epic_plan)."""

    def __init__(self, ant_xy, n_pol, kernel, grid_n, freq_hz, du=0.5, max_spectra=1000,
                 precision=EPIC_FP32, flags=0):
        L = load()
        self._ant = np.ascontiguousarray(ant_xy, np.float64)
        self._kern = np.ascontiguousarray(kernel, np.complex64)
        self.grid_n = np.ascontiguousarray(grid_n, np.int32)
        self._freq = np.ascontiguousarray(freq_hz, np.float64)
        if self._ant.ndim != 2 or self._ant.shape[1] != 2:
            raise ValueError("ant_xy must be [A][2]")
        per_antenna = bool(int(flags) & EPIC_ANTENNA_KERNELS)
        if per_antenna:
            if self._kern.ndim != 3 or self._kern.shape[0] != self._ant.shape[0] \
                    or self._kern.shape[1] != self._kern.shape[2]:
                raise ValueError("with EPIC_ANTENNA_KERNELS the kernel must be [A][K][K]")
        elif self._kern.ndim != 2 or self._kern.shape[0] != self._kern.shape[1]:
            raise ValueError("kernel must be [K][K]")
        if self.grid_n.shape != self._freq.shape:
            raise ValueError("grid_n and freq_hz must have one entry per channel")
        self.A = self._ant.shape[0]
        self.P = int(n_pol)
        self.NP = 4 if self.P == 2 else 1
        self.C = len(self._freq)
        self.K = self._kern.shape[-1]
        self.max_spectra = int(max_spectra)
        self.precision = int(precision)
        self.flags = int(flags)
        h = ctypes.c_void_p()
        rc = L.epic_plan(ctypes.byref(h), self._ant.ctypes.data, self.A, self.P, self._kern.ctypes.data,
                         self.K, self.grid_n.ctypes.data, self._freq.ctypes.data, self.C, float(du),
                         self.max_spectra, self.precision, self.flags)
        _check(rc, "epic_plan")
        self._h = h
        self.out_floats = int(L.epic_out_floats(h))

    @classmethod
    def from_workload(cls, wl, **kw):
        kw.setdefault("max_spectra", wl.T)
        return cls(wl.ant_xy, wl.n_pol, wl.kernel, wl.grid_n, wl.freq_hz, wl.du, **kw)

    @property
    def handle(self):
        return self._h.value

    def _stream(self, stream):
        return _stream_handle(stream)

    def _check_inputs(self, v, gains, device: bool):
        import torch
        if not isinstance(v, torch.Tensor) or v.dtype != torch.uint8:
            raise TypeError("v must be a torch.uint8 tensor [T][C][A][P]")
        if v.dim() != 4 or tuple(v.shape[1:]) != (self.C, self.A, self.P):
            raise ValueError(f"v must be [T][{self.C}][{self.A}][{self.P}], got {tuple(v.shape)}")
        if not v.is_contiguous():
            raise ValueError("v must be contiguous")
        if v.is_cuda != device:
            raise ValueError("v is on the wrong device for this call")
        if gains is not None:
            if gains.dtype != torch.complex64 or tuple(gains.shape) != (self.C, self.A, self.P):
                raise ValueError(f"gains must be complex64 [{self.C}][{self.A}][{self.P}]")
            if not gains.is_contiguous() or gains.is_cuda != device:
                raise ValueError("gains must be contiguous and on the same device as v")

    def image(self, v, gains=None, out=None, stream=None, delays=None):
        """Image one integration of device-resident voltages; returns (or fills)
        a flat complex64 device tensor of epic_out_floats/2 elements.  delays:
        optional float64 device tensor [T][A] of geometric delays in seconds
        (epic_image_ex, the delay-correction block of Sec. 2.2)."""
        import torch
        self._check_inputs(v, gains, device=True)
        if delays is not None:
            if (not isinstance(delays, torch.Tensor) or delays.dtype != torch.float64 or not delays.is_cuda
                    or tuple(delays.shape) != (v.shape[0], self.A) or not delays.is_contiguous()):
                raise ValueError(f"delays must be a contiguous float64 CUDA tensor [{v.shape[0]}][{self.A}]")
        if out is None:
            out = torch.empty(self.out_floats // 2, dtype=torch.complex64, device=v.device)
        elif out.dtype != torch.complex64 or out.numel() * 2 != self.out_floats or not out.is_contiguous():
            raise ValueError("out must be a contiguous complex64 tensor of the plan's output size")
        g = gains.data_ptr() if gains is not None else None
        if delays is None:
            rc = load().epic_image(self._h, v.data_ptr(), g, int(v.shape[0]), out.data_ptr(), self._stream(stream))
            _check(rc, "epic_image")
        else:
            rc = load().epic_image_ex(self._h, v.data_ptr(), g, delays.data_ptr(), int(v.shape[0]), out.data_ptr(),
                                      self._stream(stream))
            _check(rc, "epic_image_ex")
        return out

    def image_efield(self, v, gains=None, out=None, stream=None):
        """E-field images of every sample (epic_image_efield): a complex64
        device tensor [T][epic_efield_floats/2], per sample the channels packed,
        each [P][N][N] fft-shifted."""
        import torch
        self._check_inputs(v, gains, device=True)
        T = int(v.shape[0])
        per = int(load().epic_efield_floats(self._h)) // 2
        if out is None:
            out = torch.empty((T, per), dtype=torch.complex64, device=v.device)
        elif out.dtype != torch.complex64 or out.numel() != T * per or not out.is_contiguous():
            raise ValueError("out must be a contiguous complex64 tensor of T x epic_efield_floats/2 elements")
        rc = load().epic_image_efield(self._h, v.data_ptr(), gains.data_ptr() if gains is not None else None, T,
                                      out.data_ptr(), self._stream(stream))
        _check(rc, "epic_image_efield")
        return out

    def autotune(self, n_spectra, stream=None):
        """Time a few launch shapes per channel group for n_spectra and keep the
        fastest (epic_autotune); blocks until done."""
        _check(load().epic_autotune(self._h, int(n_spectra), self._stream(stream)), "epic_autotune")

    def solve_gains(self, v, l, m, n_iter=2, out=None, stream=None):
        """Per-antenna gains from one calibrator at direction cosines (l, m)
        (epic_solve_gains); returns a complex64 device tensor [C][A][P]."""
        import torch
        self._check_inputs(v, None, device=True)
        if out is None:
            out = torch.empty((self.C, self.A, self.P), dtype=torch.complex64, device=v.device)
        rc = load().epic_solve_gains(self._h, v.data_ptr(), int(v.shape[0]), float(l), float(m), int(n_iter),
                                     out.data_ptr(), self._stream(stream))
        _check(rc, "epic_solve_gains")
        return out

    def image_series(self, v, spectra_per_image, gains=None, out=None, stream=None, delays=None):
        """Time-resolved images: one image per block of spectra_per_image spectra
        (epic_image_series, or epic_image_series_ex with [T][A] float64 device
        delays); returns a [n_img, out_floats/2] complex64 tensor."""
        import torch
        self._check_inputs(v, gains, device=True)
        T = int(v.shape[0])
        if spectra_per_image < 1 or T % spectra_per_image:
            raise ValueError("n_spectra must be a positive multiple of spectra_per_image")
        if delays is not None and (not isinstance(delays, torch.Tensor) or delays.dtype != torch.float64
                                   or not delays.is_cuda or tuple(delays.shape) != (T, self.A)
                                   or not delays.is_contiguous()):
            raise ValueError(f"delays must be a contiguous float64 CUDA tensor [{T}][{self.A}]")
        n_img = T // spectra_per_image
        if out is None:
            out = torch.empty((n_img, self.out_floats // 2), dtype=torch.complex64, device=v.device)
        rc = load().epic_image_series_ex(self._h, v.data_ptr(), gains.data_ptr() if gains is not None else None,
                                         delays.data_ptr() if delays is not None else None, T,
                                         int(spectra_per_image), out.data_ptr(), self._stream(stream))
        _check(rc, "epic_image_series_ex")
        return out

    def image_host(self, v, gains=None, out=None, stream=None):
        """Host-buffer variant (epic_image_host): copies in, images, copies out."""
        import torch
        self._check_inputs(v, gains, device=False)
        if out is None:
            out = torch.empty(self.out_floats // 2, dtype=torch.complex64)
        rc = load().epic_image_host(self._h, v.data_ptr(), gains.data_ptr() if gains is not None else None,
                                    int(v.shape[0]), out.data_ptr(), self._stream(stream))
        _check(rc, "epic_image_host")
        return out

    def image_host_async(self, v, gains=None, out=None, stream=None):
        """Pipelined host-buffer variant (epic_image_host_async): queues upload,
        imaging and download and returns at once; call host_wait() before reading
        `out` or changing the inputs.  Host tensors should be pinned."""
        import torch
        self._check_inputs(v, gains, device=False)
        if out is None:
            out = torch.empty(self.out_floats // 2, dtype=torch.complex64).pin_memory()
        elif out.dtype != torch.complex64 or out.numel() * 2 != self.out_floats or not out.is_contiguous() \
                or out.is_cuda:
            raise ValueError("out must be a contiguous host complex64 tensor of the plan's output size")
        rc = load().epic_image_host_async(self._h, v.data_ptr(), gains.data_ptr() if gains is not None else None,
                                          int(v.shape[0]), out.data_ptr(), self._stream(stream))
        _check(rc, "epic_image_host_async")
        return out

    def host_wait(self):
        """Block until every queued image_host_async call's copies have finished."""
        _check(load().epic_host_wait(self._h), "epic_host_wait")

    def split(self, flat):
        """Per-channel [NP][N][N] views of a packed output."""
        res, off = [], 0
        for N in self.grid_n:
            sz = self.NP * int(N) * int(N)
            res.append(flat[off:off + sz].reshape(self.NP, int(N), int(N)))
            off += sz
        return res

    def stage_names(self):
        names = [] if self.flags & EPIC_NO_AUTOSUB else ["autopower"]
        for N in sorted(set(int(n) for n in self.grid_n)):
            names += [f"image[N={N}]", f"epilogue[N={N}]"]
        return names

    def set_profiling(self, on: bool = True):
        _check(load().epic_set_profiling(self._h, int(bool(on))), "epic_set_profiling")

    def stage_times(self):
        """{stage name: device ms} of the last epic_image call (profiling on)."""
        names = self.stage_names()
        buf = (ctypes.c_float * len(names))()
        n = load().epic_stage_times(self._h, buf, len(names))
        if n < 0:
            _check(n, "epic_stage_times")
        return {names[i]: float(buf[i]) for i in range(n)}

    def status(self) -> int:
        return load().epic_status(self._h)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().epic_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def image_static(ant_xy, n_pol, kernel, grid_n, freq_hz, du, v, gains=None, flags=0, out=None, stream=None):
    """epic_image_static: plan-free imaging with no device allocation (one grid
    side for all channels).  v, gains, out are device tensors as for Plan.image."""
    import torch
    L = load()
    ant = np.ascontiguousarray(ant_xy, np.float64)
    kern = np.ascontiguousarray(kernel, np.complex64)
    fr = np.ascontiguousarray(freq_hz, np.float64)
    C, A, P = len(fr), ant.shape[0], int(n_pol)
    if v.dtype != torch.uint8 or not v.is_cuda or not v.is_contiguous() or tuple(v.shape[1:]) != (C, A, P):
        raise ValueError(f"v must be a contiguous CUDA uint8 tensor [T][{C}][{A}][{P}]")
    if gains is not None and (gains.dtype != torch.complex64 or not gains.is_cuda or not gains.is_contiguous()
                              or tuple(gains.shape) != (C, A, P)):
        raise ValueError(f"gains must be a contiguous CUDA complex64 tensor [{C}][{A}][{P}]")
    NP = 4 if P == 2 else 1
    n_out = C * NP * int(grid_n) * int(grid_n)
    if out is None:
        out = torch.empty(n_out, dtype=torch.complex64, device=v.device)
    elif out.dtype != torch.complex64 or out.numel() != n_out or not out.is_contiguous():
        raise ValueError("out must be a contiguous complex64 tensor of C*NP*N*N elements")
    s = torch.cuda.current_stream() if stream is None else stream
    rc = L.epic_image_static(ant.ctypes.data, A, P, kern.ctypes.data, kern.shape[0], int(grid_n), fr.ctypes.data,
                             C, float(du), v.data_ptr(), gains.data_ptr() if gains is not None else None,
                             int(v.shape[0]), int(flags), out.data_ptr(), ctypes.c_void_p(s.cuda_stream))
    _check(rc, "epic_image_static")
    return out


PEAKS = {"fp32": 0, "fp32x2": 1, "fp64": 2, "fp16_tc": 3}


def measure_peak(what: str, ms: int = 100, stream=None) -> float:
    """Measured peak rate (TFLOP/s) of one arithmetic pipe (epic_measure_peak):
    'fp32', 'fp32x2' (packed FMA pairs), 'fp64' or 'fp16_tc' (dense tcgen05)."""
    out = ctypes.c_double()
    _check(load().epic_measure_peak(PEAKS[what], int(ms), ctypes.byref(out), _stream_handle(stream)),
           "epic_measure_peak")
    return out.value


def make_plan_raw(ant_xy, n_pol, kernel, grid_n, freq_hz, du=0.5, max_spectra=16, precision=EPIC_FP32,
                  flags=0):
    """Call epic_plan and return (rc, handle) without raising (for error-path tests)."""
    L = load()
    ant = np.ascontiguousarray(ant_xy, np.float64)
    kern = np.ascontiguousarray(kernel, np.complex64)
    gn = np.ascontiguousarray(grid_n, np.int32)
    fr = np.ascontiguousarray(freq_hz, np.float64)
    h = ctypes.c_void_p()
    rc = L.epic_plan(ctypes.byref(h), ant.ctypes.data, ant.shape[0], int(n_pol), kern.ctypes.data, kern.shape[0],
                     gn.ctypes.data, fr.ctypes.data, len(fr), float(du), int(max_spectra), int(precision), int(flags))
    return rc, h


class Search:
    """De-dispersion and single-pulse search of an intensity cube (epic_search_*).

    freq_hz [C], dt_s, dms [n_dm] (pc cm^-3), n_pix, n_time; widths: boxcar
    widths, powers of two up to 32; diag: EPIC_SEARCH_DIAG_* options (tests)."""

    def __init__(self, freq_hz, dt_s, dms, n_pix, n_time, widths=(1, 2, 4, 8, 16, 32), diag=0):
        L = load()
        self._f = np.ascontiguousarray(freq_hz, np.float64)
        self._dm = np.ascontiguousarray(dms, np.float64)
        mask = 0
        for w in widths:
            k = int(w).bit_length() - 1
            if int(w) != 1 << k or k > 5:
                raise ValueError("widths must be powers of two up to 32")
            mask |= 1 << k
        self.C, self.n_dm, self.n_pix, self.n_time = len(self._f), len(self._dm), int(n_pix), int(n_time)
        self._h = ctypes.c_void_p()
        rc = L.epic_search_plan(ctypes.byref(self._h), self._f.ctypes.data, self.C, float(dt_s), self._dm.ctypes.data,
                                self.n_dm, self.n_pix, self.n_time, mask | int(diag))
        _check(rc, "epic_search_plan")
        t_out, smax = ctypes.c_int(), ctypes.c_int()
        _check(L.epic_search_info(self._h, ctypes.byref(t_out), ctypes.byref(smax)), "epic_search_info")
        self.t_out, self.max_shift = t_out.value, smax.value

    def dedisperse(self, cube, strides=None, out=None, stream=None):
        """cube: float32 CUDA tensor; strides (t, c, p) in elements, default the
        contiguous [n_time][C][n_pix] layout.  Returns dd [n_dm][t_out][n_pix]."""
        import torch
        if not isinstance(cube, torch.Tensor) or cube.dtype != torch.float32 or not cube.is_cuda:
            raise TypeError("cube must be a float32 CUDA tensor")
        ts, cs, ps = strides if strides is not None else (self.C * self.n_pix, self.n_pix, 1)
        last = (self.n_time - 1) * ts + (self.C - 1) * cs + (self.n_pix - 1) * ps
        if min(ts, cs, ps) < 1 or last >= cube.numel() or not cube.is_contiguous():
            raise ValueError("cube is too small for the plan's shape and these strides")
        if out is None:
            out = torch.empty((self.n_dm, self.t_out, self.n_pix), dtype=torch.float32, device=cube.device)
        rc = load().epic_dedisperse(self._h, cube.data_ptr(), int(ts), int(cs), int(ps), out.data_ptr(),
                                    _stream_handle(stream))
        _check(rc, "epic_dedisperse")
        return out

    def single_pulse(self, dd, threshold, cand_cap=4096, stream=None):
        """Returns (best_snr, best_t, best_w [n_dm][n_pix], cand [cap][2] int32, n_cand) on the device."""
        import torch
        if (dd.dtype != torch.float32 or not dd.is_cuda or not dd.is_contiguous()
                or tuple(dd.shape) != (self.n_dm, self.t_out, self.n_pix)):
            raise ValueError(f"dd must be float32 CUDA [{self.n_dm}][{self.t_out}][{self.n_pix}]")
        dev = dd.device
        snr = torch.empty((self.n_dm, self.n_pix), dtype=torch.float32, device=dev)
        bt = torch.empty((self.n_dm, self.n_pix), dtype=torch.int32, device=dev)
        bw = torch.empty_like(bt)
        cand = torch.empty((max(int(cand_cap), 1), 2), dtype=torch.int32, device=dev)
        n = torch.empty(1, dtype=torch.int32, device=dev)
        rc = load().epic_single_pulse(self._h, dd.data_ptr(), float(threshold), snr.data_ptr(), bt.data_ptr(),
                                      bw.data_ptr(), cand.data_ptr(), int(cand_cap), n.data_ptr(),
                                      _stream_handle(stream))
        _check(rc, "epic_single_pulse")
        return snr, bt, bw, cand, n

    def status(self) -> int:
        """Sticky device status (EPIC_OK or EPIC_ERR_TIMEOUT); reading clears it."""
        return load().epic_search_status(self._h)

    def close(self):
        if self._h:
            load().epic_search_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

