"""Python binding of the teuk C ABI (include/teuk.h): argument marshalling only.

Every step of the method runs in the CUDA library ``_build/libteuk.so``; this module only
converts arguments (numpy host arrays, torch streams) and raises on error codes. There is
no CPU fallback: without the built library or a CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_NONFINITE, ERR_STATE_MISMATCH, ERR_NO_DEVICE, ERR_TIMEOUT = (
    0, -1, -2, -3, -4, -5, -6, -7)
FP64, DD, QD = 1, 2, 4

SYMBOLS = [
    "teuk_create", "teuk_destroy", "teuk_set_initial", "teuk_set_initial_pulse", "teuk_step",
    "teuk_substep", "teuk_sync", "teuk_observe", "teuk_set_observer", "teuk_read_waveform",
    "teuk_get_state", "teuk_set_state", "teuk_get_state_device", "teuk_get_coeffs",
    "teuk_get_tortoise", "teuk_info", "teuk_kernel_launches", "teuk_strerror", "teuk_last_error",
    "teuk_mw_eval", "teuk_timing", "teuk_kernel_times", "teuk_fp64_peak", "teuk_substep_noalloc",
    "teuk_tune", "teuk_batch_create", "teuk_batch_step", "teuk_batch_sync", "teuk_batch_info",
    "teuk_batch_destroy", "teuk_use_graphs", "teuk_launch_shape",
    "teuk_set_launch_shape", "teuk_read_multipoles", "teuk_substep_host_state",
    "teuk_set_dissipation", "teuk_set_engine", "teuk_engine", "teuk_set_theta_dissipation",
    "teuk_theta_dissipation", "teuk_int_peak", "teuk_test_stall_copies", "teuk_set_persistent",
    "teuk_create_slab", "teuk_get_halo_rows", "teuk_set_halo_rows", "teuk_slab_rows",
    "teuk_set_theta_filter", "teuk_theta_filter", "teuk_theta_filter_period",
]


class TeukGrid(ctypes.Structure):
    _fields_ = [
        ("rstar_min", ctypes.c_double), ("rstar_max", ctypes.c_double),
        ("n_r", ctypes.c_int32), ("n_theta", ctypes.c_int32),
        ("dt", ctypes.c_double),
        ("substeps", ctypes.c_int32), ("theta_order", ctypes.c_int32),
        ("parity", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("ko_sigma", ctypes.c_double), ("ko_theta", ctypes.c_double),
        ("theta_filter", ctypes.c_int32), ("theta_filter_period", ctypes.c_int32),
    ]


class TeukError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"teuk error {code}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load libteuk.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise TeukError(ERR_NO_DEVICE, f"CUDA library not built: {path}")
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        d, i32, i64, vp = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        dp = P(d)
        L.teuk_create.argtypes = [P(vp), d, d, i32, i32, P(TeukGrid), i32, vp]
        L.teuk_destroy.argtypes = [vp]
        L.teuk_create_slab.argtypes = [P(vp), d, d, i32, i32, P(TeukGrid), i32, vp, i32, i32]
        L.teuk_get_halo_rows.argtypes = [vp, vp, vp]
        L.teuk_set_halo_rows.argtypes = [vp, vp, vp]
        L.teuk_slab_rows.argtypes = [vp, P(i32), P(i32), P(i32)]
        L.teuk_set_initial.argtypes = [vp, dp]
        L.teuk_set_initial_pulse.argtypes = [vp, d, d, d, d, i32]
        L.teuk_step.argtypes = [vp, i64]
        L.teuk_substep.argtypes = [vp, i64]
        L.teuk_sync.argtypes = [vp]
        L.teuk_observe.argtypes = [vp, d, dp, dp]
        L.teuk_set_observer.argtypes = [vp, d, i64]
        L.teuk_read_waveform.argtypes = [vp, dp, P(i64)]
        L.teuk_read_multipoles.argtypes = [vp, i32, i32, dp, P(i64)]
        L.teuk_substep_host_state.argtypes = [vp, dp, i64]
        L.teuk_set_dissipation.argtypes = [vp, d]
        L.teuk_set_theta_dissipation.argtypes = [vp, d]
        L.teuk_theta_dissipation.argtypes = [vp]
        L.teuk_theta_dissipation.restype = d
        L.teuk_set_theta_filter.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        L.teuk_theta_filter.argtypes = [vp]
        L.teuk_theta_filter_period.argtypes = [vp]
        L.teuk_set_engine.argtypes = [vp, i32]
        L.teuk_engine.argtypes = [vp]
        L.teuk_get_state.argtypes = [vp, dp, P(i64)]
        L.teuk_set_state.argtypes = [vp, dp, i64]
        L.teuk_get_state_device.argtypes = [vp, vp]
        L.teuk_get_coeffs.argtypes = [vp, i32, dp]
        L.teuk_get_tortoise.argtypes = [vp, i32, dp]
        L.teuk_info.argtypes = [vp, P(i32), P(i32), P(i32), P(i32), dp]
        L.teuk_kernel_launches.argtypes = [vp]
        L.teuk_kernel_launches.restype = i64
        L.teuk_strerror.argtypes = [i32]
        L.teuk_strerror.restype = ctypes.c_char_p
        L.teuk_last_error.argtypes = [vp]
        L.teuk_last_error.restype = ctypes.c_char_p
        L.teuk_mw_eval.argtypes = [i32, i32, i32, dp, dp, dp, i64]
        L.teuk_timing.argtypes = [vp, i32]
        L.teuk_kernel_times.argtypes = [vp, dp, dp, P(i64), P(i64)]
        L.teuk_fp64_peak.argtypes = [dp]
        L.teuk_int_peak.argtypes = [dp]
        L.teuk_test_stall_copies.argtypes = [vp, i32, i32]
        L.teuk_set_persistent.argtypes = [vp, i32, i32, i32]
        L.teuk_substep_noalloc.argtypes = [vp, vp, vp, i64]
        L.teuk_tune.argtypes = [vp, P(i32)]
        L.teuk_batch_create.argtypes = [P(vp), P(vp), i32]
        L.teuk_batch_step.argtypes = [vp, i64]
        L.teuk_batch_sync.argtypes = [vp]
        L.teuk_batch_info.argtypes = [vp, P(i32), P(i32), P(i64), P(i64)]
        L.teuk_batch_destroy.argtypes = [vp]
        L.teuk_use_graphs.argtypes = [vp, i32]
        L.teuk_launch_shape.argtypes = [vp, P(i32), P(i32), P(i32)]
        L.teuk_set_launch_shape.argtypes = [vp, i32, i32, i32]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _addr(buf):
    """A buffer argument as a pointer: a tensor's data, an integer address, or NULL."""
    if buf is None:
        return None
    return ctypes.c_void_p(int(buf.data_ptr()) if hasattr(buf, "data_ptr") else int(buf) or None)


def _check(rc, handle=None):
    if rc != OK:
        L = lib()
        msg = L.teuk_strerror(rc).decode()
        if handle:
            detail = L.teuk_last_error(handle).decode()
            if detail:
                msg += f" ({detail})"
        raise TeukError(rc, msg)


CUDA_STREAM_LEGACY = 1  # cudaStreamLegacy: the legacy default stream


def _current_stream():
    """torch's current CUDA stream as a cudaStream_t; the default stream (handle 0) is passed
    as cudaStreamLegacy so that the library does not create a stream of its own."""
    try:
        import torch
        if torch.cuda.is_available():
            handle = torch.cuda.current_stream().cuda_stream
            return ctypes.c_void_p(handle if handle else CUDA_STREAM_LEGACY)
    except Exception:  # torch absent or without CUDA: the library makes its own stream
        pass
    return None


class Teuk:
    """One Teukolsky problem on the GPU (see include/teuk.h)."""

    def __init__(self, *, M, a, s, m, rstar_min, rstar_max, n_r, n_theta, dt=0.0, substeps=1,
                 theta_order=10, parity=0, precision=FP64, stream="current", own_rows=None,
                 ko_sigma=0.0, ko_theta=0.0, theta_filter=0, theta_filter_period=1):
        """own_rows = (own_lo, own_hi): an r* slab of the grid (teuk_create_slab); n_r is then
        the whole grid's and self.n_r the slab's local rows (owned rows and halos)."""
        L = lib()
        self.grid = TeukGrid(float(rstar_min), float(rstar_max), int(n_r), int(n_theta), float(dt),
                             int(substeps), int(theta_order), int(parity), 0, float(ko_sigma),
                             float(ko_theta), int(theta_filter), int(theta_filter_period))
        h = ctypes.c_void_p()
        st = _current_stream() if stream == "current" else stream
        if own_rows is None:
            rc = L.teuk_create(ctypes.byref(h), float(M), float(a), int(s), int(m),
                               ctypes.byref(self.grid), int(precision), st)
        else:
            rc = L.teuk_create_slab(ctypes.byref(h), float(M), float(a), int(s), int(m),
                                    ctypes.byref(self.grid), int(precision), st, int(own_rows[0]),
                                    int(own_rows[1]))
        _check(rc)
        self._h = h
        self.words = int(precision)
        self.n_theta = int(n_theta)
        self.substeps = int(substeps)
        r0, lo, hi = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(L.teuk_slab_rows(h, ctypes.byref(r0), ctypes.byref(lo), ctypes.byref(hi)), h)
        self.row0, self.own_lo, self.own_hi = r0.value, lo.value, hi.value
        nr = ctypes.c_int()
        _check(L.teuk_info(h, None, ctypes.byref(nr), None, None, None), h)
        self.n_r = nr.value

    @classmethod
    def from_problem(cls, p, precision=None, **kw):
        g = cls(M=p.M, a=p.a, s=p.s, m=p.m, rstar_min=p.rstar_min, rstar_max=p.rstar_max,
                n_r=p.n_r, n_theta=p.n_theta, dt=0.0, substeps=p.substeps,
                theta_order=p.theta_order, parity=p.parity,
                precision=precision if precision is not None else p.words,
                ko_sigma=getattr(p, "ko_sigma", 0.0), ko_theta=getattr(p, "ko_theta", 0.0),
                theta_filter=getattr(p, "theta_filter", 0),
                theta_filter_period=getattr(p, "theta_filter_period", 1), **kw)
        return g

    def close(self):
        if getattr(self, "_h", None):
            lib().teuk_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- data in / out --------------------------------------------------------------------
    def set_initial(self, planes):
        planes = np.ascontiguousarray(planes, dtype=np.float64)
        assert planes.shape == (4, self.words, self.n_r, self.n_theta), planes.shape
        _check(lib().teuk_set_initial(self._h, _dp(planes)), self._h)

    def set_initial_pulse(self, center, width, amp_re, amp_im, ell):
        _check(lib().teuk_set_initial_pulse(self._h, float(center), float(width), float(amp_re),
                                            float(amp_im), int(ell)), self._h)

    def step(self, n_outer=1):
        _check(lib().teuk_step(self._h, int(n_outer)), self._h)

    def substep(self, n=1):
        _check(lib().teuk_substep(self._h, int(n)), self._h)

    def sync(self):
        _check(lib().teuk_sync(self._h), self._h)

    def observe(self, rstar_obs):
        out = np.empty((2, self.words, self.n_theta))
        used = ctypes.c_double()
        _check(lib().teuk_observe(self._h, float(rstar_obs), _dp(out), ctypes.byref(used)), self._h)
        return out, used.value

    def set_observer(self, rstar_obs, capacity):
        _check(lib().teuk_set_observer(self._h, float(rstar_obs), int(capacity)), self._h)

    def read_waveform(self):
        n = ctypes.c_int64()
        _check(lib().teuk_read_waveform(self._h, None, ctypes.byref(n)), self._h)
        out = np.empty((n.value, 2, self.words, self.n_theta))
        if n.value:
            _check(lib().teuk_read_waveform(self._h, _dp(out), ctypes.byref(n)), self._h)
        return out

    def set_engine(self, engine):
        """Multi-word arithmetic engine: 0 FP64 error-free transforms, 1 integer engine (dd, qd)."""
        _check(lib().teuk_set_engine(self._h, int(engine)), self._h)

    @property
    def engine(self) -> int:
        return int(lib().teuk_engine(self._h))

    def set_dissipation(self, sigma):
        """r* Kreiss-Oliger dissipation once per outer step (not part of the paper's scheme;
        0 = off)."""
        _check(lib().teuk_set_dissipation(self._h, float(sigma)), self._h)

    def set_theta_dissipation(self, sigma):
        """12th-order theta Kreiss-Oliger dissipation once per outer step (not part of the
        paper's scheme; 0 = off)."""
        _check(lib().teuk_set_theta_dissipation(self._h, float(sigma)), self._h)

    @property
    def theta_dissipation(self) -> float:
        return float(lib().teuk_theta_dissipation(self._h))

    def set_theta_filter(self, l_cut, period=1):
        """Projection of every row onto the harmonics sY_lm with l < l_cut at every period-th
        outer step (not part of the paper's scheme; l_cut = 0 = off)."""
        _check(lib().teuk_set_theta_filter(self._h, int(l_cut), int(period)), self._h)

    @property
    def theta_filter(self) -> int:
        return int(lib().teuk_theta_filter(self._h))

    @property
    def theta_filter_period(self) -> int:
        return int(lib().teuk_theta_filter_period(self._h))

    def substep_host_state(self, planes, n=1):
        """n iterations with the state held in host memory (the paper's first CUDA design's
        data flow, Sec. 4): planes [4][words][n_r][n_theta], C-contiguous float64, updated
        in place (pass page-locked memory for full link speed)."""
        assert planes.flags.c_contiguous and planes.dtype == np.float64
        assert planes.shape == (4, self.words, self.n_r, self.n_theta)
        _check(lib().teuk_substep_host_state(self._h, _dp(planes), int(n)), self._h)

    def read_multipoles(self, ell_min, ell_max):
        """Multipoles c_l(t) of the recorded waveform, computed on the device in the handle's
        precision: array [n_samples][ell_max - ell_min + 1][2 (re, im)][words]."""
        n = ctypes.c_int64()
        _check(lib().teuk_read_multipoles(self._h, int(ell_min), int(ell_max), None, ctypes.byref(n)), self._h)
        out = np.empty((n.value, ell_max - ell_min + 1, 2, self.words))
        if n.value:
            _check(lib().teuk_read_multipoles(self._h, int(ell_min), int(ell_max), _dp(out), ctypes.byref(n)),
                   self._h)
        return out

    def get_state(self):
        out = np.empty((4, self.words, self.n_r, self.n_theta))
        k = ctypes.c_int64()
        _check(lib().teuk_get_state(self._h, _dp(out), ctypes.byref(k)), self._h)
        return out

    def set_state(self, planes, substeps_done=0):
        planes = np.ascontiguousarray(planes, dtype=np.float64)
        assert planes.shape == (4, self.words, self.n_r, self.n_theta)
        _check(lib().teuk_set_state(self._h, _dp(planes), int(substeps_done)), self._h)

    def get_state_device(self, dev_ptr: int):
        _check(lib().teuk_get_state_device(self._h, ctypes.c_void_p(dev_ptr)), self._h)

    def coeffs(self, which=0):
        rows = self.n_r - 1 if which else self.n_r
        out = np.empty((8, self.words, rows, self.n_theta))
        _check(lib().teuk_get_coeffs(self._h, int(which), _dp(out)), self._h)
        return out

    def tortoise_x(self, which=0):
        rows = self.n_r - 1 if which else self.n_r
        out = np.empty((self.words, rows))
        _check(lib().teuk_get_tortoise(self._h, int(which), _dp(out)), self._h)
        return out

    def info(self):
        w, nr, nt, k = (ctypes.c_int() for _ in range(4))
        dt = ctypes.c_double()
        _check(lib().teuk_info(self._h, ctypes.byref(w), ctypes.byref(nr), ctypes.byref(nt),
                               ctypes.byref(k), ctypes.byref(dt)), self._h)
        return dict(words=w.value, n_r=nr.value, n_theta=nt.value, substeps=k.value, dt=dt.value)

    def launch_shape(self):
        tx, ty, v = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().teuk_launch_shape(self._h, ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(v)),
               self._h)
        return dict(threads_theta=tx.value, rows_per_block=ty.value, variant=v.value)

    def set_launch_shape(self, threads_theta=128, rows_per_block=1, variant=0):
        _check(lib().teuk_set_launch_shape(self._h, int(threads_theta), int(rows_per_block),
                                           int(variant)), self._h)

    def set_persistent(self, rows_per_block=2, steps_per_launch=1, threads_theta=0):
        """Outer steps in persistent cooperative launches (variant 9; small problems)."""
        _check(lib().teuk_set_persistent(self._h, int(threads_theta), int(rows_per_block),
                                         int(steps_per_launch)), self._h)

    def get_halo_rows(self, lo, hi):
        """The slab's first / last owned rows into device (or page-locked host) buffers of
        [4][words][n_theta] doubles: tensors or integer addresses (None / 0 to skip)."""
        _check(lib().teuk_get_halo_rows(self._h, _addr(lo), _addr(hi)), self._h)

    def set_halo_rows(self, lo, hi):
        """The halo rows (own_lo - 1, own_hi + 1) from buffers like get_halo_rows' (None to skip)."""
        _check(lib().teuk_set_halo_rows(self._h, _addr(lo), _addr(hi)), self._h)

    def use_graphs(self, enable=True):
        _check(lib().teuk_use_graphs(self._h, 1 if enable else 0), self._h)

    def tune(self) -> int:
        """Pick the fastest step-kernel launch shape (rows per block); state is preserved."""
        r = ctypes.c_int()
        _check(lib().teuk_tune(self._h, ctypes.byref(r)), self._h)
        return r.value

    def timing(self, enable=True):
        _check(lib().teuk_timing(self._h, 1 if enable else 0), self._h)

    def kernel_times(self):
        """(ms_half, ms_full, n_half, n_full) since the last call; clears the counters."""
        a, b = ctypes.c_double(), ctypes.c_double()
        na, nb = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().teuk_kernel_times(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(na),
                                       ctypes.byref(nb)), self._h)
        return a.value, b.value, na.value, nb.value

    @property
    def kernel_launches(self) -> int:
        return int(lib().teuk_kernel_launches(self._h))


class Batch:
    """Several Teuk problems advanced together in one cooperative launch per 200 steps."""

    def __init__(self, members):
        self.members = list(members)
        arr = (ctypes.c_void_p * len(self.members))(*[m._h.value for m in self.members])
        h = ctypes.c_void_p()
        _check(lib().teuk_batch_create(ctypes.byref(h), arr, len(self.members)))
        self._h = h

    def step(self, n_outer=1):
        rc = lib().teuk_batch_step(self._h, int(n_outer))
        if rc != OK:
            raise TeukError(rc, lib().teuk_strerror(rc).decode())

    def sync(self):
        rc = lib().teuk_batch_sync(self._h)
        if rc != OK:
            raise TeukError(rc, lib().teuk_strerror(rc).decode())

    def info(self):
        g, k = ctypes.c_int(), ctypes.c_int()
        pts, nl = ctypes.c_int64(), ctypes.c_int64()
        _check(lib().teuk_batch_info(self._h, ctypes.byref(g), ctypes.byref(k), ctypes.byref(pts),
                                     ctypes.byref(nl)))
        return dict(grid=g.value, k_max=k.value, points_per_outer_step=pts.value, launches=nl.value)

    def close(self):
        if getattr(self, "_h", None):
            lib().teuk_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fp64_peak() -> float:
    """Measured FP64 pipe operations per second of the current device."""
    v = ctypes.c_double()
    _check(lib().teuk_fp64_peak(ctypes.byref(v)))
    return v.value


def int_peak() -> float:
    """Measured product-window partial products (32-bit limb multiply-add pairs) per second of
    the current device: the integer engine's roofline unit."""
    v = ctypes.c_double()
    _check(lib().teuk_int_peak(ctypes.byref(v)))
    return v.value


def mw_eval(op: int, words: int, a, b, out=None, device: bool = True):
    """Multi-word arithmetic self-test (see teuk_mw_eval): arrays are [words, n]."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.zeros_like(a) if out is None else np.ascontiguousarray(out, dtype=np.float64).copy()
    n = a.shape[1]
    _check(lib().teuk_mw_eval(int(op), int(words), 1 if device else 0, _dp(a), _dp(b), _dp(out), n))
    return out
