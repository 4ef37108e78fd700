"""CPU oracle for the Lax-Wendroff Teukolsky step (arXiv:1006.0663, Sec. 3).

TEST INFRASTRUCTURE ONLY: the slow, plain reference that the CUDA library is checked
against. Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the product: the solver is
``teuk_oracle.cpp`` (IEEE double with FMA contraction off, or GNU MPFR at 256 bits),
compiled by :func:`build` with g++ and loaded through ctypes.

Every function of the solver follows a passage of the paper (see the header of
``teuk_oracle.cpp``); the pins live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "teuk_oracle.cpp")
_HDR = os.path.join(_HERE, "mpfr_min.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libteuk_oracle.so")
_lock = threading.Lock()
_lib = None


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("M", ctypes.c_double), ("a", ctypes.c_double),
        ("s", ctypes.c_int32), ("m", ctypes.c_int32),
        ("rstar_min", ctypes.c_double), ("rstar_max", ctypes.c_double),
        ("n_r", ctypes.c_int32), ("n_theta", ctypes.c_int32),
        ("dt", ctypes.c_double),
        ("substeps", ctypes.c_int32), ("theta_order", ctypes.c_int32),
        ("parity", ctypes.c_int32),
        ("row_lo", ctypes.c_int32), ("row_hi", ctypes.c_int32),
        ("ko_sigma", ctypes.c_double),
        ("ko_theta", ctypes.c_double),
        ("theta_filter", ctypes.c_int32),
        ("theta_filter_period", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, OpenMP, no FMA contraction)."""
    with _lock:
        os.makedirs(_BUILD, exist_ok=True)
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-l:libmpfr.so.6"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        d, i32, i64, vp = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        dp = P(d)
        L.oracle_create.restype = vp
        L.oracle_create.argtypes = [P(OracleParams), i32]
        L.oracle_destroy.argtypes = [vp]
        L.oracle_rows.argtypes = [vp]
        L.oracle_set_pulse.argtypes = [vp, d, d, d, d, i32]
        L.oracle_set_state.argtypes = [vp, dp, i32]
        L.oracle_get_state.argtypes = [vp, dp, i32]
        L.oracle_get_row.argtypes = [vp, i32, dp, i32]
        L.oracle_get_coeffs.argtypes = [vp, i32, dp, i32]
        L.oracle_get_grid.argtypes = [vp, dp, dp, dp, dp, dp, dp, i32]
        L.oracle_step.argtypes = [vp, i64]
        L.oracle_substeps_done.restype = i64
        L.oracle_substeps_done.argtypes = [vp]
        L.oracle_tortoise.argtypes = [i32, d, d, dp, i32, dp, i32]
        L.oracle_inverse_tortoise.argtypes = [i32, d, d, dp, i32, dp, i32]
        L.oracle_coeffs_at.argtypes = [i32, P(OracleParams), i32, dp, dp, dp]
        L.oracle_max_rel_err.argtypes = [vp, dp, i32, i32, i32, dp, dp]
        L.oracle_theta_op.argtypes = [i32, i32, i32, i32, dp, i32, dp, i32]
        L.oracle_spin_profile.argtypes = [i32, i32, i32, i32, i32, dp, i32]
        L.oracle_set_row.argtypes = [vp, i32, dp, i32]
        L.oracle_filter_rows.argtypes = [vp]
        L.oracle_set_forcing.argtypes = [vp, d, dp, dp]
        L.oracle_fejer_weights.argtypes = [i32, i32, dp, i32]
        L.oracle_swsh.argtypes = [i32, i32, i32, i32, i32, dp, dp, i32]
        L.oracle_project.argtypes = [i32, i32, i32, i32, i32, i32, dp, i32, i64, dp, i32]
        L.oracle_set_threads.argtypes = [i32]
        L.oracle_max_threads.restype = i32
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def default_parity(m: int, s: int) -> int:
    """Axis parity of a spin-weight-s, azimuthal-m field: (-1)^(m+s).

    sY_lm is a polynomial in sin(th/2), cos(th/2) whose every term has parity (-1)^(m+s)
    under th -> -th and th -> 2 pi - th.  For s = 0 this is the paper's rule (Sec. 3.B:
    even |m| -> d_th Phi = 0, odd |m| -> Phi = 0)."""
    return 1 if (m + s) % 2 == 0 else -1


def paper_parity(m: int) -> int:
    """The paper's rule (Sec. 3.B): even |m| -> reflection +1, odd |m| -> -1."""
    return 1 if abs(m) % 2 == 0 else -1


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(lib().oracle_max_threads())


class Oracle:
    """One problem on the CPU: a window [row_lo, row_hi] of the r* grid, all theta."""

    def __init__(self, *, M, a, s, m, rstar_min, rstar_max, n_r, n_theta, dt, substeps=1,
                 theta_order=10, parity=None, row_lo=0, row_hi=None, bits=256, ko_sigma=0.0,
                 ko_theta=0.0, theta_filter=0, theta_filter_period=1):
        if parity is None:
            parity = default_parity(m, s)
        if row_hi is None:
            row_hi = n_r - 1
        self.params = OracleParams(float(M), float(a), int(s), int(m), float(rstar_min),
                                   float(rstar_max), int(n_r), int(n_theta), float(dt),
                                   int(substeps), int(theta_order), int(parity), int(row_lo),
                                   int(row_hi), float(ko_sigma), float(ko_theta), int(theta_filter),
                                   int(theta_filter_period))
        self.bits = int(bits)
        self._h = lib().oracle_create(ctypes.byref(self.params), self.bits)
        if not self._h:
            raise ValueError("oracle: invalid parameters")
        self.nrow = int(lib().oracle_rows(self._h))
        self.nth = int(n_theta)
        self.row_lo = int(row_lo)

    def close(self):
        if getattr(self, "_h", None):
            lib().oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def pulse(self, center, width, amp_re, amp_im, ell):
        rc = lib().oracle_set_pulse(self._h, float(center), float(width), float(amp_re),
                                    float(amp_im), int(ell))
        if rc != 0:
            raise ValueError("oracle: invalid pulse")

    def set_state(self, planes: np.ndarray):
        planes = np.ascontiguousarray(planes, dtype=np.float64)
        assert planes.ndim == 4 and planes.shape[0] == 4
        assert planes.shape[2:] == (self.nrow, self.nth)
        lib().oracle_set_state(self._h, _dp(planes), planes.shape[1])

    def get_state(self, words: int = 1) -> np.ndarray:
        out = np.empty((4, words, self.nrow, self.nth))
        lib().oracle_get_state(self._h, _dp(out), words)
        return out

    def get_row(self, row: int, words: int = 1) -> np.ndarray:
        out = np.empty((4, words, self.nth))
        if lib().oracle_get_row(self._h, int(row), _dp(out), words) != 0:
            raise IndexError(row)
        return out

    def set_row(self, row: int, values: np.ndarray):
        """Overwrite one window row from values [4, words, n_theta]."""
        values = np.ascontiguousarray(values, dtype=np.float64)
        assert values.shape[0] == 4 and values.shape[2] == self.nth
        if lib().oracle_set_row(self._h, int(row), _dp(values), values.shape[1]) != 0:
            raise IndexError(row)

    def set_forcing(self, omega, f_node, f_half):
        """Test-only forcing of the Pi rows for manufactured solutions (not part of the
        method): S_Pi += e^{-i omega t} F^, F^ complex arrays [nrow][n_theta] at nodes and
        [nrow-1][n_theta] at half nodes. None switches it off."""
        if f_node is None:
            lib().oracle_set_forcing(self._h, 0.0, None, None)
            return
        fn = np.ascontiguousarray(np.stack([np.real(f_node), np.imag(f_node)]), dtype=np.float64)
        fh = np.ascontiguousarray(np.stack([np.real(f_half), np.imag(f_half)]), dtype=np.float64)
        assert fn.shape == (2, self.nrow, self.nth) and fh.shape == (2, self.nrow - 1, self.nth)
        lib().oracle_set_forcing(self._h, float(omega), _dp(fn), _dp(fh))

    def coeffs(self, which: int, words: int = 1) -> np.ndarray:
        rows = self.nrow - 1 if which else self.nrow
        out = np.empty((8, words, rows, self.nth))
        lib().oracle_get_coeffs(self._h, int(which), _dp(out), words)
        return out

    def grid(self, words: int = 1):
        rn = np.empty((words, self.nrow)); xn = np.empty((words, self.nrow))
        rh = np.empty((words, self.nrow - 1)); xh = np.empty((words, self.nrow - 1))
        th = np.empty((words, self.nth)); ct = np.empty((words, self.nth))
        lib().oracle_get_grid(self._h, _dp(rn), _dp(xn), _dp(rh), _dp(xh), _dp(th), _dp(ct), words)
        return dict(rstar_node=rn, x_node=xn, rstar_half=rh, x_half=xh, theta=th, cot_theta=ct)

    def filter_rows(self):
        """Applies the theta filter (not part of the method; the `theta_filter` parameter) to
        the current state, as at the start of an outer step."""
        if lib().oracle_filter_rows(self._h) != 0:
            raise ValueError("oracle: no theta filter on this problem")

    def step(self, n_substeps: int):
        lib().oracle_step(self._h, int(n_substeps))

    @property
    def substeps_done(self) -> int:
        return int(lib().oracle_substeps_done(self._h))

    def max_rel_err(self, planes: np.ndarray, row_a: int = 0, row_b: int | None = None):
        """max |sum_words(planes) - u| / max |u| over window rows [row_a, row_b]."""
        planes = np.ascontiguousarray(planes, dtype=np.float64)
        assert planes.shape[0] == 4 and planes.shape[2:] == (self.nrow, self.nth)
        if row_b is None:
            row_b = self.nrow - 1
        err = ctypes.c_double(); umax = ctypes.c_double()
        rc = lib().oracle_max_rel_err(self._h, _dp(planes), planes.shape[1], int(row_a), int(row_b),
                                      ctypes.byref(err), ctypes.byref(umax))
        if rc != 0:
            raise ValueError("bad rows")
        return err.value, umax.value


def tortoise(M, a, x_words, bits=256, out_words=5) -> np.ndarray:
    x = np.ascontiguousarray(np.atleast_1d(x_words), dtype=np.float64)
    out = np.empty(out_words)
    if lib().oracle_tortoise(int(bits), float(M), float(a), _dp(x), len(x), _dp(out), out_words):
        raise ValueError("oracle_tortoise")
    return out


def inverse_tortoise(M, a, rstar_words, bits=256, out_words=5) -> np.ndarray:
    r = np.ascontiguousarray(np.atleast_1d(rstar_words), dtype=np.float64)
    out = np.empty(out_words)
    if lib().oracle_inverse_tortoise(int(bits), float(M), float(a), _dp(r), len(r), _dp(out),
                                     out_words):
        raise ValueError("oracle_inverse_tortoise")
    return out


def coeffs_at(M, a, s, m, x, theta, bits=256) -> np.ndarray:
    """The 8 system coefficients at points (x = r - r+, theta): [n, 8], rounded to double."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    p = OracleParams(float(M), float(a), int(s), int(m), -1.0, 1.0, 3, 6, 0.1, 1, 10, 1, 0, 2)
    out = np.empty((len(x), 8))
    if lib().oracle_coeffs_at(int(bits), ctypes.byref(p), len(x), _dp(x), _dp(th), _dp(out)):
        raise ValueError("oracle_coeffs_at")
    return out


def theta_op(f_words, *, order=10, parity=1, bits=256, out_words=5) -> np.ndarray:
    """L_th f on the cell-centred grid of len(f) cells; f is [words, n_theta] or [n_theta]."""
    f = np.ascontiguousarray(np.atleast_2d(f_words), dtype=np.float64)
    nth = f.shape[1]
    out = np.empty((out_words, nth))
    if lib().oracle_theta_op(int(bits), nth, int(order), int(parity), _dp(f), f.shape[0], _dp(out),
                             out_words):
        raise ValueError("oracle_theta_op")
    return out


def spin_profile(s, m, ell, n_theta, *, bits=256, out_words=5) -> np.ndarray:
    """The unnormalised sY_lm profile of the initial data at theta_j: [out_words, n_theta]."""
    out = np.empty((out_words, n_theta))
    if lib().oracle_spin_profile(int(bits), int(s), int(m), int(ell), int(n_theta), _dp(out),
                                 out_words):
        raise ValueError("oracle_spin_profile")
    return out


def fejer_weights(n_theta, *, bits=256, out_words=5) -> np.ndarray:
    """Fejer's first-rule weights on the cell-centred theta grid: [out_words, n_theta]."""
    out = np.empty((out_words, n_theta))
    if lib().oracle_fejer_weights(int(bits), int(n_theta), _dp(out), out_words):
        raise ValueError("oracle_fejer_weights")
    return out


def swsh(s, m, ell, theta, *, bits=256, out_words=5) -> np.ndarray:
    """Normalised spin-weighted spherical harmonic sY_lm(theta, phi = 0): [out_words, n]."""
    th = np.ascontiguousarray(np.atleast_1d(theta), dtype=np.float64)
    out = np.empty((out_words, th.size))
    if lib().oracle_swsh(int(bits), int(s), int(m), int(ell), th.size, _dp(th), _dp(out), out_words):
        raise ValueError("oracle_swsh")
    return out


def project(s, m, ell_min, ell_max, samples, *, bits=256, out_words=5) -> np.ndarray:
    """Multipoles c_l(t) = 2 pi int Phi sY_lm sin(theta) dtheta of recorded samples given as
    word expansions [n][2][words][n_theta]: [n][ell_max - ell_min + 1][2][out_words]."""
    x = np.ascontiguousarray(samples, dtype=np.float64)
    n, two, words, nth = x.shape
    out = np.empty((n, ell_max - ell_min + 1, 2, out_words))
    if lib().oracle_project(int(bits), int(s), int(m), int(nth), int(ell_min), int(ell_max), _dp(x),
                            int(words), int(n), _dp(out), out_words):
        raise ValueError("oracle_project")
    return out


def words_to_mpf(words, mp):
    """Exact sum of double words as an mpmath number (tests only)."""
    total = mp.mpf(0)
    for w in np.atleast_1d(words):
        total += mp.mpf(float(w))
    return total
