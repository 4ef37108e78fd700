"""Host-side checks of the CUDA library: it builds, loads, exports every symbol declared in
include/teuk.h, refuses bad arguments, and its multi-word arithmetic (the same header the
kernels use, compiled for the host) meets the error bounds of the published algorithms."""
import ctypes
import os
import re

import mpmath as mpm
import numpy as np
import pytest

from paper_1006_0663_gb300 import teuk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "teuk.h")).read()
    return sorted(set(re.findall(r"\b(teuk_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    L = teuk.lib()
    names = declared_symbols()
    assert len(names) >= 18
    for name in names:
        assert hasattr(L, name), name
    assert set(names) <= set(teuk.SYMBOLS) | {"teuk_create"}


def test_strerror_and_invalid_arguments():
    L = teuk.lib()
    assert L.teuk_strerror(0) == b"ok"
    assert b"invalid" in L.teuk_strerror(teuk.ERR_INVALID_ARG)
    assert b"limit" in L.teuk_strerror(teuk.ERR_TIMEOUT)
    g = teuk.TeukGrid(-10.0, 10.0, 2, 16, 0.0, 1, 10, 0, 0)  # n_r < 3
    h = ctypes.c_void_p()
    rc = L.teuk_create(ctypes.byref(h), 1.0, 0.5, -2, 2, ctypes.byref(g), 1, None)
    assert rc == teuk.ERR_INVALID_ARG
    g = teuk.TeukGrid(-10.0, 10.0, 64, 16, 0.0, 1, 10, 0, 0)
    assert L.teuk_create(ctypes.byref(h), 1.0, 1.0, -2, 2, ctypes.byref(g), 1, None) == teuk.ERR_INVALID_ARG
    assert L.teuk_create(ctypes.byref(h), 1.0, 0.5, -2, 2, ctypes.byref(g), 3, None) == teuk.ERR_INVALID_ARG
    g = teuk.TeukGrid(-10.0, 10.0, 64, 16, 0.0, 1, 4, 0, 0)  # theta order 4 unsupported
    assert L.teuk_create(ctypes.byref(h), 1.0, 0.5, -2, 2, ctypes.byref(g), 1, None) == teuk.ERR_INVALID_ARG
    n = ctypes.c_int64()
    assert L.teuk_read_multipoles(None, 0, 4, None, ctypes.byref(n)) == teuk.ERR_INVALID_ARG


def _rand_words(rng, words, n, spread=True):
    """Random normalised expansions with leading words of mixed sign and magnitude."""
    mpm.mp.prec = 400
    vals, out = [], np.zeros((words, n))
    for t in range(n):
        e = rng.integers(-30, 30) if spread else 0
        v = mpm.mpf(rng.uniform(-1, 1)) * mpm.mpf(2) ** int(e)
        for k in range(1, 6):
            v += mpm.mpf(rng.uniform(-1, 1)) * mpm.mpf(2) ** (int(e) - 53 * k)
        rest = v
        for k in range(words):
            out[k, t] = float(rest)
            rest -= out[k, t]
        vals.append(sum(mpm.mpf(float(x)) for x in out[:, t]))
    return out, vals


def _words_value(w, t):
    return sum(mpm.mpf(float(x)) for x in w[:, t])


OPS = {"add": 0, "sub": 1, "mul": 2, "div": 3, "sqrt": 4, "exp": 5, "log": 6, "acc": 7}
# relative error bounds used: dd ~ 2^-104 (JMP17: <= 4u^2 for mul, 3u^2 for accurate add),
# qd ~ 2^-205 (HLB01 quad-double bounds with margin)
BOUND = {2: 2.0 ** -101, 4: 2.0 ** -200}


@pytest.mark.parametrize("words", [2, 4])
@pytest.mark.parametrize("op", ["add", "sub", "mul", "div", "sqrt", "exp", "log"])
def test_multiword_host_vs_mpmath(words, op):
    rng = np.random.default_rng(7 + words + OPS[op])
    n = 200
    a, av = _rand_words(rng, words, n)
    b, bv = _rand_words(rng, words, n)
    if op in ("sqrt", "log"):
        a = a * np.sign(a[0])[None, :]
        av = [abs(v) for v in av]
    if op == "exp":
        a = a / 2.0 ** 30 * 40  # |x| up to ~40
        a[0] = np.clip(a[0], -700, 700)
        av = [_words_value(a, t) for t in range(n)]
    out = teuk.mw_eval(OPS[op], words, a, b, device=False)
    mpm.mp.prec = 400
    worst = 0.0
    for t in range(n):
        x, y = _words_value(a, t), _words_value(b, t)
        want = {"add": lambda: x + y, "sub": lambda: x - y, "mul": lambda: x * y,
                "div": lambda: x / y, "sqrt": lambda: mpm.sqrt(x), "exp": lambda: mpm.exp(x),
                "log": lambda: mpm.log(x)}[op]()
        got = _words_value(out, t)
        scale = abs(want)
        if op in ("add", "sub"):
            scale = abs(x) + abs(y)  # qd add is the sloppy variant (error relative to |x|+|y|)
        if op == "log":
            scale = max(abs(want), 1)
        worst = max(worst, float(abs(got - want) / scale))
    assert worst < BOUND[words] * (64 if op in ("exp", "log") else 1), worst


@pytest.mark.parametrize("words", [2, 4])
def test_dot_accumulator_host(words):
    """acc + a*b through the step kernels' accumulator: error ~ u^2 of |acc| + |a b|."""
    rng = np.random.default_rng(11 + words)
    n = 200
    a, _ = _rand_words(rng, words, n)
    b, _ = _rand_words(rng, words, n)
    c, _ = _rand_words(rng, words, n)
    out = teuk.mw_eval(OPS["acc"], words, a, b, out=c, device=False)
    worst = 0.0
    for t in range(n):
        x, y, z = _words_value(a, t), _words_value(b, t), _words_value(c, t)
        want = z + x * y
        got = _words_value(out, t)
        worst = max(worst, float(abs(got - want) / (abs(z) + abs(x * y))))
    assert worst < BOUND[words], worst


def test_no_device_is_an_error_not_a_fallback():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(teuk.TeukError) as e:
        teuk.Teuk(M=1.0, a=0.5, s=-2, m=2, rstar_min=-10, rstar_max=10, n_r=16, n_theta=16)
    assert e.value.code in (teuk.ERR_NO_DEVICE, teuk.ERR_CUDA)


@pytest.mark.parametrize("words", [2, 4])
def test_dot11_accumulator_with_cancellation_host(words):
    """The kernels' 11-term dot products (the theta stencil): weights of both signs and
    magnitude ~1e3 applied to smooth data, so that the sum cancels by ~1e3; the error stays
    at the arithmetic's level relative to sum |c_k v_k|."""
    mpm.mp.prec = 400
    n = 64
    rng = np.random.default_rng(5 + words)
    w2 = [8, -125, 1000, -6000, 42000, -73766, 42000, -6000, 1000, -125, 8]
    a = np.zeros((words, n)); b = np.zeros((words, n))
    av, bv = [], []
    for t in range(n):
        x = mpm.mpf(w2[t % 11]) / 25200 * 400 * (1 + mpm.mpf(rng.uniform(-1, 1)) * mpm.mpf(2) ** -60)
        y = mpm.cos(mpm.mpf(t) / 17) * (1 + mpm.mpf(rng.uniform(-1, 1)) * mpm.mpf(2) ** -70)
        for vals, arr, v in ((av, a, x), (bv, b, y)):
            rest = v
            for k in range(words):
                arr[k, t] = float(rest)
                rest -= arr[k, t]
            vals.append(sum(mpm.mpf(float(q)) for q in arr[:, t]))
    c = np.zeros((words, n))
    out = teuk.mw_eval(8, words, a, b, out=c, device=False)
    worst = 0.0
    for t in range(n):
        terms = [av[(t + q) % n] * bv[(t + q) % n] for q in range(11)]
        want = sum(terms)
        got = _words_value(out, t)
        worst = max(worst, float(abs(got - want) / sum(abs(x) for x in terms)))
    assert worst < BOUND[words], worst


# result, largest term (12 terms x the cut of the product window: 2^-122.4 / 2^-249.1 per
# term), larger operand
ENGINE_BOUNDS = {2: (-104, -118, -125), 4: (-208, -245, -253)}


def _rand_expansion(rng, words, e):
    v = mpm.mpf(rng.uniform(-1, 1)) * mpm.mpf(2) ** int(e)
    for k in range(1, words + 2):
        v += mpm.mpf(rng.uniform(-1, 1)) * mpm.mpf(2) ** (int(e) - 53 * k)
    out = []
    for _ in range(words):
        out.append(float(v))
        v -= mpm.mpf(out[-1])
    return out


def _val(x, t):
    return mpm.fsum(mpm.mpf(float(x[k, t])) for k in range(x.shape[0]))


@pytest.mark.parametrize("words", [2, 4])
def test_integer_engine_dot_host(words):
    """The integer engine's dot product (op 9: out + 11 products, operands with exponents spread
    over +-200 binades, zeros, repeated terms that cancel) against mpmath: the error stays within
    2^-104 (dd) / 2^-208 (qd) of the exact result plus 2^-118 / 2^-245 of the largest term."""
    mpm.mp.prec = 900
    rng = np.random.default_rng(11 + words)
    n = 160
    a = np.zeros((words, n)); b = np.zeros((words, n)); o = np.zeros((words, n))
    for t in range(n):
        a[:, t] = _rand_expansion(rng, words, rng.integers(-200, 200))
        b[:, t] = _rand_expansion(rng, words, rng.integers(-200, 200))
        o[:, t] = _rand_expansion(rng, words, rng.integers(-400, 400))
    a[:, 5] = 0; b[:, 7] = 0; o[:, 9] = 0; a[:, 40:60] = 0; o[:, 45] = 0
    a[:, 100:111] = a[:, 100:101]; b[:, 100:111] = -b[:, 100:101]
    r = teuk.mw_eval(9, words, a, b, out=o, device=False)
    er, eb, _ = ENGINE_BOUNDS[words]
    for t in range(n):
        terms = [_val(a, (t + q) % n) * _val(b, (t + q) % n) for q in range(11)] + [_val(o, t)]
        exact = mpm.fsum(terms)
        big = max(abs(x) for x in terms)
        got = _val(r, t)
        if big == 0:
            assert got == 0
            continue
        assert abs(got - exact) <= abs(exact) * mpm.mpf(2) ** er + big * mpm.mpf(2) ** eb, t
        assert abs(r[1, t]) <= np.spacing(abs(r[0, t])) / 2, t
    with pytest.raises(teuk.TeukError):
        teuk.mw_eval(9, 1, np.zeros((1, 3)), np.zeros((1, 3)), device=False)


def _words_of(v, words):
    out = []
    for _ in range(words):
        out.append(float(v))
        v -= mpm.mpf(out[-1])
    return out


@pytest.mark.parametrize("words", [2, 4])
def test_integer_engine_dot_cancellation_host(words):
    """Dot products whose exact value is far below their largest term (x y - x (y + eps) plus
    small terms, eps = 2^-80 / 2^-170 of y): the error is then governed by the bound relative
    to the largest term, N 2^-122.4 / N 2^-249.1 for N terms (the partial products a product
    window drops), and is not far below it: a window that kept fewer columns, or a bound
    claimed tighter than the window allows, fails here."""
    mpm.mp.prec = 900
    rng = np.random.default_rng(40 + words)
    n = 11  # every output sums the same 11 products (op 9 windows are circular)
    sh = 80 if words == 2 else 170
    _, eb, _ = ENGINE_BOUNDS[words]
    worst = mpm.mpf(0)
    for trial in range(40):
        a = np.zeros((words, n)); b = np.zeros((words, n)); o = np.zeros((words, n))
        x = _rand_expansion(rng, words, 0)
        y = _rand_expansion(rng, words, 0)
        eps = mpm.mpf(rng.uniform(0.5, 1.0)) * mpm.mpf(2) ** (-sh) * _val(np.array(y)[:, None], 0)
        a[:, 0] = x; b[:, 0] = y
        a[:, 1] = x; b[:, 1] = _words_of(-(_val(np.array(y)[:, None], 0) + eps), words)
        for q in range(2, n):
            a[:, q] = _rand_expansion(rng, words, -sh - 10 - int(rng.integers(0, 20)))
            b[:, q] = _rand_expansion(rng, words, 0)
        r = teuk.mw_eval(9, words, a, b, out=o, device=False)
        terms = [_val(a, q) * _val(b, q) for q in range(n)]
        exact = mpm.fsum(terms)
        big = max(abs(t) for t in terms)
        assert abs(exact) < big * mpm.mpf(2) ** (-sh + 2)
        for t in range(n):
            err = abs(_val(r, t) - exact)
            assert err <= abs(exact) * mpm.mpf(2) ** (-104 if words == 2 else -208) + big * mpm.mpf(2) ** eb, (trial, t)
            worst = max(worst, err / big)
    # the cut of the windows is visible: the error relative to the largest term is within a few
    # binades of the bound, far above the final rounding's 2^-105 |exact| share
    assert worst > mpm.mpf(2) ** (eb - 12), float(mpm.log(worst, 2))


@pytest.mark.parametrize("words", [2, 4])
def test_integer_engine_pow2_products_host(words):
    """a / 2 + b through the engine's products by powers of two (op 12: the window of 2^k v is
    v's mantissa shifted, no partial products dropped): the exact value rounded once (to the
    top 106 / 212 bits); with b = 0 or a = 0 the leading word is exactly a[0] / 2 or b[0]."""
    mpm.mp.prec = 900
    rng = np.random.default_rng(70 + words)
    n = 200
    a = np.zeros((words, n)); b = np.zeros((words, n))
    for t in range(n):
        ea = int(rng.integers(-300, 300))
        a[:, t] = _rand_expansion(rng, words, ea)
        b[:, t] = _rand_expansion(rng, words, ea + int(rng.integers(-150, 150)))
    b[:, :20] = 0.0
    a[:, 20:40] = 0.0
    r = teuk.mw_eval(12, words, a, b, device=False)
    er = -104 if words == 2 else -208
    for t in range(n):
        exact = _val(a, t) / 2 + _val(b, t)
        big = max(abs(_val(a, t)) / 2, abs(_val(b, t)))
        assert abs(_val(r, t) - exact) <= abs(exact) * mpm.mpf(2) ** er + big * mpm.mpf(2) ** -180, t
    # the leading word of a single power-of-two term is the operand's, scaled
    np.testing.assert_array_equal(r[0, :20], a[0, :20] / 2)
    np.testing.assert_array_equal(r[0, 20:40], b[0, 20:40])
    with pytest.raises(teuk.TeukError):
        teuk.mw_eval(12, 1, np.zeros((1, 3)), np.zeros((1, 3)), device=False)


@pytest.mark.parametrize("words", [2, 4])
@pytest.mark.parametrize("op", [10, 11])
def test_integer_engine_sum_host(op, words):
    """a + b and a - b through the integer engine (the smaller operand cut below the larger's
    last mantissa bit, then rounded): within 2^-104 / 2^-208 of the exact result plus
    2^-125 / 2^-253 of the larger operand; exact cancellation gives zero."""
    mpm.mp.prec = 900
    rng = np.random.default_rng(3 + op + words)
    n = 300
    a = np.zeros((words, n)); b = np.zeros((words, n))
    for t in range(n):
        ea = int(rng.integers(-60, 60))
        a[:, t] = _rand_expansion(rng, words, ea)
        b[:, t] = _rand_expansion(rng, words, ea + (int(rng.integers(-280, 280)) if t % 3 else 0))
    b[:, 10] = a[:, 10]; b[:, 11] = -a[:, 11]; a[:, 12] = 0; b[:, 13] = 0
    r = teuk.mw_eval(op, words, a, b, device=False)
    er, _, eo = ENGINE_BOUNDS[words]
    for t in range(n):
        exact = _val(a, t) + (_val(b, t) if op == 10 else -_val(b, t))
        big = max(abs(_val(a, t)), abs(_val(b, t)))
        got = _val(r, t)
        assert abs(got - exact) <= abs(exact) * mpm.mpf(2) ** er + big * mpm.mpf(2) ** eo, t
    assert r[0, 11 if op == 10 else 10] == 0.0
