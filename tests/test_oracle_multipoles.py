"""Pins of the oracle's multipole projection (Sec. 3.C, Fig. 1: the tail of each multipole l of
the field at the observer), checked against mathematics the oracle does not use:

* Fejer's first rule on the cell-centred nodes integrates x^p exactly for p < N;
* the normalised spin-weighted harmonics equal mpmath's Y_lm for s = 0 (Condon-Shortley
  phase) and the tabulated closed forms of -2Y_2m;
* they are orthonormal under the discrete projection (exact for l + l' < N);
* projection of a smooth non-polynomial field agrees with mpmath adaptive quadrature.
"""
import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")
mp = mpmath.mp


def _theta(n):
    return (np.arange(n) + 0.5) * np.pi / n


def _words(v, n=5):
    """mpmath number as n doubles: w[0] = round(v), w[k] = round(v - w[0] - ... - w[k-1])."""
    out = np.zeros(n)
    rest = mp.mpf(v)
    for k in range(n):
        out[k] = float(rest)
        rest -= mp.mpf(out[k])
    return out


def _mpf_words(w):
    total = mp.mpf(0)
    for x in w:
        total += mp.mpf(float(x))
    return total


@pytest.mark.parametrize("n", [7, 16, 33, 64])
def test_fejer_exact_on_polynomials(oracle_mod, n):
    mp.prec = 300
    w = oracle_mod.fejer_weights(n, bits=256, out_words=5)
    wm = [_mpf_words(w[:, j]) for j in range(n)]
    xs = [mp.cos((mp.mpf(j) + mp.mpf(1) / 2) * mp.pi / n) for j in range(n)]
    for p in range(n):
        q = mp.fsum(wj * xj ** p for wj, xj in zip(wm, xs))
        exact = mp.mpf(2) / (p + 1) if p % 2 == 0 else mp.mpf(0)
        assert abs(q - exact) < mp.mpf(2) ** -240, (n, p, q - exact)


def test_fejer_double_matches_256_bit(oracle_mod):
    w53 = oracle_mod.fejer_weights(40, bits=53, out_words=1)[0]
    w256 = oracle_mod.fejer_weights(40, bits=256, out_words=1)[0]
    np.testing.assert_allclose(w53, w256, rtol=1e-14, atol=1e-16)


@pytest.mark.parametrize("ell,m", [(0, 0), (1, 0), (1, 1), (2, 1), (3, -2), (5, 3), (8, 0)])
def test_swsh_spin0_is_ylm(oracle_mod, ell, m):
    mp.prec = 300
    th = _theta(13)
    y = oracle_mod.swsh(0, m, ell, th, bits=256, out_words=5)
    for j, t in enumerate(th):
        ref = mpmath.spherharm(ell, m, mp.mpf(float(t)), 0)
        assert abs(_mpf_words(y[:, j]) - ref.real) < mp.mpf(2) ** -240
        assert abs(ref.imag) < mp.mpf(2) ** -280


def test_swsh_spin_minus2_closed_forms(oracle_mod):
    mp.prec = 300
    th = _theta(11)
    forms = {
        2: lambda t: mp.sqrt(5 / (64 * mp.pi)) * (1 + mp.cos(t)) ** 2,
        0: lambda t: mp.sqrt(15 / (32 * mp.pi)) * mp.sin(t) ** 2,
        -2: lambda t: mp.sqrt(5 / (64 * mp.pi)) * (1 - mp.cos(t)) ** 2,
    }
    for m, f in forms.items():
        y = oracle_mod.swsh(-2, m, 2, th, bits=256, out_words=5)
        for j, t in enumerate(th):
            assert abs(_mpf_words(y[:, j]) - f(mp.mpf(float(t)))) < mp.mpf(2) ** -240, (m, j)


@pytest.mark.parametrize("s,m,n", [(0, 0, 24), (-2, 2, 24), (-1, 2, 19), (-2, -1, 30), (1, 3, 20)])
def test_projection_orthonormal(oracle_mod, s, m, n):
    mp.prec = 300
    lo = max(abs(s), abs(m))
    hi = lo + 6
    samples = np.zeros((hi - lo + 1, 2, 5, n))
    for i, ell in enumerate(range(lo, hi + 1)):
        for j in range(n):  # sY_l'm at the exact cell centres, as word expansions
            samples[i, 0, :, j] = _words(_swsh_mp(s, m, ell, (mp.mpf(j) + mp.mpf(1) / 2) * mp.pi / n))
        samples[i, 1] = 0.5 * samples[i, 0]   # exact scaling: imaginary part = Y / 2
    c = oracle_mod.project(s, m, lo, hi, samples, bits=256, out_words=5)
    for i in range(hi - lo + 1):
        for l in range(hi - lo + 1):
            if (lo + i) + (lo + l) >= n:
                continue
            expect = 1.0 if i == l else 0.0
            re = c[i, l, 0, 0] + c[i, l, 0, 1]
            im = c[i, l, 1, 0] + c[i, l, 1, 1]
            assert abs(re - expect) < 1e-30 and abs(im - 0.5 * expect) < 1e-30, (s, m, i, l, re, im)


def test_projection_of_smooth_field_matches_adaptive_quadrature(oracle_mod):
    mp.prec = 200
    n, s, m = 64, -2, 2

    def field(t):  # regular at both poles for s = -2, m = 2: cos^4(t/2) times a smooth factor
        return mp.cos(t / 2) ** 4 * mp.exp(mp.cos(t)) * (1 + mp.sin(t) ** 2 / 3)

    samples = np.zeros((1, 2, 5, n))
    for j in range(n):
        samples[0, 0, :, j] = _words(field((mp.mpf(j) + mp.mpf(1) / 2) * mp.pi / n))  # exact centre
    c = oracle_mod.project(s, m, 2, 6, samples, bits=256, out_words=5)
    for ell in range(2, 7):
        ref = 2 * mp.pi * mp.quad(lambda t: field(t) * _swsh_mp(s, m, ell, t) * mp.sin(t), [0, mp.pi / 2, mp.pi])
        got = _mpf_words(c[0, ell - 2, 0])
        assert abs(got - ref) < mp.mpf(10) ** -40, (ell, got - ref)


def _swsh_mp(s, m, ell, t):
    """Goldberg et al. sum in mpmath (the test's own transcription, for the quadrature)."""
    def fact(k):
        return mp.factorial(k)

    norm = (-1) ** m * mp.sqrt((2 * ell + 1) / (4 * mp.pi) * fact(ell + m) * fact(ell - m)
                                / (fact(ell + s) * fact(ell - s)))
    total = mp.mpf(0)
    for r in range(0, ell - s + 1):
        k2 = r + s - m
        if k2 < 0 or k2 > ell + s:
            continue
        c = mp.binomial(ell - s, r) * mp.binomial(ell + s, k2) * (-1) ** (ell - r - s)
        total += c * mp.sin(t / 2) ** (2 * ell - 2 * r - s + m) * mp.cos(t / 2) ** (2 * r + s - m)
    return norm * total
