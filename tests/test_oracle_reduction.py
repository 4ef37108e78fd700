"""Pin: the oracle's first-order system is the Teukolsky master equation (Eq. 1).

The paper leaves the matrices M, L, A of Eq. evln unprinted. This test starts from Eq. 1 as
printed (Sec. 3.A), substitutes the ansatz Psi = e^{i m phi~} r^3 Phi (Eq. psiphi) with
d phi~ = d phi + a/Delta dr and the tortoise derivative d/dr = (r^2+a^2)/Delta d/dr*
(Sec. 3.B), and reads off every coefficient of the resulting second-order equation with
sympy. The first-order system u_t + D u' = S with Pi = Phi_t + b Phi' (Sec. 3.B) implies

    Sigma^2 [Phi_tt - b^2 Phi'' + beta Phi_t + (c - b b' + beta b) Phi' - g L_th Phi - nu Phi]

for the same operator (times -1), so the oracle's b, c, beta = B/Sigma^2, g = Delta/Sigma^2,
nu = V/Sigma^2 are compared with the sympy-derived values at random points.
"""
import random

import mpmath as mpm
import numpy as np
import pytest

sp = pytest.importorskip("sympy")
from tests.eq1_symbolic import eq1_functions  # noqa: E402


def reduced_coefficients(s_val: int, m_val: int):
    return eq1_functions(s_val, m_val, "mpmath")


def expected_system(s, m, Mv, av, r, th):
    """b, c_R, c_I, beta_R, beta_I, g, nu_R, nu_I from the sympy coefficients of Eq. 1."""
    e_tt, e_t, e_rr, e_r, e_thth, e_th, e_0 = [f(r, th, Mv, av) for f in reduced_coefficients(s, m)]
    Delta = r**2 - 2 * Mv * r + av**2
    R = r**2 + av**2
    Sig2 = R**2 - av**2 * Delta * mpm.sin(th) ** 2
    assert abs(e_tt + Sig2) <= 1e-30 * abs(Sig2)
    # Phi'' coefficient: e_rr (R/Delta)^2 must be R^2 = Sigma^2 b^2
    assert abs(e_rr * (R / Delta) ** 2 - R**2) <= 1e-30 * R**2
    assert abs(e_th - e_thth * mpm.cot(th)) <= 1e-30 * (1 + abs(e_th))
    b_of = lambda rr: (rr**2 + av**2) / mpm.sqrt((rr**2 + av**2) ** 2 - av**2 * (rr**2 - 2 * Mv * rr + av**2) * mpm.sin(th) ** 2)
    b = b_of(r)
    bbp = b * (Delta / R) * mpm.diff(b_of, r)
    dRD = mpm.diff(lambda rr: (rr**2 + av**2) / (rr**2 - 2 * Mv * rr + av**2), r)
    beta = -e_t / Sig2
    phi_prime = e_r * (R / Delta) + e_rr * dRD
    c = bbp - beta * b - phi_prime / Sig2
    g = e_thth / Sig2
    nu = e_0 / Sig2
    return [b, c.real, c.imag, beta.real, beta.imag, g, nu.real, nu.imag]


@pytest.mark.parametrize("s,m", [(0, 0), (0, 2), (-2, 2), (-1, -3), (1, 1), (-2, -1)])
def test_coefficients_match_eq1(oracle_mod, s, m):
    mpm.mp.dps = 40
    rng = random.Random(1000 + 17 * s + m)
    for a in (0.0, 0.5, 0.9):
        rp = 1 + mpm.sqrt(1 - mpm.mpf(a) ** 2)
        xs, ths = [], []
        for _ in range(4):
            xs.append(float(rng.choice([0.05, 0.7, 3.0, 25.0]) * (0.5 + rng.random())))
            ths.append(0.15 + 2.8 * rng.random())
        got = oracle_mod.coeffs_at(1.0, a, s, m, np.array(xs), np.array(ths), bits=256)
        for k, (x, th) in enumerate(zip(xs, ths)):
            want = expected_system(s, m, mpm.mpf(1), mpm.mpf(a), rp + mpm.mpf(x), mpm.mpf(th))
            scale = max(abs(float(w)) for w in want)
            for c in range(8):
                assert abs(got[k, c] - float(want[c])) <= 1e-13 * max(abs(float(want[c])), 1e-3 * scale), \
                    (a, x, th, c, got[k, c], float(want[c]))


def test_d_matrix_signs(oracle_mod):
    """Eq. d_matrix: the Phi rows move with +b, the Pi rows with -b; b -> 1 at the horizon
    and at large r, and 0 < b <= 1 + O(a^2/r^2) everywhere."""
    got = oracle_mod.coeffs_at(1.0, 0.9, -2, 2, np.array([1e-12, 1.0, 1e4]), np.array([0.3, 1.5, 2.9]))
    b = got[:, 0]
    assert abs(b[0] - 1) < 1e-6 and abs(b[2] - 1) < 1e-6
    assert np.all(b > 0)
