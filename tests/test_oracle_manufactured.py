"""Pin: a forced manufactured solution of Eq. 1 at a != 0 (the oracle's complex couplings).

The symbolic pin (test_oracle_reduction) fixes the values of the eight coefficients of the
first-order system; this one fixes how the oracle's Lax-Wendroff step combines them with
the complex state. A smooth complex field

    Phi_ex(t, r*, theta) = e^{-i omega t} G(r*) Y(theta),
    G = exp(-((r* - c)/w)^2) e^{i kappa r*},  Y = sY_{l0 m} + (2/5) i sY_{l0+1, m}

(unnormalised Goldberg sums, so Y has the axis parity (-1)^(m+s) of the ghost cells) is
pushed through Eq. 1 as printed (tests/eq1_symbolic.py, sympy, no oracle coefficient):
E[Phi_ex] = e_tt Phi_tt + ... + e_0 Phi. With Pi = Phi_t + b Phi' the first-order system of
Sec. 3.B is equivalent to Phi_tt - b (b Phi')' - S_Pi = 0, and E = e_tt times the same
expression, so forcing the Pi rows with F = E[Phi_ex] / e_tt makes Phi_ex an exact solution
of the forced system. The oracle integrates it (Eqs. lw1, lw2 with F taken at t_n on half
nodes and t_n + dt/2 on nodes) from Phi_ex(0), Pi_ex(0); the error at t = 4 must fall by
4 +- 0.3 per halving of (dr*, dt): the scheme's 2nd order (Sec. 3.D). Conjugating any of
c, B/Sigma^2 or V/Sigma^2, or flipping the sign of any single imaginary cross term in the
assembly of S_Pi, leaves errors of order one that do not fall with refinement.
"""
import math

import numpy as np
import pytest

sp = pytest.importorskip("sympy")
from tests.eq1_symbolic import eq1_functions  # noqa: E402

M, A, S, MM = 1.0, 0.7, -1, 2
OMEGA, KAPPA, C0, WID = 0.6, 0.5, 2.0, 3.0
RMIN, RMAX = -25.0, 30.0
N_THETA, K, T_END = 32, 8, 4.0
RP = M + math.sqrt(M * M - A * A)


def _profile_functions():
    th = sp.symbols("theta", real=True)

    def goldberg(l):
        tot = 0
        for r in range(0, l - S + 1):
            c = sp.binomial(l - S, r) * sp.binomial(l + S, r + S - MM)
            if c:
                tot += ((-1) ** (l - r - S) * c * sp.sin(th / 2) ** (2 * l - 2 * r - S + MM)
                        * sp.cos(th / 2) ** (2 * r + S - MM))
        return tot

    l0 = max(abs(S), abs(MM))
    Y = goldberg(l0) + sp.Rational(2, 5) * sp.I * goldberg(l0 + 1)
    return [sp.lambdify(th, e, "numpy") for e in (Y, sp.diff(Y, th), sp.diff(Y, th, 2))]


def _radial(rs):
    """G, dG/dr*, d2G/dr*^2."""
    z = (rs - C0) / WID
    g = np.exp(-z * z) * np.exp(1j * KAPPA * rs)
    q = -2 * (rs - C0) / WID**2 + 1j * KAPPA
    return g, g * q, g * (q * q - 2 / WID**2)


def _forcing(Yf, x, rs, theta):
    """F^ = E[Phi_ex] / e_tt at t = 0 (the time dependence is e^{-i omega t})."""
    ef = eq1_functions(S, MM, "numpy")
    r = (RP + x)[:, None]
    t = theta[None, :]
    D = r * r - 2 * M * r + A * A
    R = r * r + A * A
    RD = R / D                                     # dr*/dr
    dRD = 2 * (r * D - R * (r - M)) / D**2         # d/dr (R / Delta)
    g, g1, g2 = (v[:, None] for v in _radial(rs))
    Y, Y1, Y2 = (np.broadcast_to(f(theta), theta.shape)[None, :] for f in Yf)
    e = [np.asarray(f(r, t, M, A), dtype=complex) * np.ones((len(x), len(theta))) for f in ef]
    Phi = g * Y
    E = (e[0] * (-OMEGA**2) * Phi + e[1] * (-1j * OMEGA) * Phi
         + e[2] * (g2 * RD**2 + g1 * dRD) * Y + e[3] * g1 * RD * Y
         + e[4] * g * Y2 + e[5] * g * Y1 + e[6] * Phi)
    return E / e[0]


def _exact(Yf, x, rs, theta, t):
    """Phi_ex and Pi_ex = Phi_t + b Phi' with b = (r^2 + a^2)/Sigma (Sec. 3.B)."""
    r = (RP + x)[:, None]
    D = r * r - 2 * M * r + A * A
    R = r * r + A * A
    b = R / np.sqrt(R * R - A * A * D * np.sin(theta[None, :]) ** 2)
    g, g1, _ = _radial(rs)
    Y = Yf[0](theta)[None, :]
    ph = np.exp(-1j * OMEGA * t)
    return ph * g[:, None] * Y, ph * (-1j * OMEGA * g[:, None] + b * g1[:, None]) * Y


def _run(oracle_mod, Yf, n_r):
    o = oracle_mod.Oracle(M=M, a=A, s=S, m=MM, rstar_min=RMIN, rstar_max=RMAX, n_r=n_r,
                          n_theta=N_THETA, dt=0.0, substeps=K, bits=53)
    gr = o.grid()
    theta = gr["theta"][0]
    xn, rn, xh, rh = gr["x_node"][0], gr["rstar_node"][0], gr["x_half"][0], gr["rstar_half"][0]
    o.set_forcing(OMEGA, _forcing(Yf, xn, rn, theta), _forcing(Yf, xh, rh, theta))
    Phi, Pi = _exact(Yf, xn, rn, theta, 0.0)
    st = np.stack([Phi.real, Phi.imag, Pi.real, Pi.imag])[:, None].copy()
    st[:, :, 0] = 0.0
    st[:, :, -1] = 0.0
    o.set_state(st)
    dt = 0.25 * (RMAX - RMIN) / (n_r - 1)
    n_out = int(round(T_END / dt))
    o.step(n_out * K)
    u = o.get_state()[:, 0]
    Phi, Pi = _exact(Yf, xn, rn, theta, n_out * dt)
    e_phi = np.abs((u[0] + 1j * u[1]) - Phi).max() / np.abs(Phi).max()
    e_pi = np.abs((u[2] + 1j * u[3]) - Pi).max() / np.abs(Pi).max()
    return e_phi, e_pi


def test_forced_solution_converges_at_second_order(oracle_mod):
    Yf = _profile_functions()
    errs = [_run(oracle_mod, Yf, n_r) for n_r in (111, 221, 441)]  # dr* = 1/2, 1/4, 1/8
    assert errs[0][0] < 0.1 and errs[0][1] < 0.2, errs
    for coarse, fine in zip(errs, errs[1:]):
        for c in range(2):
            assert abs(coarse[c] / fine[c] - 4.0) < 0.3, errs


def test_forcing_switches_off(oracle_mod):
    """Without forcing the hook leaves the step untouched (bit for bit)."""
    Yf = _profile_functions()
    runs = []
    for forced in (False, True):
        o = oracle_mod.Oracle(M=M, a=A, s=S, m=MM, rstar_min=RMIN, rstar_max=RMAX, n_r=23,
                              n_theta=12, dt=0.0, substeps=2, bits=53)
        o.pulse(2.0, 3.0, 0.7, 0.6, 2)
        if forced:
            gr = o.grid()
            th = gr["theta"][0]
            o.set_forcing(OMEGA, _forcing(Yf, gr["x_node"][0], gr["rstar_node"][0], th),
                          _forcing(Yf, gr["x_half"][0], gr["rstar_half"][0], th))
            o.set_forcing(0.0, None, None)
        o.step(6)
        runs.append(o.get_state())
    assert np.array_equal(runs[0], runs[1])
