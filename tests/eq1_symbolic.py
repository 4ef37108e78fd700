"""The Teukolsky master equation (Eq. 1, Sec. 3.A) reduced with sympy, for the oracle's pins.

Eq. 1 is written out as printed, the ansatz Psi = e^{i m phi~} r^3 F(t, r, theta) (Eq. psiphi,
d phi~ = d phi + a/Delta dr) is substituted, the common phase is divided out and the result
is multiplied by Delta / r^3. What is left is linear in F and its derivatives:

    E[F] = e_tt F_tt + e_t F_t + e_rr F_rr + e_r F_r + e_thth F_thth + e_th F_th + e_0 F,

derivatives in (t, r, theta). Nothing here comes from the oracle: this is the independent
side of its pins."""
import functools

import pytest

sp = pytest.importorskip("sympy")

NAMES = ("e_tt", "e_t", "e_rr", "e_r", "e_thth", "e_th", "e_0")


@functools.lru_cache(maxsize=None)
def eq1_coefficients(s_val: int, m_val: int):
    """Sympy expressions of e_tt .. e_0 in (r, theta, M, a) for spin weight s and mode m."""
    t, r, th, phi = sp.symbols("t r theta phi", real=True)
    M, a = sp.symbols("M a", positive=True)
    F = sp.Function("F")(t, r, th)
    G = sp.Function("G")(r)
    I = sp.I
    s, m = sp.Integer(s_val), sp.Integer(m_val)
    Delta = r**2 - 2 * M * r + a**2
    E0 = sp.exp(I * m * (phi + G))
    Psi = E0 * r**3 * F
    # Eq. 1 as printed in Sec. 3.A
    eq = (-((r**2 + a**2) ** 2 / Delta - a**2 * sp.sin(th) ** 2) * sp.diff(Psi, t, 2)
          - 4 * M * a * r / Delta * sp.diff(Psi, t, phi)
          - 2 * s * (r - M * (r**2 - a**2) / Delta + I * a * sp.cos(th)) * sp.diff(Psi, t)
          + Delta ** (-s) * sp.diff(Delta ** (s + 1) * sp.diff(Psi, r), r)
          + 1 / sp.sin(th) * sp.diff(sp.sin(th) * sp.diff(Psi, th), th)
          + (1 / sp.sin(th) ** 2 - a**2 / Delta) * sp.diff(Psi, phi, 2)
          + 2 * s * (a * (r - M) / Delta + I * sp.cos(th) / sp.sin(th) ** 2) * sp.diff(Psi, phi)
          - (s**2 * sp.cot(th) ** 2 - s) * Psi)
    E = eq / E0
    E = E.subs(sp.Derivative(G, (r, 2)), sp.diff(a / Delta, r)).subs(sp.Derivative(G, r), a / Delta)
    syms = sp.symbols("d_tt d_t d_rr d_r d_thth d_th d_0")
    E = E.subs({sp.Derivative(F, (t, 2)): syms[0], sp.Derivative(F, (r, 2)): syms[2],
                sp.Derivative(F, (th, 2)): syms[4]})
    E = E.subs({sp.Derivative(F, t): syms[1], sp.Derivative(F, r): syms[3],
                sp.Derivative(F, th): syms[5]})
    E = E.subs(F, syms[6])
    E = sp.expand(E)
    coeffs = [E.coeff(v) for v in syms]
    assert sp.expand(E - sum(c * v for c, v in zip(coeffs, syms))) == 0
    return (r, th, M, a), [c * Delta / r**3 for c in coeffs]


@functools.lru_cache(maxsize=None)
def eq1_functions(s_val: int, m_val: int, module: str = "mpmath"):
    """e_tt .. e_0 as callables f(r, theta, M, a) (module "mpmath" or "numpy")."""
    args, exprs = eq1_coefficients(s_val, m_val)
    return [sp.lambdify(args, e, module) for e in exprs]
