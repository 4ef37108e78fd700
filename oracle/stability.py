"""Substep count for a stable run of the Lax-Wendroff scheme (test infrastructure).

The paper states that the Lax-Wendroff iteration gives stable evolutions (Sec. 3.B) but
gives no time-step rule. The theta derivatives sit in the source S, so for a mode that is
smooth in r* the two-step iteration (Eqs. lw1, lw2) reduces to the explicit midpoint rule
u <- u + z u + z^2/2 u with z = lambda dt, whose amplification 1 + z + z^2/2 exceeds the
exact exp(z) in modulus for every imaginary z (|G|^2 = 1 + y^4/4 at z = i y). The largest
|lambda| comes from the (m + s cos th)^2 / sin^2 th potential in the cells next to the poles.

Reading adopted (not in the paper): keep dt = 0.25 dr* as the outer step and integrate it
with k Lax-Wendroff iterations of dt/k, k being the smallest integer for which the excess
growth max |G(lambda dt/k)| / |exp(lambda dt/k)| of the worst local mode, raised to the
number of iterations in the run, stays below 10.

The local operator at one r* node is the 2 n_theta x 2 n_theta complex matrix of
(Phi, Pi)_t = [[0, I], [g L_th + diag(V/Sigma^2), -diag(B/Sigma^2)]] (Phi, Pi) with the
r*-transport terms left out; L_th is the centred theta operator with parity ghosts.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

from . import Oracle


def fd_weights(offsets, deriv):
    """Exact finite-difference weights for the `deriv`-th derivative at 0 on integer offsets,
    from the Taylor moment conditions sum_q w_q q^p / p! = [p == deriv]."""
    n = len(offsets)
    A = [[Fraction(q) ** p for q in offsets] for p in range(n)]
    rhs = [Fraction(math.factorial(deriv)) if p == deriv else Fraction(0) for p in range(n)]
    # Gaussian elimination over the rationals
    M = [row[:] + [rhs[i]] for i, row in enumerate(A)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [M[i][n] / M[i][i] for i in range(n)]


def theta_matrix(theta, cot, parity, order=10):
    """Matrix of L_th f = f_thth + cot th f_th on the cell-centred grid with ghosts."""
    nth = len(theta)
    dth = math.pi / nth
    half = 5 if order == 10 else 1
    offs = list(range(-half, half + 1))
    w2 = [float(w) for w in fd_weights(offs, 2)]
    w1 = [float(w) for w in fd_weights(offs, 1)]
    L = np.zeros((nth, nth))
    for j in range(nth):
        for qi, q in enumerate(offs):
            w = w2[qi] / dth**2 + cot[j] * w1[qi] / dth
            jj = j + q
            sign = 1.0
            if jj < 0:
                jj, sign = -1 - jj, float(parity)
            elif jj >= nth:
                jj, sign = 2 * nth - 1 - jj, float(parity)
            L[j, jj] += sign * w
    return L


def local_eigenvalues(coef_row, L):
    """Eigenvalues of the local (Phi, Pi) operator at one node; coef_row is [8, n_theta]."""
    nth = L.shape[0]
    g = coef_row[5]
    nu = coef_row[6] + 1j * coef_row[7]
    beta = coef_row[3] + 1j * coef_row[4]
    A = np.zeros((2 * nth, 2 * nth), dtype=complex)
    A[:nth, nth:] = np.eye(nth)
    A[nth:, :nth] = g[:, None] * L + np.diag(nu)
    A[nth:, nth:] = -np.diag(beta)
    return np.linalg.eigvals(A)


def excess_log_growth(lams, dt_sub):
    z = lams * dt_sub
    G = 1 + z + 0.5 * z * z
    return float(np.max(np.log(np.abs(G)) - z.real))


def analyse(problem, rows_to_check=24, growth=10.0, kmax=4096):
    """Smallest k with (worst excess amplification)^(steps k) <= growth, and the worst |lambda|."""
    p = problem
    o = Oracle(M=p.M, a=p.a, s=p.s, m=p.m, rstar_min=p.rstar_min, rstar_max=p.rstar_max,
               n_r=p.n_r, n_theta=p.n_theta, dt=p.dt, substeps=1, theta_order=p.theta_order,
               parity=p.parity, bits=53)
    cf = o.coeffs(0, 1)[:, 0]  # [8, n_r, n_theta]
    grid = o.grid(1)
    theta, cot = grid["theta"][0], grid["cot_theta"][0]
    L = theta_matrix(theta, cot, p.parity, p.theta_order)
    # rank rows by a Gershgorin-type bound of the Pi <- Phi block, check the worst ones
    rowsum = np.abs(L).sum(axis=1)
    bound = (cf[5] * rowsum[None, :] + np.hypot(cf[6], cf[7])).max(axis=1)
    cand = list(np.argsort(bound)[::-1][:rows_to_check])
    cand += list(np.linspace(1, p.n_r - 2, 8).astype(int))
    lams = np.concatenate([local_eigenvalues(cf[:, i], L) for i in sorted(set(cand))])
    o.close()
    n_outer = p.steps
    for k in range(1, kmax + 1):
        if n_outer * k * excess_log_growth(lams, p.dt / k) <= math.log(growth):
            return k, float(np.max(np.abs(lams)))
    raise RuntimeError("no stable substep count below kmax")
