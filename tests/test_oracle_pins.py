"""Pins of the CPU oracle against facts that the paper and the mathematics fix.

* tortoise coordinate (Sec. 3.B): closed form r = 2M [1 + W(e^{r*/2M - 1})] at a = 0,
  and dr*/dr = (r^2 + a^2)/Delta for a != 0;
* theta operator (Sec. 3.D, 10th order; Sec. 3.B, 2nd order): convergence order on
  functions compatible with the parity ghosts, and the spin-weighted spherical harmonic
  eigen-relation (L_th - (m + s cos th)^2/sin^2 th + s) sY = -(l - s)(l + s + 1) sY;
* the initial angular profile: closed forms for (s, l, m) = (-2, 2, 2) and (0, 0, 0);
* boundaries (Sec. 3.B): zero r* rows, axis reflection symmetry;
* a -> -a with conjugate data gives the conjugate solution, bit for bit;
* windows: rows farther than n rows from a window edge agree bit for bit with the full grid
  after n Lax-Wendroff iterations (the domain of dependence used for sampled parity);
* second-order convergence in (t, r*) of the two-step scheme (Sec. 3.D: 2nd order in t, r*);
* a = 0: the theta profile stays sY_lm, and the observer signal matches a 1+1 radial
  Lax-Wendroff solver of the separated equation;
* the late-time tail of a = 0, s = 0, l = 0 decays as t^-(2l+3) (Sec. 3.C).
"""
import math

import mpmath as mpm
from fractions import Fraction

import numpy as np
import pytest

from oracle.stability import fd_weights, theta_matrix


def test_tortoise_closed_form_a0(oracle_mod):
    mpm.mp.dps = 90
    for rs in (-200.0, -50.0, -3.25, 0.0, 7.5, 150.0, 1800.0):
        x = oracle_mod.inverse_tortoise(1.0, 0.0, rs, bits=256)
        got = oracle_mod.words_to_mpf(x, mpm)
        want = 2 * mpm.lambertw(mpm.exp(mpm.mpf(rs) / 2 - 1)).real  # x = r - 2M, M = 1
        assert abs(got - want) <= mpm.mpf(2) ** -245 * abs(want), rs
        back = oracle_mod.words_to_mpf(oracle_mod.tortoise(1.0, 0.0, x, bits=256), mpm)
        assert abs(back - rs) <= mpm.mpf(2) ** -240 * max(1, abs(rs))


@pytest.mark.parametrize("a", [0.5, 0.9, 0.99])
def test_tortoise_derivative(oracle_mod, a):
    mpm.mp.dps = 90
    rp = 1 + mpm.sqrt(1 - mpm.mpf(a) ** 2)
    rm = mpm.mpf(a) ** 2 / rp
    for x0 in (1e-20, 0.3, 2.0, 40.0):
        x = mpm.mpf(x0)
        h = x * mpm.mpf(10) ** -25

        def rstar(xx):
            words = [float(xx)]
            words.append(float(xx - words[0]))
            words.append(float(xx - words[0] - words[1]))
            words.append(float(xx - words[0] - words[1] - words[2]))
            return oracle_mod.words_to_mpf(oracle_mod.tortoise(1.0, a, np.array(words), bits=256), mpm)

        d = (rstar(x + h) - rstar(x - h)) / (2 * h)
        r = rp + x
        want = (r**2 + mpm.mpf(a) ** 2) / ((r - rp) * (r - rm))
        assert abs(d - want) <= mpm.mpf(10) ** -40 * abs(want), (a, x0)


def test_fornberg_weights_10th_order():
    offs = list(range(-5, 6))
    d2 = [w * 25200 for w in fd_weights(offs, 2)]
    d1 = [w * 2520 for w in fd_weights(offs, 1)]
    assert [int(v) for v in d2] == [8, -125, 1000, -6000, 42000, -73766, 42000, -6000, 1000, -125, 8]
    assert [int(v) for v in d1] == [-2, 25, -150, 600, -2100, 0, 2100, -600, 150, -25, 2]
    assert all(v.denominator == 1 for v in d2 + d1)


def _theta_grid(n):
    return (np.arange(n) + 0.5) * math.pi / n


@pytest.mark.parametrize("order,parity", [(10, 1), (10, -1), (2, 1), (2, -1)])
def test_theta_operator_order(oracle_mod, order, parity):
    """f = cos(k th) (parity +1) or sin(k th) (parity -1): L_th f has a closed form.
    Away from the poles the error falls at the stencil's order; in the cells next to a pole
    cot th ~ 1/th multiplies the first-derivative error, which costs one order there."""
    k = 3
    errs, errs_in = [], []
    for n in (16, 32, 64):
        th = _theta_grid(n)
        if parity > 0:
            f = np.cos(k * th)
            want = -k * k * np.cos(k * th) - k * np.sin(k * th) / np.tan(th)
        else:
            f = np.sin(k * th)
            want = -k * k * np.sin(k * th) + k * np.cos(k * th) / np.tan(th)
        # f and want in 256-bit via mpmath for the smaller errors of the 10th-order case
        mpm.mp.dps = 70
        fw = np.zeros((4, n))
        ww = []
        for j in range(n):
            tj = (mpm.mpf(j) + mpm.mpf(1) / 2) * mpm.pi / n
            fv = mpm.cos(k * tj) if parity > 0 else mpm.sin(k * tj)
            for q in range(4):
                fw[q, j] = float(fv)
                fv -= fw[q, j]
            wv = (-k * k * mpm.cos(k * tj) - k * mpm.sin(k * tj) * mpm.cot(tj)) if parity > 0 else \
                 (-k * k * mpm.sin(k * tj) + k * mpm.cos(k * tj) * mpm.cot(tj))
            ww.append(wv)
        out = oracle_mod.theta_op(fw, order=order, parity=parity, bits=256)
        e = [abs(oracle_mod.words_to_mpf(out[:, j], mpm) - ww[j]) for j in range(n)]
        errs.append(float(max(e)))
        errs_in.append(float(max(e[n // 4: 3 * n // 4])))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    rates_in = [math.log2(errs_in[i] / errs_in[i + 1]) for i in range(len(errs) - 1)]
    assert min(rates_in) > order - 0.6, (errs_in, rates_in)
    assert min(rates) > order - 1.3, (errs, rates)


@pytest.mark.parametrize("s,m,l", [(-2, 2, 2), (-2, 2, 3), (0, 0, 0), (0, 1, 2), (-1, -2, 3), (-2, -1, 2)])
def test_spin_harmonic_eigenrelation(oracle_mod, s, m, l):
    """sY_lm solves the a = 0 angular Teukolsky equation: the discrete residual of
    (L_th - (m + s cos th)^2/sin^2 th + s + (l - s)(l + s + 1)) sY falls at 10th order
    (9th in the pole cells of odd-parity fields, where cot th ~ 1/th)."""
    lam = (l - s) * (l + s + 1)
    par = 1 if (m + s) % 2 == 0 else -1
    errs = []
    for n in (16, 32, 64):
        Y = oracle_mod.spin_profile(s, m, l, n, bits=256)
        LY = oracle_mod.theta_op(Y, order=10, parity=par, bits=256)
        mpm.mp.dps = 70
        res = []
        for j in range(n):
            tj = (mpm.mpf(j) + mpm.mpf(1) / 2) * mpm.pi / n
            y = oracle_mod.words_to_mpf(Y[:, j], mpm)
            ly = oracle_mod.words_to_mpf(LY[:, j], mpm)
            pot = (m + s * mpm.cos(tj)) ** 2 / mpm.sin(tj) ** 2
            res.append(abs(ly - pot * y + s * y + lam * y))
        ymax = max(abs(oracle_mod.words_to_mpf(Y[:, j], mpm)) for j in range(n))
        errs.append(float(max(res) / ymax))
    assert errs[-1] < 1e-9, errs
    if max(errs) < 1e-60:  # l = 0: a constant profile, reproduced to rounding
        return
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(rates) > 8.7, (errs, rates)


def test_spin_profile_closed_forms(oracle_mod):
    n = 12
    th = _theta_grid(n)
    Y = oracle_mod.spin_profile(-2, 2, 2, n, bits=53, out_words=1)[0]
    np.testing.assert_allclose(Y, np.cos(th / 2) ** 4, rtol=1e-14)
    Y0 = oracle_mod.spin_profile(0, 0, 0, n, bits=53, out_words=1)[0]
    np.testing.assert_array_equal(Y0, np.ones(n))
    # s = 0: sY_lm is Y_lm up to normalisation, Y_10 ~ cos th
    Y10 = oracle_mod.spin_profile(0, 0, 1, n, bits=53, out_words=1)[0]
    np.testing.assert_allclose(Y10 / Y10[0], np.cos(th) / np.cos(th[0]), rtol=1e-13)


def small_problem(**kw):
    base = dict(M=1.0, a=0.7, s=-2, m=2, rstar_min=-20.0, rstar_max=40.0, n_r=61, n_theta=16,
                dt=0.25, substeps=4)
    base.update(kw)
    return base


def test_boundaries_and_axis_symmetry(oracle_mod):
    p = small_problem(a=0.0, s=0, m=0)
    o = oracle_mod.Oracle(**p, bits=53)
    o.pulse(10.0, 3.0, 0.8, 0.6, 2)
    o.step(40)
    u = o.get_state(1)[:, 0]
    assert np.all(u[:, 0] == 0) and np.all(u[:, -1] == 0)
    # a = 0, m = 0, s = 0, l = 2: symmetric about the equator
    np.testing.assert_allclose(u, u[:, :, ::-1], rtol=0, atol=1e-13 * np.abs(u).max())


@pytest.mark.parametrize("bits", [53, 256])
def test_conjugation_symmetry(oracle_mod, bits):
    """a -> -a with A -> conj(A) gives conj(u), exactly: every imaginary coefficient carries a."""
    p = small_problem(n_r=25, n_theta=12, rstar_min=-5.0, rstar_max=19.0, substeps=2)
    o1 = oracle_mod.Oracle(**p, bits=bits)
    o2 = oracle_mod.Oracle(**dict(p, a=-p["a"]), bits=bits)
    o1.pulse(7.0, 2.0, 0.8, 0.6, 2)
    o2.pulse(7.0, 2.0, 0.8, -0.6, 2)
    n = 6 if bits > 53 else 30
    o1.step(n)
    o2.step(n)
    w = 4 if bits > 53 else 1
    u1, u2 = o1.get_state(w), o2.get_state(w)
    assert np.abs(u1).max() > 0
    np.testing.assert_array_equal(u1[0], u2[0])
    np.testing.assert_array_equal(u1[1], -u2[1])
    np.testing.assert_array_equal(u1[2], u2[2])
    np.testing.assert_array_equal(u1[3], -u2[3])


def test_window_domain_of_dependence(oracle_mod):
    p = small_problem()
    full = oracle_mod.Oracle(**p, bits=53)
    full.pulse(10.0, 3.0, 0.8, 0.6, 2)
    lo, hi, n = 14, 50, 9
    win = oracle_mod.Oracle(**p, row_lo=lo, row_hi=hi, bits=53)
    win.pulse(10.0, 3.0, 0.8, 0.6, 2)
    full.step(n)
    win.step(n)
    uf = full.get_state(1)[:, 0, lo + n:hi - n + 1]
    uw = win.get_state(1)[:, 0, n:hi - lo - n + 1]
    np.testing.assert_array_equal(uf, uw)


def test_second_order_convergence(oracle_mod):
    """Richardson: dr*, dt halved twice on nested grids -> error ratio ~ 4 (Sec. 3.D)."""
    T = 8.0
    res = []
    for lev in range(2, 5):
        n_r = 60 * 2**lev + 1
        dr = 60.0 / (n_r - 1)
        dt = 0.25 * dr
        p = dict(M=1.0, a=0.6, s=-1, m=1, rstar_min=-20.0, rstar_max=40.0, n_r=n_r, n_theta=16,
                 dt=dt, substeps=2)
        o = oracle_mod.Oracle(**p, bits=53)
        o.pulse(12.0, 4.0, 0.9, 0.7, 1)
        o.step(int(round(T / dt)) * 2)
        res.append(o.get_state(1)[:, 0, :: 2 ** (lev - 2)])
    e1 = np.abs(res[0] - res[1]).max()
    e2 = np.abs(res[1] - res[2]).max()
    assert 3.7 < e1 / e2 < 4.3, (e1, e2, e1 / e2)


def _radial_coefficients(s, m, l, r, M=1.0):
    """Separated a = 0 coefficients for Phi(t, r*) sY_lm(th) (Sec. 3.A with a = 0):
    Sigma = r^2, b = 1, Delta = r^2 - 2Mr, the angular operator replaced by its eigenvalue."""
    D = r * r - 2 * M * r
    R = r * r
    B = 2 * s * (D * r - M * r * r)
    C = 2 * r * D + 2 * s * (r - M) * R
    fp = 3 * D / (r * R)
    fpp = 6 * D * ((r - M) * r * R) / (r * r * R**3)
    V = R * R * fpp + C * fp - D * (l - s) * (l + s + 1)
    c = -(B + 6 * R * D / r + C) / R**2
    return c, B / R**2, V / R**2


def test_a0_separability_and_radial_solver(oracle_mod):
    s, m, l = -2, 2, 2
    p = dict(M=1.0, a=0.0, s=s, m=m, rstar_min=-30.0, rstar_max=60.0, n_r=181, n_theta=24,
             dt=0.125, substeps=6)
    o = oracle_mod.Oracle(**p, bits=53)
    o.pulse(15.0, 3.0, 1.0, 0.0, l)
    nsteps = 160
    o.step(nsteps * p["substeps"])
    u = o.get_state(1)[:, 0]
    Y = oracle_mod.spin_profile(s, m, l, p["n_theta"], bits=53, out_words=1)[0]
    # separability: every row is a multiple of Y
    coef = u[0] @ Y / (Y @ Y)
    dev = np.abs(u[0] - np.outer(coef, Y)).max() / np.abs(u[0]).max()
    assert dev < 1e-6, dev
    # 1+1 radial Lax-Wendroff on the separated equation
    x = o.grid(1)["x_node"][0]
    xh = o.grid(1)["x_half"][0]
    r, rh = 2.0 + x, 2.0 + xh
    cn, bn, vn = _radial_coefficients(s, m, l, r)
    chh, bh, vh = _radial_coefficients(s, m, l, rh)
    rs = o.grid(1)["rstar_node"][0]
    G = np.exp(-((rs - 15.0) / 3.0) ** 2)
    phi = G.copy()
    pi = -2 * (rs - 15.0) / 9.0 * G
    phi[[0, -1]] = 0
    pi[[0, -1]] = 0
    dr = 90.0 / 180
    h = p["dt"] / p["substeps"]
    for _ in range(nsteps * p["substeps"]):
        pb, qb = 0.5 * (phi[1:] + phi[:-1]), 0.5 * (pi[1:] + pi[:-1])
        dp, dq = (phi[1:] - phi[:-1]) / dr, (pi[1:] - pi[:-1]) / dr
        Sq = -chh * dp - bh * qb + vh * pb
        ph = pb - 0.5 * h * (dp - qb)
        qh = qb - 0.5 * h * (-dq - Sq)
        pb2, qb2 = 0.5 * (ph[1:] + ph[:-1]), 0.5 * (qh[1:] + qh[:-1])
        dp2, dq2 = (ph[1:] - ph[:-1]) / dr, (qh[1:] - qh[:-1]) / dr
        Sq2 = -cn[1:-1] * dp2 - bn[1:-1] * qb2 + vn[1:-1] * pb2
        phi[1:-1] = phi[1:-1] - h * (dp2 - qb2)
        pi[1:-1] = pi[1:-1] - h * (-dq2 - Sq2)
    np.testing.assert_allclose(coef, phi, rtol=0, atol=2e-6 * np.abs(phi).max())


def _tail_index(oracle_mod, velocity_data):
    p = dict(M=1.0, a=0.0, s=0, m=0, rstar_min=-700.0, rstar_max=900.0, n_r=3201, n_theta=8,
             dt=0.125, substeps=1)
    o = oracle_mod.Oracle(**p, bits=53)
    if velocity_data:  # Phi = 0, Phi_t = Pi = Gaussian
        rs = o.grid(1)["rstar_node"][0]
        G = np.exp(-((rs - 30.0) / 4.0) ** 2)
        G[[0, -1]] = 0
        planes = np.zeros((4, 1, p["n_r"], p["n_theta"]))
        planes[2, 0] = G[:, None]
        o.set_state(planes)
    else:  # the workloads' pulse: Gaussian Phi, zero time derivative
        o.pulse(30.0, 4.0, 1.0, 0.0, 0)
    i_obs = int(round((50.0 - p["rstar_min"]) / 0.5))
    ts, vals = [], []
    for n in range(1, 340 + 1):  # t <= 1360: no boundary reflection reaches r* = 50 before ~1450
        o.step(40)
        ts.append(n * 40 * p["dt"])
        vals.append(o.get_row(i_obs, 1)[0, 0, 0])
    ts, vals = np.array(ts), np.abs(np.array(vals))
    slope = -np.diff(np.log(vals)) / np.diff(np.log(ts))
    return slope[(ts[1:] > 1100) & (ts[1:] < 1300)]


@pytest.mark.slow
def test_schwarzschild_tail_exponent(oracle_mod):
    """a = 0, s = 0, l = 0 at a fixed observer, boundaries causally disconnected: generic
    (here: pure velocity) data decay as t^-(2l+3) = t^-3 (Sec. 3.C); time-symmetric data,
    the workloads' zero-initial-time-derivative pulse, as t^-(2l+4) = t^-4."""
    n_vel = _tail_index(oracle_mod, True)
    assert np.all(np.abs(n_vel - 3.0) < 0.05), n_vel
    n_sym = _tail_index(oracle_mod, False)
    assert np.all(np.abs(n_sym - 4.0) < 0.05), n_sym


def test_r_dissipation_step_by_linearity(oracle_mod):
    """The oracle's r* dissipation step (not part of the paper's scheme): one iteration with
    sigma minus one without equals -eps times one iteration (without) applied to the fourth
    difference of the data, eps = sigma dt / (16 dr*), rows 2 .. n_r - 3 only (the scheme is
    linear); a cubic in r* is left unchanged; sigma = 0 changes nothing."""
    n_r, nth, sigma = 23, 8, 1.5
    p = dict(M=1.0, a=0.7, s=-1, m=1, rstar_min=-10.0, rstar_max=12.0, n_r=n_r, n_theta=nth, dt=0.0,
             substeps=1, theta_order=10, parity=1)
    rng = np.random.default_rng(4)
    u = rng.uniform(-1, 1, (4, 1, n_r, nth))
    u[:, :, [0, -1]] = 0.0
    d4 = np.zeros_like(u)
    d4[:, :, 2:-2] = u[:, :, :-4] - 4 * u[:, :, 1:-3] + 6 * u[:, :, 2:-2] - 4 * u[:, :, 3:-1] + u[:, :, 4:]

    def one(state, ko):
        o = oracle_mod.Oracle(**p, bits=256, ko_sigma=ko)
        o.set_state(state)
        o.step(1)
        return o.get_state(words=4)

    def val(w):
        return np.sum(w, axis=1)  # word sums in double: the tolerance below is far above that

    with_ko, without = one(u, sigma), one(u, 0.0)
    of_d4 = one(d4, 0.0)
    eps = sigma * 0.25 / 16.0  # dt = 0.25 dr*
    lhs = (with_ko - without)
    lhs = lhs[:, 0] + lhs[:, 1] + lhs[:, 2] + lhs[:, 3]
    rhs = -eps * val(of_d4)
    assert np.abs(lhs - rhs).max() < 1e-13 * np.abs(rhs).max()
    assert np.abs(rhs).max() > 1e-3
    # a cubic in the row index is in the kernel of the fourth difference
    i = np.arange(n_r, dtype=float)
    cubic = np.zeros_like(u)
    cubic[:] = ((3 + i - 2 * i ** 2 + i ** 3) / 1024.0)[None, None, :, None]  # exact doubles
    cubic[:, :, [0, -1]] = 0.0
    # the fourth difference vanishes at rows 3 .. n_r - 4 (away from the zeroed rows 0, n_r - 1);
    # one iteration spreads a difference by one row
    np.testing.assert_array_equal(one(cubic, sigma)[:, :, 4:-4], one(cubic, 0.0)[:, :, 4:-4])


def _one_iteration(oracle_mod, p, state, ko_theta, words=4):
    o = oracle_mod.Oracle(**p, bits=256, ko_theta=ko_theta)
    o.set_state(state)
    o.step(1)
    return o.get_state(words=words)


def _wsum(w):
    return w[:, 0] + w[:, 1] + w[:, 2] + w[:, 3]


def test_theta_dissipation_sawtooth_eigenvalue(oracle_mod):
    """theta dissipation step (not part of the paper's scheme): with odd axis parity (s + m
    odd) the theta sawtooth (-1)^j continues through the ghost cells, so it is an eigenvector
    of (d^2)^6 with eigenvalue 4^6 and one step multiplies row i by
    1 - sigma c_th(i) dt / dtheta, c_th(i) = max_j sqrt(Delta/Sigma^2) (the g coefficient,
    pinned against Eq. 1). The iteration is linear, so
    step_with(u) - step_without(u) = -step_without(sigma c_th dt / dtheta u)."""
    n_r, nth, sigma = 19, 12, 0.8
    p = dict(M=1.0, a=0.6, s=-1, m=2, rstar_min=-8.0, rstar_max=10.0, n_r=n_r, n_theta=nth, dt=0.0,
             substeps=1, theta_order=10, parity=-1)
    rng = np.random.default_rng(7)
    saw = (-1.0) ** np.arange(nth)
    u = rng.uniform(0.5, 1.0, (4, 1, n_r, 1)) * saw[None, None, None, :]
    u[:, :, [0, -1]] = 0.0
    g = oracle_mod.Oracle(**p, bits=256).coeffs(0, 1)[5, 0]  # Delta / Sigma^2 at the nodes
    c_th = np.sqrt(g.max(axis=1))
    dt = 0.25 * (p["rstar_max"] - p["rstar_min"]) / (n_r - 1)
    dth = np.pi / nth
    v = u * (sigma * c_th * dt / dth)[None, None, :, None]
    v[:, :, [0, -1]] = 0.0
    lhs = _wsum(_one_iteration(oracle_mod, p, u, sigma) - _one_iteration(oracle_mod, p, u, 0.0))
    rhs = -_wsum(_one_iteration(oracle_mod, p, v, 0.0))
    assert np.abs(rhs).max() > 0.05
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()


def test_theta_dissipation_is_a_twelfth_difference(oracle_mod):
    """(d^2)^6 annihilates every polynomial of degree <= 11 in the column index: away from the
    poles (and from the columns the next iteration's 11-point theta stencil reads from there)
    the step changes nothing; together with the sawtooth eigenvalue this fixes all 13
    weights. With even parity a theta-constant row continues through the ghosts and is not
    changed anywhere."""
    n_r, nth, sigma = 9, 40, 1.0
    p = dict(M=1.0, a=0.6, s=0, m=0, rstar_min=-8.0, rstar_max=10.0, n_r=n_r, n_theta=nth, dt=0.0,
             substeps=1, theta_order=10, parity=1)
    # an exact degree-11 polynomial in j: dyadic coefficients and x = (j - 20)/16, times dyadic
    # row amplitudes; each value is a dyadic rational held exactly as two double words
    coef = [Fraction(c, 8) for c in (3, -2, 5, 1, -4, 2, 6, -3, 2, 1, -3, 4)]
    amps = [[Fraction(4 + (3 * c + 5 * i) % 5, 8) for i in range(n_r)] for c in range(4)]
    u = np.zeros((4, 2, n_r, nth))
    for c in range(4):
        for i in range(1, n_r - 1):
            for j in range(nth):
                x = Fraction(j - 20, 16)
                v = amps[c][i] * sum(ck * x ** k for k, ck in enumerate(coef))
                hi = float(v)
                lo = float(v - Fraction(hi))
                assert Fraction(hi) + Fraction(lo) == v
                u[c, 0, i, j], u[c, 1, i, j] = hi, lo
    diff = _wsum(_one_iteration(oracle_mod, p, u, sigma) - _one_iteration(oracle_mod, p, u, 0.0))
    assert np.abs(diff[:, :, :6]).max() > 1e-6          # the pole regions are changed
    assert np.abs(diff[:, :, 11:nth - 11]).max() < 1e-40  # columns 6 .. nth-7 read none of them
    rng = np.random.default_rng(8)
    const = rng.uniform(0.5, 1.0, (4, 1, n_r, 1)) * np.ones((1, 1, 1, nth))
    const[:, :, [0, -1]] = 0.0
    d0 = _wsum(_one_iteration(oracle_mod, p, const, sigma) - _one_iteration(oracle_mod, p, const, 0.0))
    assert np.abs(d0).max() < 1e-60


def test_theta_dissipation_keeps_tenth_order(oracle_mod):
    """On a smooth (regular, parity-consistent) field the step's change is
    sigma c_th dt / (4096 dtheta) (d^2)^6 u = O(dtheta^11): halving dtheta divides it by about
    2^11 (the scheme's 10th-order theta accuracy is kept)."""
    sigma = 1.0
    changes = []
    for nth in (24, 48):
        p = dict(M=1.0, a=0.0, s=0, m=0, rstar_min=-8.0, rstar_max=10.0, n_r=7, n_theta=nth, dt=0.0,
                 substeps=1, theta_order=10, parity=1)
        th = (np.arange(nth) + 0.5) * np.pi / nth
        prof = np.cos(th) ** 2 + 0.3 * np.cos(th) ** 4 * np.sin(th) ** 2  # smooth, even at both poles
        u = np.ones((4, 1, 7, 1)) * prof[None, None, None, :]
        u[:, :, [0, -1]] = 0.0
        d = _wsum(_one_iteration(oracle_mod, p, u, sigma) - _one_iteration(oracle_mod, p, u, 0.0))
        changes.append(np.abs(d).max())
    ratio = changes[0] / changes[1]
    assert 2 ** 10.3 < ratio < 2 ** 11.7, (changes, np.log2(ratio))
