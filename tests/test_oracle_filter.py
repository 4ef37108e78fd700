"""Pins of the oracle's theta filter (not part of the paper's method; `theta_filter` = l_cut).

The filter replaces every interior row by its orthogonal projection, in the discrete inner
product with Fejer's first-rule weights, onto the spin-weighted harmonics of the problem's s
and m with l < l_cut. The oracle computes it from that definition (a Gram-system solve over
its own unnormalised Goldberg profiles). Pinned here against:

* Legendre polynomials from mpmath at 256 bits (s = m = 0): a row that is a Legendre series
  keeps exactly its terms below l_cut (Fejer's rule on n_theta cell centres is exact for
  polynomials in cos(theta) of degree < n_theta);
* the normalised spin-weighted harmonics of the oracle's separate swsh() for
  (s, m) = (-2, 2), (-1, -3), (0, 1);
* projection properties: idempotence, no growth of the weighted norm, window edges and
  r* boundary rows untouched;
* its purpose: on the photon-sphere rows of a = 0.99, r* in [-100, 400] with 1024 points,
  random data grow by orders of magnitude without it and decay with l_cut = 7.
"""
import mpmath as mpm
import numpy as np
import pytest


def _oracle(oracle_mod, *, s=0, m=0, a=0.5, n_theta=32, l_cut=6, bits=256, rows=(10, 13), **kw):
    return oracle_mod.Oracle(M=1.0, a=a, s=s, m=m, rstar_min=-100.0, rstar_max=400.0, n_r=64,
                             n_theta=n_theta, dt=0.0, substeps=1, bits=bits, row_lo=rows[0],
                             row_hi=rows[1], theta_filter=l_cut, **kw)


def _words(x, n):
    """mpmath value -> n doubles whose sum approximates it."""
    out, rest = [], x
    for _ in range(n):
        d = float(rest)
        out.append(d)
        rest -= d
    return out


def test_filter_keeps_legendre_terms_below_cut_256bit(oracle_mod):
    mpm.mp.prec = 256
    nth, l_cut, deg, words = 32, 6, 20, 3
    rng = np.random.default_rng(11)
    o = _oracle(oracle_mod, n_theta=nth, l_cut=l_cut)
    xs = [mpm.cos((j + mpm.mpf(1) / 2) * mpm.pi / nth) for j in range(nth)]
    state = np.zeros((4, words, o.nrow, nth))
    want = {}
    for c in range(4):
        for i in range(o.nrow):
            b = rng.standard_normal(deg + 1)
            full = [sum(mpm.mpf(float(b[l])) * mpm.legendre(l, x) for l in range(deg + 1)) for x in xs]
            want[c, i] = [sum(mpm.mpf(float(b[l])) * mpm.legendre(l, x) for l in range(l_cut)) for x in xs]
            for j in range(nth):
                state[c, :, i, j] = _words(full[j], words)
    o.set_state(state)
    o.filter_rows()
    got = o.get_state(words=words)
    for c in range(4):
        for i in (1, 2):  # interior rows of the window
            scale = max(abs(v) for v in want[c, i])
            for j in range(nth):
                g = sum(mpm.mpf(float(got[c, k, i, j])) for k in range(words))
                assert abs(g - want[c, i][j]) <= mpm.mpf(10) ** -40 * scale, (c, i, j)
    # the frozen window edges are left as they are
    np.testing.assert_array_equal(got[:, 0, 0], state[:, 0, 0])
    np.testing.assert_array_equal(got[:, 0, -1], state[:, 0, -1])


@pytest.mark.parametrize("s,m", [(-2, 2), (-1, -3), (0, 1)])
def test_filter_keeps_spin_weighted_harmonics_below_cut(oracle_mod, s, m):
    nth = 40
    l_low = max(abs(s), abs(m))
    l_cut = l_low + 6
    o = _oracle(oracle_mod, s=s, m=m, n_theta=nth, l_cut=l_cut, parity=oracle_mod.default_parity(m, s))
    th = o.grid(1)["theta"][0]
    Y = {l: oracle_mod.swsh(s, m, l, th, out_words=1)[0] for l in range(l_low, l_low + 13)}
    rng = np.random.default_rng(5 + 7 * abs(s) + abs(m))
    state = np.zeros((4, 1, o.nrow, nth))
    want = np.zeros_like(state)
    for c in range(4):
        for i in range(o.nrow):
            b = rng.standard_normal(13)
            state[c, 0, i] = sum(b[q] * Y[l_low + q] for q in range(13))
            want[c, 0, i] = sum(b[q] * Y[l_low + q] for q in range(6)) if 0 < i < o.nrow - 1 else state[c, 0, i]
    o.set_state(state)
    o.filter_rows()
    got = o.get_state()
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    # l_cut = l_low + 1 keeps exactly the l_low term
    o1 = _oracle(oracle_mod, s=s, m=m, n_theta=nth, l_cut=l_low + 1, parity=oracle_mod.default_parity(m, s))
    o1.set_state(state)
    o1.filter_rows()
    lead = o1.get_state()[0, 0, 1]
    b0 = np.dot(lead, Y[l_low]) / np.dot(Y[l_low], Y[l_low])
    assert np.abs(lead - b0 * Y[l_low]).max() <= 1e-12 * np.abs(lead).max()


def test_filter_is_a_contracting_projection(oracle_mod):
    nth, l_cut = 48, 9
    o = _oracle(oracle_mod, s=-2, m=2, n_theta=nth, l_cut=l_cut, bits=53, rows=(0, 6))
    rng = np.random.default_rng(2)
    u = rng.standard_normal((4, 1, o.nrow, nth))
    u[:, :, 0] = 0.0  # global boundary row r* = r*_min
    o.set_state(u)
    o.filter_rows()
    once = o.get_state()
    o.filter_rows()
    twice = o.get_state()
    assert np.abs(twice - once).max() <= 1e-13 * np.abs(once).max()
    w = oracle_mod.fejer_weights(nth, out_words=1)[0]
    for c in range(4):
        for i in range(1, o.nrow - 1):
            assert np.dot(w, once[c, 0, i] ** 2) <= np.dot(w, u[c, 0, i] ** 2) * (1 + 1e-13)
    assert not once[:, 0, 0].any()
    np.testing.assert_array_equal(once[:, 0, -1], u[:, 0, -1])


def test_filter_parameter_rules(oracle_mod):
    for s, m, l_cut in [(0, 0, -1), (-2, 2, 2), (-1, -3, 3), (0, 0, 40)]:
        with pytest.raises(ValueError):
            _oracle(oracle_mod, s=s, m=m, n_theta=32, l_cut=l_cut)
    o = _oracle(oracle_mod, l_cut=0)
    with pytest.raises(ValueError):
        o.filter_rows()


def test_filter_period_schedule(oracle_mod):
    """With period 3 the filter projects at outer steps 0 and 3: four outer steps equal three
    outer steps that project at step 0 only (period 1024), then one outer step that projects
    (a fresh run with period 1 from that state); and differ from projecting every step."""
    kw = dict(M=1.0, a=0.9, s=-1, m=2, rstar_min=-30.0, rstar_max=50.0, n_r=41, n_theta=24, dt=0.0,
              substeps=3, bits=53, ko_sigma=1.0, theta_filter=6, parity=oracle_mod.default_parity(2, -1))
    rng = np.random.default_rng(9)
    u = rng.standard_normal((4, 1, 41, 24))
    u[:, :, 0] = 0.0
    u[:, :, -1] = 0.0
    runs = {}
    for period in (3, 1024, 1):
        runs[period] = oracle_mod.Oracle(theta_filter_period=period, **kw)
        runs[period].set_state(u)
    runs[3].step(4 * 3)
    runs[1].step(4 * 3)
    runs[1024].step(3 * 3)
    last = oracle_mod.Oracle(theta_filter_period=1, **kw)
    last.set_state(runs[1024].get_state())
    last.step(3)
    np.testing.assert_array_equal(runs[3].get_state(), last.get_state())
    assert not np.array_equal(runs[3].get_state(), runs[1].get_state())


def test_filter_removes_photon_sphere_growth(oracle_mod):
    """a = 0.99, s = m = 0, r* in [-100, 400] with 1024 points, k = 20, r* dissipation
    sigma = 2, theta x 32, random data on rows 150..260 (r* from -27 to 27): multipoles
    l >= 7 are trapped at r ~ 3M by the grid and grow; l_cut = 7 removes them, every outer
    step or every 8th (about 1 M)."""
    peaks = {}
    for l_cut, period in ((0, 1), (7, 1), (7, 8)):
        o = oracle_mod.Oracle(M=1.0, a=0.99, s=0, m=0, rstar_min=-100.0, rstar_max=400.0, n_r=1024,
                              n_theta=32, dt=0.0, substeps=20, bits=53, ko_sigma=2.0, row_lo=150,
                              row_hi=260, theta_filter=l_cut, theta_filter_period=period)
        rng = np.random.default_rng(3)
        u = rng.standard_normal((4, 1, o.nrow, 32))
        u[:, :, :3] = 0.0
        u[:, :, -3:] = 0.0
        o.set_state(u)
        trace = []
        for _ in range(8):
            o.step(250 * 20)  # 250 outer steps, 30.5 M
            trace.append(np.abs(o.get_state()).max())
        peaks[l_cut, period] = trace
    assert peaks[0, 1][-1] > 1e6 * peaks[0, 1][1]        # unfiltered: e^{~0.1 t}
    for period in (1, 8):
        assert peaks[7, period][-1] < 0.5 * peaks[7, period][1]  # filtered: decays
        assert peaks[0, 1][-1] > 1e6 * peaks[7, period][-1]
