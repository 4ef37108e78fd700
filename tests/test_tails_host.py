"""Host logic of the Kerr-tails study (Sec. 3.C, Fig. 1): the local power index and the
reflection-free span of the study's domain."""
import numpy as np

from paper_1006_0663_gb300 import tails, workloads


def test_local_power_index_of_exact_power_laws():
    t = np.linspace(100.0, 2000.0, 4001)
    for n in (3.0, 5.0, 7.5):
        idx = tails.local_power_index(t, 1e-30 * t ** -n, stride=4)
        assert np.nanmax(np.abs(idx - n)) < 1e-9
        assert np.isnan(idx[:4]).all() and np.isnan(idx[-4:]).all()


def test_local_power_index_with_log_correction():
    # t^-3 (1 + 10/t): the index tends to 3 from above as 3 + 10/(t + 10)
    t = np.linspace(200.0, 1500.0, 2001)
    idx = tails.local_power_index(t, t ** -3 * (1 + 10 / t), stride=2)
    ok = np.isfinite(idx)
    np.testing.assert_allclose(idx[ok], 3 + 10 / (t[ok] + 10), rtol=1e-6)


def test_zero_amplitude_gives_nan_not_inf():
    t = np.linspace(1.0, 10.0, 11)
    amp = np.ones_like(t)
    amp[5] = 0.0
    idx = tails.local_power_index(t, amp, stride=1)
    assert np.isnan(idx[4]) and np.isnan(idx[6])


def test_study_domain_is_reflection_free_for_the_whole_run():
    p = workloads.TAILS
    assert tails.reflection_free_until(p) >= p.steps * p.dt
    assert (p.s, p.m, p.ell) == (0, 0, 0) and p.words == 4
    # observer inside the domain, pulse ahead of it
    assert p.rstar_min < p.center < p.rstar_obs < p.rstar_max


def test_power_law_fit():
    t = np.linspace(500.0, 1500.0, 2001)
    assert abs(tails.power_law_fit(t, 3e-20 * t ** -7.0, 1000.0, 1450.0) - 7.0) < 1e-9
    assert tails.power_law_fit(t, np.zeros_like(t), 1000.0, 1450.0) is None


def test_velocity_data_planes():
    p = workloads.TAILS.with_(n_r=41, n_theta=8, rstar_min=-10.0, rstar_max=30.0)
    planes = tails.velocity_data(p, 4)
    assert planes.shape == (4, 4, 41, 8)
    assert not planes[:2].any() and not planes[:, 1:].any()    # Phi = 0, single-word values
    assert not planes[:, :, [0, -1]].any()                      # zero r* boundary rows
    ar, _ = p.amps
    i = int(round((p.center - p.rstar_min) / p.dr))
    assert planes[2, 0, i, 3] == ar                              # Gaussian peak, theta-constant
