"""Kerr-tails study on the GPU (Sec. 3.C, Fig. 1): invariants of the multipole split that hold
at any size, in every arithmetic, through the C ABI."""
import numpy as np
import pytest

from paper_1006_0663_gb300 import tails, teuk, workloads

pytestmark = pytest.mark.gpu

EPS = {1: 2.0 ** -52, 2: 2.0 ** -104, 4: 2.0 ** -208}


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _scalar(a, **kw):
    base = dict(M=1.0, a=a, s=0, m=0, rstar_min=-60.0, rstar_max=120.0, n_r=181, n_theta=32, dt=0.0,
                substeps=4, theta_order=10, parity=0)
    base.update(kw)
    return base


def _multipoles(p, W, steps, ell_max=8):
    g = teuk.Teuk(precision=W, **p)
    g.set_initial_pulse(10.0, 4.0, 0.9, 0.4, 0)
    g.set_observer(30.0, capacity=steps)
    g.step(steps)
    g.sync()
    return g.read_multipoles(0, ell_max)


@pytest.mark.parametrize("W", [1, 2, 4])
def test_schwarzschild_keeps_a_pure_monopole(W):
    """a = 0, s = m = 0: the discrete theta operator annihilates a theta-constant field and no
    coefficient depends on theta, so l' = 0 data stay l = 0; the projections onto l >= 1 are
    rounding-level (Fejer's rule integrates the constant times sY_l0 exactly)."""
    c = _multipoles(_scalar(0.0), W, 60)
    lead = np.hypot(c[:, :, 0, 0], c[:, :, 1, 0])
    scale = lead[:, 0].max()
    assert scale > 1e-3
    assert lead[:, 1:].max() < 64 * EPS[W] * scale, lead[:, 1:].max() / scale


@pytest.mark.parametrize("W", [1, 2, 4])
def test_kerr_couples_even_multipoles_only(W):
    """a = 0.9: the theta dependence of Sigma^2 couples l = 0 to l = 2, 4, ... (Fig. 1), while
    the problem is symmetric under theta -> pi - theta, so odd l stay at rounding level."""
    c = _multipoles(_scalar(0.9), W, 60)
    lead = np.hypot(c[:, :, 0, 0], c[:, :, 1, 0])
    scale = lead[:, 0].max()
    # even multipoles of this run (oracle, FP64): l = 2 ~ 9e-4, l = 4 ~ 4e-7, l = 6 ~ 1e-9 of l = 0
    assert lead[:, 2].max() > 1e-4 * scale
    assert lead[:, 4].max() > 1e-8 * scale
    assert lead[:, 6].max() > 1e-11 * scale
    odd = lead[:, 1::2].max()
    assert odd < 1e4 * EPS[W] * scale, odd / scale


def test_multipoles_agree_across_arithmetics():
    """The same short Kerr run in FP64, dd and qd: the l = 0 and l = 2 series agree to the
    cruder arithmetic's accuracy, dd to qd far below FP64 rounding."""
    p = _scalar(0.9)
    c1, c2, c4 = (_multipoles(p, W, 40, ell_max=2) for W in (1, 2, 4))
    ref = c4[..., 0] + c4[..., 1]
    scale = np.abs(ref).max()
    assert np.abs(c1[..., 0] - ref).max() < 1e-12 * scale
    assert np.abs((c2[..., 0] + c2[..., 1]) - ref).max() < 1e-26 * scale


def test_study_run_reports_power_indices():
    """A short prefix of the study workload through tails.run: shapes, reflection-free span
    and a finite local power index for l = 0 once the pulse has passed the observer."""
    p = workloads.TAILS
    res = tails.run(p, precision=2, ell_max=4, steps=800, tune=False)
    assert res["amp"].shape == (800, 5)
    assert res["reflection_free_until"] >= p.steps * p.dt
    n0 = tails.local_power_index(res["t"], res["amp"][:, 0], stride=8)
    assert np.isnan(n0[-8:]).all()            # centred differences need 8 samples on each side
    assert np.isfinite(n0[-40:-8]).all()
