"""The stability reading (not fixed by the paper): one outer step of the scheme as a linear map,
taken from the oracle as a black box on the 1D problem a = 0, s = m = 0, l = 0 (a theta-constant
field), and its largest eigenvalue.

With 9 iterations per dt = 0.25 dr* on dr* = 1/2 a short r* wave near the potential peak grows
as e^{0.2 t}: the iterations divide the Courant number by 9 and with it the scheme's damping of
short waves. One iteration per dt on the same grid, or the tails study's dr* = 1/8 with two
iterations, keep every eigenvalue inside the unit circle."""
import numpy as np
import pytest


def _outer_step_matrix(oracle_mod, dr, k, rmin=-30.0, rmax=40.0, nth=6):
    n_r = int(round((rmax - rmin) / dr)) + 1
    o = oracle_mod.Oracle(M=1.0, a=0.0, s=0, m=0, rstar_min=rmin, rstar_max=rmax, n_r=n_r, n_theta=nth,
                          dt=0.0, substeps=k, theta_order=10, parity=1, bits=53)
    A = np.zeros((2 * n_r, 2 * n_r))
    for col in range(2 * n_r):
        comp, i = divmod(col, n_r)
        if i in (0, n_r - 1):
            continue
        st = np.zeros((4, 1, n_r, nth))
        st[2 * comp, 0, i, :] = 1.0  # Phi_R or Pi_R, constant in theta
        o.set_state(st)
        o.step(k)
        out = o.get_state(1)[:, 0]
        A[:n_r, col] = out[0, :, 0]
        A[n_r:, col] = out[2, :, 0]
    o.close()
    return A


@pytest.mark.slow
@pytest.mark.parametrize("dr,k,stable", [(0.5, 9, False), (0.5, 1, True), (0.125, 2, True)])
def test_outer_step_spectral_radius(oracle_mod, dr, k, stable):
    A = _outer_step_matrix(oracle_mod, dr, k)
    rho = np.abs(np.linalg.eigvals(A)).max()
    rate = np.log(rho) / (0.25 * dr)  # per unit time
    if stable:
        assert rho <= 1.0 + 1e-12, (rho, rate)
    else:
        assert rate > 0.1, (rho, rate)
