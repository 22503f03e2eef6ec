"""Pins of the oracle with fixed-flux walls (Eq. 7: dT/dz = -1 at z = +-1/2, Ra
read as the flux Rayleigh number of Eq. 8).

FF1 the linear conduction profile is a fixed point with Nu = 1; FF2 a
Neumann temperature mode decays by the implicit stability function exactly;
FF3 the independent collocation solver's marginal curve tends to the classical
Ra_c = 720 as k -> 0 (rigid, insulating walls); FF4 the oracle's stage
operators have the collocation solver's growth rate at k = pi, and its onset
there; FF5 the time stepper grows at that rate; FF6 the walls' slopes stay at
-1 (Nu_b = Nu_t = 1) and the mean temperature is conserved while convecting.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.optimize import brentq
from scipy.special import jv

import linear_stability as ls
from oracle.rbc import RBC
from test_oracle_pins import conduction, cos_pi_z, implicit_stability

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")
FF = "fixed_flux"


def cos_pi_zp(N):
    """Chebyshev coefficients of cos(pi (z + 1/2)) = -sin(pi s / 2) (Jacobi-Anger)."""
    a = np.zeros(N)
    for j in range((N - 1) // 2 + 1):
        if 2 * j + 1 < N:
            a[2 * j + 1] = -2.0 * (-1) ** j * jv(2 * j + 1, np.pi / 2)
    return a


def test_FF1_conduction_is_a_fixed_point():
    r = RBC(5e4, 1.0, 2.0, 16, 16, 1e-3, bc=FF)
    X = conduction(r)
    Y, _ = r.run(X, 5)
    assert np.abs(Y.T - X.T).max() < 1e-14
    assert np.abs(Y.psi).max() == 0.0 and np.abs(Y.U).max() == 0.0
    np.testing.assert_allclose(r.nusselt(Y), 1.0, atol=1e-13)


@pytest.mark.parametrize("m", [0, 1])
def test_FF2_neumann_mode_decays_by_the_stability_function(m):
    r = RBC(0.0, 1.0, 2.0, 8, 32, 2e-3, bc=FF)
    X = conduction(r)
    a = cos_pi_zp(r.Nz)
    X.T[m] = X.T[m] + 1e-2 * a
    n = 7
    Y, _ = r.run(X, n)
    ref = implicit_stability(r.dt * -(r.k[m] ** 2 + np.pi ** 2)) ** n * 1e-2 * a
    base = conduction(r).T[m]
    np.testing.assert_allclose(Y.T[m].real - base.real, ref, rtol=0, atol=1e-15)
    # the fixed-temperature walls would not let this mode decay freely
    Z, _ = RBC(0.0, 1.0, 2.0, 8, 32, 2e-3).run(X, n)
    assert np.abs(Z.T[m].real - base.real - ref).max() > 1e-4


# the Neumann boundary rows make the collocation problem less well conditioned
# than the Dirichlet one: at 32 points it is converged to about 1e-7
NC = 32


def fixed_flux_onset():
    with open(os.path.join(os.path.dirname(__file__), "golden", "fixed_flux_onset.txt")) as f:
        return float(next(l for l in f if l.strip() and not l.startswith("#")).split()[0])


def test_FF3_collocation_marginal_curve_tends_to_720():
    Ra0 = fixed_flux_onset()
    r2 = ls.critical_Ra(0.2, N=NC, bc=FF, lo=500.0, hi=3000.0)
    r1 = ls.critical_Ra(0.1, N=NC, bc=FF, lo=500.0, hi=3000.0)
    assert Ra0 < r1 < r2 < Ra0 + 2.0
    assert abs((r2 - Ra0) / (r1 - Ra0) - 4.0) < 0.05               # approaches the limit like k^2
    assert abs(r1 - (r2 - r1) / 3.0 - Ra0) < 0.01                  # Richardson limit k -> 0


def oracle_linear_eigs_ff(r, m):
    """Eigenvalues of the oracle's linearised stage operators at mode m, with its
    fixed-flux temperature rows."""
    Nz, k = r.Nz, r.k[m]
    MT, LT = r.ops_T(k)
    MP, LP, Cpl = r.ops_psi(k)
    A = np.zeros((2 * Nz, 2 * Nz), dtype=complex)
    B = np.zeros_like(A)
    A[: Nz - 2, :Nz] = LT
    A[: Nz - 2, Nz:] = -1j * k * r.S2
    B[: Nz - 2, :Nz] = MT
    A[Nz - 2, :Nz] = r.T_bc_lo
    A[Nz - 1, :Nz] = r.T_bc_hi
    A[Nz : 2 * Nz - 4, :Nz] = Cpl
    A[Nz : 2 * Nz - 4, Nz:] = LP
    B[Nz : 2 * Nz - 4, Nz:] = MP
    A[2 * Nz - 4, Nz:] = r.bc_val_lo
    A[2 * Nz - 3, Nz:] = r.bc_val_hi
    A[2 * Nz - 2, Nz:] = r.bc_slope_lo
    A[2 * Nz - 1, Nz:] = r.bc_slope_hi
    w = sla.eig(A, B, right=False)
    w = w[np.isfinite(w)]
    return w[np.abs(w) < 1e8]


@pytest.mark.parametrize("Ra", [900.0, 1100.0, 5000.0])
def test_FF4_oracle_operators_match_collocation_growth_rate(Ra):
    r = RBC(Ra, 1.0, 2.0, 4, 40, 1e-3, bc=FF)
    s_oracle = np.max(oracle_linear_eigs_ff(r, 1).real)
    s_coll = ls.max_growth(Ra, np.pi, N=NC, bc=FF)
    assert abs(s_oracle - s_coll) < 1e-6 * max(1.0, abs(s_coll))


def test_FF4_onset_at_k_pi():
    def sig(Ra):
        return np.max(oracle_linear_eigs_ff(RBC(Ra, 1.0, 2.0, 4, 32, 1e-3, bc=FF), 1).real)
    Ra_pi = brentq(sig, 900.0, 1300.0, xtol=1e-8)
    assert abs(Ra_pi - ls.critical_Ra(np.pi, N=NC, bc=FF, lo=500.0, hi=3000.0)) < 1e-3
    assert fixed_flux_onset() < Ra_pi < ls.critical_Ra(np.pi)         # below the fixed-T onset


def test_FF5_time_stepper_growth_rate_matches_eigenvalue():
    Ra, dt = 2000.0, 2e-3
    r = RBC(Ra, 1.0, 2.0, 4, 24, dt, bc=FF)
    X = conduction(r)
    X.T[1] = 1e-9 * cos_pi_z(r.Nz)           # even in z, like the leading mode
    X, _ = r.run(X, 150)
    a0 = np.abs(X.T[1]).max()
    X, _ = r.run(X, 100)
    rate = np.log(np.abs(X.T[1]).max() / a0) / (100 * dt)
    sigma = ls.max_growth(Ra, np.pi, N=NC, bc=FF)
    assert sigma > 0
    assert abs(rate - sigma) < 2e-3 * abs(sigma), (rate, sigma)


def test_FF6_wall_slopes_and_mean_temperature_while_convecting():
    r = RBC(2e4, 1.0, 2.0, 16, 24, 2e-3, bc=FF)
    X = conduction(r)
    X.T[1] = 1e-2 * cos_pi_zp(r.Nz)
    n = np.arange(r.Nz)
    mean0 = 0.5 * np.sum(X.T[0].real[::2] * 2.0 / (1.0 - n[::2] ** 2))   # <T>_V = (1/2) int T_0 ds
    X, _ = r.run(X, 200)
    _, nb, nt = r.nusselt(X)
    assert abs(nb - 1.0) < 1e-12 and abs(nt - 1.0) < 1e-12
    assert np.abs(X.psi).max() > 1e-3                                  # it convects
    mean = 0.5 * np.sum(X.T[0].real[::2] * 2.0 / (1.0 - n[::2] ** 2))
    assert abs(mean - mean0) < 1e-7
