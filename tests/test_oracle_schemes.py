"""Lower-order coarse steppers (Sec. 3.6): ARS(2,2,2) and ARS(1,1,1), the two
smaller IMEX Runge-Kutta pairs of the family RK443 belongs to.

S1 structure and order conditions of each pair: explicit first stage, constant
   implicit diagonal, row sums equal to the abscissae, stiffly accurate; order 2
   for RK222 (each part and the coupling conditions) and order 1 for RK111.
S2 L-stability of the implicit parts: R(z) -> 0 as z -> -inf.
S3 the oracle's time stepper on linear diffusion (one temperature mode, and the
   mean flow with Pr != 1): the decay per step equals the closed-form stability
   function of the implicit part, 1/(1 - z) for backward Euler and
   (1 + (1 - 2 g) z)/(1 - g z)^2 for ARS(2,2,2) with g = 1 - 1/sqrt(2),
   derived by hand from the two stage equations.
S4 observed order of convergence on a convecting state: 2 and 1.
S5 the default scheme is RK443, unchanged bit for bit.
"""
import math

import numpy as np
import pytest

from oracle.rbc import RBC, SCHEMES
from test_oracle_pins import conduction, cos_pi_z

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

G = 1.0 - 1.0 / math.sqrt(2.0)
ORDER = {"RK443": 3, "RK222": 2, "RK111": 1}


def dot(a, b):
    return sum(x * y for x, y in zip(a, b))


def matvec(A, v):
    return [dot(row, v) for row in A]


@pytest.mark.parametrize("name", ["RK222", "RK111"])
def test_S1_structure_and_order_conditions(name):
    c, AI, AE = SCHEMES[name]
    s = len(AI)
    assert len(AE) == s and len(c) == s
    for i in range(s):
        assert abs(sum(AI[i]) - c[i]) < 1e-15 and abs(sum(AE[i]) - c[i]) < 1e-15
        assert all(AE[i][j] == 0 for j in range(i, s))          # explicit part explicit
        assert all(AI[i][j] == 0 for j in range(i + 1, s))      # implicit part lower triangular
        assert AI[i][0] == 0                                    # explicit first stage
    assert all(abs(AI[i][i] - AI[1][1]) < 1e-16 for i in range(1, s))   # one stage matrix
    bI, bE = AI[-1], AE[-1]                                     # stiffly accurate
    for b in (bI, bE):
        assert abs(sum(b) - 1) < 1e-15
    if ORDER[name] >= 2:
        for b in (bI, bE):
            assert abs(dot(b, c) - 0.5) < 1e-15
        # the pair's coupling conditions for order 2 (the same abscissae)
        assert abs(dot(bI, matvec(AE, [1.0] * s)) - 0.5) < 1e-15
        assert abs(dot(bE, matvec(AI, [1.0] * s)) - 0.5) < 1e-15
    else:
        assert abs(dot(bI, c) - 0.5) > 0.1                      # first order only


def stability(AI, z):
    s = len(AI)
    Y = np.linalg.solve(np.eye(s) - z * np.array(AI, dtype=float), np.ones(s))
    return Y[-1]


@pytest.mark.parametrize("name", ["RK443", "RK222", "RK111"])
def test_S2_implicit_parts_are_L_stable(name):
    AI = SCHEMES[name][1]
    assert abs(stability(AI, -1e12)) < 1e-10
    for z in (-0.1, -1.0, -10.0, -100.0):
        assert abs(stability(AI, z)) < 1.0


def closed_form_R(name, z):
    if name == "RK111":
        return 1.0 / (1.0 - z)
    return (1.0 + (1.0 - 2.0 * G) * z) / (1.0 - G * z) ** 2


@pytest.mark.parametrize("name", ["RK222", "RK111"])
def test_S3_temperature_mode_decays_by_the_closed_form(name):
    r = RBC(0.0, 1.0, 2.0, 8, 32, 2e-3, scheme=name)
    X = conduction(r)
    a = cos_pi_z(r.Nz)
    X.T[1] = 1e-2 * a
    n = 7
    Y, _ = r.run(X, n)
    z = r.dt * -(r.k[1] ** 2 + np.pi ** 2)
    ref = closed_form_R(name, z) ** n * 1e-2 * a
    np.testing.assert_allclose(Y.T[1].real, ref, rtol=0, atol=1e-15)
    assert np.abs(Y.T[1].imag).max() < 1e-17
    np.testing.assert_allclose(Y.T[0], X.T[0], atol=1e-15)


@pytest.mark.parametrize("name", ["RK222", "RK111"])
def test_S3_mean_flow_decays_by_the_closed_form_with_Pr(name):
    Pr = 2.5
    r = RBC(0.0, Pr, 2.0, 8, 32, 1e-3, scheme=name)
    X = conduction(r)
    a = cos_pi_z(r.Nz)
    X.U = 0.3 * a
    n = 6
    Y, _ = r.run(X, n)
    ref = closed_form_R(name, r.dt * (-Pr * np.pi ** 2)) ** n * 0.3 * a
    np.testing.assert_allclose(Y.U, ref, atol=1e-14)


def _convect(dt, scheme):
    r = RBC(5e3, 1.0, 2.0, 16, 16, dt, scheme=scheme)
    X = conduction(r)
    X.T[1] = 0.05 * cos_pi_z(r.Nz)
    X.T[2] = 0.02j * cos_pi_z(r.Nz)
    Y, _ = r.run(X, int(round(0.024 / dt)))
    return Y


@pytest.fixture(scope="module")
def reference_run():
    return _convect(0.024 / 1536, "RK443")


@pytest.mark.parametrize("name", ["RK222", "RK111"])
def test_S4_observed_order_of_convergence(name, reference_run):
    ref = reference_run
    errs = []
    for dt in (0.024 / 48, 0.024 / 96, 0.024 / 192):
        Y = _convect(dt, name)
        errs.append(max(np.abs(Y.T - ref.T).max(), np.abs(Y.psi - ref.psi).max()))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    p = ORDER[name]
    assert np.all(np.abs(orders - p) < 0.05), (errs, orders)


def test_S5_default_scheme_is_rk443():
    a = RBC(5e3, 1.0, 2.0, 16, 16, 1e-4)
    b = RBC(5e3, 1.0, 2.0, 16, 16, 1e-4, scheme="RK443")
    assert a.stages == 4 and a.gamma == 0.5
    X = conduction(a)
    X.T[1] = 0.05 * cos_pi_z(a.Nz)
    Ya, _ = a.run(X, 5)
    Yb, _ = b.run(X, 5)
    assert np.array_equal(Ya.T, Yb.T) and np.array_equal(Ya.psi, Yb.psi) and np.array_equal(Ya.U, Yb.U)
    with pytest.raises(ValueError):
        RBC(5e3, 1.0, 2.0, 16, 16, 1e-4, scheme="RK332")
