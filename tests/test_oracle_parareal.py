"""P6: Parareal pins (Eq. 20, Sec. 3.1, Fig. 7 caption: with as many iterations as
slices the Parareal solution is the serial fine one)."""
import numpy as np
import pytest

from oracle.parareal import dahlquist_closed_form, parareal
from oracle.rbc import RBC, prolong, restrict
from paper_2001_01609_gb300.inputs import initial_temperature

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


class Scalar:
    def __init__(self, v):
        self.v = v

    def __add__(self, o):
        return Scalar(self.v + o.v)

    def __sub__(self, o):
        return Scalar(self.v - o.v)


def test_dahlquist_matches_closed_form():
    lam, dT, N, K = -1.3 + 0.4j, 0.25, 8, 5
    f = np.exp(lam * dT)                     # exact fine propagator
    g = 1.0 / (1.0 - lam * dT)               # backward Euler coarse
    res = parareal(Scalar(1.0 + 0j), N, lambda U: (Scalar(f * U.v), 0.0), lambda U: Scalar(g * U.v),
                   K, lambda a, b: abs(a.v - b.v) / abs(a.v))
    for n in range(N + 1):
        assert abs(res["U"][n].v - dahlquist_closed_form(1.0, f, g, n, K)) < 1e-14
    for n in range(K + 1):
        assert abs(res["U"][n].v - f ** n) < 1e-14       # exact on the first K slices


def make_rbc(nsteps_f=4, nsteps_c=2):
    fine = RBC(3e4, 1.0, 2.0, 16, 16, 2e-3)
    coarse = RBC(3e4, 1.0, 2.0, 8, 8, 4e-3)
    U0 = fine.from_grid(initial_temperature(16, 16, seed=0, amplitude=0.3))

    def F(U):
        return fine.run(U, nsteps_f)

    def G(U):
        return prolong(coarse.run(restrict(U, 8, 8), nsteps_c)[0], 16, 16)

    def diff(a, b):
        return fine.l2_T(a - b) / fine.l2_T(a)

    return fine, U0, F, G, diff


def test_parareal_iterate_k_is_serial_fine_on_first_k_slices_bitwise():
    fine, U0, F, G, diff = make_rbc()
    N, K = 4, 2
    res = parareal(U0, N, F, G, K, diff)
    serial = [U0]
    for n in range(N):
        serial.append(F(serial[-1])[0])
    for n in range(K + 1):
        for a, b in zip(res["U"][n].arrays(), serial[n].arrays()):
            assert np.array_equal(a, b)
    # and not on later slices (the coarse propagator is really coarser)
    assert diff(res["U"][N], serial[N]) > 1e-8
    full = parareal(U0, N, F, G, N, diff)
    for a, b in zip(full["U"][N].arrays(), serial[N].arrays()):
        assert np.array_equal(a, b)


def test_parareal_with_G_equal_F_converges_in_one_iteration():
    fine, U0, F, G, diff = make_rbc()
    res = parareal(U0, 3, F, lambda U: F(U)[0], 2, diff)
    assert res["defects"][1] == 0.0


def test_parareal_defect_decreases_and_nu_window():
    fine, U0, F, G, diff = make_rbc()
    res = parareal(U0, 4, F, G, 3, diff, nu_window=(2, 2 * 4 * 2e-3))
    assert res["defects"][2] < res["defects"][0]
    assert len(res["nus"]) == 3 and all(np.isfinite(res["nus"]))
    stop = parareal(U0, 4, F, G, 4, diff, criterion="defect", tol=res["defects"][1] * 1.0001)
    assert stop["k"] == 2
