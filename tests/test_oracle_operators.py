"""Pins of the oracle's z-operators against library routines and closed forms."""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as C
from scipy.special import eval_gegenbauer

from oracle import ultraspherical as us
from oracle.rbc import RBC

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")
RNG = np.random.default_rng(7)
S = np.linspace(-0.97, 0.99, 23)


def gegen_series(coef, lam, s):
    return sum(c * eval_gegenbauer(n, lam, s) for n, c in enumerate(coef))


@pytest.mark.parametrize("lam", [1, 2, 3, 4])
def test_conversion_chain_matches_gegenbauer(lam):
    N = 14
    a = np.zeros(N)
    a[: N - 2 * lam] = RNG.standard_normal(N - 2 * lam)   # room so truncation is exact
    b = us.convert_chain(lam, N) @ a
    np.testing.assert_allclose(gegen_series(b, lam, S), C.chebval(S, a), rtol=0, atol=1e-12)


@pytest.mark.parametrize("lam", [1, 2, 4])
def test_derivative_matches_chebder(lam):
    N = 12
    a = RNG.standard_normal(N)
    b = us.derivative(lam, N) @ a
    ref = C.chebval(S, C.chebder(a, m=lam))
    np.testing.assert_allclose(gegen_series(b, lam, S), ref, rtol=1e-12, atol=1e-9)


def test_S4D2_is_second_derivative_in_C4():
    N = 16
    a = np.zeros(N)
    a[:10] = RNG.standard_normal(10)
    b = us.convert_C(3, N) @ us.convert_C(2, N) @ us.derivative(2, N) @ a
    np.testing.assert_allclose(gegen_series(b, 4, S), C.chebval(S, C.chebder(a, 2)), atol=1e-10)


def test_boundary_rows():
    N = 11
    a = RNG.standard_normal(N)
    for side in (-1.0, 1.0):
        assert abs(us.value_row(N, side) @ a - C.chebval(side, a)) < 1e-12
        assert abs(us.slope_row(N, side) @ a - C.chebval(side, C.chebder(a))) < 1e-10


def test_gram_matrix_by_gauss_legendre():
    N = 9
    x, w = np.polynomial.legendre.leggauss(40)
    V = C.chebvander(x, N - 1)
    np.testing.assert_allclose(us.cheb_gram(N), V.T @ (w[:, None] * V), atol=1e-13)


def test_clenshaw_curtis_weights_exact_for_low_degree():
    r = RBC(1e4, 1.0, 2.0, 8, 16, 1e-3)
    sp = np.cos(np.pi * np.arange(r.Mz) / (r.Mz - 1))
    for deg in range(0, r.Mz):
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)             # int_{-1}^{1} s^deg ds
        assert abs(np.dot(r.cc_weights, sp ** deg) - exact) < 1e-12


def test_padded_transforms_roundtrip():
    r = RBC(1e4, 1.0, 2.0, 12, 10, 1e-3)
    c = RNG.standard_normal((r.nm, r.Nz)) + 1j * RNG.standard_normal((r.nm, r.Nz))
    c[0] = c[0].real
    g = r._spec_to_padded_grid(c)
    np.testing.assert_allclose(r._padded_grid_to_spec(g), c, atol=1e-12)


def test_native_grid_roundtrip_and_streamfunction():
    r = RBC(1e4, 1.0, 2.0, 12, 10, 1e-3)
    X = r.zero_state()
    X.T = RNG.standard_normal(X.T.shape) + 1j * RNG.standard_normal(X.T.shape)
    X.T[0] = X.T[0].real
    X.psi[1:] = RNG.standard_normal(X.psi[1:].shape) + 1j * RNG.standard_normal(X.psi[1:].shape)
    X.U = RNG.standard_normal(r.Nz)
    Tg, ug, wg = r.to_grid(X)
    Y = r.from_grid(Tg, ug, wg)
    np.testing.assert_allclose(Y.T, X.T, atol=1e-12)
    np.testing.assert_allclose(Y.psi, X.psi, atol=1e-12)
    np.testing.assert_allclose(Y.U, X.U, atol=1e-12)
    # u = d_z psi, w = -d_x psi checked by finite differences of the evaluated field
    x = np.linspace(0, 2, 7)[:, None]
    z = np.linspace(-0.45, 0.45, 5)[None, :]

    def psi_at(xx, zz):
        tot = np.zeros(np.broadcast(xx, zz).shape)
        for m in range(r.nm):
            fac = 1.0 if m == 0 else 2.0
            tot = tot + fac * (C.chebval(2 * zz, X.psi[m]) * np.exp(1j * r.k[m] * xx)).real
        return tot

    def w_at(xx, zz):
        tot = np.zeros(np.broadcast(xx, zz).shape)
        for m in range(1, r.nm):
            tot = tot + 2.0 * (C.chebval(2 * zz, -1j * r.k[m] * X.psi[m]) * np.exp(1j * r.k[m] * xx)).real
        return tot

    h = 1e-5
    fd = -(psi_at(x + h, z) - psi_at(x - h, z)) / (2 * h)
    np.testing.assert_allclose(w_at(x, z), fd, atol=1e-5)
