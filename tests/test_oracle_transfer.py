"""Pins of the oracle's grid transfers of the coarse propagator (Sec. 3.6: the
coarse solver runs on a grid reduced by the coarsening factor; reading: both
grids share the Fourier x Chebyshev basis, so restriction truncates the
coefficient arrays and prolongation zero-pads them).

The fields are evaluated point by point from their definition
f(x, z) = sum_{|m| < Nx/2} sum_n f_mn T_n(2z) exp(i k_m x) (f_{-m} = conj f_m),
with u = d psi/dz + U(z) and w = -d psi/dx, by brute-force sums, independently
of the oracle's transforms.

* Restriction is the orthogonal projection onto the coarse space in the
  Chebyshev-weighted inner product (Fourier truncation is the L2 projection in
  x, Chebyshev truncation the projection with the weight (1 - s^2)^(-1/2)):
  the residual f - R f is orthogonal to every coarse basis function, for the
  fields whose coefficients are stored (T, psi and the mean flow U; w = -d psi/dx
  too, the x-derivative not mixing modes).  The inner products are
  Gauss-Chebyshev and uniform-x quadratures, exact here.
* Prolongation represents the same function: the coarse and the prolonged
  state agree at arbitrary points, for T, u (mean flow included), w, psi, U.
* R(P(X)) = X exactly.
"""
import numpy as np
import pytest

from oracle import rbc as orbc
from paper_2001_01609_gb300.inputs import initial_temperature

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

LX = 2.0


def cheb_T(n_max, s):
    """T_0..T_{n_max-1} at the points s (three-term recurrence), shape (n_max, len(s))."""
    s = np.asarray(s, dtype=np.float64)
    T = np.zeros((n_max, s.size))
    T[0] = 1.0
    if n_max > 1:
        T[1] = s
    for n in range(2, n_max):
        T[n] = 2.0 * s * T[n - 1] - T[n - 2]
    return T


def cheb_dT(n_max, s):
    """d T_n / ds at the points s, from T_n' = n U_{n-1} (second kind, by recurrence)."""
    s = np.asarray(s, dtype=np.float64)
    U = np.zeros((n_max, s.size))
    U[0] = 1.0
    if n_max > 1:
        U[1] = 2.0 * s
    for n in range(2, n_max):
        U[n] = 2.0 * s * U[n - 1] - U[n - 2]
    d = np.zeros((n_max, s.size))
    for n in range(1, n_max):
        d[n] = n * U[n - 1]
    return d


def evaluate(X, x, z):
    """(T, u, w, psi, U) of the state X at the points (x[i], z[i]), by brute-force sums."""
    nm, Nz = X.T.shape
    s = 2.0 * np.asarray(z)
    Tn, dTn = cheb_T(Nz, s), cheb_dT(Nz, s)
    T = np.zeros(len(x))
    u = np.zeros(len(x))
    w = np.zeros(len(x))
    psi = np.zeros(len(x))
    for m in range(nm):
        k = 2.0 * np.pi * m / LX
        e = np.exp(1j * k * np.asarray(x))
        c = 1.0 if m == 0 else 2.0                      # f_m e^{ikx} + conj, real part
        tz = X.T[m] @ Tn
        pz = X.psi[m] @ Tn
        dpz = 2.0 * (X.psi[m] @ dTn)                    # d/dz = 2 d/ds
        T += c * np.real(tz * e)
        if m > 0:
            psi += c * np.real(pz * e)
            u += c * np.real(dpz * e)
            w += c * np.real(-1j * k * pz * e)
    U = X.U @ Tn                                        # mean flow
    return T, u + U, w, psi, U


def fine_state(Nx, Nz, seed):
    rng = np.random.default_rng(seed)
    r = orbc.RBC(1e5, 1.0, LX, Nx, Nz, 1e-3)
    X = r.from_grid(initial_temperature(Nx, Nz, seed=seed, amplitude=0.3))
    # give psi and the mean flow content of their own (from_grid keeps them zero for w = u = 0)
    nm = Nx // 2
    X.psi = (rng.standard_normal((nm, Nz)) + 1j * rng.standard_normal((nm, Nz))) / (1.0 + np.arange(Nz)) ** 2
    X.psi[0] = 0.0
    X.U = rng.standard_normal(Nz) / (1.0 + np.arange(Nz)) ** 2
    return X


def weighted_projection(f_of, Nx, nm_c, nz_c, Q):
    """<f, e^{i k_m x} T_n(s)> over x in [0, Lx) (uniform, Nx points) and s with the
    Chebyshev weight (Gauss-Chebyshev, Q points), for m < nm_c, n < nz_c."""
    xs = LX * np.arange(Nx) / Nx
    q = np.arange(Q)
    s = np.cos(np.pi * (q + 0.5) / Q)
    wq = np.pi / Q
    xx, ss = np.meshgrid(xs, s, indexing="ij")
    vals = f_of(xx.ravel(), 0.5 * ss.ravel()).reshape(Nx, Q)
    Tn = cheb_T(nz_c, s)
    out = np.zeros((nm_c, nz_c), dtype=complex)
    for m in range(nm_c):
        e = np.exp(-1j * 2.0 * np.pi * m / LX * xs)
        out[m] = (e @ vals) @ Tn.T * wq
    return out


@pytest.mark.parametrize("fine_grid,coarse_grid", [((16, 12), (8, 8)), ((24, 16), (12, 10)), ((16, 16), (16, 8))])
def test_restriction_residual_is_orthogonal_to_the_coarse_space(fine_grid, coarse_grid):
    (Nx, Nz), (Nxc, Nzc) = fine_grid, coarse_grid
    X = fine_state(Nx, Nz, seed=5)
    Xc = orbc.restrict(X, Nxc, Nzc)
    assert Xc.T.shape == (Nxc // 2, Nzc) and Xc.psi.shape == (Nxc // 2, Nzc) and Xc.U.shape == (Nzc,)
    Q = Nz + 6
    for field in (0, 2, 3, 4):          # T, w, psi, U
        def resid(x, z, field=field):
            return evaluate(X, x, z)[field] - evaluate(Xc, x, z)[field]

        def full(x, z, field=field):
            return evaluate(X, x, z)[field]
        p_res = weighted_projection(resid, Nx, Nxc // 2, Nzc, Q)
        p_full = weighted_projection(full, Nx, Nxc // 2, Nzc, Q)
        assert np.abs(p_full).max() > 1e-3                     # the field has coarse content
        assert np.abs(p_res).max() < 1e-12 * np.abs(p_full).max(), field


@pytest.mark.parametrize("coarse_grid,fine_grid", [((8, 8), (16, 12)), ((12, 10), (24, 16))])
def test_prolongation_represents_the_same_fields(coarse_grid, fine_grid):
    (Nxc, Nzc), (Nx, Nz) = coarse_grid, fine_grid
    Xc = fine_state(Nxc, Nzc, seed=11)
    Xf = orbc.prolong(Xc, Nx, Nz)
    assert Xf.T.shape == (Nx // 2, Nz) and Xf.U.shape == (Nz,)
    rng = np.random.default_rng(3)
    x = rng.uniform(0.0, LX, 64)
    z = rng.uniform(-0.5, 0.5, 64)
    for a, b in zip(evaluate(Xc, x, z), evaluate(Xf, x, z)):
        assert np.abs(a).max() > 1e-3
        assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()


def test_restrict_of_prolong_is_the_identity_bitwise():
    Xc = fine_state(12, 10, seed=13)
    Xc.T[0] = Xc.T[0].real
    back = orbc.restrict(orbc.prolong(Xc, 24, 16), 12, 10)
    for a, b in zip(back.arrays(), Xc.arrays()):
        assert np.array_equal(a, b)
