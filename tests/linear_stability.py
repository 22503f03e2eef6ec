"""Independent linear-stability solver for the onset pin (Sec. 3.3).

Not part of the oracle: a separate Chebyshev *collocation* discretisation
(Gauss-Lobatto differentiation matrices, boundary rows replacing equations) of
the Boussinesq equations linearised about the conduction state T = 1/2 - z,
u = 0, in the same variables (psi, T) and units as Eqs. 3-6:

    sigma lap_k psi = Pr lap_k^2 psi - i k Pr Ra theta
    sigma theta     = lap_k theta + (-dT0/dz) w = lap_k theta - i k psi,

psi = psi' = 0 and theta = 0 on z = +-1/2 (fixed temperature, Eq. 6), or
theta' = 0 there (fixed flux, Eq. 7: the conduction profile has the same
slope, so only the temperature boundary rows change).  It shares no code with
``oracle``.  Chandrasekhar's marginal curve for two rigid walls has its minimum
Ra_c = 1707.76 at k_c = 3.117; the paper reports agreement within 0.1%.  With
fixed flux at two rigid walls the marginal curve decreases to Ra_c = 720 as
k -> 0 (Sparrow, Goldstein & Jonsson 1964; Hurle, Jakeman & Pike 1967).
"""
import numpy as np
import scipy.linalg as sla
from scipy.optimize import brentq, minimize_scalar


def cheb_collocation(N):
    """Trefethen's Chebyshev differentiation matrix on x_j = cos(pi j / N)."""
    x = np.cos(np.pi * np.arange(N + 1) / N)
    c = np.ones(N + 1)
    c[0] = c[-1] = 2.0
    c *= (-1.0) ** np.arange(N + 1)
    X = np.tile(x, (N + 1, 1)).T
    dX = X - X.T
    D = np.outer(c, 1.0 / c) / (dX + np.eye(N + 1))
    D -= np.diag(D.sum(axis=1))
    return D, x


def growth_rates(Ra, k, Pr=1.0, N=40, bc="fixed_T"):
    """All finite eigenvalues sigma of the linearised problem at wavenumber k."""
    D, s = cheb_collocation(N)
    Dz = 2.0 * D                       # z = s/2
    I = np.eye(N + 1)
    lap = Dz @ Dz - k * k * I
    n = N + 1
    A = np.zeros((2 * n, 2 * n), dtype=complex)
    B = np.zeros((2 * n, 2 * n), dtype=complex)
    A[:n, :n] = Pr * lap @ lap
    A[:n, n:] = -1j * k * Pr * Ra * I
    B[:n, :n] = lap
    A[n:, :n] = -1j * k * I
    A[n:, n:] = lap
    B[n:, n:] = I
    # boundary rows: psi(+-1) = 0, psi'(+-1) = 0 (rows 0, 1, N-1, N of the psi block), theta(+-1) = 0
    for r, row in ((0, I[0]), (N, I[N]), (1, Dz[0]), (N - 1, Dz[N])):
        A[r, :] = 0.0
        B[r, :] = 0.0
        A[r, :n] = row
    for r, j in ((n, 0), (n + N, N)):
        A[r, :] = 0.0
        B[r, :] = 0.0
        if bc == "fixed_T":
            A[r, n + j] = 1.0
        else:
            A[r, n:] = Dz[j]
    w = sla.eig(A, B, right=False)
    w = w[np.isfinite(w)]
    return w[np.abs(w) < 1e8]


def max_growth(Ra, k, Pr=1.0, N=40, bc="fixed_T"):
    return np.max(growth_rates(Ra, k, Pr, N, bc).real)


def critical_Ra(k, Pr=1.0, N=40, bc="fixed_T", lo=1000.0, hi=5000.0):
    """Ra at which the leading growth rate crosses zero for wavenumber k."""
    return brentq(lambda Ra: max_growth(Ra, k, Pr, N, bc), lo, hi, xtol=1e-10)


def critical_point(Pr=1.0, N=40):
    """(k_c, Ra_c) minimising the marginal curve."""
    r = minimize_scalar(lambda k: critical_Ra(k, Pr, N), bounds=(2.5, 3.8), method="bounded",
                        options={"xatol": 1e-6})
    return r.x, r.fun
