"""Chebyshev / ultraspherical (Gegenbauer) operators for the z-direction.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper discretises z with Chebyshev polynomials (Sec. 3.2) and treats the
linear terms implicitly; it does not say how the boundary conditions enter.  The
reading used throughout this repository is the ultraspherical tau method of
Olver & Townsend (2013): an equation of differential order lambda is written in
the C^(lambda) basis, its last lambda rows are replaced by boundary rows.

All operators act on Chebyshev-T coefficient vectors a (f(s) = sum_n a_n T_n(s),
s in [-1, 1]) and are returned as dense N x N matrices (slow, plain).
"""
from math import factorial

import numpy as np


def convert_T_to_C1(N):
    """S_0: T-coefficients -> C^(1)-coefficients of the same function.

    T_0 = C^(1)_0, T_1 = C^(1)_1 / 2, T_n = (C^(1)_n - C^(1)_{n-2}) / 2.
    """
    S = np.zeros((N, N))
    S[0, 0] = 1.0
    for j in range(1, N):
        S[j, j] = 0.5
    for j in range(N - 2):
        S[j, j + 2] = -0.5
    return S


def convert_C(lam, N):
    """S_lam: C^(lam)-coefficients -> C^(lam+1)-coefficients (lam >= 1).

    C^(lam)_n = lam / (n + lam) * (C^(lam+1)_n - C^(lam+1)_{n-2}).
    """
    S = np.zeros((N, N))
    for j in range(N):
        S[j, j] = lam / (j + lam)
        if j + 2 < N:
            S[j, j + 2] = -lam / (j + lam + 2)
    return S


def convert_chain(lam, N):
    """S_{lam-1} ... S_1 S_0: T-coefficients -> C^(lam)-coefficients."""
    S = convert_T_to_C1(N)
    for l in range(1, lam):
        S = convert_C(l, N) @ S
    return S


def derivative(lam, N):
    """D_lam: T-coefficients of f -> C^(lam)-coefficients of d^lam f / ds^lam.

    d^lam T_n / ds^lam = 2^(lam-1) (lam-1)! n C^(lam)_{n-lam}.
    """
    D = np.zeros((N, N))
    c = 2.0 ** (lam - 1) * factorial(lam - 1)
    for j in range(N - lam):
        D[j, j + lam] = c * (j + lam)
    return D


def value_row(N, side):
    """Row r with r @ a = f(side), side = +1 or -1: T_n(+-1) = (+-1)^n."""
    return np.array([float(side) ** n for n in range(N)])


def slope_row(N, side):
    """Row r with r @ a = df/ds(side): T_n'(+-1) = (+-1)^(n+1) n^2."""
    return np.array([float(side) ** (n + 1) * n * n for n in range(N)])


def cheb_derivative_matrix(N):
    """Dense N x N matrix of d/ds acting on T-coefficients (result in T basis)."""
    D = np.zeros((N, N))
    for n in range(N):
        e = np.zeros(N)
        e[n] = 1.0
        d = np.polynomial.chebyshev.chebder(e)
        D[: len(d), n] = d
    return D


def cheb_gram(N):
    """G_ab = int_{-1}^{1} T_a T_b ds (exact): products T_a T_b = (T_{a+b} + T_|a-b|)/2."""
    G = np.zeros((N, N))
    for a in range(N):
        for b in range(N):
            if (a + b) % 2 == 0:
                G[a, b] = 1.0 / (1.0 - (a + b) ** 2) + 1.0 / (1.0 - (a - b) ** 2)
    return G
