"""Reindexing between the oracle's State and the C ABI's spectral state layout.

Pure data movement, no arithmetic of the method: the ABI state is
double X[2][Nz][Nx/2][2] (field T / psi, Chebyshev n, Fourier m, re/im) with the
mean flow U in the m = 0 slot of psi (include/rbc.h).
"""
import numpy as np

from oracle.rbc import State


def to_abi(X):
    nm, Nz = X.T.shape
    a = np.zeros((2, Nz, nm, 2))
    a[0, :, :, 0] = X.T.real.T
    a[0, :, :, 1] = X.T.imag.T
    P = X.psi.copy()
    P[0] = X.U
    a[1, :, :, 0] = P.real.T
    a[1, :, :, 1] = P.imag.T
    return a


def from_abi(a):
    a = np.asarray(a)
    T = (a[0, :, :, 0] + 1j * a[0, :, :, 1]).T.copy()
    P = (a[1, :, :, 0] + 1j * a[1, :, :, 1]).T.copy()
    U = P[0].real.copy()
    P[0] = 0.0
    return State(T, P, U)


def max_rel_diff(A, B):
    """max |A - B| over all coefficients / max |B|."""
    d = max(np.abs(A.T - B.T).max(), np.abs(A.psi - B.psi).max(), np.abs(A.U - B.U).max())
    s = max(np.abs(B.T).max(), np.abs(B.psi).max(), np.abs(B.U).max())
    return d / s
