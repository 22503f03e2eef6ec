"""Parareal iteration with defect and Nusselt stopping norms.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Eq. 20: U_{n+1}^{k+1} = G(t_{n+1}, t_n, U_n^{k+1}) + F(t_{n+1}, t_n, U_n^k)
                         - G(t_{n+1}, t_n, U_n^k),
with U_0^k = U_0 and U^0 from one serial coarse sweep (Sec. 3.1).  Reading: the
sum is formed as F + (G_new - G_old), so that a slice whose input did not change
gets exactly F (bitwise) - the paper notes that after as many iterations as
slices the solution is the serial fine one.
"""
import numpy as np


def parareal(U0, nslices, F, G, max_iters, diff_norm, nu_window=None,
             criterion="fixed", tol=0.0, summarize=None, change=None):
    """Run Parareal.

    F(U) -> (U_end, nu_integral); G(U) -> U_end; states support + and -.
    diff_norm(a, b) -> ||a - b|| / ||a||.  nu_window = (first slice, window
    length) for Nu_k = sum of the Nu_V integrals over those slices / length.
    With ``summarize``, F returns (U_end, integrals) of any kind and
    Nu_k = summarize(list of the window slices' integrals) instead.

    criterion: "fixed" (max_iters iterations, the paper's Sec. 3.7 practice),
    "defect" (stop at the first k with Defect_k <= tol), "nu" (stop at the
    first k with |Nu_k - Nu_{k-1}| / |Nu_k| <= tol) or "stat" (stop at the
    first k with change(Nu_k, Nu_{k-1}) <= tol, for summaries of several
    statistics; Sec. 5.2).

    Returns dict(U=list of U_n^k, k=iterations done, defects=[...], nus=[...],
    F=list of the last F results, serial_coarse=U^0).
    """
    N = nslices
    U = [U0]
    Gold = []
    for n in range(N):
        g = G(U[n])
        Gold.append(g)
        U.append(g)
    U_coarse = list(U)
    Fres = [None] * N
    Inu = [0.0] * N
    defects, nus = [], []
    k_done = 0
    for k in range(1, max_iters + 1):
        for n in range(k - 1, N):
            Fres[n], Inu[n] = F(U[n])
        if nu_window is not None:
            n0, length = nu_window
            nus.append(sum(Inu[n0:]) / length if summarize is None else summarize(Inu[n0:]))
        Unew = [U0]
        for n in range(N):
            gnew = G(Unew[n])
            Unew.append(Fres[n] + (gnew - Gold[n]))
            Gold[n] = gnew
        defects.append(max(diff_norm(Unew[n], U[n]) for n in range(1, N + 1)))
        U = Unew
        k_done = k
        if criterion == "defect" and defects[-1] <= tol:
            break
        if criterion == "nu" and len(nus) >= 2 and abs(nus[-1] - nus[-2]) <= tol * abs(nus[-1]):
            break
        if criterion == "stat" and len(nus) >= 2 and change(nus[-1], nus[-2]) <= tol:
            break
    return dict(U=U, k=k_done, defects=defects, nus=nus, F=Fres, serial_coarse=U_coarse)


def dahlquist_closed_form(u0, f, g, n, k):
    """U_n^k for y' = lam y with exact per-slice factors f (fine) and g (coarse).

    Expanding Eq. 20 on a scalar linear problem gives
    U_n^k = sum_{j=0}^{min(k,n)} binom(n, j) (f - g)^j g^(n-j) u0.
    """
    from math import comb
    return sum(comb(n, j) * (f - g) ** j * g ** (n - j) for j in range(min(k, n) + 1)) * u0
