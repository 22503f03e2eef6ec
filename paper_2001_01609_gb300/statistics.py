"""Time statistics of the consistency checks of Sec. 2.2, and Parareal with a
statistical stopping rule (Sec. 3.7, Sec. 5.2), driven through the C ABI.

Every field operation runs in the CUDA library: the fine and coarse steps
(rbc_step_batch), restriction, prolongation and the correction of Eq. 20
(rbc_restrict, rbc_prolong, rbc_parareal_correct), the defect norms
(rbc_l2_diff) and the per-state averages (rbc_diagnostics).  The host keeps the
trapezoid time integrals of the sampled averages (a few hundred numbers per
slice and sample) and forms the final ratios.

Quantities (Sec. 2.2): the characteristic speed U = mean <u^2 + w^2>_V^(1/2)
and Re = U / Pr (velocities in units of kappa / L; the paper's Pr = 1 gives
Re = U); Nu_V, Nu_b, Nu_t (Eqs. 9-11); Nu_int (Eq. 13); buoyancy production
P = Ra mean <w T>_V and viscous dissipation eps_U = |mean <u . lap u>_V|
(Eq. 14) with the balance |P - eps_U| / P (Eq. 15); T_rms(z) (Eq. 16) with
T_rms^2 = mean <T^2>_x - (mean <T>_x)^2; delta_T, the height above the bottom
wall of the T_rms peak over the padded points of the lower half (nearest the
wall on a tie), and N_BL, the interior native Lobatto points within delta_T
of the wall; delta_t = 1 / (2 Nu_V) (Eq. 17, L = 1).

Sampling: the averages are taken every ``every`` fine steps and at the end of
each slice; time means are trapezoid integrals over the samples divided by the
sampled duration.

Statistical stopping (the rule the paper leaves open): iteration k's fine
sweep, launched from U^(k-1), gives time means over the averaging window (the
second half of the slices by default); stop at the first k >= 2 at which every
one of (Nu_V, Nu_b, Nu_t, Re, P, eps_U) changed by at most ``tol`` relative to
iteration k - 1.  As with the library's own iteration, k stops at nslices,
where the fine trajectories are the serial fine ones.
"""
import math

import numpy as np

from . import rbc

STAT_QUANTITIES = ("NuV", "Nub", "Nut", "Re", "P", "eps_U")
STAT, FIXED = "stat", "fixed"


def padded_z(Nz):
    """z of the padded Lobatto points of rbc_diagnostics' profiles (descending)."""
    Mz = 3 * Nz // 2
    return 0.5 * np.cos(np.pi * np.arange(Mz) / (Mz - 1))


def sample_values(diag, Mz):
    """Per-state sampled quantities from rbc_diagnostics rows (B, 6 + 2 Mz):
    [U, <u.lap u>_V, <wT>_V, Nu_V, Nu_b, Nu_t, <T>_x (Mz), <T^2>_x (Mz)]."""
    d = np.asarray(diag, dtype=np.float64)
    v = d.copy()
    v[:, 0] = np.sqrt(d[:, 0])
    Tm, Tv = d[:, 6:6 + Mz], d[:, 6 + Mz:6 + 2 * Mz]
    v[:, 6 + Mz:] = Tv + Tm * Tm
    return v


def sampled_run(prop, states, nsteps, every):
    """Advance the B states by nsteps steps in place (on the current stream),
    sampling the Sec. 2.2 averages at steps 0, every, 2 every, ... and nsteps.
    Returns the trapezoid time integrals (B, 6 + 2 Mz) in sample_values'
    column order."""
    if every < 1:
        raise ValueError("every must be at least 1")
    Mz = 3 * prop.Nz // 2
    prev = sample_values(prop.diagnostics(states).cpu().numpy(), Mz)
    acc = np.zeros_like(prev)
    s = 0
    while s < nsteps:
        c = min(every, nsteps - s)
        prop.step_batch(states, c)
        cur = sample_values(prop.diagnostics(states).cpu().numpy(), Mz)
        acc += (0.5 * c * prop.dt) * (prev + cur)
        prev = cur
        s += c
    return acc


def boundary_layer(Trms, zp, Nz):
    """(delta_T, N_BL) from T_rms at the padded points zp."""
    lower = np.nonzero(zp < 0.0)[0]
    up = lower[np.argsort(zp[lower])]              # from the bottom wall upwards
    vals = Trms[up]
    if not np.any(vals > 0.0):
        return float("nan"), 0
    delta = float(zp[up[int(np.argmax(vals))]] + 0.5)
    j = np.arange(1, Nz - 1)
    dist = 0.5 - 0.5 * np.cos(np.pi * j / (Nz - 1))
    return delta, int(np.count_nonzero(dist <= delta))


def averages(integrals, duration, Ra, Pr, Nz):
    """Time means and the Sec. 2.2 checks from the summed integrals of one or
    more trajectories (rows are added) over `duration`."""
    I = np.asarray(integrals, dtype=np.float64)
    if I.ndim == 2:
        I = I.sum(axis=0)
    Mz = 3 * Nz // 2
    m = I / duration
    U, eps, wT, NuV, Nub, Nut = (float(x) for x in m[:6])
    Tm, T2 = m[6:6 + Mz], m[6 + Mz:6 + 2 * Mz]
    Trms = np.sqrt(np.maximum(T2 - Tm * Tm, 0.0))
    P, eps_U = Ra * wT, abs(eps)
    delta_T, N_BL = boundary_layer(Trms, padded_z(Nz), Nz)
    return dict(U=U, Re=U / Pr, NuV=NuV, Nub=Nub, Nut=Nut,
                Nu_int=max(abs(Nub - NuV), abs(Nub - Nut), abs(NuV - Nut)) / NuV,
                P=P, eps_U=eps_U, balance=abs(P - eps_U) / P if P != 0.0 else float("nan"),
                Trms=Trms, delta_T=delta_T, N_BL=N_BL, delta_t=0.5 / NuV, duration=duration)


def stat_change(new, old, quantities=STAT_QUANTITIES):
    """Largest relative change of the statistical quantities between two iterations."""
    return max(abs(new[q] - old[q]) / abs(new[q]) for q in quantities)


def _whole_steps(length, dt):
    q = length / dt
    n = round(q)
    if n < 1 or abs(q - n) > 1e-9 * n:
        raise ValueError(f"slice length {length} is not a whole number of steps of {dt}")
    return int(n)


class StatisticalParareal:
    """Parareal (Eq. 20) over [t0, t1] with nslices slices, sampling the Sec. 2.2
    averages along every fine sweep and stopping on their time means."""

    def __init__(self, fine, coarse, t0, t1, nslices, every, tol=1e-2, window_first=None, criterion=STAT,
                 lib=rbc):
        if criterion not in (STAT, FIXED):
            raise ValueError(f"criterion {criterion!r}")
        if nslices < 1 or every < 1:
            raise ValueError("nslices and every must be at least 1")
        self.fine, self.coarse, self.lib = fine, coarse, lib
        self.N, self.every, self.tol, self.criterion = nslices, every, tol, criterion
        slice_len = (t1 - t0) / nslices
        self.nf = _whole_steps(slice_len, fine.dt)
        self.nc = _whole_steps(slice_len, coarse.dt)
        self.window_first = nslices // 2 if window_first is None else window_first
        if not 0 <= self.window_first < nslices:
            raise ValueError("window_first outside the slices")
        self.window = (nslices - self.window_first) * self.nf * fine.dt

    def iterate(self, U0, U, max_iters):
        """Run up to max_iters iterations from U0 into U (nslices + 1 states), on
        the current stream.

        Returns dict(status, k, defects, stats): stats[k-1] are the time means
        of iteration k's fine trajectories (from U^(k-1)) over the window.
        status: RBC_OK when the rule was met (always for the fixed count),
        RBC_ENOTCONVERGED when the iterations ran out, RBC_EDIVERGED on a
        non-finite state."""
        import torch
        F, G, lib, N = self.fine, self.coarse, self.lib, self.N
        U[0].copy_(U0)
        Gold = G.new_states(N, U.device)
        g = G.new_states(1, U.device)
        for n in range(N):                                   # U^0: the serial coarse sweep
            lib.restrict(F, G, U[n:n + 1], g)
            G.step_batch(g, self.nc)
            Gold[n].copy_(g[0])
            lib.prolong(F, G, g, U[n + 1:n + 2])
        Fres = F.new_states(N, U.device)
        K = 6 + 2 * (3 * F.Nz // 2)
        integ = np.zeros((N, K))
        Uold = F.new_states(N + 1, U.device)
        norms = torch.zeros(2 * (N + 1), dtype=torch.float64, device=U.device)
        defects, stats = [], []
        status, k = rbc.RBC_ENOTCONVERGED, 0
        for k in range(1, min(max_iters, N) + 1):
            n0 = k - 1                                       # slices n < k - 1 are exact already
            Fres[n0:].copy_(U[n0:N])
            integ[n0:] = sampled_run(F, Fres[n0:], self.nf, self.every)
            stats.append(averages(integ[self.window_first:], self.window, F.Ra, F.Pr, F.Nz))
            Uold.copy_(U)
            for n in range(n0, N):
                lib.restrict(F, G, U[n:n + 1], g)
                G.step_batch(g, self.nc)
                lib.parareal_correct(F, G, Fres[n:n + 1], g, Gold[n:n + 1], U[n + 1:n + 2])
                Gold[n].copy_(g[0])
            lib.l2_diff(F, U, Uold, norms[:N + 1])
            lib.l2_diff(F, U, None, norms[N + 1:])
            nrm = norms.cpu().numpy()
            defect = 0.0
            for n in range(1, N + 1):
                a, b = nrm[n], nrm[N + 1 + n]
                if not (math.isfinite(a) and math.isfinite(b)):
                    return dict(status=rbc.RBC_EDIVERGED, k=k, defects=defects, stats=stats)
                if b > 0.0:
                    defect = max(defect, math.sqrt(a / b))
            defects.append(defect)
            if self.criterion == STAT and k >= 2 and stat_change(stats[-1], stats[-2]) <= self.tol:
                status = rbc.RBC_OK
                break
        else:
            if self.criterion == FIXED:
                status = rbc.RBC_OK
        return dict(status=status, k=k, defects=defects, stats=stats)
