"""Time-averaged statistics and the consistency checks of Sec. 2.2, and a
statistical stopping rule for Parareal (Sec. 3.7, Sec. 5.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 2.2 assesses a run by time averages (the overbar) of volume and plane
averages:

* the characteristic speed U = mean of <u^2 + w^2>_V^(1/2); with velocities in
  units of kappa / L, Re = U / Pr (the paper's Pr = 1 gives Re = U);
* Nu_V, Nu_b, Nu_t (Eqs. 9-11) and Nu_int, their largest pairwise difference
  relative to Nu_V (Eq. 13);
* buoyancy production P = Ra mean <w T>_V against viscous dissipation
  eps_U = |mean <u . lap u>_V| (Eq. 14), checked as |P - eps_U| / P (Eq. 15);
* T_rms(z) (Eq. 16), whose peak height above the bottom wall is the thermal
  boundary-layer thickness delta_T, and N_BL, the number of grid points inside
  it (at least 6, Sec. 2.2); Eq. 17 relates delta_t = 1 / (2 Nu) (L = 1).

Readings (the paper gives no sampling rule or time-integration rule):

* diagnostics are sampled every ``every`` time steps and at the end of each
  trajectory; time means are trapezoid integrals over the samples divided by
  the sampled duration;
* Eq. 16 as printed takes the square root of a square; read as the RMS
  fluctuation about the time-mean plane average:
  T_rms(z)^2 = mean <T^2>_x - (mean <T>_x)^2;
* delta_T is the distance from the bottom wall of the largest T_rms over the
  padded Lobatto points of the lower half (the first such point from the wall
  on a tie); N_BL counts the interior native Lobatto points no farther than
  delta_T from the wall;
* statistical stopping (the paper leaves the rule open, Sec. 3.7 and
  Sec. 5.2): stop at the first iteration k >= 2 whose time means of
  (Nu_V, Nu_b, Nu_t, Re, P, eps_U) over the averaging window all changed by at
  most ``tol`` relative to iteration k - 1.
"""
import numpy as np

SCALARS = ("sqrtKE2", "eps", "wT", "NuV", "Nub", "Nut")
PROFILES = ("Tm", "T2")
STAT_QUANTITIES = ("NuV", "Nub", "Nut", "Re", "P", "eps_U")


def sample(rbc, X):
    """The sampled quantities of one state (Sec. 2.2): scalars and two profiles."""
    d = rbc.diagnostics(X)
    return dict(sqrtKE2=np.sqrt(d["KE2"]), eps=d["eps"], wT=d["wT"], NuV=d["nu"][0], Nub=d["nu"][1],
                Nut=d["nu"][2], Tm=d["Tm"], T2=d["Tv"] + d["Tm"] ** 2)


def run_sampled(rbc, X, nsteps, every):
    """Advance X by nsteps time steps, sampling at steps 0, every, 2 every, ...
    and nsteps; returns (X_end, integrals): the trapezoid time integral of each
    sampled quantity and the duration "T"."""
    if every < 1:
        raise ValueError("every >= 1")
    prev = sample(rbc, X)
    acc = {q: 0.0 * v for q, v in prev.items()}
    s = 0
    while s < nsteps:
        c = min(every, nsteps - s)
        for _ in range(c):
            X, _ = rbc.step(X)
        cur = sample(rbc, X)
        h = c * rbc.dt
        for q in acc:
            acc[q] = acc[q] + 0.5 * h * (prev[q] + cur[q])
        prev = cur
        s += c
    acc["T"] = nsteps * rbc.dt
    return X, acc


def combine(integrals):
    """Integrals of consecutive trajectories (time slices) added up."""
    out = {q: 0.0 * v for q, v in integrals[0].items()}
    for I in integrals:
        for q in out:
            out[q] = out[q] + I[q]
    return out


def lobatto_distance(Nz):
    """Distance from the bottom wall of the interior native points (Lz = 1)."""
    j = np.arange(1, Nz - 1)
    return 0.5 - 0.5 * np.cos(np.pi * j / (Nz - 1))


def boundary_layer(Trms, zp, Nz):
    """(delta_T, N_BL) from a T_rms profile at the padded points zp (descending z)."""
    lower = np.nonzero(zp < 0.0)[0]
    order = lower[np.argsort(zp[lower])]            # from the bottom wall upwards
    vals = Trms[order]
    if not np.any(vals > 0.0):
        return float("nan"), 0
    i = int(np.argmax(vals))                          # first maximum from the wall
    delta = float(zp[order[i]] + 0.5)
    return delta, int(np.count_nonzero(lobatto_distance(Nz) <= delta))


def averages(I, Ra, Pr, zp, Nz):
    """Time means and the consistency checks of Sec. 2.2 from summed integrals."""
    D = I["T"]
    m = {q: I[q] / D for q in SCALARS + PROFILES}
    NuV, Nub, Nut = m["NuV"], m["Nub"], m["Nut"]
    U = m["sqrtKE2"]
    P = Ra * m["wT"]
    eps_U = abs(m["eps"])
    Trms = np.sqrt(np.maximum(m["T2"] - m["Tm"] ** 2, 0.0))
    delta_T, N_BL = boundary_layer(Trms, zp, Nz)
    return dict(U=U, Re=U / Pr, NuV=NuV, Nub=Nub, Nut=Nut,
                Nu_int=max(abs(Nub - NuV), abs(Nub - Nut), abs(NuV - Nut)) / NuV,
                P=P, eps_U=eps_U, balance=abs(P - eps_U) / P if P != 0.0 else float("nan"),
                Trms=Trms, delta_T=delta_T, N_BL=N_BL, delta_t=0.5 / NuV, duration=D)


def stat_change(new, old, quantities=STAT_QUANTITIES):
    """Largest relative change of the statistical quantities between iterations."""
    return max(abs(new[q] - old[q]) / abs(new[q]) for q in quantities)
