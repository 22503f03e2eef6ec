"""Time-step stability survey of one propagator (reading R9 of the configs).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  The paper prints no
time steps; it reports that the largest stable step met its accuracy criteria
(Sec. 3.4).  This script runs the oracle from the seeded initial condition with
a given dt until t_end or until the state blows up (non-finite, or a
coefficient above 1e6), printing Nu_V along the way, so that a halving ladder
of dt values can be checked.

    python -m oracle.survey_dt Ra Nx Nz dt t_end [seed]
"""
import sys
import time

import numpy as np

from oracle.rbc import RBC
from paper_2001_01609_gb300.inputs import initial_temperature


def survey(Ra, Nx, Nz, dt, t_end, seed=0, report_every=0.05):
    o = RBC(Ra, 1.0, 2.0, Nx, Nz, dt)
    X = o.from_grid(initial_temperature(Nx, Nz, seed=seed))
    nsteps = int(round(t_end / dt))
    every = max(1, int(round(report_every / dt)))
    t0 = time.time()
    for s in range(nsteps):
        X, nu = o.step(X)
        big = max(np.abs(X.T).max(), np.abs(X.psi).max())
        if not np.isfinite(big) or big > 1e6:
            print(f"BLOWUP at step {s + 1} t={(s + 1) * dt:.5f}", flush=True)
            return False
        if (s + 1) % every == 0:
            print(f"t={(s + 1) * dt:.4f} Nu_V={nu:.6f} max|psi|={np.abs(X.psi).max():.4e} "
                  f"wall={time.time() - t0:.0f}s", flush=True)
    print(f"STABLE to t={t_end}", flush=True)
    return True


if __name__ == "__main__":
    a = sys.argv[1:]
    survey(float(a[0]), int(a[1]), int(a[2]), float(a[3]), float(a[4]), int(a[5]) if len(a) > 5 else 0)
