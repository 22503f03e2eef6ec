"""Largest stable time step on a halving ladder, run with the CUDA propagator.

The paper prints no time steps; it used the largest stable one (Sec. 3.4).  For
grids where the CPU checker is too slow to follow a run through the initial
plume burst, this runs one slice from the seeded initial condition with each
dt of the ladder dt0, dt0/2, ... until t_end, and reports the first dt whose
run stays finite.

    python -m paper_2001_01609_gb300.survey Ra Nx Nz dt0 t_end [--mixed] [--rungs R]
"""
import argparse
import json

import numpy as np


def stable_dt(Ra, Nx, Nz, dt0, t_end, mixed=False, rungs=8, seed=0, chunk=500):
    import torch
    from . import build
    build.build()
    from . import rbc
    from .inputs import initial_temperature
    prec = rbc.RBC_MIXED if mixed else rbc.RBC_FP64
    log = []
    dt = dt0
    for _ in range(rungs):
        F = rbc.Propagator(Ra, 1.0, 2.0, Nx, Nz, dt, precision=prec)
        st = F.new_states(1)
        F.set_state(st[0], initial_temperature(Nx, Nz, seed=seed))
        n = int(round(t_end / dt))
        done, ok = 0, True
        while done < n:
            k = min(chunk, n - done)
            F.step_batch(st, k)
            done += k
            if F.check_diverged() != rbc.RBC_OK or not torch.isfinite(st).all() or st.abs().max().item() > 1e6:
                ok = False
                break
        nu = F.nusselt(st[0])[0] if ok else float("nan")
        log.append(dict(dt=dt, stable=ok, t_reached=done * dt, nu_v=nu))
        F.close()
        if ok:
            return dt, log
        dt *= 0.5
    return None, log


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("Ra", type=float)
    ap.add_argument("Nx", type=int)
    ap.add_argument("Nz", type=int)
    ap.add_argument("dt0", type=float)
    ap.add_argument("t_end", type=float)
    ap.add_argument("--mixed", action="store_true")
    ap.add_argument("--rungs", type=int, default=8)
    a = ap.parse_args()
    dt, log = stable_dt(a.Ra, a.Nx, a.Nz, a.dt0, a.t_end, a.mixed, a.rungs)
    print(json.dumps(dict(Ra=a.Ra, grid=f"{a.Nx}x{a.Nz}", mixed=a.mixed, stable_dt=dt, ladder=log)))


if __name__ == "__main__":
    main()
