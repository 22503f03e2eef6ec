"""The serving scheduler on the host, with a toy propagator standing in for the
library (tests/fake_propagator.py): every request's iterates, defects and Nu
values must equal those of the plain Parareal iteration (Eq. 20) run by the
oracle's driver with the same propagators, whatever the mix, the chunking of
the fine sweeps and the memory limit."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import fake_propagator as fake  # noqa: E402
from oracle.parareal import parareal  # noqa: E402
from paper_2001_01609_gb300 import rbc, serving  # noqa: E402


def classes(Nx, Nz, precision):
    return serving.ClassConfig(Nx, Nz, precision, 0.01, 0.02, 12, 6, Nx // 2, Nz // 2)


def engine(**kw):
    base = dict(max_iters=3, f_chunk=5, class_config=classes, keep_states=True, device="cpu", lib=fake,
                runtime=fake.HostRuntime(), mem_limit=1 << 40, bmax=64)
    base.update(kw)
    return serving.Engine(**base)


def initial(eng, r):
    cls = eng._class(r.key)
    u = cls.fine.new_states(1)
    g = np.random.Generator(np.random.PCG64(r.seed))
    cls.fine.set_state(u[0], 0.5 + 0.3 * g.standard_normal((r.Nz, r.Nx)))
    r.U0 = u[0]
    return r


def reference(eng, r, criterion="fixed", tol=0.0, max_iters=3):
    """Eq. 20 by the oracle's driver, with the toy fine and coarse propagators."""
    cfg = eng.config_for(r.key)
    Fp = fake.FakePropagator(r.Ra, 1.0, 2.0, r.Nx, r.Nz, cfg.dt_fine)
    Gp = fake.FakePropagator(r.Ra, 1.0, 2.0, cfg.coarse_Nx, cfg.coarse_Nz, cfg.dt_coarse)

    def F(U):
        X = U.clone()[None]
        nu = torch.zeros(1, dtype=torch.float64)
        Fp.step_batch(X, cfg.nf, nu)
        return X[0], float(nu[0])

    def G(U):
        c = Gp.new_states(1)
        fake.restrict(Fp, Gp, U[None], c)
        Gp.step_batch(c, cfg.nc)
        out = Fp.new_states(1)
        fake.prolong(Fp, Gp, c, out)
        return out[0]

    def diff(a, b):
        return math.sqrt(float(((a[0] - b[0]) ** 2).sum()) / float((a[0] ** 2).sum()))

    N = r.nslices
    t0, t1 = eng.interval(r)
    win = (t1 - t0) * (N - N // 2) / N
    return parareal(r.U0.clone(), N, F, G, min(max_iters, N), diff, nu_window=(N // 2, win),
                    criterion=criterion, tol=tol)


def requests(n=9, seed=0):
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        Nx, Nz = [(16, 8), (32, 16)][int(g.integers(2))]
        out.append(serving.Request(rid=i, Ra=float(10 ** g.uniform(3.5, 4.5)), Nx=Nx, Nz=Nz,
                                   nslices=int(g.integers(2, 9)), precision=int(g.integers(2)),
                                   arrival=0.0, seed=100 + i))
    return out


@pytest.mark.parametrize("f_chunk", [12, 5, 1])
def test_each_request_matches_plain_parareal(f_chunk):
    eng = engine(f_chunk=f_chunk)
    reqs = [initial(eng, r) for r in requests()]
    eng.run(reqs, deadline=60)
    for r in reqs:
        ref = reference(eng, r)
        assert r.status == rbc.RBC_OK and r.k_done == ref["k"]
        for n in range(r.nslices + 1):
            assert torch.equal(r.U[n], ref["U"][n]), (r.rid, n)
        assert r.defects == ref["defects"]
        # the oracle's driver sums the slices with Python's compensated sum(); the
        # engine, like the library, adds them in slice order
        np.testing.assert_allclose(r.nus, ref["nus"], rtol=1e-14 if f_chunk >= 12 else 1e-13)


def test_fine_batches_and_coarse_ticks_are_shared():
    eng = engine()
    reqs = [initial(eng, r) for r in requests()]
    eng.run(reqs, deadline=60)
    fb = sum(c.launches["f_batches"] for c in eng.classes.values())
    gt = sum(c.launches["g_ticks"] for c in eng.classes.values())
    # solo, each request needs ceil(12/5) fine launches per iteration and one coarse tick per slice per sweep
    solo_f = sum(3 * r.k_done for r in reqs)
    solo_g = sum(r.nslices * (r.k_done + 1) for r in reqs)
    assert fb < solo_f and gt < solo_g
    assert max(max(c.fine.batches) for c in eng.classes.values()) > max(r.nslices for r in reqs)
    assert eng.peak_active == len(reqs)


@pytest.mark.parametrize("criterion,tol", [("defect", 1e-3), ("nu", 1e-4)])
def test_stopping_criteria_match_plain_parareal(criterion, tol):
    crit = {"defect": rbc.CRIT_DEFECT, "nu": rbc.CRIT_NU}[criterion]
    eng = engine(criterion=crit, tol=tol, max_iters=6, f_chunk=12)
    reqs = [initial(eng, r) for r in requests(6, seed=3)]
    eng.run(reqs, deadline=60)
    for r in reqs:
        ref = reference(eng, r, criterion, tol, max_iters=6)
        assert r.k_done == ref["k"], r.rid
        assert r.defects == ref["defects"]
        converged = (ref["defects"][-1] <= tol) if criterion == "defect" else (
            len(ref["nus"]) >= 2 and abs(ref["nus"][-1] - ref["nus"][-2]) <= tol * abs(ref["nus"][-1]))
        assert r.status == (rbc.RBC_OK if converged else rbc.RBC_ENOTCONVERGED)


def test_memory_limit_bounds_admission_and_keeps_results():
    free = engine()
    base = [initial(free, r) for r in requests()]
    free.run(base, deadline=60)
    lim = engine()
    reqs = [initial(lim, r) for r in requests()]
    need = sorted(lim.request_bytes(r) for r in reqs)
    lim.mem_limit = lim.committed + need[-1]              # one large request at a time
    lim.run(reqs, deadline=60)
    assert lim.peak_committed <= lim.mem_limit
    assert lim.peak_active < len(reqs)
    for a, b in zip(base, reqs):
        assert torch.equal(a.U, b.U) and a.defects == b.defects
    with pytest.raises(RuntimeError):
        tiny = engine(mem_limit=1)
        tiny.run([initial(tiny, requests(1)[0])], deadline=10)


def test_arrivals_are_honoured_and_latency_reported():
    eng = engine()
    reqs = [initial(eng, r) for r in requests(4, seed=7)]
    for i, r in enumerate(reqs):
        r.arrival = 0.05 * i
    eng.run(reqs, deadline=60)
    for r in reqs:
        assert r.t_admit >= r.arrival and r.t_done >= r.t_admit and r.latency > 0
    st = serving.latency_stats(reqs)
    assert st["p50_s"] <= st["p99_s"] <= st["max_s"]
    assert serving.dof_steps(reqs, eng) == sum(
        2 * r.Nx * r.Nz * 12 * sum(r.nslices - (k - 1) for k in range(1, r.k_done + 1)) for r in reqs)


def test_deadline_stops_a_loop_that_cannot_progress():
    eng = engine(runtime=fake.HostRuntime(event_done=lambda: False))
    r = initial(eng, requests(1)[0])
    with pytest.raises(RuntimeError, match="deadline"):
        eng.run([r], deadline=0.5)


class _Diverging(fake.FakePropagator):
    """Steps that turn a state non-finite when its Ra is above a threshold."""

    def one_step(self, X, ra):
        Y = super().one_step(X, ra)
        return Y * float("inf") if ra > 4e4 else Y


def test_a_diverging_request_is_reported_and_the_others_finish():
    lib = type("lib", (), dict(Propagator=_Diverging, restrict=fake.restrict, prolong=fake.prolong,
                               parareal_correct=fake.parareal_correct, l2_diff=fake.l2_diff))
    eng = engine(lib=lib)
    reqs = [initial(eng, r) for r in requests(5, seed=11)]
    reqs[2].Ra = 5e4
    eng.run(reqs, deadline=60)
    assert reqs[2].status == rbc.RBC_EDIVERGED and reqs[2].k_done == 0
    base = engine()
    ok = [initial(base, r) for r in requests(5, seed=11)]
    del ok[2]
    base.run(ok, deadline=60)
    for a, b in zip([r for i, r in enumerate(reqs) if i != 2], ok):
        assert b.status == rbc.RBC_OK and torch.equal(a.U, b.U)
