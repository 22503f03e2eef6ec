"""Host side of the Sec. 2.2 statistics and the statistical Parareal driver.

* The product's time means, ratios and boundary-layer count equal the
  oracle's (oracle/statistics.py, written separately) on the same integrals.
* StatisticalParareal, run on the oracle behind the propagator interface
  (tests/oracle_backend.py), reproduces oracle.parareal with the statistical
  criterion: the same iterates U^k (bit for bit), defects, time statistics,
  iteration count and status.
"""
import numpy as np
import pytest
import torch

import oracle_backend as ob
from oracle import statistics as ost
from oracle.parareal import parareal
from oracle.rbc import RBC, prolong, restrict
from paper_2001_01609_gb300 import rbc
from paper_2001_01609_gb300 import statistics as pst
from paper_2001_01609_gb300.inputs import initial_temperature

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def to_oracle_integrals(row, Mz, duration):
    return dict(sqrtKE2=row[0], eps=row[1], wT=row[2], NuV=row[3], Nub=row[4], Nut=row[5],
                Tm=row[6:6 + Mz], T2=row[6 + Mz:6 + 2 * Mz], T=duration)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_averages_match_the_oracle(seed):
    g = np.random.default_rng(seed)
    Nz, Ra, Pr = 24, 3e5, 0.8
    Mz = 3 * Nz // 2
    B, D = 3, 0.7
    I = np.zeros((B, 6 + 2 * Mz))
    I[:, 0] = g.uniform(1, 50, B)
    I[:, 1] = -g.uniform(1e3, 5e3, B)
    I[:, 2] = g.uniform(0.01, 0.05, B)
    I[:, 3:6] = g.uniform(2.0, 2.2, (B, 3))
    I[:, 6:6 + Mz] = g.uniform(0.2, 0.3, (B, Mz))
    I[:, 6 + Mz:] = I[:, 6:6 + Mz] ** 2 / (D / B) + g.uniform(1e-4, 1e-2, (B, Mz))
    p = pst.averages(I, D, Ra, Pr, Nz)
    o = ost.averages(ost.combine([to_oracle_integrals(r, Mz, D / B) for r in I]), Ra, Pr,
                     RBC(Ra, Pr, 2.0, 16, Nz, 1e-3).padded_z(), Nz)
    for q in ("U", "Re", "NuV", "Nub", "Nut", "Nu_int", "P", "eps_U", "balance", "delta_t", "duration"):
        assert abs(p[q] - o[q]) <= 1e-13 * abs(o[q]), q
    np.testing.assert_allclose(p["Trms"], o["Trms"], rtol=1e-10)
    assert p["delta_T"] == o["delta_T"] and p["N_BL"] == o["N_BL"]


def test_sample_values_layout():
    Mz = 6
    d = np.arange(2 * (6 + 2 * Mz), dtype=float).reshape(2, -1) + 1.0
    v = pst.sample_values(d, Mz)
    np.testing.assert_array_equal(v[:, 0], np.sqrt(d[:, 0]))
    np.testing.assert_array_equal(v[:, 1:6 + Mz], d[:, 1:6 + Mz])
    np.testing.assert_array_equal(v[:, 6 + Mz:], d[:, 6 + Mz:] + d[:, 6:6 + Mz] ** 2)


def setup(N=3, nf=6, nc=3, every=4):
    Ra = 3e4
    F = ob.OracleProp(Ra, 1.0, 2.0, 16, 16, 2e-3)
    G = ob.OracleProp(Ra, 1.0, 2.0, 8, 8, 4e-3)
    U0 = F.new_states(1)
    F.set_state(U0[0], initial_temperature(16, 16, seed=0, amplitude=0.3))
    t1 = N * nf * F.dt

    def oF(X):
        return ost.run_sampled(F.o, X, nf, every)

    def oG(X):
        return prolong(G.o.run(restrict(X, 8, 8), nc)[0], 16, 16)

    def diff(a, b):
        return F.o.l2_T(a - b) / F.o.l2_T(a)

    zp = F.o.padded_z()

    def summarize(Is):
        return ost.averages(ost.combine(Is), Ra, 1.0, zp, 16)

    return F, G, U0, t1, oF, oG, diff, summarize


@pytest.mark.parametrize("criterion,tol,max_iters", [("fixed", 0.0, 3), ("stat", 0.05, 3), ("stat", 1e-12, 2)])
def test_driver_reproduces_the_oracle_iteration(criterion, tol, max_iters):
    from layout import from_abi, to_abi
    N = 3
    F, G, U0, t1, oF, oG, diff, summarize = setup(N)
    P = pst.StatisticalParareal(F, G, 0.0, t1, N, every=4, tol=tol, window_first=1, criterion=criterion, lib=ob)
    U = F.new_states(N + 1)
    res = P.iterate(U0[0], U, max_iters)
    ref = parareal(from_abi(U0[0].numpy()), N, oF, oG, max_iters, diff, nu_window=(1, None),
                   criterion=criterion, tol=tol, summarize=summarize, change=ost.stat_change)
    assert res["k"] == ref["k"]
    for n in range(N + 1):
        np.testing.assert_array_equal(U[n].numpy(), to_abi(ref["U"][n]))
    np.testing.assert_allclose(res["defects"], ref["defects"], rtol=1e-13)
    for a, b in zip(res["stats"], ref["nus"]):
        for q in pst.STAT_QUANTITIES + ("Nu_int", "balance"):
            assert abs(a[q] - b[q]) <= 1e-12 * abs(b[q]), q
        assert a["N_BL"] == b["N_BL"]
    if criterion == "fixed":
        assert res["status"] == rbc.RBC_OK
    elif tol == 0.05:
        assert res["k"] == 2 and res["status"] == rbc.RBC_OK
    else:
        assert res["status"] == rbc.RBC_ENOTCONVERGED


def test_driver_checks_its_arguments():
    F, G, U0, t1, *_ = setup()
    with pytest.raises(ValueError):
        pst.StatisticalParareal(F, G, 0.0, t1, 3, every=0, lib=ob)
    with pytest.raises(ValueError):
        pst.StatisticalParareal(F, G, 0.0, t1, 3, every=2, window_first=3, lib=ob)
    with pytest.raises(ValueError):
        pst.StatisticalParareal(F, G, 0.0, t1 * 1.001, 3, every=2, lib=ob)
    with pytest.raises(ValueError):
        pst.StatisticalParareal(F, G, 0.0, t1, 3, every=2, criterion="nu", lib=ob)


def test_sampled_run_partial_last_chunk():
    F, *_ = setup()
    X = F.new_states(2)
    F.set_state(X[0], initial_temperature(16, 16, seed=1, amplitude=0.3))
    F.set_state(X[1], initial_temperature(16, 16, seed=2, amplitude=0.3))
    from layout import from_abi
    refs = [ost.run_sampled(F.o, from_abi(X[b].numpy()), 7, 3)[1] for b in range(2)]
    I = pst.sampled_run(F, X, 7, 3)
    Mz = F.o.Mz
    for b in range(2):
        np.testing.assert_allclose(I[b, :6], [refs[b][q] for q in ost.SCALARS], rtol=1e-13)
        np.testing.assert_allclose(I[b, 6:6 + Mz], refs[b]["Tm"], rtol=1e-13, atol=1e-18)
        np.testing.assert_allclose(I[b, 6 + Mz:], refs[b]["T2"], rtol=1e-13)


def test_single_slice_is_exact_after_one_iteration():
    """N = 1: the first fine sweep starts from U0 itself, so U_1^1 is the serial fine
    state and the statistics are those of the one fine trajectory."""
    from layout import from_abi, to_abi
    F, G, U0, _, oF, *_ = setup(N=1)
    t1 = 6 * F.dt
    P = pst.StatisticalParareal(F, G, 0.0, t1, 1, every=4, lib=ob, criterion="fixed")
    U = F.new_states(2)
    res = P.iterate(U0[0], U, 5)
    assert res["k"] == 1 and res["status"] == rbc.RBC_OK and P.window_first == 0
    Xend, I = oF(from_abi(U0[0].numpy()))
    np.testing.assert_array_equal(U[1].numpy(), to_abi(Xend))
    ref = ost.averages(I, F.Ra, F.Pr, F.o.padded_z(), F.Nz)
    for q in pst.STAT_QUANTITIES:
        assert abs(res["stats"][0][q] - ref[q]) <= 1e-13 * abs(ref[q]), q


def test_sampling_interval_longer_than_a_slice():
    """every > steps per slice: one trapezoid over each slice's end points."""
    F, *_ = setup()
    X = F.new_states(1)
    F.set_state(X[0], initial_temperature(16, 16, seed=3, amplitude=0.3))
    from layout import from_abi
    ref = ost.run_sampled(F.o, from_abi(X[0].numpy()), 5, 5)[1]
    I = pst.sampled_run(F, X, 5, 50)
    np.testing.assert_allclose(I[0, :6], [ref[q] for q in ost.SCALARS], rtol=1e-13)


def test_statistical_rule_runs_out_at_the_slice_count():
    """With an unreachable tolerance the rule is not met; iterations stop at k = N."""
    F, G, U0, t1, *_ = setup(N=2)
    P = pst.StatisticalParareal(F, G, 0.0, 2 * 6 * F.dt, 2, every=3, tol=0.0, lib=ob)
    U = F.new_states(3)
    res = P.iterate(U0[0], U, 10)
    assert res["k"] == 2 and res["status"] == rbc.RBC_ENOTCONVERGED and len(res["stats"]) == 2
