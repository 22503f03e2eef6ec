"""Sec. 2.2 diagnostics and the statistical Parareal driver on the GPU.

* rbc_diagnostics against the oracle's diagnostics (padded-grid products and
  x-means there, Clenshaw-Curtis in z) on random states of several grids;
  the same bits for every batch size and for both handle precisions (the
  transforms run in FP64); B = 0 and bad arguments.
* StatisticalParareal on the library against oracle.parareal with the
  statistical criterion; with the fixed count it reproduces the library's own
  parareal_iterate bit for bit (chunked fine sweeps take the same steps).
"""
import numpy as np
import pytest

from layout import from_abi, max_rel_diff, to_abi
from oracle import statistics as ost
from oracle.parareal import parareal
from oracle.rbc import RBC, prolong, restrict
from paper_2001_01609_gb300.inputs import initial_temperature

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::DeprecationWarning")]


@pytest.fixture(scope="module")
def rbc():
    from paper_2001_01609_gb300 import build
    build.build()
    from paper_2001_01609_gb300 import rbc as r
    r.load()
    assert torch.cuda.is_available()
    return r


def random_states(o, B, seed):
    g = np.random.default_rng(seed)
    out = []
    for b in range(B):
        X = o.from_grid(initial_temperature(o.Nx, o.Nz, seed=seed + b, amplitude=0.4),
                        0.3 * g.standard_normal((o.Nz, o.Nx)), 0.3 * g.standard_normal((o.Nz, o.Nx)))
        out.append(X)
    return out


def oracle_row(o, X):
    d = o.diagnostics(X)
    return np.concatenate([[d["KE2"], d["eps"], d["wT"]], d["nu"], d["Tm"], d["Tv"]])


@pytest.mark.parametrize("Nx,Nz", [(32, 16), (64, 20), (16, 36), (128, 64)])
def test_diagnostics_match_oracle(rbc, Nx, Nz):
    o = RBC(2e5, 0.9, 2.0, Nx, Nz, 1e-3)
    Xs = random_states(o, 3, seed=Nx + Nz)
    F = rbc.Propagator(2e5, 0.9, 2.0, Nx, Nz, 1e-3)
    st = F.new_states(len(Xs))
    for b, X in enumerate(Xs):
        st[b].copy_(torch.from_numpy(to_abi(X)))
    out = F.diagnostics(st)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    Mz = 3 * Nz // 2
    assert got.shape == (3, 6 + 2 * Mz) and F.diag_size == 6 + 2 * Mz
    for b, X in enumerate(Xs):
        ref = oracle_row(o, X)
        for q in range(3):
            assert abs(got[b, q] - ref[q]) < 1e-11 * abs(ref[q]), (b, q)
        np.testing.assert_allclose(got[b, 3:6], ref[3:6], rtol=0, atol=1e-11 * max(1.0, np.abs(ref[3:6]).max()))
        np.testing.assert_allclose(got[b, 6:6 + Mz], ref[6:6 + Mz], rtol=0, atol=1e-13)
        np.testing.assert_allclose(got[b, 6 + Mz:], ref[6 + Mz:], rtol=1e-11, atol=1e-15)
    # one state at a time and the mixed-precision handle: the same bits
    Fm = rbc.Propagator(2e5, 0.9, 2.0, Nx, Nz, 1e-3, precision=rbc.RBC_MIXED)
    outm = Fm.diagnostics(st)
    for b in range(len(Xs)):
        assert torch.equal(F.diagnostics(st[b:b + 1])[0], out[b])
    assert torch.equal(outm, out)


def test_diagnostics_conduction_and_arguments(rbc):
    F = rbc.Propagator(1e6, 1.0, 2.0, 32, 16, 1e-3)
    st = F.new_states(2)
    T = 0.5 - (-0.5 * np.cos(np.pi * np.arange(16) / 15))[:, None] * np.ones((1, 32))
    F.set_state(st[0], T)
    F.set_state(st[1], T)
    d = F.diagnostics(st).cpu().numpy()
    assert np.abs(d[:, :3]).max() < 1e-28
    np.testing.assert_allclose(d[:, 3:6], 1.0, atol=1e-12)
    empty = F.new_states(0)
    out = torch.zeros((0, F.diag_size), dtype=torch.float64, device="cuda")
    F.diagnostics(empty, out=out)
    with pytest.raises(rbc.RBCError):
        rbc._check(rbc.load().rbc_diagnostics(F.h, None, 1, None, None))


def small_problem(N=3, nf=6, nc=3, every=4):
    Ra = 3e4
    fo = RBC(Ra, 1.0, 2.0, 16, 16, 2e-3)
    co = RBC(Ra, 1.0, 2.0, 8, 8, 4e-3)
    X0 = fo.from_grid(initial_temperature(16, 16, seed=0, amplitude=0.3))
    zp = fo.padded_z()

    def oF(X):
        return ost.run_sampled(fo, X, nf, every)

    def oG(X):
        return prolong(co.run(restrict(X, 8, 8), nc)[0], 16, 16)

    def diff(a, b):
        return fo.l2_T(a - b) / fo.l2_T(a)

    def summarize(Is):
        return ost.averages(ost.combine(Is), Ra, 1.0, zp, 16)

    return Ra, X0, N * nf * fo.dt, oF, oG, diff, summarize


@pytest.mark.parametrize("criterion,tol", [("stat", 0.05), ("fixed", 0.0)])
def test_statistical_parareal_matches_oracle(rbc, criterion, tol):
    from paper_2001_01609_gb300 import statistics as pst
    N = 3
    Ra, X0, t1, oF, oG, diff, summarize = small_problem(N)
    F = rbc.Propagator(Ra, 1.0, 2.0, 16, 16, 2e-3)
    G = rbc.Propagator(Ra, 1.0, 2.0, 8, 8, 4e-3)
    P = pst.StatisticalParareal(F, G, 0.0, t1, N, every=4, tol=tol, window_first=1, criterion=criterion)
    U0 = F.new_states(1)
    U0[0].copy_(torch.from_numpy(to_abi(X0)))
    U = F.new_states(N + 1)
    res = P.iterate(U0[0], U, 3)
    ref = parareal(X0, N, oF, oG, 3, diff, nu_window=(1, None), criterion=criterion, tol=tol,
                   summarize=summarize, change=ost.stat_change)
    assert res["k"] == ref["k"] and res["status"] == rbc.RBC_OK
    for n in range(N + 1):
        assert max_rel_diff(from_abi(U[n].cpu().numpy()), ref["U"][n]) < 1e-11, n
    np.testing.assert_allclose(res["defects"], ref["defects"], rtol=1e-8)
    for a, b in zip(res["stats"], ref["nus"]):
        for q in pst.STAT_QUANTITIES + ("Nu_int", "balance"):
            assert abs(a[q] - b[q]) <= 1e-10 * abs(b[q]), q


def test_statistical_parareal_fixed_equals_library_parareal(rbc):
    from paper_2001_01609_gb300 import statistics as pst
    N, nf, nc = 4, 10, 5
    F = rbc.Propagator(5e4, 1.0, 2.0, 32, 16, 1e-3)
    G = rbc.Propagator(5e4, 1.0, 2.0, 16, 8, 2e-3)
    t1 = N * nf * 1e-3
    U0 = F.new_states(1)
    F.set_state(U0[0], initial_temperature(32, 16, seed=5, amplitude=0.3))
    U = F.new_states(N + 1)
    res = pst.StatisticalParareal(F, G, 0.0, t1, N, every=3, criterion="fixed").iterate(U0[0], U, 2)
    Ulib = F.new_states(N + 1)
    st, k, de, _ = rbc.Parareal(F, G, 0.0, t1, N).iterate(U0[0], Ulib, 2)
    assert st == rbc.RBC_OK and k == 2 and res["k"] == 2
    assert torch.equal(U, Ulib)
    np.testing.assert_allclose(res["defects"], de, rtol=1e-14)
