"""Sec. 2.2 diagnostics and the statistical Parareal driver on the GPU.

* rbc_diagnostics against the oracle's diagnostics (padded-grid products and
  x-means there, Clenshaw-Curtis in z) on random states of several grids;
  the same bits for every batch size and for both handle precisions (the
  transforms run in FP64); B = 0 and bad arguments.
* rbc_step_batch_sampled (the sampled time integrals of Sec. 2.2) against the
  oracle's sampled run.
* parareal_iterate with sampling and RBC_CRIT_STAT against oracle.parareal with
  the statistical criterion; sampling changes no iterate.
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


def oracle_rows(I, Mz):
    """The oracle's integrals in rbc_step_batch_sampled's column order."""
    return np.concatenate([[I[q] for q in ost.SCALARS], I["Tm"], I["T2"]])


@pytest.mark.parametrize("nsteps,every", [(7, 3), (5, 50), (6, 1)])
def test_sampled_run_matches_oracle(rbc, nsteps, every):
    """rbc_step_batch_sampled: states and trapezoid integrals of the sampled
    averages (a partial last interval, an interval longer than the run, every
    step) against the oracle's sampled run, state by state."""
    Nx, Nz, Ra = 16, 16, 3e4
    o = RBC(Ra, 1.0, 2.0, Nx, Nz, 2e-3)
    F = rbc.Propagator(Ra, 1.0, 2.0, Nx, Nz, 2e-3)
    Xs = [o.from_grid(initial_temperature(Nx, Nz, seed=s, amplitude=0.3)) for s in (1, 2)]
    st = F.new_states(2)
    for b, X in enumerate(Xs):
        st[b].copy_(torch.from_numpy(to_abi(X)))
    nu = torch.zeros(2, dtype=torch.float64, device="cuda")
    stat = F.step_batch_sampled(st, nsteps, every, nu=nu)
    torch.cuda.synchronize()
    got = stat.cpu().numpy()
    Mz = 3 * Nz // 2
    for b, X in enumerate(Xs):
        Xend, I = ost.run_sampled(o, X, nsteps, every)
        assert max_rel_diff(from_abi(st[b].cpu().numpy()), Xend) < 1e-12
        ref = oracle_rows(I, Mz)
        np.testing.assert_allclose(got[b], ref, rtol=1e-11, atol=1e-15 * np.abs(ref).max())
        _, integ = o.run(X, nsteps)
        assert abs(nu[b].item() - integ) <= 1e-11 * abs(integ)
    with pytest.raises(rbc.RBCError):
        F.step_batch_sampled(st, 3, 0)


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


@pytest.mark.parametrize("criterion,tol,max_iters,depth", [("stat", 0.05, 3, 2), ("fixed", 0.0, 3, 0),
                                                           ("stat", 1e-12, 2, 1)])
def test_statistical_parareal_matches_oracle(rbc, criterion, tol, max_iters, depth):
    """parareal_iterate with the sampled statistics and RBC_CRIT_STAT against
    oracle.parareal with the statistical rule: the same iteration count and
    status, iterates, defects and window statistics."""
    N = 3
    Ra, X0, t1, oF, oG, diff, summarize = small_problem(N)
    F = rbc.Propagator(Ra, 1.0, 2.0, 16, 16, 2e-3)
    G = rbc.Propagator(Ra, 1.0, 2.0, 8, 8, 4e-3)
    crit = rbc.CRIT_STAT if criterion == "stat" else rbc.CRIT_FIXED
    P = rbc.Parareal(F, G, 0.0, t1, N, crit, tol)
    P.set_sampling(4, window_first=1)
    P.set_depth(depth)
    U0 = F.new_states(1)
    U0[0].copy_(torch.from_numpy(to_abi(X0)))
    U = F.new_states(N + 1)
    st, k, defects, nus = P.iterate(U0[0], U, max_iters)
    ref = parareal(X0, N, oF, oG, max_iters, diff, nu_window=(1, None), criterion=criterion, tol=tol,
                   summarize=summarize, change=ost.stat_change)
    assert k == ref["k"]
    if criterion == "stat" and tol < 1e-6:
        assert st == rbc.RBC_ENOTCONVERGED
    else:
        assert st == rbc.RBC_OK
    for n in range(N + 1):
        assert max_rel_diff(from_abi(U[n].cpu().numpy()), ref["U"][n]) < 1e-11, n
    np.testing.assert_allclose(defects, ref["defects"], rtol=1e-8)
    got = rbc.stat_summary(16, Ra, 1.0, P.stat_means())
    last = ref["nus"][-1]
    for q in ("NuV", "Nub", "Nut", "Re", "P", "eps_U", "Nu_int", "balance", "delta_t"):
        assert abs(got[q] - last[q]) <= 1e-10 * abs(last[q]), q
    assert got["N_BL"] == last["N_BL"] and got["delta_T"] == pytest.approx(last["delta_T"], abs=1e-14)
    # T_rms^2 = <T^2> - <T>^2 cancels at the walls (T fixed there): compare the squares
    np.testing.assert_allclose(got["Trms"] ** 2, last["Trms"] ** 2, rtol=1e-8, atol=1e-13)


def test_sampled_parareal_iterates_equal_the_unsampled_ones(rbc):
    """Sampling the statistics changes no state: the iterates equal
    parareal_iterate's without sampling bit for bit (the Nu integrals are
    summed per sampling interval, so only their last bits may differ)."""
    N, nf, nc = 4, 10, 5
    F = rbc.Propagator(5e4, 1.0, 2.0, 32, 16, 1e-3)
    G = rbc.Propagator(5e4, 1.0, 2.0, 16, 8, 2e-3)
    t1 = N * nf * 1e-3
    U0 = F.new_states(1)
    F.set_state(U0[0], initial_temperature(32, 16, seed=5, amplitude=0.3))
    U = F.new_states(N + 1)
    P = rbc.Parareal(F, G, 0.0, t1, N)
    P.set_sampling(3)
    st, k, de, nus = P.iterate(U0[0], U, 2)
    Ulib = F.new_states(N + 1)
    st2, k2, de2, nus2 = rbc.Parareal(F, G, 0.0, t1, N).iterate(U0[0], Ulib, 2)
    assert st == st2 == rbc.RBC_OK and k == k2 == 2
    assert torch.equal(U, Ulib)
    np.testing.assert_array_equal(de, de2)
    np.testing.assert_allclose(nus, nus2, rtol=1e-13)
    with pytest.raises(rbc.RBCError):
        rbc.Parareal(F, G, 0.0, t1, N, rbc.CRIT_STAT, 0.01).set_sampling(0)
