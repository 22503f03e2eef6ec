"""Pins of the oracle's Sec. 2.2 diagnostics and time statistics.

D1 conduction state, D2 a polynomial state whose averages follow by exact
polynomial algebra, D3 the kinetic-energy budget d<|u|^2>/dt = 2 Pr (P + <u.lap u>)
along the oracle's own dynamics (ties the signs and factors of P and eps to
Eq. 3), D4 <u.lap u>_V = -<omega^2>_V (integration by parts, no-slip walls)
against the exact Chebyshev Gram matrix, D5 plane mean and variance of T by
brute force, D6 Nu_int and the P / eps_U balance of Eqs. 13-15 on steady rolls,
D7 the trapezoid time integrals against the closed-form decay of pure
diffusion, D8 the boundary-layer point count, D9 statistical Parareal at
k = N equals the serial fine statistics bitwise.
"""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as C
from numpy.polynomial import polynomial as Pn

from oracle import statistics as st
from oracle.parareal import parareal
from oracle.rbc import RBC, prolong, restrict
from oracle import ultraspherical as us
from paper_2001_01609_gb300.inputs import initial_temperature
from test_oracle_pins import conduction, cos_pi_z, implicit_stability

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def cheb(p, N):
    cc = C.poly2cheb(p.coef)
    c = np.zeros(N, dtype=cc.dtype)
    c[: len(cc)] = cc
    return c


def polynomial_state(r, A=0.3, B=0.2, Cc=0.1, D=0.05):
    """psi = A sin(k x) g(s), U = B (1 - s^2), T = T0(s) + Cc cos(k x) h(s), k = k_1.

    Returns the state and its averages from exact polynomial integration
    (d/dz = 2 d/ds, <f>_V = (1/2) int_{-1}^{1} <f>_x ds)."""
    N = r.Nz
    g = Pn.Polynomial([1, 0, -2, 0, 1])                      # (1 - s^2)^2: psi = psi' = 0 at the walls
    U = B * Pn.Polynomial([1, 0, -1])
    h = Pn.Polynomial([1, 0, -1])
    T0 = Pn.Polynomial([0.5 + D, -0.5, -D])                 # T0(-1) = 1, T0(1) = 0
    X = r.zero_state()
    X.psi[1] = -0.5j * A * cheb(g, N)                          # sin(kx) = (e^{ikx} - e^{-ikx}) / 2i
    X.U = cheb(U, N)
    X.T[0] = cheb(T0, N)
    X.T[1] = 0.5 * Cc * cheb(h, N)
    k = r.k[1]
    g1, g2, g3 = g.deriv(1), g.deriv(2), g.deriv(3)
    vol = lambda p: 0.5 * (p.integ()(1.0) - p.integ()(-1.0))
    # u = 2 A sin(kx) g' + U, w = -A k cos(kx) g; lap u = A sin(kx)(8 g''' - 2 k^2 g') + 4 U'',
    # lap w = -A k cos(kx)(4 g'' - k^2 g); x-means of sin^2 and cos^2 are 1/2
    KE2 = vol(2 * A ** 2 * g1 ** 2 + U ** 2 + 0.5 * A ** 2 * k ** 2 * g ** 2)
    eps = vol(A ** 2 * g1 * (8 * g3 - 2 * k ** 2 * g1) + 4 * U * U.deriv(2)
              + 0.5 * A ** 2 * k ** 2 * g * (4 * g2 - k ** 2 * g))
    wT = vol(-0.5 * A * k * Cc * g * h)
    nu = (1.0 + wT, -2.0 * T0.deriv(1)(-1.0), -2.0 * T0.deriv(1)(1.0))
    return X, dict(KE2=KE2, eps=eps, wT=wT, nu=nu, T0=T0, Tv=lambda s: 0.5 * Cc ** 2 * h(s) ** 2)


def test_D1_conduction_state():
    r = RBC(1e6, 1.0, 2.0, 16, 16, 1e-3)
    d = r.diagnostics(conduction(r))
    assert d["KE2"] == 0.0 and d["eps"] == 0.0 and d["wT"] == 0.0
    np.testing.assert_allclose(d["nu"], 1.0, atol=1e-13)
    np.testing.assert_allclose(d["Tm"], 0.5 - r.padded_z(), atol=1e-15)
    assert np.abs(d["Tv"]).max() < 1e-30


@pytest.mark.parametrize("Nx,Nz", [(8, 16), (12, 10)])
def test_D2_polynomial_state_closed_form(Nx, Nz):
    r = RBC(3e4, 1.0, 2.0, Nx, Nz, 1e-3)
    X, ex = polynomial_state(r)
    d = r.diagnostics(X)
    for q in ("KE2", "eps", "wT"):
        assert abs(d[q] - ex[q]) < 1e-13 * max(1.0, abs(ex[q])), q
    np.testing.assert_allclose(d["nu"], ex["nu"], rtol=0, atol=1e-13)
    s = 2.0 * r.padded_z()
    np.testing.assert_allclose(d["Tm"], ex["T0"](s), atol=1e-15)
    np.testing.assert_allclose(d["Tv"], ex["Tv"](s), atol=1e-16)


def test_D3_kinetic_energy_budget_along_the_dynamics():
    """Dotting Eq. 3 (times Pr) with u: d<u^2 + w^2>_V/dt = 2 Pr (Ra <wT>_V + <u.lap u>_V);
    pressure and advection integrate to zero.  Checked during the growth of the
    first rolls (Ra = 1e4, Pr = 0.7), with a five-point difference in time."""
    energy_budget("fixed_T", 30)


def test_D3_kinetic_energy_budget_with_fixed_flux():
    """The same budget with fixed-flux walls (it does not involve the temperature
    boundary condition)."""
    energy_budget("fixed_flux", 28)


def energy_budget(bc, nsteps):
    Pr = 0.7
    r = RBC(1e4, Pr, 2.0, 16, 32, 5e-3, bc=bc)
    X = conduction(r)
    X.T[1] = 1e-3 * cos_pi_z(r.Nz)
    for _ in range(nsteps):
        X, _ = r.step(X)
    h = RBC(1e4, Pr, 2.0, 16, 32, 1e-5, bc=bc)
    Xs = [X]
    for _ in range(4):
        Xs.append(h.step(Xs[-1])[0])
    ke = [h.diagnostics(x)["KE2"] for x in Xs]
    d = h.diagnostics(Xs[2])
    rate = (ke[0] - 8 * ke[1] + 8 * ke[3] - ke[4]) / (12 * h.dt)
    P, eps = h.Ra * d["wT"], d["eps"]
    assert P > 1e3 and abs(P + eps) > 0.3 * P                  # a transient, far from balance
    assert abs(rate / (2 * Pr) - (P + eps)) < 1e-6 * P


def test_D4_viscous_term_is_minus_enstrophy():
    """<u.lap u>_V = -<omega^2>_V for fields vanishing at the walls; the right side
    from the exact Gram matrix of omega's coefficients, Parseval in x."""
    g = np.random.default_rng(3)
    r = RBC(1e5, 1.0, 2.0, 12, 16, 1e-3)
    X = r.zero_state()
    wall2 = Pn.Polynomial([1, 0, -2, 0, 1])
    for m in range(1, r.nm):
        q = Pn.Polynomial(g.standard_normal(4) + 1j * g.standard_normal(4))
        X.psi[m] = cheb(wall2 * q, r.Nz)
    X.U = cheb(Pn.Polynomial([1, 0, -1]) * Pn.Polynomial(g.standard_normal(3)), r.Nz)
    eps = r.diagnostics(X)["eps"]
    G = us.cheb_gram(r.Nz)
    ik = 1j * r.k[:, None]
    u = X.psi @ r.Dz.T
    u[0] = X.U
    w = -ik * X.psi
    w[0] = 0.0
    om = ik * w - u @ r.Dz.T
    ens = sum((1.0 if m == 0 else 2.0) * (om[m].conj() @ G @ om[m]).real for m in range(r.nm)) * 0.5
    assert abs(eps + ens) < 1e-12 * ens


def test_D5_plane_mean_and_variance_by_brute_force():
    r = RBC(1e5, 1.0, 2.0, 10, 12, 1e-3)
    g = np.random.default_rng(8)
    X = r.zero_state()
    X.T = g.standard_normal(X.T.shape) + 1j * g.standard_normal(X.T.shape)
    X.T[0] = X.T[0].real
    d = r.diagnostics(X)
    x = r.Lx * np.arange(64) / 64
    s = 2.0 * r.padded_z()
    Tg = np.zeros((len(s), len(x)))
    for m in range(r.nm):
        Tg += (1.0 if m == 0 else 2.0) * np.outer(C.chebval(s, X.T[m]), np.exp(1j * r.k[m] * x)).real
    np.testing.assert_allclose(d["Tm"], Tg.mean(axis=1), atol=1e-12)
    np.testing.assert_allclose(d["Tv"], Tg.var(axis=1), rtol=1e-12)


def test_D6_consistency_checks_on_steady_rolls():
    """Eq. 12 and Eq. 14 hold for a steady state: Nu_V = Nu_b = Nu_t and P = eps_U,
    up to the spatial error of the 16 x 16 grid."""
    r = RBC(1e4, 1.0, 2.0, 16, 16, 5e-3)
    X = conduction(r)
    X.T[1] = 1e-3 * cos_pi_z(r.Nz)
    X, _ = r.run(X, 500)
    X, I = st.run_sampled(r, X, 20, 5)
    a = st.averages(I, r.Ra, r.Pr, r.padded_z(), r.Nz)
    assert a["NuV"] > 2.0 and a["Re"] > 10.0
    assert a["Nu_int"] < 3e-3
    assert a["balance"] < 2e-4
    assert a["N_BL"] >= 1 and 0.0 < a["delta_T"] < 0.5


def test_D7_trapezoid_integrals_of_pure_diffusion():
    """Ra = 0: a temperature mode decays by R(dt lam) per step (P2), so the plane
    variance at step n is Tv_0 R^(2n); a mean flow decays by R(-dt Pr pi^2), so
    <U^2>^(1/2) is scaled by |R|^n.  Samples at steps 0, 3, 6, 9, 10."""
    r = RBC(0.0, 2.5, 2.0, 8, 32, 2e-3)
    X = conduction(r)
    X.T[1] = 1e-2 * cos_pi_z(r.Nz)
    rT = implicit_stability(r.dt * -(r.k[1] ** 2 + np.pi ** 2))
    Tv0 = r.diagnostics(X)["Tv"]
    _, I = st.run_sampled(r, X, 10, 3)
    steps = [0, 3, 6, 9, 10]
    exp = sum(0.5 * (b - a) * r.dt * Tv0 * (rT ** (2 * a) + rT ** (2 * b)) for a, b in zip(steps, steps[1:]))
    Tm0 = r.diagnostics(X)["Tm"]
    np.testing.assert_allclose(I["Tm"], 10 * r.dt * Tm0, rtol=1e-13, atol=1e-30)
    np.testing.assert_allclose(I["T2"] - 10 * r.dt * Tm0 ** 2, exp, rtol=1e-9, atol=2e-17)
    assert I["T"] == 10 * r.dt and I["sqrtKE2"] == 0.0
    Y = conduction(r)
    Y.U = 0.3 * cos_pi_z(r.Nz)
    rU = implicit_stability(r.dt * -(r.Pr * np.pi ** 2))
    k0 = np.sqrt(r.diagnostics(Y)["KE2"])
    _, J = st.run_sampled(r, Y, 10, 3)
    expU = sum(0.5 * (b - a) * r.dt * k0 * (abs(rU) ** a + abs(rU) ** b) for a, b in zip(steps, steps[1:]))
    assert abs(J["sqrtKE2"] - expU) < 1e-12 * expU


def test_D8_boundary_layer_points():
    r = RBC(1e6, 1.0, 2.0, 16, 32, 1e-3)
    zp = r.padded_z()
    zd = zp + 0.5
    prof = np.exp(-((zd - 0.061) / 0.03) ** 2) + np.exp(-((0.5 - zp - 0.07) / 0.03) ** 2)
    delta, nbl = st.boundary_layer(prof, zp, r.Nz)
    lower = zd[zp < 0]
    assert delta == lower[np.argmin(abs(lower - 0.061))]
    count = 0
    for j in range(1, r.Nz - 1):
        if 0.5 - 0.5 * np.cos(np.pi * j / (r.Nz - 1)) <= delta:
            count += 1
    assert nbl == count and 3 <= nbl <= 8
    assert st.boundary_layer(np.zeros(r.Mz), zp, r.Nz)[1] == 0


def stat_problem(N=3, nf=10, nc=5, every=5):
    fine = RBC(3e4, 1.0, 2.0, 16, 16, 2e-3)
    coarse = RBC(3e4, 1.0, 2.0, 8, 8, 4e-3)
    U0 = fine.from_grid(initial_temperature(16, 16, seed=0, amplitude=0.3))
    zp = fine.padded_z()

    def F(U):
        return st.run_sampled(fine, U, nf, every)

    def G(U):
        return prolong(coarse.run(restrict(U, 8, 8), nc)[0], 16, 16)

    def diff(a, b):
        return fine.l2_T(a - b) / fine.l2_T(a)

    def summarize(Is):
        return st.averages(st.combine(Is), fine.Ra, fine.Pr, zp, fine.Nz)

    return fine, U0, F, G, diff, summarize


def test_D9_statistical_parareal_at_k_equal_N_is_serial_fine():
    fine, U0, F, G, diff, summarize = stat_problem()
    N = 3
    res = parareal(U0, N, F, G, N, diff, nu_window=(1, None), summarize=summarize)
    serial, Is = U0, []
    for n in range(N):
        serial, I = F(serial)
        Is.append(I)
    ref = summarize(Is[1:])
    last = res["nus"][-1]
    for q in st.STAT_QUANTITIES + ("Nu_int", "balance", "N_BL"):
        assert last[q] == ref[q], q
    np.testing.assert_array_equal(last["Trms"], ref["Trms"])
    # the statistics move between iterations until the fine trajectories are exact
    assert st.stat_change(res["nus"][1], res["nus"][0]) > 0.0


def test_D9_statistical_criterion_stops_when_the_statistics_settle():
    fine, U0, F, G, diff, summarize = stat_problem()
    N = 3
    # G = F: U^0 is already the serial fine solution, so iterations 1 and 2 see the
    # same trajectories and the rule stops at k = 2 with no change
    res = parareal(U0, N, F, lambda U: F(U)[0], 3, diff, nu_window=(1, None), criterion="stat", tol=1e-12,
                   summarize=summarize, change=st.stat_change)
    assert res["k"] == 2 and st.stat_change(res["nus"][1], res["nus"][0]) == 0.0
    res = parareal(U0, N, F, G, 3, diff, nu_window=(1, None), criterion="stat", tol=1e-14,
                   summarize=summarize, change=st.stat_change)
    assert res["k"] == 3
