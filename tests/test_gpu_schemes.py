"""Lower-order coarse steppers (Sec. 3.6) on the GPU: ARS(2,2,2) and ARS(1,1,1)
against the oracle's same schemes, through the C ABI.

Tolerances as for RK443: 1e-11 relative (max norm over all coefficients) for a
few FP64 steps on small grids, 1e-10 for Parareal, the stated 1e-5 for the
mixed mode.  A one-stage scheme writes the new state into the step-start
buffer inside the stage that reads it, so its batch-shape and eager-launch
invariances are checked bit for bit as well.
"""
import numpy as np
import pytest

from layout import from_abi, max_rel_diff, to_abi
from oracle.parareal import parareal as oracle_parareal
from oracle.rbc import RBC, prolong, restrict
from paper_2001_01609_gb300.inputs import initial_temperature

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::DeprecationWarning")]

NAMES = {1: "RK222", 2: "RK111"}


@pytest.fixture(scope="module")
def rbc():
    from paper_2001_01609_gb300 import build
    build.build()
    from paper_2001_01609_gb300 import rbc as r
    r.load()
    assert torch.cuda.is_available()
    return r


def put(states, b, X):
    states[b].copy_(torch.from_numpy(to_abi(X)))


def get(states, b):
    return from_abi(states[b].cpu().numpy())


def developed(o, seed):
    X = o.from_grid(initial_temperature(o.Nx, o.Nz, seed=seed, amplitude=0.3, Lx=o.Lx))
    for _ in range(3):
        X, _ = o.step(X)
    return X


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("Nx,Nz,Ra,dt", [(16, 18, 1e5, 1e-4), (64, 32, 1e6, 2e-5), (32, 64, 3e5, 2e-5)])
def test_few_steps_match_oracle(rbc, scheme, Nx, Nz, Ra, dt):
    o = RBC(Ra, 1.0, 2.0, Nx, Nz, dt, scheme=NAMES[scheme])
    X0 = developed(o, seed=Nx + Nz + scheme)
    F = rbc.Propagator(Ra, 1.0, 2.0, Nx, Nz, dt, scheme=scheme)
    st = F.new_states(1)
    put(st, 0, X0)
    nu = torch.zeros(1, dtype=torch.float64, device="cuda")
    F.step_batch(st, 5, nu)
    assert F.check_diverged() == rbc.RBC_OK
    ref, integ = o.run(X0, 5)
    assert max_rel_diff(get(st, 0), ref) < 1e-11
    assert abs(nu.item() - integ) < 1e-11 * abs(integ)


@pytest.mark.parametrize("scheme", [1, 2])
def test_mixed_precision_within_stated_tolerance(rbc, scheme):
    Nx, Nz, Ra, dt = 256, 64, 1e6, 1e-5
    o = RBC(Ra, 1.0, 2.0, Nx, Nz, dt, scheme=NAMES[scheme])
    X0 = developed(o, seed=5)
    F = rbc.Propagator(Ra, 1.0, 2.0, Nx, Nz, dt, precision=rbc.RBC_MIXED, scheme=scheme)
    st = F.new_states(1)
    put(st, 0, X0)
    F.step_batch(st, 4)
    assert F.check_diverged() == rbc.RBC_OK
    ref, _ = o.run(X0, 4)
    assert max_rel_diff(get(st, 0), ref) < 1e-5


@pytest.mark.parametrize("scheme", [1, 2])
def test_batch_shapes_and_eager_launches_give_identical_bits(rbc, scheme):
    Nx, Nz, B, steps = 32, 16, 160, 3
    F = rbc.Propagator(2e4, 1.0, 2.0, Nx, Nz, 2e-4, scheme=scheme)
    E = rbc.Propagator(2e4, 1.0, 2.0, Nx, Nz, 2e-4, scheme=scheme, eager=True)
    st = F.new_states(B)
    for b in range(B):
        F.set_state(st[b], initial_temperature(Nx, Nz, seed=300 + b, amplitude=0.3))
    picks = (0, B // 2 - 3, B - 1)
    solo = [st[b:b + 1].clone() for b in picks]
    eager = [st[b:b + 1].clone() for b in picks]
    nu = torch.zeros(B, dtype=torch.float64, device="cuda")
    F.step_batch(st, steps, nu)
    for s1, e1, b in zip(solo, eager, picks):
        nu1 = torch.zeros(1, dtype=torch.float64, device="cuda")
        F.step_batch(s1, steps, nu1)
        assert torch.equal(s1[0], st[b]), b
        assert torch.equal(nu1[0], nu[b]), b
        E.step_batch(e1, steps)
        assert torch.equal(e1[0], st[b]), b


def test_rk443_default_is_unchanged(rbc):
    F = rbc.Propagator(2e4, 1.0, 2.0, 32, 16, 2e-4)
    G = rbc.Propagator(2e4, 1.0, 2.0, 32, 16, 2e-4, scheme=rbc.RBC_RK443)
    a, b = F.new_states(1), G.new_states(1)
    F.set_state(a[0], initial_temperature(32, 16, seed=4, amplitude=0.3))
    b.copy_(a)
    F.step_batch(a, 4)
    G.step_batch(b, 4)
    assert torch.equal(a, b)
    with pytest.raises(rbc.RBCError):
        rbc.Propagator(2e4, 1.0, 2.0, 32, 16, 2e-4, scheme=3)


@pytest.mark.parametrize("scheme", [1, 2])
def test_parareal_with_lower_order_coarse_matches_oracle(rbc, scheme):
    """F: RK443 on the fine grid; G: the lower-order scheme on the coarse grid."""
    Ra, Nf, Zf, Nc, Zc = 3e4, 32, 16, 16, 8
    dtf, dtc, N, T = 2e-3, 2e-3, 4, 0.064
    fo = RBC(Ra, 1.0, 2.0, Nf, Zf, dtf)
    co = RBC(Ra, 1.0, 2.0, Nc, Zc, dtc, scheme=NAMES[scheme])
    nf, nc = int(round(T / N / dtf)), int(round(T / N / dtc))
    U0 = fo.from_grid(initial_temperature(Nf, Zf, seed=0, amplitude=0.3))
    K = 3
    ores = oracle_parareal(U0, N, lambda U: fo.run(U, nf), lambda U: prolong(co.run(restrict(U, Nc, Zc), nc)[0], Nf, Zf),
                           K, lambda a, b: fo.l2_T(a - b) / fo.l2_T(a), nu_window=(N // 2, T / 2))
    F = rbc.Propagator(Ra, 1.0, 2.0, Nf, Zf, dtf)
    G = rbc.Propagator(Ra, 1.0, 2.0, Nc, Zc, dtc, scheme=scheme)
    P = rbc.Parareal(F, G, 0.0, T, N)
    u0 = F.new_states(1)
    put(u0, 0, U0)
    U = F.new_states(N + 1)
    st, k, defects, nus = P.iterate(u0[0], U, K)
    assert st == rbc.RBC_OK and k == K
    for n in range(N + 1):
        assert max_rel_diff(get(U, n), ores["U"][n]) < 1e-10
    np.testing.assert_allclose(defects, ores["defects"], rtol=1e-8)
    np.testing.assert_allclose(nus, ores["nus"], rtol=1e-10)
