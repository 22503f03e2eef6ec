"""Fixed-flux walls (Eq. 7) on the GPU against the FP64 oracle.

* a few steps from a developed state match the oracle's fixed-flux scheme,
  on grids that take the dense small-system solve and the banded recurrence;
* the linear conduction profile stays exact, with Nu_b = Nu_t = 1;
* mixed precision stays within its stated tolerance;
* handles of different boundary conditions cannot be combined in Parareal.
"""
import numpy as np
import pytest

from layout import from_abi, max_rel_diff, to_abi
from oracle.rbc import RBC
from paper_2001_01609_gb300.inputs import initial_temperature

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::DeprecationWarning")]
FF = "fixed_flux"


@pytest.fixture(scope="module")
def rbc():
    from paper_2001_01609_gb300 import build
    build.build()
    from paper_2001_01609_gb300 import rbc as r
    r.load()
    assert torch.cuda.is_available()
    return r


def developed(o, seed, amp=0.3, steps=3):
    X = o.from_grid(initial_temperature(o.Nx, o.Nz, seed=seed, amplitude=amp, Lx=o.Lx))
    for _ in range(steps):
        X, _ = o.step(X)
    return X


@pytest.mark.parametrize("Nx,Nz,Ra", [(32, 16, 3e4), (64, 48, 2e5), (16, 10, 1e5)])
def test_fixed_flux_steps_match_oracle(rbc, Nx, Nz, Ra):
    dt = 2e-4
    o = RBC(Ra, 1.0, 2.0, Nx, Nz, dt, bc=FF)
    X0 = developed(o, seed=Nx + Nz)
    F = rbc.Propagator(Ra, 1.0, 2.0, Nx, Nz, dt, bc=rbc.RBC_FIXED_FLUX)
    st = F.new_states(1)
    st[0].copy_(torch.from_numpy(to_abi(X0)))
    nu = torch.zeros(1, dtype=torch.float64, device="cuda")
    F.step_batch(st, 4, nu)
    assert F.check_diverged() == rbc.RBC_OK
    ref, integ = o.run(X0, 4)
    assert max_rel_diff(from_abi(st[0].cpu().numpy()), ref) < 1e-11
    assert abs(nu.item() - integ) < 1e-11 * abs(integ)
    nb, nt = F.nusselt(st[0])[1:]
    assert abs(nb - 1.0) < 1e-11 and abs(nt - 1.0) < 1e-11
    # the fixed-temperature scheme gives another state from the same input
    G = rbc.Propagator(Ra, 1.0, 2.0, Nx, Nz, dt)
    s2 = G.new_states(1)
    s2[0].copy_(torch.from_numpy(to_abi(X0)))
    G.step_batch(s2, 4)
    assert max_rel_diff(from_abi(s2[0].cpu().numpy()), ref) > 1e-6


def test_fixed_flux_conduction_state_stays_exact(rbc):
    F = rbc.Propagator(1e5, 1.0, 2.0, 32, 16, 1e-3, bc=rbc.RBC_FIXED_FLUX)
    st = F.new_states(1)
    z = -0.5 * np.cos(np.pi * np.arange(16) / 15)
    F.set_state(st[0], (0.5 - z)[:, None] * np.ones((1, 32)))
    before = st.clone()
    F.step_batch(st, 10)
    assert (st - before).abs().max().item() < 1e-12
    np.testing.assert_allclose(F.nusselt(st[0]), 1.0, atol=1e-12)


def test_fixed_flux_mixed_precision_within_tolerance(rbc):
    Nx, Nz, Ra, dt = 64, 32, 1e5, 1e-4
    o = RBC(Ra, 1.0, 2.0, Nx, Nz, dt, bc=FF)
    X0 = developed(o, seed=9)
    F = rbc.Propagator(Ra, 1.0, 2.0, Nx, Nz, dt, precision=rbc.RBC_MIXED, bc=rbc.RBC_FIXED_FLUX)
    st = F.new_states(1)
    st[0].copy_(torch.from_numpy(to_abi(X0)))
    F.step_batch(st, 4)
    ref, _ = o.run(X0, 4)
    assert max_rel_diff(from_abi(st[0].cpu().numpy()), ref) < 1e-5


def test_boundary_conditions_must_match(rbc):
    F = rbc.Propagator(1e4, 1.0, 2.0, 32, 16, 1e-3, bc=rbc.RBC_FIXED_FLUX)
    G = rbc.Propagator(1e4, 1.0, 2.0, 16, 8, 2e-3)
    with pytest.raises(rbc.RBCError):
        rbc.Parareal(F, G, 0.0, 0.04, 4)
    a, b = F.new_states(1), G.new_states(1)
    with pytest.raises(rbc.RBCError):
        rbc.restrict(F, G, a, b)
    with pytest.raises(rbc.RBCError):
        rbc.Propagator(1e4, 1.0, 2.0, 32, 16, 1e-3, bc=2)
