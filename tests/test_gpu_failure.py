"""Failure detection on the GPU without a fault: the bounded mbarrier waits of
the mixed-precision tensor-core kernels give up, the library reports
RBC_ETIMEOUT, leaves the states concerned as they were, and the context stays
usable.

The mixed mode runs its z transforms on the tensor cores on grids with at
least 64 Chebyshev coefficients, so the tests use 64 x 64.  The test lowers
the wait limit to 0 polls (rbc_set_wait_limit), so that every
such wait gives up at once: a wait that nothing will end, made to run out.  The
kernels then still drain the tensor-core work they issued (with the default
limit) before they free tensor memory, so nothing is left in flight.
"""
import numpy as np
import pytest

from paper_2001_01609_gb300.inputs import initial_temperature

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbc():
    from paper_2001_01609_gb300 import build
    build.build()
    from paper_2001_01609_gb300 import rbc as r
    r.load()
    assert torch.cuda.is_available()
    return r


class lowered_wait_limit:
    def __init__(self, rbc, polls):
        self.rbc, self.polls = rbc, polls

    def __enter__(self):
        torch.cuda.synchronize()
        self.rbc.set_wait_limit(self.polls)

    def __exit__(self, *exc):
        torch.cuda.synchronize()
        self.rbc.set_wait_limit(-1)


def mixed_states(rbc, Nx, Nz, B, seed0=30):
    F = rbc.Propagator(1e5, 1.0, 2.0, Nx, Nz, 1e-4, precision=rbc.RBC_MIXED)
    st = F.new_states(B)
    for b in range(B):
        F.set_state(st[b], initial_temperature(Nx, Nz, seed=seed0 + b, amplitude=0.3))
    return F, st


@pytest.mark.parametrize("eager", [False, True])
def test_wait_timeout_reports_etimeout_and_leaves_the_states_unchanged(rbc, eager):
    Nx, Nz = 64, 64
    F, st = mixed_states(rbc, Nx, Nz, 3)
    if eager:
        F = rbc.Propagator(1e5, 1.0, 2.0, Nx, Nz, 1e-4, precision=rbc.RBC_MIXED, eager=True)
    F.step_batch(st, 2)                       # a normal call first: graphs captured, workspace sized
    assert F.check_diverged() == rbc.RBC_OK
    before = st.clone()
    nu = torch.zeros(3, dtype=torch.float64, device="cuda")
    with lowered_wait_limit(rbc, 0):
        F.step_batch(st, [4, 1, 3], nu)
        assert F.check_diverged() == rbc.RBC_ETIMEOUT
        assert torch.equal(st, before)
        with pytest.raises(rbc.RBCError) as e:
            F.nusselt(st[0])
        assert e.value.status == rbc.RBC_ETIMEOUT
    # the states of the failed call stay flagged until the next call; the
    # context is usable
    assert F.check_diverged() == rbc.RBC_ETIMEOUT
    F.step_batch(st, 3)
    assert F.check_diverged() == rbc.RBC_OK
    G, ref = mixed_states(rbc, Nx, Nz, 3)
    G.step_batch(ref, 2)
    G.step_batch(ref, 3)
    assert torch.equal(st, ref)               # as if the failed call had not happened


def test_fp64_handles_have_no_bounded_waits(rbc):
    F = rbc.Propagator(1e5, 1.0, 2.0, 32, 16, 1e-4)
    st = F.new_states(1)
    F.set_state(st[0], initial_temperature(32, 16, seed=3, amplitude=0.3))
    with lowered_wait_limit(rbc, 0):
        F.step_batch(st, 2)
        assert F.check_diverged() == rbc.RBC_OK


def test_parareal_reports_a_wait_timeout(rbc):
    Fm = rbc.Propagator(1e5, 1.0, 2.0, 64, 64, 1e-4, precision=rbc.RBC_MIXED)
    Gm = rbc.Propagator(1e5, 1.0, 2.0, 32, 32, 2e-4, precision=rbc.RBC_MIXED)
    U0 = Fm.new_states(1)
    Fm.set_state(U0[0], initial_temperature(64, 64, seed=5, amplitude=0.3))
    U = Fm.new_states(5)
    P = rbc.Parareal(Fm, Gm, 0.0, 4 * 8e-4, 4)
    with lowered_wait_limit(rbc, 0):
        status, k, _, _ = P.iterate(U0, U, 2)
    assert status == rbc.RBC_ETIMEOUT
    status, k, defects, _ = P.iterate(U0, U, 2)
    assert status == rbc.RBC_OK and k == 2 and np.isfinite(defects).all()
