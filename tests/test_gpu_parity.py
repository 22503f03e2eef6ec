"""Parity of the CUDA propagator and Parareal (through the C ABI) with the FP64 oracle.

Tolerance: 1e-10 relative for FP64 runs (the all-FP64 target); a few steps on
small grids are held to 1e-11.  Max-norm over all spectral coefficients,
relative to the largest coefficient.
"""
import numpy as np
import pytest

from layout import from_abi, max_rel_diff, to_abi
from oracle.parareal import parareal as oracle_parareal
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


def put(states, b, X):
    states[b].copy_(torch.from_numpy(to_abi(X)))


def get(states, b):
    return from_abi(states[b].cpu().numpy())


def developed_state(o, seed, amp=0.3, steps=3):
    """A nonlinear state: strong seeded perturbation, a few oracle steps."""
    X = o.from_grid(initial_temperature(o.Nx, o.Nz, seed=seed, amplitude=amp, Lx=o.Lx))
    for _ in range(steps):
        X, _ = o.step(X)
    return X


@pytest.mark.parametrize("Nx,Nz", [(64, 32), (16, 10), (8, 18)])
def test_set_state_matches_oracle_transform(rbc, Nx, Nz):
    o = RBC(1e4, 1.0, 2.0, Nx, Nz, 1e-3)
    F = rbc.Propagator(1e4, 1.0, 2.0, Nx, Nz, 1e-3)
    Tg = initial_temperature(Nx, Nz, seed=4, amplitude=0.2)
    g = np.random.default_rng(1)
    ug, wg = g.standard_normal((Nz, Nx)), g.standard_normal((Nz, Nx))
    st = F.new_states(1)
    F.set_state(st[0], Tg, ug, wg)
    ref = o.from_grid(Tg, ug, wg)
    assert max_rel_diff(get(st, 0), ref) < 1e-12
    T2, u2, w2 = F.get_state(st[0])
    To, uo, wo = o.to_grid(ref)
    for a, b in ((T2, To), (u2, uo), (w2, wo)):
        assert np.abs(a - b).max() < 1e-11 * max(1.0, np.abs(b).max())


@pytest.mark.parametrize("Nx,Nz,Ra", [(16, 18, 1e5), (32, 16, 3e4), (8, 10, 2e5), (64, 32, 1e6)])
def test_few_steps_match_oracle(rbc, Nx, Nz, Ra):
    dt = 2e-4
    o = RBC(Ra, 1.0, 2.0, Nx, Nz, dt)
    X0 = developed_state(o, seed=Nx + Nz)
    F = rbc.Propagator(Ra, 1.0, 2.0, Nx, Nz, dt)
    st = F.new_states(1)
    put(st, 0, X0)
    nu = torch.zeros(1, dtype=torch.float64, device="cuda")
    F.step_batch(st, 4, nu)
    assert F.check_diverged() == rbc.RBC_OK
    ref, integ = o.run(X0, 4)
    assert max_rel_diff(get(st, 0), ref) < 1e-11
    assert abs(nu.item() - integ) < 1e-11 * abs(integ)


@pytest.mark.parametrize("Nx,Nz,Ra,dt,steps", [(64, 128, 1e6, 2e-6, 2), (16, 256, 1e7, 2e-7, 2),
                                                 (256, 128, 1e8, 1.5625e-7, 2)])
def test_long_chebyshev_expansions_match_oracle(rbc, Nx, Nz, Ra, dt, steps):
    """Nz = 128 and 256: the band recurrences of the stage solve run over 64 and
    128 unknowns per parity, at wavenumbers up to pi (Nx/2 - 1)."""
    o = RBC(Ra, 1.0, 2.0, Nx, Nz, dt)
    X0 = developed_state(o, seed=Nz + 1, amp=0.3, steps=1)
    F = rbc.Propagator(Ra, 1.0, 2.0, Nx, Nz, dt)
    st = F.new_states(1)
    put(st, 0, X0)
    F.step_batch(st, steps)
    ref, _ = o.run(X0, steps)
    assert max_rel_diff(get(st, 0), ref) < 1e-10


def test_config0_single_slice_parity_over_1000_steps(rbc):
    """Ra = 1e4, 64 x 32, dt = 1e-3, seeded IC (seed 0): one slice of t in [0, 1]."""
    o = RBC(1e4, 1.0, 2.0, 64, 32, 1e-3)
    Tg = initial_temperature(64, 32, seed=0)
    F = rbc.Propagator(1e4, 1.0, 2.0, 64, 32, 1e-3)
    st = F.new_states(1)
    F.set_state(st[0], Tg)
    X0 = o.from_grid(Tg)
    assert max_rel_diff(get(st, 0), X0) < 1e-13
    nu = torch.zeros(1, dtype=torch.float64, device="cuda")
    F.step_batch(st, 1000, nu)
    ref, integ = o.run(X0, 1000)
    assert max_rel_diff(get(st, 0), ref) < 1e-10
    assert abs(nu.item() - integ) < 1e-10 * abs(integ)
    nv = F.nusselt(st[0])
    no = o.nusselt(ref)
    assert np.allclose(nv, no, rtol=1e-10, atol=0)


def test_batched_uneven_steps_equal_solo_runs_and_oracle(rbc):
    Nx, Nz, Ra, dt = 32, 18, 5e4, 5e-4
    o = RBC(Ra, 1.0, 2.0, Nx, Nz, dt)
    F = rbc.Propagator(Ra, 1.0, 2.0, Nx, Nz, dt)
    Xs = [developed_state(o, seed=s, steps=1) for s in range(4)]
    nsteps = [7, 0, 3, 5]
    st = F.new_states(4)
    for b, X in enumerate(Xs):
        put(st, b, X)
    nu = torch.zeros(4, dtype=torch.float64, device="cuda")
    F.step_batch(st, nsteps, nu)
    for b, X in enumerate(Xs):
        solo = F.new_states(1)
        put(solo, 0, X)
        nus = torch.zeros(1, dtype=torch.float64, device="cuda")
        F.step_batch(solo, nsteps[b], nus)
        assert torch.equal(solo[0], st[b])                 # batch-invariant, bitwise
        assert nus.item() == nu[b].item()
        ref, integ = o.run(X, nsteps[b])
        assert max_rel_diff(get(st, b), ref) < 1e-11
        assert abs(nu[b].item() - integ) <= 1e-11 * max(abs(integ), 1e-30)
    assert torch.equal(st[1].cpu(), torch.from_numpy(to_abi(Xs[1])))   # 0 steps: untouched


@pytest.mark.parametrize("precision,Nx,Nz,B", [(0, 32, 16, 160), (1, 32, 16, 160), (1, 64, 64, 40), (2, 64, 64, 40)])
def test_small_and_large_batch_kernel_shapes_give_identical_bits(rbc, precision, Nx, Nz, B):
    """A batch of 160 states takes the large-batch launch shapes (one row kernel
    block per row, 16-mode solve tiles, 32-mode z-forward tiles); one state
    alone takes the small-batch shapes (a cluster of five CTAs per row,
    single-mode tiles).  The arithmetic is the same, so are the bits (with the
    tensor-core transforms of the mixed mode too, at 64 x 64)."""
    steps = 3
    F = rbc.Propagator(2e4, 1.0, 2.0, Nx, Nz, 2e-4, precision)
    st = F.new_states(B)
    for b in range(B):
        F.set_state(st[b], initial_temperature(Nx, Nz, seed=100 + b, amplitude=0.3))
    picks = (0, B // 2 - 3, B - 1)
    solo = [st[b:b + 1].clone() for b in picks]
    nu = torch.zeros(B, dtype=torch.float64, device="cuda")
    F.step_batch(st, steps, nu)
    for s1, b in zip(solo, picks):
        nu1 = torch.zeros(1, dtype=torch.float64, device="cuda")
        F.step_batch(s1, steps, nu1)
        assert torch.equal(s1[0], st[b]), b
        assert torch.equal(nu1[0], nu[b]), b


def test_eager_launches_equal_graph_loop(rbc):
    """rbc_opts.eager (every kernel launched from the host) gives the bits of
    the device-side step loop, alone and inside Parareal."""
    Ra, Nf, Zf, Nc, Zc, dtf, dtc = 3e4, 32, 16, 16, 8, 2e-3, 4e-3
    N, nf = 4, 6
    out = []
    for eager in (False, True):
        F = rbc.Propagator(Ra, 1.0, 2.0, Nf, Zf, dtf, eager=eager)
        G = rbc.Propagator(Ra, 1.0, 2.0, Nc, Zc, dtc, eager=eager)
        u0 = F.new_states(1)
        F.set_state(u0[0], initial_temperature(Nf, Zf, seed=9, amplitude=0.3))
        st = u0.clone()
        F.step_batch(st, 7)
        U = F.new_states(N + 1)
        s, k, d, nus = rbc.Parareal(F, G, 0.0, N * nf * dtf, N).iterate(u0[0], U, 2)
        assert s == rbc.RBC_OK and k == 2
        out.append((st, U, d, nus))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    np.testing.assert_array_equal(out[0][2], out[1][2])
    np.testing.assert_array_equal(out[0][3], out[1][3])


def test_nusselt_and_l2_match_oracle(rbc):
    o = RBC(2e5, 1.0, 2.0, 32, 24, 1e-3)
    X = developed_state(o, seed=7, amp=0.5, steps=4)
    F = rbc.Propagator(2e5, 1.0, 2.0, 32, 24, 1e-3)
    st = F.new_states(1)
    put(st, 0, X)
    assert np.allclose(F.nusselt(st[0]), o.nusselt(X), rtol=1e-12, atol=1e-13)
    assert abs(F.l2_temperature(st[0]) - o.l2_T(X)) < 1e-12 * o.l2_T(X)


def test_conduction_state_stays_exact(rbc):
    # exact conduction coefficients (T = 1/2 - z, nothing else): at Ra = 1e8 any
    # roundoff in the m >= 1 modes would grow, so the state is set spectrally
    F = rbc.Propagator(1e8, 1.0, 2.0, 64, 32, 1e-4)
    st = F.new_states(1)
    st[0, 0, 0, 0, 0] = 0.5
    st[0, 0, 1, 0, 0] = -0.5
    before = st.clone()
    F.step_batch(st, 20)
    assert (st - before).abs().max().item() < 1e-14
    nv, nb, nt = F.nusselt(st[0])
    assert abs(nv - 1) < 1e-13 and abs(nb - 1) < 1e-12 and abs(nt - 1) < 1e-12


def test_config1_full_size_batched_launch_sampled_slices(rbc):
    """Ra = 1e6, 256 x 64, 32 slices in one launch; slices 0 and 31 checked."""
    Nx, Nz, Ra, dt = 256, 64, 1e6, 2e-4
    o = RBC(Ra, 1.0, 2.0, Nx, Nz, dt)
    F = rbc.Propagator(Ra, 1.0, 2.0, Nx, Nz, dt)
    B = 32
    st = F.new_states(B)
    for b in range(B):
        F.set_state(st[b], initial_temperature(Nx, Nz, seed=100 + b, amplitude=0.3))
    X0 = {b: get(st, b) for b in (0, B - 1)}
    F.step_batch(st, 3)
    assert F.check_diverged() == rbc.RBC_OK
    for b, X in X0.items():
        ref, _ = o.run(X, 3)
        assert max_rel_diff(get(st, b), ref) < 1e-10


def test_nonfinite_state_is_reported(rbc):
    F = rbc.Propagator(1e4, 1.0, 2.0, 16, 16, 1e-3)
    st = F.new_states(2)
    F.set_state(st[0], initial_temperature(16, 16, seed=0))
    F.set_state(st[1], initial_temperature(16, 16, seed=1))
    st[1, 0, 3, 2, 0] = float("nan")
    F.step_batch(st, 2)
    assert F.check_diverged() == rbc.RBC_EDIVERGED
    assert torch.isfinite(st[0]).all()
    F.step_batch(st[:1], 1)
    assert F.check_diverged() == rbc.RBC_OK


def test_empty_batch_and_zero_steps(rbc):
    F = rbc.Propagator(1e4, 1.0, 2.0, 16, 16, 1e-3)
    st = F.new_states(2)
    F.set_state(st[0], initial_temperature(16, 16, seed=0))
    before = st.clone()
    F.step_batch(st[:0], 3)
    F.step_batch(st, [0, 0])
    assert torch.equal(st, before)


def parareal_case():
    Ra, Nf, Zf, Nc, Zc = 3e4, 32, 16, 16, 8
    dtf, dtc, N, T = 2e-3, 4e-3, 4, 0.064
    return Ra, Nf, Zf, Nc, Zc, dtf, dtc, N, T


def test_parareal_matches_oracle_and_is_exact_on_first_k_slices(rbc):
    Ra, Nf, Zf, Nc, Zc, dtf, dtc, N, T = parareal_case()
    fo, co = RBC(Ra, 1.0, 2.0, Nf, Zf, dtf), RBC(Ra, 1.0, 2.0, Nc, Zc, dtc)
    nf, nc = int(round(T / N / dtf)), int(round(T / N / dtc))
    U0 = fo.from_grid(initial_temperature(Nf, Zf, seed=0, amplitude=0.3))
    K = 3
    ores = oracle_parareal(U0, N, lambda U: fo.run(U, nf), lambda U: prolong(co.run(restrict(U, Nc, Zc), nc)[0], Nf, Zf),
                           K, lambda a, b: fo.l2_T(a - b) / fo.l2_T(a), nu_window=(N // 2, T / 2))
    F = rbc.Propagator(Ra, 1.0, 2.0, Nf, Zf, dtf)
    G = rbc.Propagator(Ra, 1.0, 2.0, Nc, Zc, dtc)
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
    # exactness: U_n^K equals the GPU serial fine solution bitwise for n <= K
    ser = F.new_states(1)
    put(ser, 0, U0)
    for n in range(1, K + 1):
        F.step_batch(ser, nf)
        assert torch.equal(ser[0], U[n]), n


def test_parareal_stopping_criteria(rbc):
    Ra, Nf, Zf, Nc, Zc, dtf, dtc, N, T = parareal_case()
    F = rbc.Propagator(Ra, 1.0, 2.0, Nf, Zf, dtf)
    G = rbc.Propagator(Ra, 1.0, 2.0, Nc, Zc, dtc)
    u0 = F.new_states(1)
    F.set_state(u0[0], initial_temperature(Nf, Zf, seed=0, amplitude=0.3))
    U = F.new_states(N + 1)
    st, k, d, nus = rbc.Parareal(F, G, 0.0, T, N).iterate(u0[0], U, 4)
    tol = d[1] * 1.0001
    expect = 1 + min(i for i in range(len(d)) if d[i] <= tol)
    Pd = rbc.Parareal(F, G, 0.0, T, N, rbc.CRIT_DEFECT, tol)
    st2, k2, d2, _ = Pd.iterate(u0[0], U, 4)
    assert st2 == rbc.RBC_OK and k2 == expect
    np.testing.assert_array_equal(d2, d[:k2])          # deterministic rerun
    Pn = rbc.Parareal(F, G, 0.0, T, N, rbc.CRIT_NU, 1e-30)
    st3, k3, _, _ = Pn.iterate(u0[0], U, 2)
    assert st3 == rbc.RBC_ENOTCONVERGED and k3 == 2
    with pytest.raises(rbc.RBCError):
        rbc.Parareal(F, G, 0.0, T * 1.0001, N)          # not a whole number of steps


@pytest.mark.parametrize("precision", [0, 1])
def test_parareal_schedule_does_not_change_results(rbc, precision):
    """The overlap of the coarse, fine and correction sweeps (fine groups of
    1, 2, 4 or all slices, growing groups, one or two fine streams, coarse
    priority on or off) changes timing only: iterates, defects and Nu agree
    bit for bit; after nslices iterations U is the serial fine solution."""
    Ra, Nf, Zf, Nc, Zc, dtf, dtc = 3e4, 32, 16, 16, 8, 2e-3, 4e-3
    N, nf = 6, 8
    T = N * nf * dtf
    F = rbc.Propagator(Ra, 1.0, 2.0, Nf, Zf, dtf, precision)
    G = rbc.Propagator(Ra, 1.0, 2.0, Nc, Zc, dtc, precision)
    u0 = F.new_states(1)
    F.set_state(u0[0], initial_temperature(Nf, Zf, seed=2, amplitude=0.3))
    out = []
    for sched in ((N, N, 1, 0, 0), (1, 1, 1, 0, 0), (2, 2, 2, 1, 0), (4, 1, 2, 0, 0), (4, 2, 1, 1, 0),
                  (2, 1, 2, 1, 40)):
        P = rbc.Parareal(F, G, 0.0, T, N)
        P.set_schedule(*sched)
        assert (P.coarse_sms > 0) == (sched[4] > 0)
        U = F.new_states(N + 1)
        st, k, d, nus = P.iterate(u0[0], U, 3)
        assert st == rbc.RBC_OK and k == 3
        out.append((U, d, nus))
    for U, d, nus in out[1:]:
        assert torch.equal(U, out[0][0])
        np.testing.assert_array_equal(d, out[0][1])
        np.testing.assert_array_equal(nus, out[0][2])
    # iterations enqueued ahead of the one being evaluated: timing only
    for depth in (0, 1, 3, 6):
        P = rbc.Parareal(F, G, 0.0, T, N)
        P.set_depth(depth)
        U = F.new_states(N + 1)
        st, k, d, nus = P.iterate(u0[0], U, 3)
        assert st == rbc.RBC_OK and k == 3
        assert torch.equal(U, out[0][0])
        np.testing.assert_array_equal(d, out[0][1])
        np.testing.assert_array_equal(nus, out[0][2])
    # a criterion met while later iterations run ahead: they are stopped and
    # dropped, the result is iterate k, and the next call starts clean
    d3 = out[0][1]
    tol = d3[1] * 1.0001
    expect = 1 + min(i for i in range(len(d3)) if d3[i] <= tol)
    Pd = rbc.Parareal(F, G, 0.0, T, N, rbc.CRIT_DEFECT, tol)
    Pd.set_depth(3)
    Ud = F.new_states(N + 1)
    P2 = rbc.Parareal(F, G, 0.0, T, N)
    U2 = F.new_states(N + 1)
    P2.iterate(u0[0], U2, expect)
    for _ in range(2):
        st, k, d, _ = Pd.iterate(u0[0], Ud, N)
        assert st == rbc.RBC_OK and k == expect
        assert torch.equal(Ud, U2)
    with pytest.raises(rbc.RBCError):
        Pd.set_depth(7)
    # more iterations than slices: stops at k = N with the serial fine solution
    P = rbc.Parareal(F, G, 0.0, T, N)
    U = F.new_states(N + 1)
    st, k, d, _ = P.iterate(u0[0], U, N + 2)
    assert st == rbc.RBC_OK and k == N
    ser = F.new_states(1)
    ser.copy_(u0[0:1])
    for n in range(1, N + 1):
        F.step_batch(ser, nf)
        assert torch.equal(ser[0], U[n]), n
    for bad in ((0, 1, 1, 0, 0), (2, 3, 1, 0, 0), (2, 1, 5, 0, 0), (2, 1, 1, 2, 0), (2, 1, 1, 0, -1)):
        with pytest.raises(rbc.RBCError):
            P.set_schedule(*bad)


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("Nx,Nz,Ra", [(64, 32, 1e5), (32, 18, 2e5), (64, 64, 3e5), (256, 64, 1e6)])
def test_mixed_precision_few_steps_within_stated_tolerance(rbc, Nx, Nz, Ra, precision):
    """RBC_MIXED: FP32 transforms and products, FP64 solves and RK combination
    (the z transforms on tensor cores from Nz = 64, on CUDA cores below).
    RBC_MIXED_BF16: the same with BF16 instead of TF32 hi/lo operands in the
    tensor-core transforms (about 16 bits of each operand).

    Stated tolerance: 1e-5 relative to the largest coefficient after 4 steps
    (FP32 rounding of the explicit terms, ~1e-7, enters the state through
    dt * F and is not amplified over a few steps).
    """
    dt = 1e-4 if Ra < 1e6 else 1e-5
    o = RBC(Ra, 1.0, 2.0, Nx, Nz, dt)
    X0 = developed_state(o, seed=Nx + 7)
    F = rbc.Propagator(Ra, 1.0, 2.0, Nx, Nz, dt, precision=precision)
    st = F.new_states(1)
    put(st, 0, X0)
    nu = torch.zeros(1, dtype=torch.float64, device="cuda")
    F.step_batch(st, 4, nu)
    assert F.check_diverged() == rbc.RBC_OK
    ref, integ = o.run(X0, 4)
    err = max_rel_diff(get(st, 0), ref)
    print(f"precision {precision} {Nx}x{Nz} Ra={Ra:g}: state rel err {err:.3e}, Nu integral rel err "
          f"{abs(nu.item() - integ) / abs(integ):.3e}")
    assert err < 1e-5
    assert abs(nu.item() - integ) < 1e-5 * abs(integ)
    # the FP64 path on the same input is much closer
    F64 = rbc.Propagator(Ra, 1.0, 2.0, Nx, Nz, dt)
    st64 = F64.new_states(1)
    put(st64, 0, X0)
    F64.step_batch(st64, 4)
    assert max_rel_diff(get(st64, 0), ref) < 1e-11 < err


@pytest.mark.parametrize("precision,Nx,Nz,B", [(0, 64, 32, 5), (1, 64, 64, 12), (2, 64, 64, 12), (0, 128, 32, 1)])
def test_autotuned_shapes_give_identical_bits(rbc, precision, Nx, Nz, B):
    """rbc_autotune only picks launch shapes: a handle with the tuned shapes gives
    the bits of one with the heuristics."""
    F = rbc.Propagator(2e4, 1.0, 2.0, Nx, Nz, 2e-4, precision)
    T = rbc.Propagator(2e4, 1.0, 2.0, Nx, Nz, 2e-4, precision)
    t_heur, t_best = T.autotune(B)
    assert 0 < t_best <= t_heur
    shapes = T.tuned_shapes(B)
    assert len(shapes) == 6
    a, b = F.new_states(B), T.new_states(B)
    for i in range(B):
        F.set_state(a[i], initial_temperature(Nx, Nz, seed=40 + i, amplitude=0.3))
    b.copy_(a)
    na = torch.zeros(B, dtype=torch.float64, device="cuda")
    nb = torch.zeros(B, dtype=torch.float64, device="cuda")
    F.step_batch(a, 4, na)
    T.step_batch(b, 4, nb)
    assert torch.equal(a, b) and torch.equal(na, nb)
    assert F.check_diverged() == T.check_diverged() == rbc.RBC_OK


@pytest.mark.parametrize("precision,Nx,Nz,B", [(0, 32, 16, 6), (1, 64, 64, 3), (2, 128, 64, 2), (1, 256, 64, 4)])
def test_pinned_launch_shapes_give_identical_bits(rbc, precision, Nx, Nz, B):
    """rbc_set_shapes: every valid combination of the row kernel's form, block
    size and shared-memory layout (full or lean), the solve tile and the
    z-forward tile gives the bits of the heuristics; invalid shapes are refused."""
    ref = rbc.Propagator(2e4, 1.0, 2.0, Nx, Nz, 2e-4, precision)
    a = ref.new_states(B)
    for i in range(B):
        ref.set_state(a[i], initial_temperature(Nx, Nz, seed=70 + i, amplitude=0.3))
    start = a.clone()
    na = torch.zeros(B, dtype=torch.float64, device="cuda")
    ref.step_batch(a, 3, na)
    cases = [(0, 0, 0, 0, 0, 0), (0, 0, 0, 0, 0, 1), (0, 0, 0, 0, 1024, 1), (0, 0, 0, 1, 0, -1),
             (1, 4, 1, 0, 512, 0), (16, 32, 8, 0, 256, 1), (2, 8, 2, -1, 0, -1)]
    for sh in cases:
        T = rbc.Propagator(2e4, 1.0, 2.0, Nx, Nz, 2e-4, precision)
        T.set_shapes(B, sh)
        assert T.tuned_shapes(B) == sh
        b = start.clone()
        nb = torch.zeros(B, dtype=torch.float64, device="cuda")
        T.step_batch(b, 3, nb)
        assert torch.equal(a, b) and torch.equal(na, nb), sh
        T.close()
    for bad in ((3, 0, 0, 0, 0, 0), (0, 0, 0, 2, 0, 0), (0, 0, 0, 0, 300, 0), (0, 0, 0, 0, 0, 2)):
        with pytest.raises(rbc.RBCError):
            ref.set_shapes(B, bad)
