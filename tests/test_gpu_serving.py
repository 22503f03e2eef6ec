"""Serving path on the GPU: per-state Rayleigh numbers, the Parareal building
blocks of the C ABI, and the continuous-batching engine.

* rbc_step_batch_ra against the FP64 oracle run at each state's Ra.
* rbc_restrict / rbc_prolong / rbc_parareal_correct / rbc_l2_diff against the
  oracle's truncation, zero-padding and L2 norm (Eq. 20, Sec. 3.6-3.7).
* A request served alone reproduces the library's own parareal_iterate
  bitwise; every request served in a mix (several grids, precisions, Ra and
  slice counts, chunked fine batches, memory-limited admission) reproduces its
  solo result bitwise.
"""
import numpy as np
import pytest

from layout import from_abi, max_rel_diff, to_abi
from oracle.rbc import RBC, prolong as o_prolong, restrict as o_restrict
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


def test_per_state_rayleigh_matches_oracle(rbc):
    Nx, Nz, dt, steps = 32, 18, 1e-4, 5
    ras = [1e4, 5e4, 2e5]
    F = rbc.Propagator(1.0, 1.0, 2.0, Nx, Nz, dt)      # the handle's own Ra is not used
    st = F.new_states(len(ras))
    X0 = []
    for b, Ra in enumerate(ras):
        o = RBC(Ra, 1.0, 2.0, Nx, Nz, dt)
        X = o.from_grid(initial_temperature(Nx, Nz, seed=b, amplitude=0.3))
        X0.append(X)
        put(st, b, X)
    F.step_batch(st, steps, ra=ras)
    torch.cuda.synchronize()
    for b, Ra in enumerate(ras):
        o = RBC(Ra, 1.0, 2.0, Nx, Nz, dt)
        ref, _ = o.run(X0[b], steps)
        assert max_rel_diff(get(st, b), ref) < 1e-11, Ra
        # same arithmetic as a handle created with that Ra
        H = rbc.Propagator(Ra, 1.0, 2.0, Nx, Nz, dt)
        one = H.new_states(1)
        put(one, 0, X0[b])
        H.step_batch(one, steps)
        assert torch.equal(one[0], st[b])
    with pytest.raises(rbc.RBCError):
        F.step_batch(st, 1, ra=[1e4, -1.0, 1e4])


def test_parareal_building_blocks_match_oracle(rbc):
    Nf, Zf, Nc, Zc = 32, 18, 16, 10
    F = rbc.Propagator(1e4, 1.0, 2.0, Nf, Zf, 1e-3)
    G = rbc.Propagator(1e4, 1.0, 2.0, Nc, Zc, 2e-3)
    fo = RBC(1e4, 1.0, 2.0, Nf, Zf, 1e-3)
    B = 3
    g = np.random.default_rng(5)
    fine = F.new_states(B)
    Xf = []
    for b in range(B):
        X = fo.from_grid(initial_temperature(Nf, Zf, seed=10 + b, amplitude=0.5), g.standard_normal((Zf, Nf)),
                         g.standard_normal((Zf, Nf)))
        Xf.append(X)
        put(fine, b, X)
    coarse = G.new_states(B)
    rbc.restrict(F, G, fine, coarse)
    back = F.new_states(B)
    rbc.prolong(F, G, coarse, back)
    torch.cuda.synchronize()
    for b in range(B):
        rc = o_restrict(Xf[b], Nc, Zc)
        np.testing.assert_array_equal(to_abi(rc), coarse[b].cpu().numpy())
        np.testing.assert_array_equal(to_abi(o_prolong(rc, Nf, Zf)), back[b].cpu().numpy())
    # U = F + (prolong(Gnew) - prolong(Gold)), in that order, elementwise
    Gn, Go = G.new_states(B), G.new_states(B)
    Gn.copy_(torch.randn_like(Gn))
    Go.copy_(torch.randn_like(Go))
    U = F.new_states(B)
    rbc.parareal_correct(F, G, fine, Gn, Go, U)
    Pn, Po = F.new_states(B), F.new_states(B)
    rbc.prolong(F, G, Gn, Pn)
    rbc.prolong(F, G, Go, Po)
    torch.cuda.synchronize()
    expect = fine.cpu().numpy() + (Pn.cpu().numpy() - Po.cpu().numpy())
    np.testing.assert_array_equal(U.cpu().numpy(), expect)
    # squared L2 norms of T and of T differences
    out = torch.zeros(B, dtype=torch.float64, device="cuda")
    rbc.l2_diff(F, fine, None, out)
    out2 = torch.zeros(B, dtype=torch.float64, device="cuda")
    rbc.l2_diff(F, fine, back, out2)
    torch.cuda.synchronize()
    for b in range(B):
        np.testing.assert_allclose(out[b].item(), fo.l2_T(Xf[b]) ** 2, rtol=1e-12)
        d = fo.l2_T(Xf[b] - o_prolong(o_restrict(Xf[b], Nc, Zc), Nf, Zf)) ** 2
        np.testing.assert_allclose(out2[b].item(), d, rtol=1e-10, atol=1e-14)
    with pytest.raises(rbc.RBCError):
        rbc.restrict(G, F, coarse, fine)                 # "coarse" finer than "fine"


def small_classes(Nx, Nz, precision):
    from paper_2001_01609_gb300.serving import ClassConfig
    return ClassConfig(Nx, Nz, precision, 2.5e-4, 5e-4, 20, 10, Nx // 2, Nz // 2)


def make_u0(rbc, eng, req, amp=0.3):
    cls = eng._class(req.key)
    u = cls.fine.new_states(1)
    cls.fine.set_state(u[0], initial_temperature(req.Nx, req.Nz, seed=req.seed, amplitude=amp))
    req.U0 = u[0]
    return req


def test_serving_single_request_equals_library_parareal(rbc):
    from paper_2001_01609_gb300 import serving
    eng = serving.Engine(max_iters=3, f_chunk=20, class_config=small_classes, keep_states=True)
    req = serving.Request(rid=0, Ra=3e4, Nx=64, Nz=32, nslices=6, seed=3)
    make_u0(rbc, eng, req)
    eng.run([req], deadline=120)
    assert req.status == rbc.RBC_OK and req.k_done == 3
    cfg = eng.config_for(req.key)
    F = rbc.Propagator(req.Ra, 1.0, 2.0, 64, 32, cfg.dt_fine)
    G = rbc.Propagator(req.Ra, 1.0, 2.0, 32, 16, cfg.dt_coarse)
    t0, t1 = eng.interval(req)
    P = rbc.Parareal(F, G, t0, t1, req.nslices)
    U = F.new_states(req.nslices + 1)
    st, k, d, nus = P.iterate(req.U0, U, 3)
    assert st == rbc.RBC_OK and k == 3
    assert torch.equal(U, req.U)
    np.testing.assert_array_equal(np.array(req.defects), d)
    np.testing.assert_array_equal(np.array(req.nus), nus)
    eng.close()


def mix(serving):
    """Requests over two grids and both precisions, with arrivals close together."""
    reqs = []
    spec = [(64, 32, 0, 3e4, 6), (32, 16, 1, 1e4, 4), (64, 32, 1, 5e4, 5), (32, 16, 0, 2e4, 7),
            (64, 32, 0, 4e4, 3), (32, 16, 0, 5e3, 5), (64, 32, 1, 2e4, 8)]
    for i, (Nx, Nz, prec, Ra, N) in enumerate(spec):
        reqs.append(serving.Request(rid=i, Ra=Ra, Nx=Nx, Nz=Nz, nslices=N, precision=prec,
                                    arrival=0.0 if i < 4 else 0.001 * i, seed=20 + i))
    return reqs


@pytest.mark.parametrize("limited", [False, True])
def test_serving_mix_equals_solo_bitwise(rbc, limited):
    from paper_2001_01609_gb300 import serving
    kw = dict(max_iters=3, f_chunk=7, class_config=small_classes, keep_states=True)
    solo_eng = serving.Engine(**kw)
    solo = mix(serving)
    for r in solo:
        make_u0(rbc, solo_eng, r)
        r.arrival = 0.0
        solo_eng.run([r], deadline=120)
        assert r.status == rbc.RBC_OK and r.k_done == min(3, r.nslices)
    eng = serving.Engine(**kw)
    reqs = mix(serving)
    for r in reqs:
        make_u0(rbc, eng, r)
    if limited:
        # room for the class buffers plus the two largest requests at a time
        need = sorted(eng.request_bytes(r) for r in reqs)
        eng.mem_limit = eng.committed + need[-1] + need[-2]
    eng.run(reqs, deadline=300)
    if limited:
        assert eng.peak_committed <= eng.mem_limit
        assert eng.peak_active < len(reqs)
    else:
        assert eng.peak_active >= 3                        # requests really shared the batches
    for a, b in zip(solo, reqs):
        assert b.status == a.status and b.k_done == a.k_done
        assert torch.equal(a.U, b.U), a.rid
        assert a.defects == b.defects and a.nus == b.nus, a.rid
    st = serving.latency_stats(reqs)
    assert 0 < st["p50_s"] <= st["p99_s"]
    eng.close()
    solo_eng.close()
