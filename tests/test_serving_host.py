"""Host-side logic of the serving engine (no GPU): the resolution rule that
assigns grids, the dt ladder, the request stream and the memory accounting."""
import math

import numpy as np
import pytest

pytest.importorskip("torch")
from paper_2001_01609_gb300 import rbc, serving  # noqa: E402


@pytest.mark.parametrize("Ra,ok,too_coarse", [(1e5, 32, 16), (1e6, 64, 32), (1e7, 64, 32)])
def test_boundary_layer_rule_reproduces_table1(Ra, ok, too_coarse):
    """Table 1 (N_BL >= 6 column): Ra = 1e5 needs Nz = 32, 1e6 and 1e7 need Nz = 64."""
    assert serving.boundary_layer_points(Ra, ok) >= serving.MIN_BL_POINTS
    assert serving.boundary_layer_points(Ra, too_coarse) < serving.MIN_BL_POINTS


def test_boundary_layer_points_brute_force():
    for Ra in (1e4, 3e6, 1e8):
        nu = serving.NU_FIT_A * Ra ** serving.NU_FIT_B
        delta = 1.0 / (2.0 * nu)
        for Nz in (16, 32, 64, 128, 256):
            z = [-0.5 * math.cos(math.pi * j / (Nz - 1)) for j in range(Nz)]
            cnt = sum(1 for zj in z[1:-1] if zj + 0.5 <= delta)
            assert serving.boundary_layer_points(Ra, Nz) == cnt


def test_adequate_grids_and_max_ra_are_consistent():
    for Nz in (32, 64, 128):
        r = serving.max_adequate_ra(Nz)
        assert serving.boundary_layer_points(r, Nz) >= 6
        assert serving.boundary_layer_points(r * 1.01, Nz) < 6
    assert serving.adequate_grids(1e8) == [(512, 128), (1024, 256)]
    assert serving.adequate_grids(1e4) == list(serving.SERVING_GRIDS)


def test_stable_dt_ladder():
    # measured stable points lie at or above the rule's value
    assert serving.stable_dt(64, 1e6) <= 1.25e-5
    assert serving.stable_dt(128, 1e7) <= 7.8125e-7
    for Nz, ra in ((32, 1e5), (256, 1e8)):
        dt = serving.stable_dt(Nz, ra)
        j = math.log2(1e-3 / dt)
        assert abs(j - round(j)) < 1e-9                    # on the halving ladder
        assert dt <= 40.0 / (Nz * Nz * math.sqrt(ra)) < 2 * dt
    assert serving.stable_dt(64, 1e7) < serving.stable_dt(64, 1e6) < serving.stable_dt(32, 1e6)


def test_request_stream_is_seeded_and_within_ranges():
    a = serving.make_requests(256, seed=4, rate=10.0)
    b = serving.make_requests(256, seed=4, rate=10.0)
    assert [(r.Ra, r.Nx, r.Nz, r.nslices, r.precision, r.arrival) for r in a] == \
           [(r.Ra, r.Nx, r.Nz, r.nslices, r.precision, r.arrival) for r in b]
    arr = np.array([r.arrival for r in a])
    assert np.all(np.diff(arr) > 0)
    # Poisson arrivals: mean gap 1/rate within sampling error
    assert abs(np.diff(arr).mean() - 0.1) < 0.03
    for r in a:
        assert 1e4 <= r.Ra <= 1e8 and 4 <= r.nslices <= 64
        assert (r.Nx, r.Nz) in serving.adequate_grids(r.Ra)
        assert r.precision in (rbc.RBC_FP64, rbc.RBC_MIXED)
    assert 0.3 < np.mean([r.precision == rbc.RBC_MIXED for r in a]) < 0.7
    logra = np.log10([r.Ra for r in a])
    assert abs(logra.mean() - 6.0) < 0.3


def test_run_bytes_counts_every_buffer():
    N, Sf, Sc, nch = 10, 1000, 250, 3
    # U and Uold (N+1 each), F (N), Gold (N coarse), Nu integrals and norms
    assert serving.run_bytes(N, Sf, Sc, nch) == 2 * 11 * Sf + 10 * Sf + 10 * Sc + (3 * 10 + 22) * 8


def test_default_class_config_whole_steps():
    for Nx, Nz in serving.SERVING_GRIDS:
        c = serving.default_class_config(Nx, Nz, rbc.RBC_FP64)
        assert c.nf * c.dt_fine == pytest.approx(c.nc * c.dt_coarse, rel=1e-15)
        assert (c.coarse_Nx, c.coarse_Nz) == (Nx // 2, Nz // 2)
