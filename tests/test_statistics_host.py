"""rbc_stat_summary (host arithmetic of the library: the quantities of Sec. 2.2
from time means) against the oracle's averages, written separately
(oracle/statistics.py), on the same integrals.  No device is needed."""
import numpy as np
import pytest

from oracle import statistics as ost
from oracle.rbc import RBC
from paper_2001_01609_gb300 import rbc

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def to_oracle_integrals(row, Mz, duration):
    return dict(sqrtKE2=row[0], eps=row[1], wT=row[2], NuV=row[3], Nub=row[4], Nut=row[5],
                Tm=row[6:6 + Mz], T2=row[6 + Mz:6 + 2 * Mz], T=duration)


@pytest.mark.parametrize("seed,Nz", [(0, 24), (1, 16), (2, 40)])
def test_stat_summary_matches_the_oracle(seed, Nz):
    g = np.random.default_rng(seed)
    Ra, Pr = 3e5, 0.8
    Mz = 3 * Nz // 2
    B, D = 3, 0.7
    I = np.zeros((B, 6 + 2 * Mz))
    I[:, 0] = g.uniform(1, 50, B)
    I[:, 1] = -g.uniform(1e3, 5e3, B)
    I[:, 2] = g.uniform(0.01, 0.05, B)
    I[:, 3:6] = g.uniform(2.0, 2.2, (B, 3))
    I[:, 6:6 + Mz] = g.uniform(0.2, 0.3, (B, Mz))
    I[:, 6 + Mz:] = I[:, 6:6 + Mz] ** 2 / (D / B) + g.uniform(1e-4, 1e-2, (B, Mz))
    o = ost.averages(ost.combine([to_oracle_integrals(r, Mz, D / B) for r in I]), Ra, Pr,
                     RBC(Ra, Pr, 2.0, 16, Nz, 1e-3).padded_z(), Nz)
    means = I.sum(axis=0) / sum([D / B] * B)
    p = rbc.stat_summary(Nz, Ra, Pr, means)
    for q in ("U", "Re", "NuV", "Nub", "Nut", "Nu_int", "P", "eps_U", "balance", "delta_t"):
        assert abs(p[q] - o[q]) <= 1e-13 * abs(o[q]), q
    np.testing.assert_allclose(p["Trms"], o["Trms"], rtol=1e-10)
    assert p["delta_T"] == pytest.approx(o["delta_T"], abs=1e-15) and p["N_BL"] == o["N_BL"]


def test_stat_summary_of_a_conduction_profile():
    """No fluctuation: T_rms = 0, so there is no boundary-layer peak."""
    Nz = 16
    Mz = 3 * Nz // 2
    zp = 0.5 * np.cos(np.pi * np.arange(Mz) / (Mz - 1))
    m = np.zeros(6 + 2 * Mz)
    m[3:6] = 1.0
    m[6:6 + Mz] = 0.5 - zp
    m[6 + Mz:] = (0.5 - zp) ** 2
    p = rbc.stat_summary(Nz, 1e3, 1.0, m)
    assert p["NuV"] == 1.0 and p["Nu_int"] == 0.0 and np.isnan(p["delta_T"]) and p["N_BL"] == 0
    assert np.all(p["Trms"] == 0.0)
    with pytest.raises(rbc.RBCError):
        rbc.stat_summary(7, 1e3, 1.0, np.zeros(6 + 2 * 10))
