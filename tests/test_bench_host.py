"""bench.py's host helpers: the fine-group starts it mirrors from
parareal_iterate's schedule, the derived slice arithmetic of its workloads, the
DRAM-traffic guard, and the coarsening study's slice arithmetic."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("N,group,first,expect", [
    (32, 8, 2, [0, 2, 6, 14, 22, 30, 32]),
    (32, 32, 32, [0, 32]),
    (5, 2, 1, [0, 1, 3, 5]),
    (4, 1, 1, [0, 1, 2, 3, 4]),
])
def test_fine_group_starts(N, group, first, expect):
    assert bench.fine_group_starts(N, group, first) == expect


def test_workloads_are_whole_steps():
    for name, w in bench.WORKLOADS.items():
        d = bench.derived(w)
        assert abs(d["nc"] * d["dtc"] - d["slice_len"]) < 1e-12 * d["slice_len"], name
        assert d["dof"] == 2 * w["Nx"] * w["Nz"]


def test_traffic_guard_follows_the_sources(monkeypatch):
    import hashlib
    h = hashlib.sha256()
    for f in bench.NCU_TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    monkeypatch.setattr(bench, "NCU_TRAFFIC_SHA256", h.hexdigest())
    assert bench.ncu_traffic("coarse:k_rows") == bench.NCU_TRAFFIC["coarse:k_rows"]
    monkeypatch.setattr(bench, "NCU_TRAFFIC_SHA256", "0" * 64)
    assert bench.ncu_traffic("coarse:k_rows") is None


def test_study_slices_are_whole_steps():
    s = bench.STUDY
    T = s["total_steps"] * s["dt"]
    for N in s["slices"]:
        assert s["total_steps"] % N == 0
        for _, _, dtc in s["coarse"]:
            q = T / N / dtc
            assert abs(q - round(q)) < 1e-9 * q


def test_traffic_is_keyed_by_the_sampled_batch():
    # the recorded sources are the committed ones, and every fine entry names its batch
    assert bench.ncu_traffic("coarse:k_solve") == bench.NCU_TRAFFIC["coarse:k_solve"]
    for k in bench.NCU_TRAFFIC:
        assert k.startswith("coarse:") or "@" in k, k
    assert bench.ncu_traffic("fine:k_rows@2") == bench.NCU_TRAFFIC["fine:k_rows@2"]
    assert bench.ncu_traffic("fine:k_rows@7") is None
