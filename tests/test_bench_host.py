"""Host logic of bench.py (CPU): the stored ncu DRAM traffic of a kernel is
reported only while the kernel's sources are the ones it was taken on."""
import hashlib
import os

import pytest

pytest.importorskip("torch")


def _sha(sources):
    import bench
    d = hashlib.sha256()
    for f in sources:
        with open(os.path.join(bench.ROOT, "paper_0810_1119_gb300", "csrc", f), "rb") as fh:
            d.update(fh.read())
    return d.hexdigest()[:16]


def test_traffic_figure_is_null_once_a_source_changes(monkeypatch):
    import bench
    entry = dict(bench.TRAFFIC["mean_win"])
    monkeypatch.setitem(bench.TRAFFIC, "mean_win", dict(entry, sha=_sha(entry["sources"])))
    assert bench._traffic("mean_win") == entry["bytes_per_launch"]
    monkeypatch.setitem(bench.TRAFFIC, "mean_win", dict(entry, sha="0" * 16))
    assert bench._traffic("mean_win") is None
    assert bench._traffic("no_such_kernel") is None


def test_per_position_traffic_scales_with_the_run(monkeypatch):
    import bench
    entry = dict(bench.TRAFFIC["dense_mean"])
    monkeypatch.setitem(bench.TRAFFIC, "dense_mean", dict(entry, sha=_sha(entry["sources"])))
    assert bench._traffic("dense_mean", 1000) == pytest.approx(1000 * entry["bytes_per_pair"])
