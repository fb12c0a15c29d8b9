"""Host-side bookkeeping of bench.py (no GPU): grouping of the profiled phases
into kernel functions, algorithmic bytes and the dominant-kernel roofline."""
import importlib.util
import os
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_update_instances_are_one_kernel(bench):
    m = types.SimpleNamespace(n_prisms=1000, n_tri=50)
    # momentum and tracers are two instances of k_update: together they dominate
    r = dict(phases={"ext2d": (3.0, 90), "momentum": (2.0, 2), "tracers": (2.0, 2), "hpg": (0.5, 2)})
    head, allk = bench.rooflines(r, m, "split", "mixed", "no_capture_workload", 6657.6, "measured")
    assert head["kernel"] == "k_update"
    assert allk["k_update"]["launches"] == 4
    per = bench.phase_bytes("momentum", m, 4, 0)
    assert head["alg_bytes_per_launch"] == pytest.approx(per)
    assert head["achieved"] == pytest.approx(per * 4 / 4e-3 / 1e9)
    assert head["frac"] == pytest.approx(head["achieved"] / 6657.6)
    assert head["traffic"] is None                     # no capture for this source
    assert allk["k_ext2d"]["launch_ms"] == pytest.approx(3.0 / 90, abs=1e-5)   # rounded to 10 ns


def test_ext2d_bytes_depend_on_the_form(bench):
    m = types.SimpleNamespace(n_prisms=1000, n_tri=50)
    assert bench.phase_bytes("ext2d", m, 4, 20) == 50 * 492.0
    assert bench.phase_bytes("ext2d", m, 8, 20) == 50 * 736.0


def test_persistent_2d_launch_counts_its_rk_stages(bench):
    # one persistent launch per split stage runs all its RK stages: the 2D bytes
    # follow the stage count, not the launch count
    m = types.SimpleNamespace(n_prisms=1_000_000, n_tri=50_000)
    r = dict(phases={"ext2d": (1.8, 2), "momentum": (2.0, 2)}, rk2d_stages=90)
    _, allk = bench.rooflines(r, m, "split", "mixed", "w", 6657.6, "measured")
    assert allk["k_ext2d"]["launches"] == 2
    assert allk["k_ext2d"]["achieved"] == pytest.approx(90 * 50_000 * 492.0 / 1.8e-3 / 1e9, rel=1e-3)


def test_traffic_needs_the_same_sources(bench, monkeypatch):
    m = types.SimpleNamespace(n_prisms=1000, n_tri=50)
    r = dict(phases={"momentum": (2.0, 2), "tracers": (2.0, 2)})
    monkeypatch.setitem(bench.TRAFFIC, ("k_update", "mixed", "w"), dict(bytes=123.0, src="stale"))
    head, _ = bench.rooflines(r, m, "split", "mixed", "w", 6657.6, "measured")
    assert head["traffic"] is None
    monkeypatch.setitem(bench.TRAFFIC, ("k_update", "mixed", "w"),
                        dict(bytes=123.0, src=bench.kernel_src_hash()))
    head, _ = bench.rooflines(r, m, "split", "mixed", "w", 6657.6, "measured")
    assert head["traffic"] == 123.0
