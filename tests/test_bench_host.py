"""Host logic of bench.py (no GPU): the committed closest-hit ncu summary
was taken from the kernel sources in the tree (else the bench line's DRAM
traffic would silently drop to null), it carries the figures the bench
reads, and the roofline arithmetic is algorithmic bytes per ray x rays per
launch / launch time, against the probe's peak."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_profile_matches_kernel_sources():
    prof = bench.read_profile()
    assert prof.get("kernel_sources_sha") == bench.kernel_hash(), \
        "profiles/k_trace_closest_large_nave.txt was captured from other kernel sources: capture it again"
    for key in ("dram_bytes_per_ray", "l1_throughput_pct", "l1_hit_rate_pct", "lts_throughput_pct",
                "warps_active_pct", "rays_traced", "dram_bytes_read", "dram_bytes_write"):
        assert key in prof, key
    # the per-ray figure is the capture's DRAM bytes over its rays
    per_ray = (float(prof["dram_bytes_read"]) + float(prof["dram_bytes_write"])) / float(prof["rays_traced"])
    assert float(prof["dram_bytes_per_ray"]) == pytest.approx(per_ray, rel=2e-3)


class _FakeRenderer:
    def __init__(self, l2_gbs):
        self.l2 = l2_gbs

    def probe_l2(self):
        return self.l2


def test_trace_roofline_arithmetic():
    counts = {"nodes_visited": 41_000, "tris_tested": 2_000, "ext_rays": 1_000,
              "shadow_nodes_visited": 20_000, "shadow_tris_tested": 1_500, "shadow_rays": 1_000}
    # 10 launches, 2e7 rays, 13 ms in all
    roof = bench.trace_roofline(_FakeRenderer(20_000.0), counts, ms_trace=13.0, n_trace=10, ext_rays=2e7,
                                prof_ok_traffic=80.0)
    bytes_per_ray = 41.0 * 32 + 2.0 * 48 + 32 + 8
    assert roof["algorithmic_bytes_per_ray"] == pytest.approx(bytes_per_ray)
    assert roof["launch_ms"] == pytest.approx(1.3)
    assert roof["rays_per_launch"] == pytest.approx(2e6)
    achieved = 2e6 * bytes_per_ray / 1.3e-3 / 1e9
    assert roof["achieved"] == pytest.approx(achieved)
    assert roof["frac"] == pytest.approx(achieved / 20_000.0)
    assert roof["traffic"] == pytest.approx(80.0 * 2e6)
    assert roof["sun_child_slots_per_ray"] == pytest.approx(20.0)
    # no valid capture: no traffic figure
    assert bench.trace_roofline(_FakeRenderer(20_000.0), counts, 13.0, 10, 2e7)["traffic"] is None
