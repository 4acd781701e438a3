"""Host logic of the benchmark (no GPU): the roofline arithmetic, the per-shape
DRAM-traffic lookup tied to the kernel sources' hash, and the split of the
batch into end-to-end pipeline contexts."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_roofline_arithmetic():
    kt = {"fast": {"launches": 4, "ms": 8.0, "cell_updates": 4.0e9},
          "general": {"launches": 4, "ms": 2.0, "cell_updates": 1.0e8}}
    r = bench.roofline_of(kt, (99, 99, 99))          # a shape with no measured traffic
    # 1e9 cell-updates per 2 ms launch at 20 flops each = 10 TFLOP/s
    assert abs(r["achieved"] - 10.0) < 1e-9
    peak = 2 * 128 * 152 * 2070e6 / 1e12
    assert abs(r["peak"] - peak) < 1e-9 and abs(r["frac"] - 10.0 / peak) < 1e-12
    assert r["traffic"] is None and r["bound"] == "alu"
    assert abs(r["share_of_batched_time"] - 0.8) < 1e-12
    assert bench.roofline_of({"fast": {"launches": 0, "ms": 0.0, "cell_updates": 0}}, (20, 24, 7)) is None


def test_traffic_lookup_follows_the_sources_hash():
    """The committed summary is read only for the shapes it lists and only while
    the kernel sources hash to the recorded value."""
    got = bench.measured_traffic((20, 24, 7))
    path = os.path.join(bench.ROOT, "profiles", "fast_kernel_crystal.md")
    text = open(path).read()
    if bench.kernel_source_hash() in text:
        assert got is not None and 0.5 < got < 2.5
        r = bench.roofline_of({"fast": {"launches": 1, "ms": 1.0, "cell_updates": 1.0e9}}, (20, 24, 7))
        assert abs(r["traffic"] - got * 1.0e9) < 1.0
    else:
        assert got is None
    assert bench.measured_traffic((1, 2, 3)) is None


def test_e2e_split_keeps_every_instance_once():
    """The pipeline split (bench.e2e_groups, used by e2e_pipelined): contiguous
    groups of about equal cells covering every instance exactly once."""
    rng = np.random.default_rng(3)
    cells = np.exp(rng.uniform(np.log(4096), np.log(262144), size=4096)).astype(np.int64)
    groups = bench.e2e_groups(cells, bench.E2E_PARTS)
    assert np.array_equal(np.concatenate(groups), np.arange(len(cells)))
    sizes = np.array([cells[g].sum() for g in groups])
    assert len(groups) == bench.E2E_PARTS and sizes.max() < 1.05 * sizes.mean()
