"""The committed ncu figures that bench.py reports as DRAM traffic belong to
the kernels in the tree: each entry of profiles/step_traffic.json carries
the hash of the sources of its kernels, and the entries bench.py reads must
match the current sources (no GPU needed)."""
import json
import os

import pytest

from paper_1411_7051_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _traffic():
    with open(os.path.join(ROOT, "profiles", "step_traffic.json")) as fh:
        return json.load(fh)


@pytest.mark.parametrize("tag,files", [("StoreF32", build.STEP_KERNEL_FILES),
                                       ("StoreF16", build.STEP_KERNEL_FILES),
                                       ("adjoint", build.ADJOINT_KERNEL_FILES),
                                       ("batch_fp16", build.BATCH_KERNEL_FILES),
                                       ("batch_fp32", build.BATCH_KERNEL_FILES)])
def test_traffic_matches_the_kernel_sources(tag, files):
    e = _traffic()[tag]
    assert e["source_hash"] == build.kernel_hash(files), (
        f"profiles/step_traffic.json[{tag}] was captured on other kernel sources: "
        "capture it again (its command is in the entry)")
    assert e["command"].startswith("ncu ") and "--clock-control none" in e["command"]


def test_traffic_per_update_is_plausible():
    """DRAM bytes a lattice update against the algorithmic bytes (80 B FP32,
    44 B FP16, 109.5 B for the adjoint's reverse step): below them only by
    what the 129 MB L2 can hold back, never far above (re-reads; the
    batched instances 512 and 1024 wide read their row padding too)."""
    t = _traffic()
    for tag, algo in (("StoreF32", 80.0), ("StoreF16", 44.0), ("adjoint", 109.5),
                      ("batch_fp16", 44.0), ("batch_fp32", 80.0)):
        per = t[tag]["dram_bytes_per_launch"] / t[tag]["nodes"]
        held = 129e6 / t[tag]["nodes"]
        assert algo - held - 1.0 <= per <= algo * 1.05, (tag, per)


def test_bench_reports_batch_traffic_only_for_the_captured_instances():
    """bench.py's batch roofline takes the committed traffic for the instance
    set it was captured on (same node count) and reports null otherwise, and
    never for the non-staged shapes."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    e = _traffic()["batch_fp16"]
    r = dict(ms=0.71 * 300, nodes=e["nodes"], bpu=44.0, staged=True)
    roof = bench.batch_roofline(r, 300, 6795.8, "measured", "fp16")
    assert roof["traffic"] == e["dram_bytes_per_launch"]
    assert roof["traffic_per_update"] == pytest.approx(e["dram_bytes_per_launch"] / e["nodes"])
    assert bench.batch_roofline(dict(r, nodes=e["nodes"] + 1), 300, 6795.8, "measured",
                                "fp16")["traffic"] is None
    assert bench.batch_roofline(dict(r, staged=False), 300, 6795.8, "measured",
                                "fp16")["traffic"] is None
