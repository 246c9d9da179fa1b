"""Host logic of bench.py's roofline traffic lookup: a committed ncu summary
supplies DRAM bytes per launch only for the kernel source and the kernel
variant it was taken on."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def write_summary(root, workload, tag, khash, variant, traffic):
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)
    lines = ["# summary", "", f"kernel_source_sha256_16: {khash}"]
    if variant is not None:
        lines.append(f"variant: {variant}")
    lines += ["", f"traffic_bytes_per_launch: {traffic}", ""]
    with open(os.path.join(root, "profiles", f"ncu_collide_stream_{workload}_{tag}.txt"), "w") as f:
        f.write("\n".join(lines))


@pytest.fixture
def fake_root(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0123456789abcdef")
    return str(tmp_path)


def test_traffic_needs_matching_source_and_variant(fake_root):
    write_summary(fake_root, "large", "f16", "0123456789abcdef", "tma_ws8x2", 1176899072)
    assert bench.ncu_traffic("large", 1, "tma_ws8x2") == 1176899072.0
    assert bench.ncu_traffic("large", 1, "tma_ws7x3") is None      # another variant
    assert bench.ncu_traffic("large", 2, "tma_ws8x2") is None      # no BF16 summary
    write_summary(fake_root, "large", "f32", "fedcba9876543210", "reg4_l2pf", 2379443968)
    assert bench.ncu_traffic("large", 0, "reg4_l2pf") is None      # another kernel source
    write_summary(fake_root, "paper", "f32", "0123456789abcdef", None, 49539584)
    assert bench.ncu_traffic("paper", 0, "reg2") is None           # variant not recorded


def test_committed_summaries_name_a_known_variant():
    names = set(bench.VARIANT_NAMES.values())
    prof = os.path.join(ROOT, "profiles")
    found = 0
    for f in sorted(os.listdir(prof)):
        if f.startswith("ncu_collide_stream_") and f.endswith(".txt"):
            txt = open(os.path.join(prof, f)).read()
            if "traffic_bytes_per_launch:" not in txt:
                continue
            found += 1
            v = [ln.split(":", 1)[1].strip() for ln in txt.splitlines() if ln.startswith("variant:")]
            assert len(v) == 1 and v[0] in names, f
    assert found >= 3
