"""Host logic of bench.py that needs no GPU.

The DRAM traffic and the warp-instruction count the benchmark line reports
come from committed ncu summaries, and only while the kernel source still
matches the digest recorded with them: a change to the code (not to its
comments or layout) must turn them into null rather than let a stale count be
reported for a new kernel.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _profile_with_digest(tmp_path, digest):
    p = tmp_path / "profiles"
    p.mkdir()
    (p / "k.md").write_text("# summary\nwarp_instructions_per_iteration: 1.5e6\n"
                            "traffic_bytes_per_iteration: 4096\n"
                            f"fw.cu code digest: {digest}\n")
    return p


def test_digest_ignores_comments_and_layout_but_not_code(tmp_path):
    a = tmp_path / "a.cu"
    a.write_text("int f(int x) {\n  return x + 1;  // one more\n}\n")
    b = tmp_path / "b.cu"
    b.write_text("/* the successor */ int f(int x)\n{ return x + 1; }\n")
    c = tmp_path / "c.cu"
    c.write_text("int f(int x) { return x + 2; }\n")
    assert bench.code_digest(str(a)) == bench.code_digest(str(b))
    assert bench.code_digest(str(a)) != bench.code_digest(str(c))


def test_ncu_figures_only_for_the_code_they_were_taken_on(tmp_path, monkeypatch):
    src = tmp_path / "fw.cu"
    src.write_text("__global__ void k() {}\n")
    _profile_with_digest(tmp_path, bench.code_digest(str(src)))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic(str(src), "k.md") == 4096.0
    assert bench.ncu_figure(str(src), "k.md", "warp_instructions_per_iteration") == 1.5e6
    assert bench.ncu_figure(str(src), "k.md", "no_such_figure") is None
    assert bench.ncu_traffic(str(src), "missing.md") is None
    src.write_text("__global__ void k() { int x = 1; }\n")      # the kernel changed
    assert bench.ncu_traffic(str(src), "k.md") is None
    assert bench.ncu_figure(str(src), "k.md", "warp_instructions_per_iteration") is None


def test_committed_resident_profiles_carry_their_figures():
    for name in ("fw_resident_chunglu1e5.md", "fw_resident_f32_chunglu1e5.md"):
        text = open(os.path.join(ROOT, "profiles", name)).read()
        for field in ("warp_instructions_per_iteration:", "traffic_bytes_per_iteration:",
                      "fw.cu code digest:"):
            assert field in text, (name, field)
