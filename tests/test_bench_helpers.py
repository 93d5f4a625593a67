"""Host-side helpers of the benchmark, on CPU: the guard that reports ncu
traffic figures only while the kernels' code is the code that was captured
(comment edits keep them, code edits drop them to null), and the naming of
the page kernel a plan shape runs."""
import os
import shutil
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _hash_of(root, kernel="k_points_ws"):
    saved = bench.ROOT
    try:
        bench.ROOT = root
        return bench.kernel_source_hash(kernel)
    finally:
        bench.ROOT = saved


def test_traffic_guard_ignores_comments_but_not_code(tmp_path):
    src = os.path.join(ROOT, "paper_2604_12625_gb300", "csrc")
    dst = tmp_path / "paper_2604_12625_gb300" / "csrc"
    dst.mkdir(parents=True)
    files = sorted({f for fs in bench.KERNEL_SOURCES.values() for f in fs})
    for f in files:
        shutil.copy(os.path.join(src, f), dst / f)
    h0 = _hash_of(str(tmp_path))
    assert h0 == bench.kernel_source_hash("k_points_ws")
    hyb = _hash_of(str(tmp_path), "k_hybrid_pages_tc")
    f = dst / bench.KERNEL_SOURCES["k_points_ws"][0]
    text = f.read_text()
    f.write_text("// a new comment line\n" + text.replace("\n", "\n  /* block */ ", 1))
    assert _hash_of(str(tmp_path)) == h0            # comments and spacing only
    f.write_text(text + "\nstatic int ndgi_extra_symbol;\n")
    assert _hash_of(str(tmp_path)) != h0            # code changed
    assert _hash_of(str(tmp_path), "k_hybrid_pages_tc") == hyb   # another kernel's sources: its figure stays


def test_traffic_figures_scale_or_drop():
    # a figure is reported (scaled by units) while its sources match, and null once they do not
    for name, rec in bench.NCU_TRAFFIC.items():
        got = bench.traffic_for(name, 2 * rec["units"])
        h = bench.kernel_source_hash(name)
        assert got == (2 * (rec["read"] + rec["write"]) if rec["src"] == h else None), name
        assert os.path.exists(os.path.join(ROOT, rec["profile"])), rec["profile"]
    assert bench.traffic_for("no_such_kernel", 1) is None


def test_page_kernel_names():
    assert bench.page_kernel((1, 1, 8, 1)) == "k_pages_ws"
    assert bench.page_kernel([0, 1, 4, 1]) == "k_pages_tc"
    assert bench.page_kernel((2, 1, 2, 2)) == "k_pages_tc"
