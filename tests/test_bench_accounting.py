"""The bench's roofline accounting (host logic, no GPU): algorithmic bytes and
scattered L2 operations per kernel class, the ncu kernel-name classes, and
the DRAM traffic summary built from an ncu CSV."""
import csv
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _stats(n, m, **kw):
    st = {"n": n, "m": m, "m_active": [m, m, 1000, 10], "sv_hooks": [0, 500, 40, 2], "bfs_edges_inspected": 0,
          "sv_sample_stride": 1}
    st.update(kw)
    return st


def test_degree_and_labels_bytes():
    st = _stats(1 << 20, 1 << 24)
    # read every pair (2 ids of w bytes), write n counters
    assert bench.alg_bytes("degree", st, 4) == 2 * 4 * (1 << 24) + 4 * (1 << 20)
    assert bench.alg_bytes("degree", st, 8) == 2 * 8 * (1 << 24) + 4 * (1 << 20)
    # read the parents, write the labels of the id width
    assert bench.alg_bytes("finalize", st, 8) == 4 * (1 << 20) + 8 * (1 << 20)
    assert bench.l2_ops("degree", st) == (2.0 * (1 << 24), "red_add")
    # the shared-memory form makes no L2 increments
    assert bench.l2_ops("degree", dict(st, degree_form=4))[0] == 0.0
    assert bench.l2_ops("degree", dict(st, degree_form=3))[0] == 2.0 * (1 << 24)


def test_first_pass_variants():
    n, m = 1 << 20, 1 << 24
    # plain first pass with the pre-check read (2m/n = 32: hubs)
    st = _stats(n, m)
    assert bench.alg_bytes("sv_first", st, 4) == 2 * 4 * m + 4 * m
    assert bench.l2_ops("sv_first", st) == (1.0 * m, "gather")
    # sparse graph (2m/n < 4): an atomicMin per pair, no pre-check read
    sp = _stats(m, m)
    assert bench.l2_ops("sv_first", sp) == (1.0 * m, "red_min")
    # the front end: two passes over one tile of pairs in 32
    fe = _stats(n, m, sv_sample_stride=32)
    assert bench.alg_bytes("sv_first", fe, 4) == pytest.approx((4 * 4 + 16) * m / 32)
    assert bench.l2_ops("sv_first", fe) == (4.0 * m / 32, "gather")


def test_gather_passes_count_survivors():
    n, m = 1 << 20, 1 << 24
    st = _stats(n, m)
    kept = st["m_active"][2]
    assert bench.alg_bytes("sv_gather_input", st, 4) == 2 * 4 * m + 8 * m + 12 * kept
    assert bench.l2_ops("sv_gather_input", st) == (2.0 * m + kept, "gather")
    # iterations over the list: 16 bytes read per active pair, 12 per survivor
    assert bench.alg_bytes("sv_gather_list", st, 4) == 16 * 1000 + 12 * 10 + 16 * 10
    assert bench.alg_bytes("sv_shortcut", st, 4) == 12 * sum(st["sv_hooks"])


@pytest.mark.parametrize("name,cls", [
    ("void ccg::k_degree_hubs<int, 24576, 1024, 1>(const T1 *, long long)", "degree"),
    ("ccg::k_hub_select(const unsigned int *)", "degree"),
    ("void ccg::k_degree<long>(const T1 *)", "degree"),
    ("void ccg::k_degree_partition<int, unsigned short>(const T1 *, long long)", "degree"),
    ("ccg::k_degree_window_smem(const unsigned short *, unsigned long long)", "degree"),
    ("void ccg::k_degree_split<int, unsigned int>(const T1 *, long long)", "degree"),
    ("ccg::k_degree_split_batch(const int *, long long)", "degree"),
    ("ccg::k_degree_window_batch(const unsigned int *, const long *)", "degree"),
    ("ccg::k_bwin_plan(const long *, const long *, int)", "degree"),
    ("ccg::k_degree_window_hook(const unsigned long long *, unsigned long long)", "degree"),
    ("void ccg::k_sv_sample<int, 2>(const T1 *)", "sv_first"),
    ("void ccg::k_sv_pass<int, 0, 0, 0>(const T1 *)", "sv_first"),
    ("void ccg::k_sv_pass<long, 2, 1, 1>(const T1 *)", "sv_gather_input"),
    ("void ccg::k_sv_pass<unsigned int, 2, 1, 1>(const T1 *)", "sv_gather_list"),
    ("void ccg::k_sv_pass<long, 4, 0, 0>(const T1 *)", "sv_first"),
    ("void ccg::k_sv_pass<int, 1, 1, 1>(const T1 *)", "sv_first"),
    ("void ccg::k_sv_pass<unsigned int, 1, 1, 1>(const T1 *)", "sv_first"),
    ("void ccg::k_sv_pass<int, 3, 1, 1>(const T1 *)", None),
    ("void ccg::k_sv_pass_batch<0>(const int *)", None),
    ("void ccg::k_finalize_batch(unsigned int *)", "finalize"),
    ("ccg::k_shortcut_all(unsigned int *)", "sv_shortcut"),
    ("void ccg::k_finalize<int>(unsigned int *)", "finalize"),
    ("ccg::k_ks_select(const unsigned int *)", "ks"),
    ("void at::vectorized_elementwise_kernel<4>(int)", None),
])
def test_kernel_classes(name, cls):
    assert bench.kernel_class(name) == cls


def test_traffic_summary_per_call(tmp_path):
    """Two calls captured: the class bytes are summed and divided by the calls
    (the histogram kernel runs once per call)."""
    rows = [["ID", "Kernel Name", "Metric Name", "Metric Value"]]
    launches = [("ccg::k_hist(x)", 100, 20), ("void ccg::k_degree_hubs<int>(x)", 1000, 10),
                ("ccg::k_hub_select(x)", 50, 0), ("ccg::k_hist(x)", 100, 20),
                ("void ccg::k_degree_hubs<int>(x)", 1000, 10), ("ccg::k_hub_select(x)", 50, 0)]
    for i, (name, rd, wr) in enumerate(launches):
        rows.append([str(i), name, "dram__bytes_read.sum", str(rd)])
        rows.append([str(i), name, "dram__bytes_write.sum", str(wr)])
        rows.append([str(i), name, "gpu__time_duration.sum", "1000"])
    p = tmp_path / "cap.csv"
    with open(p, "w", newline="") as f:
        f.write("==PROF== preamble line\n")
        csv.writer(f, quoting=csv.QUOTE_ALL).writerows(rows)
    out = bench.ncu_summary(str(p), "rmat22", {"rmat24": 4.0}, "cmd")
    assert out["calls"] == 2
    assert out["traffic_per_call"]["rmat22"]["degree"] == pytest.approx((1000 + 10 + 50) * 2 / 2)
    assert out["traffic_per_call"]["rmat22"]["hist"] == pytest.approx(120.0)
    assert out["traffic_per_call"]["rmat24"]["degree"] == pytest.approx(4 * 1060.0)
    json.dumps(out)


def test_traffic_summary_of_one_kernel_class(tmp_path):
    """A capture of one class (ncu -k): the calls are given, not counted."""
    rows = [["ID", "Kernel Name", "Metric Name", "Metric Value"]]
    for i in range(3):
        rows.append([str(i), "void ccg::k_degree_hubs<int>(x)", "dram__bytes_read.sum", "900"])
        rows.append([str(i), "void ccg::k_degree_hubs<int>(x)", "dram__bytes_write.sum", "30"])
    p = tmp_path / "cap.csv"
    with open(p, "w", newline="") as f:
        csv.writer(f, quoting=csv.QUOTE_ALL).writerows(rows)
    with pytest.raises(SystemExit):
        bench.ncu_summary(str(p), "rmat22", {}, "cmd")
    out = bench.ncu_summary(str(p), "rmat22", {}, "cmd", calls=3)
    assert out["traffic_per_call"]["rmat22"]["degree"] == pytest.approx(930.0)


def test_class_capture_is_tied_to_that_class_sources(tmp_path, monkeypatch):
    """A one-class summary holds the hash of that class's sources only: it
    stays valid when another class's kernel file changes, is void when its
    own files change, and serves no other class."""
    rows = [["ID", "Kernel Name", "Metric Name", "Metric Value"]]
    for i in range(2):
        rows.append([str(i), "void ccg::k_degree_hubs<int>(x)", "dram__bytes_read.sum", "900"])
        rows.append([str(i), "void ccg::k_degree_hubs<int>(x)", "dram__bytes_write.sum", "100"])
        rows.append([str(10 + i), "ccg::k_hist(x)", "dram__bytes_read.sum", "5"])
    p = tmp_path / "cap.csv"
    with open(p, "w", newline="") as f:
        csv.writer(f, quoting=csv.QUOTE_ALL).writerows(rows)
    out = bench.ncu_summary(str(p), "rmat22", {}, "cmd", calls=2, kernel_cls="degree")
    assert out["kernel_class"] == "degree" and set(out["traffic_per_call"]["rmat22"]) == {"degree"}
    assert out["sources_hash"] == bench.sources_hash("degree") != bench.sources_hash()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "ncu_traffic.json").write_text(json.dumps(out))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    src = tmp_path / "paper_1607_06156_gb300" / "csrc"
    src.mkdir(parents=True)
    for f in set(bench.KERNEL_FILES) | set(bench.CLASS_FILES["degree"]):
        (src / f).write_bytes(open(os.path.join(ROOT, "paper_1607_06156_gb300", "csrc", f), "rb").read())
    assert bench.ncu_traffic("degree", "rmat22") == pytest.approx(1000.0)
    assert bench.ncu_traffic("hist", "rmat22") is None
    (src / "k_sv.cu").write_text("// another class changed")
    assert bench.ncu_traffic("degree", "rmat22") == pytest.approx(1000.0)
    (src / "k_degree.cu").write_text("// the class's own kernel changed")
    assert bench.ncu_traffic("degree", "rmat22") is None


def test_traffic_file_with_one_record_per_class(tmp_path, monkeypatch):
    """A traffic file may hold one capture per kernel class ("classes"): each
    class is served from its own record and voided by its own sources only."""
    recs = {}
    for cls, name, rd in (("degree", "void ccg::k_degree_split<int, unsigned int>(x)", 700),
                          ("sv_gather_input", "void ccg::k_sv_pass<int, 2, 1, 1>(x)", 400)):
        rows = [["ID", "Kernel Name", "Metric Name", "Metric Value"]]
        for i in range(2):
            rows.append([str(i), name, "dram__bytes_read.sum", str(rd)])
            rows.append([str(i), name, "dram__bytes_write.sum", "100"])
        p = tmp_path / f"{cls}.csv"
        with open(p, "w", newline="") as f:
            csv.writer(f, quoting=csv.QUOTE_ALL).writerows(rows)
        recs[cls] = bench.ncu_summary(str(p), "rmat24", {}, "cmd", calls=2, kernel_cls=cls)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "ncu_traffic.json").write_text(json.dumps({"classes": recs}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    src = tmp_path / "paper_1607_06156_gb300" / "csrc"
    src.mkdir(parents=True)
    for f in set(bench.KERNEL_FILES) | set(bench.CLASS_FILES["degree"]) | set(bench.CLASS_FILES["sv_gather_input"]):
        (src / f).write_bytes(open(os.path.join(ROOT, "paper_1607_06156_gb300", "csrc", f), "rb").read())
    assert bench.ncu_traffic("degree", "rmat24") == pytest.approx(800.0)
    assert bench.ncu_traffic("sv_gather_input", "rmat24") == pytest.approx(500.0)
    assert bench.ncu_traffic("hist", "rmat24") is None
    (src / "k_sv.cu").write_text("// the gather pass changed")
    assert bench.ncu_traffic("sv_gather_input", "rmat24") is None
    assert bench.ncu_traffic("degree", "rmat24") == pytest.approx(800.0)
