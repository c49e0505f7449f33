"""The C-ABI library builds, loads without a GPU and exports every symbol the header declares."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cc_gb300.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(cc_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("cc_create", "cc_destroy", "cc_labels", "cc_labels_batched", "cc_get_stats", "cc_strerror",
              "cc_default_options", "cc_degree_distribution", "cc_ks_statistic"):
        assert f in names


def test_library_exports_every_declared_symbol():
    from paper_1607_06156_gb300 import _build

    try:
        path = _build.build()
    except (RuntimeError, FileNotFoundError) as e:  # nvcc missing on this host
        pytest.skip(f"cannot build: {e}")
    lib = ctypes.CDLL(path)
    for f in declared_functions():
        assert hasattr(lib, f), f
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(cc_\w+)", out))
    assert set(declared_functions()) <= exported


def test_no_gpu_calls_fail_cleanly():
    """Without touching compute: option defaults and status strings work."""
    import paper_1607_06156_gb300 as cc

    cc.lib()
    o = cc.default_options()
    assert o.id_bytes == 4 and abs(o.ks_tau - 0.05) < 1e-15 and o.ks_min_tail == 50 and o.ks_min_span == 10.0
    assert cc.strerror(0) == "ok"
    assert "outside" in cc.strerror(2)


def test_ctypes_structs_match_the_header(tmp_path):
    """The binding's ctypes structs have the C structs' sizes and field offsets
    (a C program compiled against the header prints them)."""
    import shutil

    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    import paper_1607_06156_gb300 as cc

    checks = {"cc_options": (cc.Options, ["ks_tau", "ks_min_span", "profile", "bfs_mode"]),
              "cc_stats": (cc.Stats, ["ks_d", "m_active", "ms_degree", "launches", "kernel_ms", "sv_hooks",
                                      "ms_features", "batch_unroll", "batch_grid_mult"]),
              "cc_l2_rates": (cc.L2Rates, ["gather", "atom_min", "table_words", "grid"])}
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "cc_gb300.h"', "int main(void) {"]
    for name, (_, fields) in checks.items():
        src.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f in fields:
            src.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    src.append("return 0; }")
    c = tmp_path / "sizes.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for name, (cls, fields) in checks.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f in fields:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)
