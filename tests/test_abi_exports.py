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


def _run_c(tmp_path, body: list[str]) -> dict:
    """Compile a C program against the header and return its "key value" lines."""
    import shutil

    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "cc_gb300.h"', "int main(void) {"]
    src += body + ["return 0; }"]
    c = tmp_path / "probe.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return dict(line.split() for line in out.splitlines())


def test_ctypes_structs_match_the_header(tmp_path):
    """Every field of the binding's ctypes structs sits at the C struct's
    offset with the C field's size, and the structs have the C sizes."""
    import paper_1607_06156_gb300 as cc

    structs = {"cc_options": cc.Options, "cc_stats": cc.Stats, "cc_l2_rates": cc.L2Rates}
    body = []
    for name, cls in structs.items():
        body.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            body.append(f'printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
            body.append(f'printf("{name}.{f}.size %zu\\n", sizeof((({name} *)0)->{f}));')
    got = _run_c(tmp_path, body)
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            field = getattr(cls, f)
            assert int(got[f"{name}.{f}"]) == field.offset, (name, f)
            assert int(got[f"{name}.{f}.size"]) == field.size, (name, f)


def test_binding_constants_match_the_header(tmp_path):
    """Status codes, route policies, fault bits, array bounds, the kernel-class
    order and the network sizes the binding mirrors are the header's."""
    import paper_1607_06156_gb300 as cc

    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    kclasses = re.findall(r"\bCC_K_(\w+)\s*=\s*(\d+)", text)
    order = [name.lower() for name, v in sorted(kclasses, key=lambda t: int(t[1])) if name != "COUNT"]
    assert order == cc.KERNELS
    consts = {"CC_K_COUNT": cc.K_COUNT, "CC_MAX_SV_ITERS_RECORDED": cc.MAX_SV_ITERS_RECORDED,
              "CC_MLP_IN": cc.MLP_IN, "CC_MLP_HIDDEN": cc.MLP_HIDDEN, "CC_MLP_OUT": cc.MLP_OUT,
              "CC_MLP_PARAMS": cc.MLP_PARAMS, "CC_FAULT_ALLOC": cc.FAULT_ALLOC,
              "CC_FAULT_ITER_CAP": cc.FAULT_ITER_CAP, "CC_ROUTE_AUTO": cc.ROUTES["auto"],
              "CC_ROUTE_LEARNED": cc.ROUTES["learned"], "CC_ROUTE_FORCE_BFS": cc.ROUTES["bfs"],
              "CC_ROUTE_FORCE_SV": cc.ROUTES["sv"]}
    consts.update({name: code for code, name in cc.STATUS.items()})
    got = _run_c(tmp_path, [f'printf("{k} %lld\\n", (long long)({k}));' for k in consts])
    for k, v in consts.items():
        assert int(got[k]) == v, k


def _prototypes():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    pat = r"^\s*((?:const\s+)?[A-Za-z_]\w*\s*\**)\s*(cc_\w+)\s*\(([^)]*)\)\s*;"
    return {m.group(2): (m.group(1).strip(), [p.strip() for p in m.group(3).split(",") if p.strip()])
            for m in re.finditer(pat, text, flags=re.M)}


def test_binding_argtypes_match_the_prototypes():
    """Each function's ctypes argtypes have the header prototype's arity and,
    parameter by parameter, the same kind (pointer, 32- or 64-bit integer,
    float, double); cc_status returns are read as int."""
    import paper_1607_06156_gb300 as cc

    L = cc.lib()
    scalar = {"int": ctypes.c_int, "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64, "float": ctypes.c_float,
              "double": ctypes.c_double, "cc_status": ctypes.c_int}
    protos = _prototypes()
    assert set(protos) == set(declared_functions())
    for name, (ret, params) in protos.items():
        fn = getattr(L, name)
        assert len(fn.argtypes) == len(params), name
        for p, at in zip(params, fn.argtypes):
            if "*" in p:
                assert at is ctypes.c_void_p or issubclass(at, ctypes._Pointer), (name, p)
            else:
                ctype = p.rsplit(None, 1)[0]
                assert ctypes.sizeof(at) == ctypes.sizeof(scalar[ctype]), (name, p)
                assert (at in (ctypes.c_float, ctypes.c_double)) == (ctype in ("float", "double")), (name, p)
        if ret == "cc_status":
            assert fn.restype is ctypes.c_int, name
        else:
            assert ret.endswith("*") and fn.restype is ctypes.c_char_p, name


def test_argument_errors_return_before_any_device_call():
    """The boundary's argument checks run on the host before any CUDA call:
    a null context, negative sizes, ids past the limits, missing pointers and
    bad options each give their status with no device present."""
    import paper_1607_06156_gb300 as cc

    L = cc.lib()
    ARG, EDGE, UNSUP = 1, 2, 7
    v = ctypes.c_void_p
    buf = ctypes.create_string_buffer(64)
    p = ctypes.cast(buf, v)
    assert L.cc_default_options(None) == ARG
    assert L.cc_create(None, None, 0) == ARG
    o = cc.default_options()
    for field, bad in (("id_bytes", 3), ("ks_tau", -1.0), ("route_policy", 9)):
        o2 = cc.default_options()
        setattr(o2, field, bad)
        out = v()
        assert L.cc_create(ctypes.byref(out), ctypes.byref(o2), 0) == ARG, field
        assert not out.value
    assert L.cc_set_options(None, ctypes.byref(o)) == ARG
    assert L.cc_destroy(None) == 0
    assert L.cc_get_stats(None, ctypes.byref(cc.Stats())) == ARG
    for f in (L.cc_labels, L.cc_labels_host, L.cc_labels_tuple_sv):
        assert f(None, p, 10, 5, p, None) == ARG
    assert L.cc_labels_batched(None, p, p, p, 1, 10, 10, p, None) == ARG
    assert L.cc_ks_statistic_batched(None, p, p, p, 1, 10, 10, p, p, p, p, p, p, None) == ARG
    assert L.cc_degree_distribution(None, p, 10, 5, p, p, 4, None) == ARG
    assert L.cc_ks_statistic(None, p, 4, p, None) == ARG
    assert L.cc_route_features(None, p, 10, 5, p, None) == ARG
    assert L.cc_set_predictor(None, p, 0.5) == ARG
    assert L.cc_measure_l2_rates(None, None, None) == ARG
    # the library-owned scratch entry point needs no context
    assert L.cc_labels_static(p, 3, 10, 5, p, None) == ARG
    assert L.cc_labels_static(p, 4, -1, 5, p, None) == ARG
    assert L.cc_labels_static(p, 4, 0, 0, p, None) == 0
    assert L.cc_labels_static(p, 4, 0, 1, p, None) == EDGE
    assert L.cc_labels_static(p, 4, (1 << 20) + 1, 5, p, None) == UNSUP
    assert L.cc_labels_static(p, 4, 10, (1 << 21) + 1, p, None) == UNSUP
    assert L.cc_labels_static(None, 4, 10, 5, p, None) == ARG
    assert L.cc_mlp_forward(None, p, 4, p, None) == ARG
    assert L.cc_mlp_forward(p, p, 0, p, None) == ARG
    assert L.cc_mlp_backward(p, p, p, p, p, 4, ctypes.c_float(0.1), p, p, p, None, None) == ARG
    assert L.cc_mlp_adam(p, p, p, p, 10, 1e-3, 0.9, 0.999, 1e-8, 0, None) == ARG
    for s in range(8):
        assert cc.strerror(s)


def test_unknown_option_names_are_refused():
    """A misspelt option raises before the context is created instead of
    being dropped silently."""
    import paper_1607_06156_gb300 as cc

    with pytest.raises(TypeError, match="profle"):
        cc.Engine(profle=1)
    o = cc.default_options()
    cc._set_options(o, {"profile": 1, "sv_sample_stride": 8})
    assert o.profile == 1 and o.sv_sample_stride == 8
    with pytest.raises(TypeError):
        cc._set_options(o, {"reserved": 0})
