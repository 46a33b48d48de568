"""CPU-only checks of the boundary: the library builds for sm_103a, loads,
and exports every function include/spamm.h declares; the Python binding
covers the same names.  No compute calls (there is no GPU here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "spamm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(spamm_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1203_1692_gb300 import build
    return build.build()


def test_header_declares_the_abi():
    names = declared_functions()
    for need in ("spamm_create", "spamm_build_norms", "spamm_multiply", "spamm_stats",
                 "spamm_destroy", "spamm_tree_destroy", "spamm_last_error"):
        assert need in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (spamm_\w+)", out))
    assert exported == set(declared_functions())


def test_binding_covers_the_abi(libpath):
    from paper_1203_1692_gb300 import _abi
    assert set(_abi.SIGNATURES) == set(declared_functions())
    _abi.lib()


def test_config_default_through_the_abi(libpath):
    from paper_1203_1692_gb300 import _abi
    c = _abi.spamm_config_default()
    assert (c.leaf, c.precision, c.checked) == (16, 0, 1)
    assert c.tie_rel == 1e-6


def test_create_rejects_bad_config_before_touching_the_gpu(libpath):
    from paper_1203_1692_gb300 import _abi
    L = _abi.lib()
    h = ctypes.c_void_p()
    c = _abi.spamm_config_default()
    c.leaf = 24
    assert L.spamm_create(ctypes.byref(h), None, ctypes.byref(c)) == _abi.SPAMM_ERR_INVALID_ARG
    c = _abi.spamm_config_default()
    c.precision = 9
    assert L.spamm_create(ctypes.byref(h), None, ctypes.byref(c)) == _abi.SPAMM_ERR_INVALID_ARG
    c = _abi.spamm_config_default()
    c.tie_rel = 0.7
    assert L.spamm_create(ctypes.byref(h), None, ctypes.byref(c)) == _abi.SPAMM_ERR_INVALID_ARG
    c = _abi.spamm_config_default()
    c.pool_bytes = -1
    assert L.spamm_create(ctypes.byref(h), None, ctypes.byref(c)) == _abi.SPAMM_ERR_INVALID_ARG


def test_no_cpu_fallback_when_library_missing(tmp_path, monkeypatch):
    from paper_1203_1692_gb300 import _abi
    monkeypatch.setattr(_abi, "_lib", None)
    monkeypatch.setattr(_abi, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="missing"):
        _abi.lib()


def test_kernels_target_sm103a(libpath):
    """The build compiles SASS for sm_103a (checked through the build flags;
    the binary itself is not inspected)."""
    from paper_1203_1692_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_slice_cull_config_is_validated_before_the_gpu(libpath):
    from paper_1203_1692_gb300 import _abi
    L = _abi.lib()
    h = ctypes.c_void_p()
    for leaf, prec, sl, want in [(64, _abi.SPAMM_PREC_FP32, 16, _abi.SPAMM_ERR_UNSUPPORTED),
                                 (16, _abi.SPAMM_PREC_TF32X3, 16, _abi.SPAMM_ERR_UNSUPPORTED),
                                 (64, _abi.SPAMM_PREC_TF32X3, 8, _abi.SPAMM_ERR_INVALID_ARG),
                                 (64, _abi.SPAMM_PREC_TF32X3, 32, _abi.SPAMM_ERR_INVALID_ARG)]:
        c = _abi.spamm_config_default()
        c.leaf, c.precision, c.slice = leaf, prec, sl
        assert L.spamm_create(ctypes.byref(h), None, ctypes.byref(c)) == want


def test_tier_config_is_validated_before_the_gpu(libpath):
    """Precision chosen by norm needs a split precision and 0 <= tier_bits
    <= 40; invalid combinations are refused before any CUDA call."""
    from paper_1203_1692_gb300 import _abi
    L = _abi.lib()
    h = ctypes.c_void_p()
    for prec, bits in [(_abi.SPAMM_PREC_FP32, 10), (_abi.SPAMM_PREC_TF32, 10),
                       (_abi.SPAMM_PREC_F16X3, -1), (_abi.SPAMM_PREC_F16X3, 41),
                       (_abi.SPAMM_PREC_BF16X3, 1000)]:
        c = _abi.spamm_config_default()
        c.leaf, c.precision, c.tier_bits = 64, prec, bits
        assert L.spamm_create(ctypes.byref(h), None, ctypes.byref(c)) == \
            _abi.SPAMM_ERR_INVALID_ARG


def test_ctypes_structs_match_the_header(tmp_path):
    """The binding's spamm_config and spamm_stats_t have the C layout: every
    field at the offset gcc gives it from include/spamm.h, and the same size
    (a field added on one side only would shift the rest)."""
    from paper_1203_1692_gb300 import _abi
    structs = {"spamm_config": _abi.spamm_config, "spamm_stats_t": _abi.spamm_stats_t}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "spamm.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in cls._fields_:
            lines.append(f'    printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                        str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n"):
        if line:
            cname, field, val = line.split()
            got[(cname, field)] = int(val)
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f in cls._fields_:
            assert got[(cname, f[0])] == getattr(cls, f[0]).offset, (cname, f[0])
