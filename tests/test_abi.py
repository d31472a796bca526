"""The C-ABI library builds, loads and exports every function include/ccl.h
declares; argument checks that return before any CUDA call behave as
documented. No GPU is needed."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"CCL_API\s+[\w\s\*]*?\b(ccl_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__ as g
    return g._build_module().build()


def test_header_declares_the_boundary():
    names = _declared("ccl.h")
    for required in ("ccl_label", "ccl_label_batched", "ccl_sync", "ccl_validate", "ccl_context_create",
                     "ccl_server_create", "ccl_server_submit", "ccl_server_wait", "ccl_label_host"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (ccl_\w+)", out))
    declared = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            declared |= set(_declared(h))
    assert declared, "no declarations parsed"
    assert declared <= exported, declared - exported
    lib = ctypes.CDLL(lib_path)
    for name in declared:
        assert hasattr(lib, name)


def test_status_strings_and_argument_checks(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.ccl_status_string.restype = ctypes.c_char_p
    assert lib.ccl_status_string(0) == b"CCL_OK"
    assert lib.ccl_status_string(5) == b"CCL_ERR_NONCONVERGED"
    assert lib.ccl_status_string(99) == b"CCL_ERR_UNKNOWN"
    assert lib.ccl_version() == 100
    # NULL context / handles: rejected before any CUDA call
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.ccl_label.argtypes = [P, I32, I64, P, P, P, P, P]
    assert lib.ccl_label(None, 10, 0, None, None, None, None, None) == 1
    lib.ccl_sync.argtypes = [P, P, I64]
    assert lib.ccl_sync(None, None, 0) == 1
    lib.ccl_server_submit.argtypes = [P, P, P]
    assert lib.ccl_server_submit(None, None, None) == 1
    lib.ccl_context_create.argtypes = [P, ctypes.c_int]
    assert lib.ccl_context_create(None, 0) == 1


def test_binding_names_match_the_abi(lib_path):
    import paper_1603_08357_gb300 as ccl
    for name in _declared("ccl.h"):
        assert hasattr(ccl, name), name
    assert ccl.LIB_PATH == lib_path


def test_binding_structs_and_constants_match_the_header(tmp_path):
    """Every ctypes struct of the binding has the C struct's size and field
    offsets, and every CCL_* constant the binding exports has the header's
    value (a C program built against include/ccl.h prints them)."""
    import paper_1603_08357_gb300.binding as b
    structs = [b.ccl_run_stats, b.ccl_server_config, b.ccl_request, b.ccl_server_stats]
    consts = sorted(n for n in dir(b) if re.fullmatch(r"CCL_[A-Z0-9_]+", n) and isinstance(getattr(b, n), int))
    assert "CCL_OK" in consts and "CCL_OPT_ANALYSIS_ORDER" in consts
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "ccl.h")).read(), flags=re.S)
    in_header = set(re.findall(r"\b(CCL_[A-Z0-9_]+)\s*=", text))
    in_header |= set(re.findall(r"#define\s+(CCL_[A-Z0-9_]+)\s+\d+", text))
    assert in_header and in_header <= set(consts), in_header - set(consts)   # the binding has them all
    lines = ["#include <ccl.h>", "#include <stddef.h>", "#include <stdio.h>", "int main(void) {"]
    for cls in structs:
        name = cls.__name__
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    for c in consts:
        lines.append(f'    printf("const {c} %lld\\n", (long long)({c}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            *key, val = ln.split(" ")
            got[" ".join(key)] = int(val)
    for cls in structs:
        name = cls.__name__
        assert got[f"{name} size"] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[f"{name} {field}"] == getattr(cls, field).offset, (name, field)
    for c in consts:
        assert got[f"const {c}"] == getattr(b, c), c


def test_binding_has_every_entry_point():
    """The Python binding offers every C entry point under its C name."""
    import paper_1603_08357_gb300.binding as b
    declared = _declared("ccl.h")
    assert len(declared) >= 20
    assert [d for d in declared if not callable(getattr(b, d, None))] == []


def test_site_count_limit_rejected_before_any_cuda_call(lib_path):
    """n_sites above CCL_MAX_SITES (2^31 - 4097) is refused by the argument
    checks, before the device is touched (the allocation-free entry needs no
    context, so this runs without a GPU)."""
    import paper_1603_08357_gb300.binding as b
    assert b.CCL_MAX_SITES == 2 ** 31 - 4097
    lib = ctypes.CDLL(lib_path)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.ccl_label_noalloc.argtypes = [I32, I64, P, P, P, P, P]
    for n in (b.CCL_MAX_SITES + 1, 2 ** 31 - 1):
        assert lib.ccl_label_noalloc(n, 0, 16, None, None, 16, None) == b.CCL_ERR_INVALID_ARGUMENT
