"""The C ABI library builds, loads and exports every entry point of include/mehdg.h (no GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mehdg.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2302_10917_gb300 import LIB_PATH, _build, load_library
    if not os.path.exists(LIB_PATH):
        _build.build()
    return load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hdg_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hdg_create", "hdg_condense", "hdg_apply", "hdg_solve", "hdg_recover", "hdg_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2302_10917_gb300 import LIB_PATH
    out = subprocess.run(["nm", "-D", "--defined-only", LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hdg_[a-z_0-9]+)$", out, flags=re.M))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_library_is_sm103a_only():
    from paper_2302_10917_gb300 import LIB_PATH
    res = subprocess.run(["/usr/local/cuda/bin/cuobjdump", "--list-elf", LIB_PATH], capture_output=True, text=True)
    if res.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    archs = set(re.findall(r"sm_(\d+a?)", res.stdout))
    assert archs == {"103a"}, archs


def test_argument_validation_without_gpu(lib):
    from paper_2302_10917_gb300 import HDG_ERR_ARG, MeshDesc
    d = MeshDesc()
    d.n, d.m, d.p = 0, 2, 2
    d.kappa0, d.tau_len = 1.0, 1.0
    h = ctypes.c_void_p()
    assert lib.hdg_create(ctypes.byref(d), None, ctypes.byref(h)) == HDG_ERR_ARG
    assert not h.value
    d.n, d.p = 2, 9
    assert lib.hdg_create(ctypes.byref(d), None, ctypes.byref(h)) == HDG_ERR_ARG
    d.p, d.bc[1] = 2, 1          # Neumann sides are not accepted
    assert lib.hdg_create(ctypes.byref(d), None, ctypes.byref(h)) == HDG_ERR_ARG
    d.bc[1], d.kappa0 = 0, -1.0
    assert lib.hdg_create(ctypes.byref(d), None, ctypes.byref(h)) == HDG_ERR_ARG
    assert lib.hdg_create(None, None, ctypes.byref(h)) == HDG_ERR_ARG
    assert lib.hdg_last_error(None) == b"null context"
    lib.hdg_destroy(None)


def _null_args(fn):
    args = []
    for t in fn.argtypes or []:
        if t in (ctypes.c_int, ctypes.c_int64, ctypes.c_uint, ctypes.c_size_t, ctypes.c_long):
            args.append(0)
        elif t in (ctypes.c_double, ctypes.c_float):
            args.append(0.0)
        else:
            args.append(None)
    return args


def test_every_entry_point_refuses_a_null_context(lib):
    """Each call that takes a context returns HDG_ERR_ARG for NULL (and NULL
    arguments) before any device work: no crash, no CUDA call."""
    from paper_2302_10917_gb300 import EXPORTED, HDG_ERR_ARG
    skip = {"hdg_create", "hdg_last_error", "hdg_destroy"}
    checked = 0
    for name in EXPORTED:
        if name in skip:
            continue
        fn = getattr(lib, name)
        assert fn.argtypes, name
        assert fn(*_null_args(fn)) == HDG_ERR_ARG, name
        checked += 1
    assert checked == len(EXPORTED) - len(skip)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without the built library the package raises instead of computing."""
    import paper_2302_10917_gb300 as pkg
    monkeypatch.setattr(pkg, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        pkg.load_library(str(tmp_path / "libmehdg.so"))


def test_no_cpu_path_without_a_gpu():
    """On a machine without a CUDA device a problem cannot be created (there is no CPU route)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2302_10917_gb300 import Problem
    with pytest.raises(RuntimeError):
        Problem(2, 2, 2)
