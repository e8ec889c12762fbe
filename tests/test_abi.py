"""The C-ABI library builds, loads without a GPU, and exports every declared symbol."""
import ctypes
import os
import re

import pytest

from paper_2603_28907_gb300 import build as B
from paper_2603_28907_gb300 import mt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "mt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mt_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return ctypes.CDLL(B.OUT)


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    names = set(declared_symbols())
    bound = set(mt.SIGNATURES) | {"mt_last_error", "mt_server_last_error"}
    assert names == bound, names ^ bound


def test_build_targets_sm103a_only():
    flags = B._flags(False)
    assert flags[:2] == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert sum(1 for f in flags if f == "-gencode") == 1


def test_create_fails_cleanly_without_gpu(lib):
    """With no usable device mt_create returns an error code and a message (no abort)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cfg = mt.Config(1, 64, 1.0, 1e4, 150.0, 0.01, 0.99, 0.1)
    lib.mt_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(mt.Config),
                              ctypes.c_void_p]
    lib.mt_last_error.restype = ctypes.c_char_p
    lib.mt_last_error.argtypes = [ctypes.c_void_p]
    h = ctypes.c_void_p()
    st = lib.mt_create(ctypes.byref(h), 0, ctypes.byref(cfg), None)
    assert st == -4  # MT_ECUDA
    assert h.value is None
    assert b"device" in lib.mt_last_error(None)


def test_create_rejects_bad_config(lib):
    lib.mt_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(mt.Config),
                              ctypes.c_void_p]
    h = ctypes.c_void_p()
    for bad in (mt.Config(7, 64, 1.0, 1e4, 150.0, 0.01, 0.99, 0.1),
                mt.Config(1, 0, 1.0, 1e4, 150.0, 0.01, 0.99, 0.1),
                mt.Config(1, 64, -1.0, 1e4, 150.0, 0.01, 0.99, 0.1),
                mt.Config(1, 64, 1.0, 1e4, 150.0, 0.01, 1.0, 0.1)):
        assert lib.mt_create(ctypes.byref(h), 0, ctypes.byref(bad), None) == -1  # MT_EINVAL


def test_null_context_calls_return_einval(lib):
    lib.mt_logpost.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p]
    assert lib.mt_logpost(None, 1, None, None, None) == -1
    assert lib.mt_destroy(None) == 0


def test_bounds_checked_variant_builds_with_the_same_abi(lib):
    """libmt_checked.so (MT_BOUNDS_CHECK) compiles, loads without a GPU and
    exports the same symbols as the production library."""
    path = B.build(checked=True)
    assert path == B.OUT_CHECKED and path != B.OUT
    chk = ctypes.CDLL(path)
    for n in declared_symbols():
        assert hasattr(chk, n), n


def test_server_calls_fail_cleanly_without_gpu(lib):
    """The serving calls return error codes with a message (no abort) when
    there is no device or no server."""
    import torch
    lib.mt_server_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_size_t,
                                     ctypes.c_int]
    lib.mt_server_last_error.restype = ctypes.c_char_p
    lib.mt_server_last_error.argtypes = [ctypes.c_void_p]
    h = ctypes.c_void_p()
    assert lib.mt_server_create(ctypes.byref(h), 0, 0, 1) == -1        # no budget
    assert lib.mt_server_create(ctypes.byref(h), 0, 1 << 30, 0) == -1  # no slot
    if not torch.cuda.is_available():
        assert lib.mt_server_create(ctypes.byref(h), 0, 1 << 30, 1) == -4  # MT_ECUDA
        assert h.value is None
        assert b"device" in lib.mt_server_last_error(None)
    lib.mt_server_submit.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.mt_server_cancel.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    lib.mt_server_stats.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.mt_server_submit(None, None, None) == -1
    assert lib.mt_server_cancel(None, 1) == -1
    assert lib.mt_server_stats(None, None) == -1
    lib.mt_server_destroy.argtypes = [ctypes.c_void_p]
    assert lib.mt_server_destroy(None) == 0


def test_binding_fails_loudly_without_the_library(monkeypatch):
    """No fallback: with the library missing, the binding raises."""
    monkeypatch.setattr(mt, "_lib", None)
    monkeypatch.setattr(mt, "LIB_PATH", os.path.join(ROOT, "no_such_dir", "libmt.so"))
    with pytest.raises(RuntimeError, match="missing"):
        mt.load()


def test_header_is_self_contained_c_and_cpp():
    """include/mt.h compiles on its own as C99 and as C++11, warnings as errors."""
    import shutil
    import subprocess
    if not shutil.which("gcc") or not shutil.which("g++"):
        pytest.skip("no host compiler")
    hdr = os.path.join(ROOT, "include", "mt.h")
    for cc, lang, std in (("gcc", "c", "-std=c99"), ("g++", "c++", "-std=c++11")):
        r = subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                            "-x", lang, hdr], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_plain_c_client_links_and_calls(lib, tmp_path):
    """A C99 program that includes only mt.h links against libmt.so, can take
    the address of every declared call, and gets a status code back from
    mt_create (MT_ECUDA without a device)."""
    import shutil
    import subprocess
    import torch
    if not shutil.which("gcc"):
        pytest.skip("no host compiler")
    names = declared_symbols()
    src = ["#include <stdio.h>", '#include "mt.h"', "int main(void) {",
           "    void *fns[] = {" + ", ".join(f"(void *)&{n}" for n in names) + "};",
           "    mt_config cfg = {MT_PREC_F32, 64, 1.0, 1e4, 150.0, 0.01, 0.99, 0.1};",
           "    mt_ctx *ctx = NULL;",
           "    mt_status st = mt_create(&ctx, 0, &cfg, NULL);",
           '    printf("%d %d\\n", (int)st, (int)(sizeof fns / sizeof fns[0]));',
           "    if (ctx) mt_destroy(ctx);",
           "    return 0;", "}"]
    c = tmp_path / "client.c"
    c.write_text("\n".join(src) + "\n")
    exe = tmp_path / "client"
    libdir = os.path.dirname(B.OUT)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", str(c), "-I", os.path.join(ROOT, "include"),
                        "-L", libdir, "-l:" + os.path.basename(B.OUT), f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    st, n = map(int, out.stdout.split())
    assert n == len(names)
    assert st == (0 if torch.cuda.is_available() else -4)
