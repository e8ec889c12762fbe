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


def _header_prototypes():
    txt = open(os.path.join(ROOT, "include", "mt.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    protos = {}
    for m in re.finditer(r"MT_API\s+[\w\s\*]*?\b(mt_[a-z_0-9]+)\s*\(([^)]*)\)", txt):
        params = [p.strip() for p in m.group(2).split(",") if p.strip() and p.strip() != "void"]
        protos[m.group(1)] = params
    return protos


def _ctype_class(param):
    """Broad class of a C parameter: 'ptr:<pointee>' or the scalar type."""
    p = re.sub(r"\bconst\b", "", param)
    if "[" in p:                                  # an array parameter is a pointer
        p = p.split()[0] + " *"
    if "*" in p:
        pointee = p.split("*")[0].split()
        return "ptr:" + (pointee[-1] if pointee else "")
    return p.split()[0]


def test_binding_signatures_match_the_header():
    """Every ctypes signature has the header's arity, and each argument the
    header's scalar type (int, double, int64_t, uint64_t, size_t) or a
    pointer (with the pointee type where the binding names one)."""
    import ctypes as C
    scalar = {"int": C.c_int, "double": C.c_double, "int64_t": C.c_int64, "uint64_t": C.c_uint64,
              "size_t": C.c_size_t}
    pointee = {"double": C.c_double, "int": C.c_int, "int64_t": C.c_int64}
    protos = _header_prototypes()
    for name, args in mt.SIGNATURES.items():
        params = protos[name]
        assert len(params) == len(args), (name, params, args)
        for p, a in zip(params, args):
            k = _ctype_class(p)
            if k.startswith("ptr:"):
                assert a is C.c_void_p or hasattr(a, "_type_") and issubclass(a, C._Pointer), (name, p, a)
                t = k[4:]
                if a is not C.c_void_p and t in pointee:
                    assert a._type_ is pointee[t], (name, p, a)
            else:
                assert a is scalar[k], (name, p, a)


def test_struct_layouts_match_the_header(tmp_path):
    """sizeof and every field offset of the ABI structs, as a C compiler lays
    them out, equal the binding's ctypes structures."""
    import ctypes as C
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("no host compiler")
    structs = {"mt_config": mt.Config, "mt_request": mt.Request, "mt_request_info": mt.RequestInfo,
               "mt_server_stats_t": mt.ServerStats}
    src = ["#include <stdio.h>", "#include <stddef.h>", '#include "mt.h"', "int main(void) {"]
    for cname, cls in structs.items():
        src.append(f'    printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for f, _ in cls._fields_:
            src.append(f'    printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    src += ["    return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", str(c), "-I", os.path.join(ROOT, "include"),
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {(a, b): int(v) for a, b, v in (l.split() for l in out if l)}
    for cname, cls in structs.items():
        assert got[(cname, "sizeof")] == C.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_run_traced_reads_the_state_after_every_super_step():
    """Context.run_traced (host loop over the ABI calls): one super-step per
    mt_run, then mt_get_state into that super-step's row of each trace."""
    import numpy as np
    calls = []
    ctx = object.__new__(mt.Context)
    ctx.run = lambda kernel, step, n_super, n_within: calls.append(("run", kernel, step, n_super, n_within))
    ctx.get_state = lambda h, ll, lp, acc: calls.append(("state", h, ll.base is not None, lp.shape, acc))
    ll, lp = np.zeros((3, 5)), np.zeros((3, 5))
    ctx.run_traced(mt.KERNEL_RW, 0.01, 3, 10, ll, lp)
    assert calls[0::2] == [("run", mt.KERNEL_RW, 0.01, 1, 10)] * 3
    assert all(c[0] == "state" and c[1] is None and c[2] and c[3] == (5,) and c[4] is None
               for c in calls[1::2])
