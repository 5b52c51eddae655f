"""The Python binding's structures against the C header.

`paper_2508_08702_gb300/msp.py` passes `msp_opts` and `msp_stats` by
pointer; a field missing, misplaced or of the wrong width there would shift
every later field without any error.  These tests compile a small C program
against include/msp.h with the host compiler and compare the field names,
order, offsets and sizes with the ctypes structures, and check that every
default the header documents in brackets is what msp_default_opts() writes.
The argument and return types the binding declares for every function are
compared with the header's prototypes the same way.  No device is needed.
"""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "msp.h")

C_TYPES = {"int64_t": ctypes.c_int64, "int32_t": ctypes.c_int32, "uint64_t": ctypes.c_uint64,
           "int": ctypes.c_int, "double": ctypes.c_double}


def header_struct(name):
    """[(C type, field name, bracketed default or None)] of `typedef struct {...} name;`."""
    src = open(HEADER).read()
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", src)
    assert m, name
    fields = []
    for line in m.group(1).splitlines():
        f = re.match(r"\s*(int64_t|int32_t|uint64_t|int|double)\s+(\w+)\s*;(.*)", line)
        if f:
            d = re.search(r"/\*\s*\[([^\]]+)\]", f.group(3))
            fields.append((f.group(1), f.group(2), d.group(1) if d else None))
    return fields


def msp():
    from paper_2508_08702_gb300 import msp as M
    return M


@pytest.mark.parametrize("name", ["msp_opts", "msp_stats"])
def test_binding_fields_follow_the_header(name):
    py = getattr(msp(), name)
    hdr = header_struct(name)
    assert [n for _, n, _ in hdr] == [n for n, _ in py._fields_]
    for (ctype, fname, _), (pname, ptype) in zip(hdr, py._fields_):
        assert ctypes.sizeof(C_TYPES[ctype]) == ctypes.sizeof(ptype), fname


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    """Offsets and sizes of both structures as the host C compiler lays them out."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no host C compiler")
    d = tmp_path_factory.mktemp("layout")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "msp.h"', "int main(void) {"]
    for name in ("msp_opts", "msp_stats"):
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for _, f, _ in header_struct(name):
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    lay = {}
    for line in out.splitlines():
        s, f, v = line.split()
        lay[(s, f)] = int(v)
    return lay


@pytest.mark.parametrize("name", ["msp_opts", "msp_stats"])
def test_binding_offsets_equal_the_c_layout(c_layout, name):
    py = getattr(msp(), name)
    assert ctypes.sizeof(py) == c_layout[(name, "size")]
    for fname, _ in py._fields_:
        assert getattr(py, fname).offset == c_layout[(name, fname)], fname


def _value(text):
    t = text.strip()
    if "<<" in t:
        a, b = t.split("<<")
        return int(a, 0) << int(b, 0)
    try:
        return int(t, 0)
    except ValueError:
        return float(t)


def test_documented_defaults_are_the_library_defaults():
    from paper_2508_08702_gb300 import build
    try:
        path = build.build()
    except (RuntimeError, FileNotFoundError) as e:   # no nvcc on this machine
        pytest.skip(f"cannot build the CUDA library here: {e}")
    lib = ctypes.CDLL(path)
    o = msp().msp_opts()
    lib.msp_default_opts(ctypes.byref(o))
    documented = [(f, d) for _, f, d in header_struct("msp_opts")]
    assert all(d is not None for _, d in documented), [f for f, d in documented if d is None]
    for f, d in documented:
        assert getattr(o, f) == _value(d), (f, d, getattr(o, f))


SCALARS = {"int": ctypes.c_int, "int64_t": ctypes.c_int64, "uint64_t": ctypes.c_uint64,
           "double": ctypes.c_double, "float": ctypes.c_float, "size_t": ctypes.c_size_t}


def header_prototypes():
    """{name: (return type text, [parameter type texts])} of the MSP_API functions."""
    src = re.sub(r"/\*.*?\*/", " ", open(HEADER).read(), flags=re.S)
    out = {}
    for ret, name, params in re.findall(r"MSP_API\s+([\w\s\*]+?)\s*\b(msp_\w+)\s*\(([^)]*)\)\s*;", src):
        ps = [" ".join(p.split()) for p in params.split(",")]
        ps = [] if ps == ["void"] else ps
        # drop the parameter name, keep the type
        types = [re.sub(r"\s*\b\w+$", "", p) if not p.endswith("*") else p for p in ps]
        out[name] = (" ".join(ret.split()), types)
    return out


def _matches(ctext, ct):
    """Whether ctypes type ct passes a C parameter or return value of type ctext."""
    t = ctext.replace("const ", "").strip()
    if t.endswith("*"):
        if t == "char *":
            return ct is ctypes.c_char_p
        return ct is ctypes.c_void_p or (isinstance(ct, type) and issubclass(ct, ctypes._Pointer))
    if t in ("msp_status", "int"):
        return ct is ctypes.c_int
    return ct is SCALARS[t]


def test_binding_signatures_follow_the_header():
    from paper_2508_08702_gb300 import build
    try:
        build.build()
    except (RuntimeError, FileNotFoundError) as e:   # no nvcc on this machine
        pytest.skip(f"cannot build the CUDA library here: {e}")
    L = msp().load()
    protos = header_prototypes()
    assert len(protos) == len(re.findall(r"^MSP_API", open(HEADER).read(), re.M))
    for name, (ret, params) in protos.items():
        fn = getattr(L, name)
        assert fn.argtypes is not None, name
        assert len(fn.argtypes) == len(params), (name, params)
        for ctext, ct in zip(params, fn.argtypes):
            assert _matches(ctext, ct), (name, ctext, ct)
        if ret == "void":
            assert fn.restype is None, name
        else:
            assert _matches(ret, fn.restype), (name, ret, fn.restype)


def test_header_compiles_as_c_and_cpp(tmp_path):
    """include/msp.h stands alone in C99 and in C++11 (its extern "C" block
    gives the C++ declarations C linkage)."""
    import shutil
    for compiler, std, ext in (("gcc", "-std=c99", "c"), ("g++", "-std=c++11", "cpp")):
        cc = shutil.which(compiler)
        if not cc:
            pytest.skip(f"no {compiler}")
        src = tmp_path / f"use.{ext}"
        src.write_text('#include "msp.h"\nint main(void) { msp_opts o; (void)o; return 0; }\n')
        subprocess.run([cc, std, "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                        "-c", str(src), "-o", str(tmp_path / f"use_{ext}.o")], check=True)
    # the C++ compile sees C linkage: no mangled msp_ names in an object that calls one
    src = tmp_path / "call.cpp"
    src.write_text('#include "msp.h"\nint f() { return msp_mlp_param_count(); }\n')
    obj = tmp_path / "call.o"
    subprocess.run([shutil.which("g++"), "-std=c++11", "-I", os.path.join(ROOT, "include"), "-c", str(src),
                    "-o", str(obj)], check=True)
    nm = shutil.which("nm")
    if nm:
        syms = subprocess.run([nm, str(obj)], check=True, capture_output=True, text=True).stdout
        assert " msp_mlp_param_count" in syms and "_Z19msp_mlp_param_countv" not in syms
