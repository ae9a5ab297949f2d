"""The C ABI library builds, loads without a GPU, exports every declared symbol, and
rejects invalid descriptors before touching the device."""
import ctypes
import os
import re

import pytest

from paper_2306_09760_gb300 import build as wbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    wbuild.build()
    from paper_2306_09760_gb300 import wcns
    return wcns


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(inc, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(wcns_[a-z0-9_]+)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("wcns_init", "wcns_rhs", "wcns_step", "wcns_adjoint_step", "wcns_batch_init",
                     "wcns_batch_step", "wcns_reduce", "wcns_sync_status", "wcns_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    L = lib.load()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings_and_defaults(lib):
    assert lib.wcns_status_string(0) == "ok"
    assert "argument" in lib.wcns_status_string(1)
    p = lib.wcns_default_params(lib.WCNS_EULER, lib.WCNS_F64)
    assert p.weights == lib.WEIGHTS["FE"] and p.flux == lib.FLUXES["HLLC"]
    assert p.xi == 1e6 and p.kappa == 0.5 and p.eps == 1e-40
    p32 = lib.wcns_default_params(lib.WCNS_EULER, lib.WCNS_F32)
    assert p32.eps == 1e-30
    with pytest.raises(lib.WcnsError):
        lib.wcns_default_params(7, 0)


def _grid(lib, **kw):
    g = lib.wcns_grid()
    g.ndim, g.nvar, g.dtype, g.nx, g.ny, g.pitch = 1, 3, 0, 100, 1, 128
    g.lo[0], g.hi[0] = 0.0, 1.0
    g.bc[0] = 1
    for k, v in kw.items():
        setattr(g, k, v)
    return g


@pytest.mark.parametrize("bad", [dict(pitch=100), dict(pitch=64), dict(nx=0), dict(ny=0), dict(ndim=3),
                                 dict(nvar=2), dict(dtype=5), dict(reserved=1)])
def test_init_rejects_bad_grid_without_gpu(lib, bad):
    p = lib.wcns_default_params(lib.WCNS_EULER, lib.WCNS_F64)
    with pytest.raises(lib.WcnsError) as e:
        lib.wcns_init(_grid(lib, **bad), p)
    assert e.value.status == lib.WCNS_ERR_ARG


def test_init_rejects_bad_params_without_gpu(lib):
    g = _grid(lib)
    for field, val, code in (("z_p", 3, 1), ("weights", 9, 1), ("eps", 0.0, 1), ("system", 0, 5),
                             ("integrator", 2, 1), ("family", 2, 1)):
        p = lib.wcns_default_params(lib.WCNS_EULER, lib.WCNS_F64)
        setattr(p, field, val)
        with pytest.raises(lib.WcnsError) as e:
            lib.wcns_init(g, p)
        assert e.value.status == code, field
    # single precision JS weights need eps^2 to stay a normal float
    g32 = _grid(lib, dtype=1)
    p = lib.make_params(lib.WCNS_EULER, lib.WCNS_F32, weights="JS")
    with pytest.raises(lib.WcnsError):
        lib.wcns_init(g32, p)


def test_batch_init_rejects_bad_layout_without_gpu(lib):
    import numpy as np
    p = lib.make_params(lib.WCNS_EULER, lib.WCNS_F64)
    for offs, sizes, total in (([0, 50], [100, 100], 200),   # overlapping problems
                               ([0, 150], [100, 100], 200),  # past the end
                               ([0], [0], 10)):              # empty problem
        with pytest.raises(lib.WcnsError) as e:
            lib.wcns_batch_init(np.array(offs), np.array(sizes), total, 0.0, 1.0, 1, p, lib.WCNS_F64)
        assert e.value.status == lib.WCNS_ERR_ARG
    with pytest.raises(lib.WcnsError) as e:
        lib.wcns_batch_init(np.array([0]), np.array([10]), 10, 0.0, 1.0, 1, p, lib.WCNS_F64, tile=100)
    assert e.value.status == lib.WCNS_ERR_ARG


def test_every_unit_is_built_and_every_family_instantiated():
    """Each .cu file under csrc is a build unit, and each kernel family (x sweeps per
    variable count, y sweeps, adjoints, the banded 2D stage, the rest) is instantiated exactly once per
    element type, so no launcher is left undefined or defined twice at link time."""
    csrc = os.path.join(ROOT, "paper_2306_09760_gb300", "csrc")
    units = sorted(f for f in os.listdir(csrc) if f.endswith(".cu"))
    assert units == sorted(wbuild.UNITS)
    seen = {}
    for f in units:
        for m in re.finditer(r"^WCNS_INSTANTIATE_(X|Y|ADJ|BAND|MISC)\((float|double)(?:, (\d))?\)", open(os.path.join(csrc, f)).read(), re.M):
            key = (m.group(1), m.group(2), m.group(3))
            assert key not in seen, (key, f, seen.get(key))
            seen[key] = f
    for t in ("float", "double"):
        for fam in (("X", t, "1"), ("X", t, "3"), ("X", t, "4"), ("Y", t, None), ("ADJ", t, None), ("BAND", t, None),
                    ("MISC", t, None)):
            assert fam in seen, fam
    assert len(seen) == 14


def test_binding_structures_match_the_header_layout():
    """The binding's ctypes descriptors (wcns_grid, wcns_params, wcns_faces) have the C
    header's size and field offsets: a C program compiled against include/wcns.h prints
    sizeof and offsetof of every field the binding declares."""
    import shutil
    import subprocess
    import tempfile
    from paper_2306_09760_gb300 import wcns
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [wcns.wcns_grid, wcns.wcns_params, wcns.wcns_faces]
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "wcns.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, *_ in st._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", exe, src],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        out = subprocess.run([exe], capture_output=True, text=True, timeout=30).stdout
    c_layout = {}
    for line in out.split("\n"):
        if line.strip():
            a, b, v = line.split()
            c_layout[(a, b)] = int(v)
    for st in structs:
        name = st.__name__
        assert c_layout[(name, "size")] == ctypes.sizeof(st), name
        for field, *_ in st._fields_:
            assert c_layout[(name, field)] == getattr(st, field).offset, (name, field)


def _header_prototypes():
    """name -> (return type, [parameter types]) for every function declared in include/*.h."""
    protos = {}
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if not fn.endswith(".h"):
            continue
        text = re.sub(r"/\*.*?\*/", "", open(os.path.join(inc, fn)).read(), flags=re.S)
        for m in re.finditer(r"^\s*((?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**)\s*(wcns_[a-z0-9_]+)\s*\(([^)]*)\)\s*;",
                             text, re.M):
            params = []
            for p in m.group(3).split(","):
                p = " ".join(p.split())
                if p in ("", "void"):
                    continue
                typ = re.sub(r"\s*\b[A-Za-z_][A-Za-z0-9_]*$", "", p)  # drop the parameter name
                params.append(typ.replace(" *", "*"))
            protos[m.group(2)] = (" ".join(m.group(1).split()).replace(" *", "*"), params)
    return protos


def test_binding_signatures_match_the_header_prototypes(lib):
    """Every entry point's ctypes restype and argtypes agree with its C prototype: scalars
    by exact type, pointers to scalars or descriptors by pointee (or as a void pointer),
    opaque handles and buffers as void pointers, out-handles as pointers to them."""
    L = lib.load()
    scalars = {"double": ctypes.c_double, "int32_t": ctypes.c_int32, "int64_t": ctypes.c_int64,
               "wcns_status": ctypes.c_int}
    structs = {"wcns_grid": lib.wcns_grid, "wcns_params": lib.wcns_params, "wcns_faces": lib.wcns_faces}

    def matches(ctype, ct):
        base = ctype.replace("const ", "").strip()
        if base in scalars:
            return ct is scalars[base]
        if base == "void":
            return ct is None
        if base == "char*":
            return ct is ctypes.c_char_p
        if base in ("void*", "wcns_ctx*", "wcns_batch*"):
            return ct is ctypes.c_void_p
        if base in ("wcns_ctx**", "wcns_batch**"):
            return ct is ctypes.POINTER(ctypes.c_void_p)
        if base.endswith("*") and base.count("*") == 1:
            pointee = base[:-1]
            want = scalars.get(pointee) or structs.get(pointee)
            if pointee == "uint64_t":
                want = ctypes.c_uint64
            return want is not None and (ct is ctypes.c_void_p or ct is ctypes.POINTER(want))
        return False

    protos = _header_prototypes()
    assert len(protos) == len(declared_functions())
    for name, (ret, params) in protos.items():
        f = getattr(L, name)
        assert matches(ret, f.restype), (name, ret, f.restype)
        assert f.argtypes is not None and len(f.argtypes) == len(params), (name, params, f.argtypes)
        for i, (p, ct) in enumerate(zip(params, f.argtypes)):
            assert matches(p, ct), (name, i, p, ct)
