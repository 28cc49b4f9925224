"""The C-ABI library builds for sm_103a, loads, and exports every entry
point include/hfdib.h declares (no compute calls: no GPU needed)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hfdib.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hfdib_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2606_06135_gb300 import build
    return build.build()


def test_header_declares_the_path():
    names = declared_functions()
    for need in ("hfdib_create", "hfdib_simple_sweep", "hfdib_solve_steady", "hfdib_get_field",
                 "hfdib_destroy"):
        assert need in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hfdib_[a-z_0-9]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binds(libpath):
    from paper_2606_06135_gb300 import hfdib
    lib = hfdib.load_library(libpath)
    for n in declared_functions():
        assert hasattr(lib, n)
    o = hfdib.default_options()
    assert o.urf_u == 0.7 and o.urf_p == 0.3 and o.urf_turb == 0.85 and o.n_u == 2
    assert lib.hfdib_error_string(-1) == b"invalid argument"


def test_create_rejects_bad_arguments_without_touching_the_gpu(libpath):
    import ctypes as C
    from paper_2606_06135_gb300 import hfdib
    lib = hfdib.load_library(libpath)
    h = C.c_void_p()
    g = hfdib.Grid(1, 4, 1, 0, 0, 0, 1, 1, 1)      # nx < 2
    bc = hfdib.Bc()
    rc = lib.hfdib_create(C.byref(g), C.c_void_p(8), None, 1, 100.0, C.byref(bc), None, None, C.byref(h))
    assert rc == -1
    g = hfdib.Grid(4, 4, 1, 0, 0, 0, 1, 1, 1)
    rc = lib.hfdib_create(C.byref(g), C.c_void_p(8), None, 7, 100.0, C.byref(bc), None, None, C.byref(h))
    assert rc == -1                                   # bad model
    rc = lib.hfdib_create(C.byref(g), C.c_void_p(8), None, 2, 100.0, C.byref(bc), None, None, C.byref(h))
    assert rc == -1                                   # SST without wall distance


def test_force_and_wall_shear_reject_null_handles_without_touching_the_gpu(libpath):
    import ctypes as C
    import numpy as np
    from paper_2606_06135_gb300 import hfdib
    lib = hfdib.load_library(libpath)
    out = np.zeros(6)
    assert lib.hfdib_ib_force(None, out.ctypes.data) == -1
    n = C.c_int64(-5)
    assert lib.hfdib_wall_shear(None, 2, None, C.byref(n)) == -1
    assert n.value == -5


def _header_structs():
    """typedef struct { ... } name; of include/hfdib.h as name -> [(field,
    c type, array length)], comments removed, in declaration order."""
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct\s*\{(.*?)\}\s*(\w+)\s*;", src, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            ctype, names = decl.split(" ", 1)
            for nm in names.split(","):
                nm = nm.strip()
                m = re.match(r"(\w+)(?:\[(\d+)\])?$", nm)
                fields.append((m.group(1), ctype, int(m.group(2)) if m.group(2) else 1))
        out[name] = fields
    return out


def test_binding_structs_match_the_header():
    """The ctypes mirrors of hfdib_grid, hfdib_bc, hfdib_options and
    hfdib_tune list the header's fields in the same order with the same types
    (an options field added on one side only would shift every later one)."""
    import ctypes as C
    from paper_2606_06135_gb300 import hfdib
    ctype_of = {"int32_t": C.c_int32, "double": C.c_double}
    structs = _header_structs()
    for cname, pyc in (("hfdib_grid", hfdib.Grid), ("hfdib_bc", hfdib.Bc), ("hfdib_options", hfdib.Options),
                       ("hfdib_tune", hfdib.Tune)):
        want = structs[cname]
        got = pyc._fields_
        assert [f[0] for f in got] == [w[0] for w in want], cname
        for (fname, ftype), (_, ctype, n) in zip(got, want):
            base = ctype_of[ctype]
            expect = base * n if n > 1 else base
            assert ftype == expect or (n > 1 and ftype._type_ == base and ftype._length_ == n), (cname, fname)


def test_set_allocator_rejects_half_a_hook(libpath):
    """hfdib_set_allocator takes both callbacks or neither (no GPU touched)."""
    from paper_2606_06135_gb300 import hfdib
    lib = hfdib.load_library(libpath)
    keep = hfdib.FREE_FN(lambda p, n, s, c: None)
    assert lib.hfdib_set_allocator(hfdib.ALLOC_FN(), keep, None) == -1
    keep2 = hfdib.ALLOC_FN(lambda n, s, c: None)
    assert lib.hfdib_set_allocator(keep2, hfdib.FREE_FN(), None) == -1
    assert lib.hfdib_set_allocator(hfdib.ALLOC_FN(), hfdib.FREE_FN(), None) == 0
