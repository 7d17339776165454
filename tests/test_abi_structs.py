"""The ctypes structures of the binding declare the fields of include/lbm.h's structures, with the
same names, in the same order and with matching C types, so that the binding and the library agree
on every offset (checked on the CPU, without loading the library)."""
import ctypes as C
import keyword
import os
import re

import pytest

from paper_2606_20646_b300 import lbm

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "lbm.h")
STRUCTS = ["lbm_grid", "lbm_shape", "lbm_material", "lbm_group", "lbm_levelset", "lbm_bc", "lbm_options",
           "lbm_info", "lbm_kernel_time", "lbm_tuning", "lbm_diag"]

# C scalar and pointer spellings of the header -> the ctypes type the binding must use
_SCALAR = {"int": C.c_int, "double": C.c_double, "long long": C.c_longlong, "size_t": C.c_size_t,
           "float": C.c_float}


def _c_fields(name):
    """(field, C type, array length) of `typedef struct name { ... } name;` in declaration order."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    m = re.search(r"typedef struct %s\s*\{(.*?)\}\s*%s\s*;" % (name, name), text, flags=re.S)
    assert m, name
    out = []
    for decl in m.group(1).split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        first, *rest = [d.strip() for d in decl.split(",")]
        mm = re.match(r"(const\s+)?([A-Za-z_][A-Za-z_ ]*?)\s*(\*?)\s*([A-Za-z_]\w*)(\[(\d+)\])?$", first)
        assert mm, (name, decl)
        ctype = mm.group(2).strip() + (" *" if mm.group(3) else "")
        names = [(mm.group(4), mm.group(6))]
        for r in rest:
            rr = re.match(r"(\*?)\s*([A-Za-z_]\w*)(\[(\d+)\])?$", r)
            assert rr, (name, decl)
            names.append((rr.group(2), rr.group(4)))
        for n, length in names:
            out.append((n, ctype, int(length) if length else None))
    return out


@pytest.mark.parametrize("name", STRUCTS)
def test_binding_structures_match_the_header(name):
    fields = _c_fields(name)
    py = getattr(lbm, name)._fields_
    # a C field named after a Python keyword is spelled with a trailing underscore in the binding
    pynames = [f[0][:-1] if f[0].endswith("_") and keyword.iskeyword(f[0][:-1]) else f[0] for f in py]
    assert pynames == [f[0] for f in fields], name
    for (pname, ptype), (cname, ctype, length) in zip(py, fields):
        if ctype.endswith("*"):
            assert issubclass(ptype, (C.c_void_p, C._Pointer)) or ptype in (C.c_void_p, C.c_char_p), (name, cname)
            continue
        want = _SCALAR.get(ctype)
        if want is None:       # a nested structure or an enum-typed int
            continue
        if length:
            assert issubclass(ptype, C.Array) and ptype._length_ == length and ptype._type_ == want, (name, cname)
        else:
            assert ptype == want, (name, cname, ptype, want)
