"""The ctypes structures of the binding mirror the C header's irk_options,
irk_kernel_options and irk_stats field for field (names, order and C types), so that a struct
passed across the ABI has the library's layout."""
import ctypes
import os
import re

from paper_1701_07181_gb300 import irk

HEADER = os.path.join(os.path.dirname(__file__), "..", "include", "irk_gb300.h")

CTYPE = {"int": ctypes.c_int, "double": ctypes.c_double, "long long": ctypes.c_longlong,
         "void *": ctypes.c_void_p, "const double *": ctypes.POINTER(ctypes.c_double),
         "const int32_t *": ctypes.POINTER(ctypes.c_int32)}


def header_fields(name):
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    end = src.index("} %s;" % name)
    start = src.rindex("typedef struct {", 0, end) + len("typedef struct {")
    fields = []
    for decl in src[start:end].split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        mm = re.match(r"((?:const )?(?:long long|int32_t|double|int|void)\s*\*?)\s*(.*)", decl)
        assert mm, decl
        ctype = mm.group(1).replace(" *", " *").strip()
        if ctype.endswith("*") and not ctype.endswith(" *"):
            ctype = ctype[:-1].strip() + " *"
        for nm in mm.group(2).split(","):
            nm = nm.strip()
            if nm.startswith("*"):
                ctype, nm = ctype + " *", nm[1:].strip()
            fields.append((nm, ctype))
    return fields


def same_type(a, b):
    return ctypes.sizeof(a) == ctypes.sizeof(b) and getattr(a, "_type_", None) == getattr(b, "_type_", None)


def test_options_mirror_header():
    hdr = header_fields("irk_options")
    py = [(n, t) for n, t in irk.Options._fields_]
    assert [n for n, _ in hdr] == [n for n, _ in py]
    for (n, ct), (_, pt) in zip(hdr, py):
        assert same_type(CTYPE[ct], pt), (n, ct, pt)


def test_stats_mirror_header():
    hdr = header_fields("irk_stats")
    py = [(n, t) for n, t in irk.Stats._fields_]
    assert [n for n, _ in hdr] == [n for n, _ in py]
    for (n, ct), (_, pt) in zip(hdr, py):
        assert same_type(CTYPE[ct], pt), (n, ct, pt)


def test_kernel_options_mirror_header():
    hdr = header_fields("irk_kernel_options")
    py = [(n, t) for n, t in irk.KernelOptions._fields_]
    assert [n for n, _ in hdr] == [n for n, _ in py]
    for (n, ct), (_, pt) in zip(hdr, py):
        assert same_type(CTYPE[ct], pt), (n, ct, pt)
