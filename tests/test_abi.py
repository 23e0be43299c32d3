"""The C-ABI library loads and exports every entry point include/discos.h
declares; host-side logic of the library (the F^P table builder) agrees with
the oracle.  No GPU needed."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "discos.h")).read()
    return sorted(set(re.findall(r"\b(discos_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2204_14167_gb300 import build as b
    b.build()
    from paper_2204_14167_gb300 import _lib
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "discos_create" in names and "discos_step" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_2204_14167_gb300 import _lib
    assert set(_declared()) == set(_lib.EXPORTS)


@pytest.mark.parametrize("kernel,psi,n", [(0, 4.0, 16), (1, 4.0, 8)])
def test_fp_table_host_matches_oracle(lib, kernel, psi, n):
    """Sec. II.B.1 table: the library's host builder (its own lattice Green's
    function and quadrature) against the oracle's."""
    import paper_2204_14167_gb300 as dg
    from oracle import greens
    a = np.array(dg.fp_table(kernel, psi, n))
    b = greens.fp_table(kernel, psi, n)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


def test_invalid_table_arguments(lib):
    import ctypes
    out = (ctypes.c_double * 4)()
    assert lib.discos_fp_table(7, 6, 8.0, 4.0, 3, out) != 0
    assert lib.discos_fp_table(0, 6, 8.0, -1.0, 3, out) != 0


def test_binding_rejects_bad_arrays():
    """The Python binding refuses arrays the library would read past or
    misread (host tensors, wrong type, too few elements, non-contiguous)
    before any library call."""
    import pytest
    torch = pytest.importorskip("torch")
    import paper_2204_14167_gb300 as dg
    dg._need(None, 10, torch.float32, "q")                        # optional argument
    for bad in (torch.zeros(10), torch.zeros(5, dtype=torch.float32), torch.zeros(20, dtype=torch.float32)[::2]):
        with pytest.raises(ValueError):
            dg._need(bad, 10, torch.float32, "q")                 # on the host, short, or strided


def _c_offsets(struct, fields):
    """offsetof() of each field and sizeof() of the struct, from a tiny C
    program compiled against include/discos.h with the host compiler."""
    import shutil
    import subprocess
    import tempfile
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(ROOT, "include")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "discos.h"', "int main(void) {"]
    lines.append(f'  printf("size %zu\\n", sizeof({struct}));')
    for f in fields:
        lines.append(f'  printf("{f} %zu\\n", offsetof({struct}, {f}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "l.c"), os.path.join(d, "l")
        open(src, "w").write("\n".join(lines))
        subprocess.run([cc, "-I", inc, src, "-o", exe], check=True, capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (l.split() for l in out.splitlines())}


@pytest.mark.parametrize("pystruct,cstruct", [("Config", "discos_config"), ("Batch", "discos_batch")])
def test_binding_struct_layout_matches_header(pystruct, cstruct):
    """The ctypes mirrors of the C structs have the header's field offsets
    and size, so the library reads every field the binding writes."""
    import ctypes
    from paper_2204_14167_gb300 import _lib
    S = getattr(_lib, pystruct)
    names = [f[0] for f in S._fields_]
    c = _c_offsets(cstruct, names)
    assert c["size"] == ctypes.sizeof(S)
    for n in names:
        assert c[n] == getattr(S, n).offset, n


def _prototypes():
    """(name, return type, [parameter types]) of every function the header
    declares, comments stripped."""
    src = open(os.path.join(ROOT, "include", "discos.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    out = []
    for m in re.finditer(r"([A-Za-z_][A-Za-z_0-9 \*]*?)\b(discos_[a-z_0-9]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
        params = " ".join(m.group(3).split())
        types = []
        if params != "void":
            for p in params.split(","):
                p = p.strip()
                # drop the parameter name: the last identifier when it follows a type
                t = re.sub(r"\s*\b[A-Za-z_][A-Za-z_0-9]*$", "", p) if re.search(r"[\s\*][A-Za-z_]\w*$", p) else p
                types.append(" ".join(t.replace("*", " * ").split()))
        ret = " ".join(m.group(1).replace("*", " * ").split())
        out.append((m.group(2), ret, types))
    return out


def _ctype_kind(t):
    """The ctypes class family one C parameter type must be bound with."""
    import ctypes
    if "*" in t or t in ("discos_alloc_fn", "discos_free_fn"):
        return "pointer"
    scalar = {"int": ctypes.c_int, "int64_t": ctypes.c_int64, "double": ctypes.c_double, "float": ctypes.c_float,
              "unsigned": ctypes.c_uint, "size_t": ctypes.c_size_t, "long long": ctypes.c_longlong}
    return scalar[t.replace("const ", "")]


def _is_pointer_type(ct):
    import ctypes
    return ct in (ctypes.c_void_p, ctypes.c_char_p) or issubclass(ct, ctypes._Pointer)


def test_binding_prototypes_match_header(lib):
    """Every entry point is called with the header's number of arguments,
    each bound with a matching ctypes type (a pointer for a pointer, the
    same integer width, double for double), and returns what the header
    says: a wrong width or a missing argument would hand the library garbage."""
    import ctypes
    protos = _prototypes()
    assert len(protos) == len(_declared())
    for name, ret, types in protos:
        fn = getattr(lib, name)
        if types:
            assert fn.argtypes is not None and len(fn.argtypes) == len(types), name
            for i, (t, ct) in enumerate(zip(types, fn.argtypes)):
                kind = _ctype_kind(t)
                if kind == "pointer":
                    assert _is_pointer_type(ct), (name, i, t, ct)
                else:
                    assert ct is kind or ctypes.sizeof(ct) == ctypes.sizeof(kind) and ct._type_ == kind._type_, \
                        (name, i, t, ct)
        else:
            assert not fn.argtypes, name
        if ret == "discos_status":
            assert fn.restype is ctypes.c_int, name
        elif ret == "const char *":
            assert fn.restype is ctypes.c_char_p, name
        elif ret == "long long":
            assert fn.restype is ctypes.c_longlong, name
        else:
            raise AssertionError(f"{name}: unexpected return type {ret!r}")
