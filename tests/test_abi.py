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
