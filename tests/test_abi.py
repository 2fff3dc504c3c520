"""The C-ABI library loads and exports every function include/*.h declares.

No compute call is made here (no GPU needed): only host-side helpers that
touch no device state run.
"""

import ctypes
import glob
import os
import re

import numpy as np
import pytest

from conftest import read_golden

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2601_00976_gb300 import _build, nmc
    if not os.path.exists(nmc.LIB_PATH):
        _build.build()
    return ctypes.CDLL(nmc.LIB_PATH)


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?(?:int|void|char|double)\s*\*?\s*(\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("collision_solve", "opacity_interp", "nmc_create", "nmc_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_the_same_symbols():
    from paper_2601_00976_gb300 import nmc
    assert set(nmc.EXPORTS) <= set(declared_functions())


def test_default_params(lib):
    from paper_2601_00976_gb300 import nmc
    p = nmc.default_params()
    assert p.tol_inner == 1e-10 and p.m_inner == 3 and p.precision == nmc.FP64
    assert p.d_min == 1e-30 and p.final_q == 1 and p.proc_mask == 15


@pytest.mark.parametrize("row", read_golden("energy_grids.txt"))
def test_library_geometric_grid_matches_table(lib, row):
    from paper_2601_00976_gb300 import nmc
    edges, alpha = nmc.geometric_edges(int(row[1]), float(row[3]), 300.0)
    assert abs(alpha - float(row[2])) <= 1e-12 * alpha
    assert float(f"{np.diff(edges)[-1]:.3g}") == pytest.approx(float(row[4]), rel=1e-12)


def test_geometric_grid_rejects_bad_arguments(lib):
    from paper_2601_00976_gb300 import nmc
    with pytest.raises(ValueError):
        nmc.geometric_edges(0, 1.0)
    with pytest.raises(ValueError):
        nmc.geometric_edges(10, 40.0)   # 10 * 40 > 300


def test_create_rejects_null_arguments(lib):
    from paper_2601_00976_gb300 import nmc
    L = nmc.load_library()
    h = ctypes.c_void_p()
    assert L.nmc_create(None, None, ctypes.byref(h)) == nmc.NMC_EINVAL
    assert not h.value
    assert L.nmc_create(None, None, None) == nmc.NMC_EINVAL
    assert L.nmc_last_error(None) == b"no context"


def test_grid_nodes_helper(lib):
    """Context-free node energies and weights agree with the oracle grid."""
    from paper_2601_00976_gb300 import nmc
    from oracle import grid as ogrid
    for nq in (1, 2, 3):
        edges, _ = ogrid.geometric_edges(16, 1.875)
        eps, w2, w3 = nmc.grid_nodes(edges, nq)
        g = ogrid.EnergyGrid(edges, nq)
        assert np.allclose(eps, g.eps, rtol=1e-15)
        assert np.allclose(w2, g.W2, rtol=1e-13)
        assert np.allclose(w3, g.W3, rtol=1e-13)


def test_ctypes_structs_match_the_header(tmp_path):
    """The binding's ctypes mirrors of nmc_grid, nmc_tables and nmc_params have the header's
    field offsets and sizes (compiled with the host C compiler)."""
    import shutil
    import subprocess
    from paper_2601_00976_gb300 import nmc
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {"nmc_grid": nmc.Grid, "nmc_tables": nmc.Tables, "nmc_params": nmc.Params}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nmc.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'    printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for field, _ in py._fields_:
            lines.append(f'    printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c = {(a, b): int(v) for a, b, v in (ln.split() for ln in out if ln)}
    for cname, py in structs.items():
        assert c[(cname, "sizeof")] == ctypes.sizeof(py), cname
        for field, _ in py._fields_:
            assert c[(cname, field)] == getattr(py, field).offset, (cname, field)
