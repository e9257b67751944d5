"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function that include/louvain.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "louvain.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(louvain_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2301_12390_gb300 import louvain
    return louvain.LIB_PATH


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("louvain_create", "louvain_load_csr", "louvain_run", "louvain_get_membership",
                     "louvain_get_modularity", "louvain_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib_path):
    from paper_2301_12390_gb300 import louvain
    bound = {name for name, _, _ in louvain.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_default_options_are_the_papers(lib_path):
    from paper_2301_12390_gb300 import default_options
    o = default_options()
    assert (o.tolerance, o.tolerance_decline, o.pass_tolerance) == (0.01, 10.0, 0.0)
    assert (o.max_iterations, o.max_passes, o.mode) == (20, 10, 0)


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the header struct's size and
    each field at the header's offset (a C program built against
    include/louvain.h prints them)."""
    import shutil
    import subprocess
    from paper_2301_12390_gb300 import louvain as L
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"louvain_options": L.Options, "louvain_stats": L.Stats, "louvain_pass_info": L.PassInfo,
               "louvain_server_config": L.ServerConfig, "louvain_server_result": L.ServerResult}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "louvain.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for field in cls._fields_:
            lines.append(f'  printf("{cname} {field[0]} %zu\\n", offsetof({cname}, {field[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {(a, b): int(c) for a, b, c in (ln.split() for ln in out if ln)}
    for cname, cls in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for field in cls._fields_:
            assert got[(cname, field[0])] == getattr(cls, field[0]).offset, (cname, field[0])


def test_arena_sizing_without_a_device(lib_path):
    """louvain_arena_bytes sizes a context's device arena by a dry run (no GPU
    needed): 68 bytes per CSR entry (input, two coarse copies, relabelled rows,
    global tables) and a few hundred per vertex, growing with both."""
    from paper_2301_12390_gb300.louvain import arena_bytes
    n, e = 1_000_000, 10_000_000
    b = arena_bytes(n, e)
    per_entry = (arena_bytes(n, 2 * e) - b) / e
    per_vertex = (arena_bytes(2 * n, e) - b) / n
    assert abs(per_entry - 68) < 0.5, per_entry
    assert 300 < per_vertex < 450, per_vertex
    assert arena_bytes(0, 0) < arena_bytes(10_000, 0) < arena_bytes(10_000, 10_000)   # (allocations are rounded)
