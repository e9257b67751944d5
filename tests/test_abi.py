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
