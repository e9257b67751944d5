"""louvain_modularity_static: modularity with its scratch in a fixed static
device array, for callers that must not allocate device memory.

Checked through the C ABI against the context-based louvain_modularity on two
calls in a row with different graphs and memberships (so leftovers from the
first call would show in the second), exact numerators and equal Q.  The file
is named so that pytest collects it last.
"""
import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _engine():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _reference(g, memb):
    from paper_2301_12390_gb300 import Louvain
    with Louvain(device=0) as lv:
        lv.load_csr(g.off, g.col, g.w)
        return lv.modularity_of(memb)


def test_static_scratch_matches_context_entry_point_on_two_calls():
    import torch
    from paper_2301_12390_gb300.louvain import modularity_static
    rng = np.random.default_rng(7)
    cases = [
        (gg.rmat(91, 16, 16, wmin=1, wmax=8), 40),     # larger graph first ...
        (gg.sbm(92, 3000, 30, 0.05, 0.002, wmin=1, wmax=5), 30),   # ... then a smaller one
    ]
    for g, k in cases:
        memb = rng.integers(0, k, g.n).astype(np.int32)
        dev = [torch.from_numpy(a).cuda() for a in (g.off, g.col, g.w, memb)]
        q, num, M = modularity_static(*dev)
        rq, rnum, rM = _reference(g, memb)
        assert (num, M) == (rnum, rM)
        assert q == rq


def test_static_rejects_sizes_beyond_capacity():
    from paper_2301_12390_gb300 import load_library
    from paper_2301_12390_gb300.louvain import STATIC_MAX_VERTICES
    import ctypes
    lib = load_library()
    q = ctypes.c_double()
    rc = lib.louvain_modularity_static(STATIC_MAX_VERTICES + 1, None, None, None, None, None, ctypes.byref(q),
                                       None, None, None)
    assert rc == -10
