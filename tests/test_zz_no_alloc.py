"""louvain_modularity_static: modularity with its scratch in a fixed static
device array, for callers that must not allocate device memory (an allocator
that already owns the free memory, a memory plan fixed up front, or streams
that cannot take the device-wide synchronisation of cudaMalloc / cudaFree).

Checked through the C ABI against the context-based louvain_modularity and
against the oracle's exact numerator, on two calls in a row with different
graphs and memberships (so leftovers of the first call would show in the
second), on the default stream and on a stream of its own; and its rejections:
a size beyond the fixed capacity, null pointers, a membership outside [0, n),
a column outside [0, n) and decreasing offsets (the kernels check each before
they index with it).  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

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


def _cases():
    rng = np.random.default_rng(7)
    out = []
    for g, k in [(gg.rmat(91, 16, 16, wmin=1, wmax=8), 40),            # larger graph first ...
                 (gg.sbm(92, 3000, 30, 0.05, 0.002, wmin=1, wmax=5), 30)]:  # ... then a smaller one
        out.append((g, rng.integers(0, k, g.n).astype(np.int32)))
    return out


@pytest.mark.parametrize("on_stream", [False, True])
def test_static_scratch_matches_context_entry_point_on_two_calls(on_stream):
    import torch
    from paper_2301_12390_gb300.louvain import modularity_static
    stream = torch.cuda.Stream() if on_stream else None
    for g, memb in _cases():
        dev = [torch.from_numpy(a).cuda() for a in (g.off, g.col, g.w, memb)]
        if stream is not None:
            stream.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(stream):
                q, num, M = modularity_static(*dev, stream=stream)
        else:
            q, num, M = modularity_static(*dev)
        rq, rnum, rM = _reference(g, memb)
        assert (num, M) == (rnum, rM)
        assert q == rq
        oq, onum, oM = oracle.modularity(g.off, g.col, g.w, memb)
        assert (num, M) == (onum, oM)
        assert q == oq


def test_static_empty_graph():
    import torch
    from paper_2301_12390_gb300.louvain import modularity_static
    z64 = torch.zeros(1, dtype=torch.int64, device="cuda")
    e32 = torch.zeros(0, dtype=torch.int32, device="cuda")
    assert modularity_static(z64, e32, e32, e32) == (0.0, 0, 0)


def test_static_rejects_sizes_beyond_capacity_and_null_pointers():
    import ctypes
    import torch
    from paper_2301_12390_gb300 import load_library
    from paper_2301_12390_gb300.louvain import STATIC_MAX_VERTICES
    lib = load_library()
    q = ctypes.c_double()
    rc = lib.louvain_modularity_static(STATIC_MAX_VERTICES + 1, None, None, None, None, None, ctypes.byref(q),
                                       None, None, None)
    assert rc == -10
    g, memb = _cases()[1]
    off, col, w, mb = [torch.from_numpy(a).cuda() for a in (g.off, g.col, g.w, memb)]
    ptrs = [off.data_ptr(), col.data_ptr(), w.data_ptr(), mb.data_ptr()]
    for k in range(4):   # each of the four device pointers null in turn
        args = list(ptrs)
        args[k] = None
        rc = lib.louvain_modularity_static(g.n, *args, None, ctypes.byref(q), None, None, None)
        assert rc == -1, k


def test_static_rejects_bad_membership_columns_and_offsets():
    """Each bad input is caught by a check that runs before the value is used
    as an index, so the call returns an error and the context stays usable."""
    import torch
    from paper_2301_12390_gb300 import LouvainError
    from paper_2301_12390_gb300.louvain import modularity_static
    g, memb = _cases()[1]
    off, col, w, mb = [torch.from_numpy(a).cuda() for a in (g.off, g.col, g.w, memb)]
    bad = mb.clone()
    bad[g.n // 2] = g.n          # a membership outside [0, n)
    with pytest.raises(LouvainError) as e:
        modularity_static(off, col, w, bad)
    assert e.value.code == -1
    bad = mb.clone()
    bad[0] = -3
    with pytest.raises(LouvainError) as e:
        modularity_static(off, col, w, bad)
    assert e.value.code == -1
    badc = col.clone()
    badc[g.nnz // 3] = g.n       # a column outside [0, n)
    with pytest.raises(LouvainError) as e:
        modularity_static(off, badc, w, mb)
    assert e.value.code == -3
    badc[g.nnz // 3] = -1
    with pytest.raises(LouvainError) as e:
        modularity_static(off, badc, w, mb)
    assert e.value.code == -3
    bado = off.clone()           # row 10 ends before it starts; every offset stays within the buffers
    bado[11] = bado[10] - 1
    with pytest.raises(LouvainError) as e:
        modularity_static(bado, col, w, mb)
    assert e.value.code == -3
    # the device is still usable, and the array's leftovers do not leak into the next call
    q, num, M = modularity_static(off, col, w, mb)
    oq, onum, oM = oracle.modularity(g.off, g.col, g.w, memb)
    assert (num, M, q) == (onum, oM, oq)


def test_static_binding_checks_types():
    import torch
    from paper_2301_12390_gb300.louvain import modularity_static
    g, memb = _cases()[1]
    off, col, w, mb = [torch.from_numpy(a).cuda() for a in (g.off, g.col, g.w, memb)]
    with pytest.raises(TypeError):
        modularity_static(off.to(torch.int32), col, w, mb)
    with pytest.raises(TypeError):
        modularity_static(off, col, w, mb.cpu())
