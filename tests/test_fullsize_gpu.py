"""Full-size checks at the benchmark configurations, in the launch configuration
bench.py times (asynchronous, pruning on, automatic vertex classes).

R-MAT scale 22 and the 4096^2 road grid: the oracle (single-threaded C)
finishes each in seconds to a minute, so the whole result is checked, not a
sample: asynchronous Q no lower than the oracle's minus 0.01 and the reported
exact numerator equal to the membership's recomputed one; synchronous (four
vertex classes) bit-exact with the oracle.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from engine_util import engine_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _engine():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def rmat22():
    return gg.rmat(0x5EED + 1, 22, 16, 0.57, 0.19, 0.19, wmin=1, wmax=8)


def test_rmat22_async_quality(rmat22):
    g = rmat22
    got = engine_run(g, mode=1, prune=1)
    ref = oracle.louvain(g.off, g.col, g.w, mode=oracle.ASYNC, prune=1)
    assert got["q"] >= ref.Q - 0.01, (got["q"], ref.Q)
    _, num, M = oracle.modularity(g.off, g.col, g.w, got["top"])
    assert got["exact"] == (num, M)


def test_rmat22_sync_bit_exact(rmat22):
    g = rmat22
    got = engine_run(g, mode=0, prune=1, subrounds=4)
    ref = oracle.louvain(g.off, g.col, g.w, mode=oracle.SYNC, prune=1, subrounds=4)
    assert got["iters"] == list(ref.iterations)
    assert np.array_equal(got["top"], ref.top)
    assert got["exact"] == (ref.q_num, ref.M)


def test_road4096_async_quality():
    g = gg.grid_road(0x5EED + 2, 4096, 0.1, 0.001, wmin=1, wmax=100)
    got = engine_run(g, mode=1, prune=1)
    ref = oracle.louvain(g.off, g.col, g.w, mode=oracle.ASYNC, prune=1)
    assert got["q"] >= ref.Q - 0.01, (got["q"], ref.Q)
