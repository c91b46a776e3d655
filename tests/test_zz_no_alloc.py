"""npcf_pair_counts_noalloc against the oracle and the context-based entry point.

The allocation-free entry point serves callers that cannot call cudaMalloc: processes
whose device memory belongs entirely to another allocator, and plug-ins that must not grow
their memory footprint per call. Its per-shell pair counts are exact integers, so they are
compared bit for bit with the oracle's counts (the same FP32 neighbour rule) and with
npcf_accumulate + npcf_pair_counts. Two calls in a row on different catalogs check that
the shared fixed scratch is cleared between calls; bad positions must be reported through
the documented UINT64_MAX sentinel, and a correct call right after a bad one must count
again.
"""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

SENTINEL = np.uint64(0xFFFFFFFFFFFFFFFF)


@pytest.fixture(scope="module")
def torch_dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_08722_gb300 import build
    build()
    oracle.build()
    return torch, torch.device("cuda:0")


def _catalog(n, side, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, side, size=(n, 3)).astype(np.float32)


def _context_counts(torch, dev, pos, w, edges, box):
    from paper_2105_08722_gb300._lib import NPCF
    est = NPCF(2, (3,), edges, box)
    est.accumulate(torch.from_numpy(pos).to(dev), torch.from_numpy(w).to(dev))
    counts = est.pair_counts()
    est.close()
    return counts


def _noalloc(torch, dev, pos, edges, box):
    from paper_2105_08722_gb300 import _lib
    lib = _lib.load()
    nr = len(edges) - 1
    stream = torch.cuda.current_stream(dev).cuda_stream
    tpos = torch.from_numpy(np.ascontiguousarray(pos)).to(dev)
    out = torch.full((nr,), 987654321, dtype=torch.int64, device=dev)  # must be overwritten
    st = lib.npcf_pair_counts_noalloc(ctypes.c_void_p(tpos.data_ptr()), len(pos), nr,
                                      edges.ctypes.data, box, ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(stream))
    assert st == _lib.NPCF_OK, lib.npcf_last_error(None)
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint64).copy()


@pytest.mark.parametrize("box", [300.0, 0.0])
def test_noalloc_counts_equal_oracle_and_context_on_two_calls(torch_dev, box):
    torch, dev = torch_dev
    edges = np.linspace(5.0, 60.0, 9)
    for call, (n, seed) in enumerate([(20000, 11), (7001, 12)]):
        pos = _catalog(n, 300.0, seed)
        want = oracle.pair_counts(pos, edges, box)
        ctx = _context_counts(torch, dev, pos, np.ones(n, np.float32), edges, box)
        got = _noalloc(torch, dev, pos, edges, box)
        assert want.sum() > 0
        assert np.array_equal(got, want), (call, got, want)
        assert np.array_equal(ctx, want), (call, ctx, want)


def test_noalloc_counts_with_zero_and_negative_weights_match_context(torch_dev):
    """The counts do not depend on the weights: a catalog with ~10 % zero weights and mixed
    signs gives the same counts through npcf_accumulate as without weights."""
    torch, dev = torch_dev
    edges = np.linspace(5.0, 60.0, 9)
    n = 9000
    pos = _catalog(n, 300.0, 21)
    rng = np.random.default_rng(22)
    w = rng.uniform(-1.5, 1.5, n).astype(np.float32)
    w[rng.random(n) < 0.1] = 0.0
    want = oracle.pair_counts(pos, edges, 300.0)
    assert np.array_equal(_noalloc(torch, dev, pos, edges, 300.0), want)
    assert np.array_equal(_context_counts(torch, dev, pos, w, edges, 300.0), want)


@pytest.mark.parametrize("box,bad", [(300.0, "outside"), (300.0, "nan"), (0.0, "nan")])
def test_noalloc_reports_bad_positions_then_counts_again(torch_dev, box, bad):
    torch, dev = torch_dev
    edges = np.linspace(5.0, 60.0, 9)
    pos = _catalog(5000, 300.0, 31)
    badpos = pos.copy()
    if bad == "outside":
        badpos[1234, 1] = 300.0   # periodic positions must lie in [0, box)
    else:
        badpos[1234, 2] = np.nan
    got = _noalloc(torch, dev, badpos, edges, box)
    assert np.all(got == SENTINEL), got
    # the next call on good positions is not affected by the flagged one
    assert np.array_equal(_noalloc(torch, dev, pos, edges, box), oracle.pair_counts(pos, edges, box))


def test_noalloc_rejects_catalogs_beyond_its_fixed_scratch(torch_dev):
    from paper_2105_08722_gb300 import _lib
    lib = _lib.load()
    edges = np.linspace(5.0, 60.0, 9)
    st = lib.npcf_pair_counts_noalloc(None, (1 << 18) + 1, 8, edges.ctypes.data, 300.0,
                                      ctypes.c_void_p(8), None)
    assert st == _lib.NPCF_EINVAL
    assert b"exceed" in lib.npcf_last_error(None)
