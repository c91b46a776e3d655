"""npcf_pair_counts_noalloc against the context-based entry point.

The allocation-free entry point serves callers that cannot call cudaMalloc (code running
during CUDA-graph capture, processes whose device memory belongs to another allocator).
Its per-shell pair counts must equal those of npcf_accumulate + npcf_pair_counts, which
are exact integers, so the comparison is bit-exact. Two calls in a row on different
catalogs check that the shared fixed scratch is cleared between calls.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_08722_gb300 import build
    build()
    return torch, torch.device("cuda:0")


def _catalog(n, side, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, side, size=(n, 3)).astype(np.float32)


def _context_counts(torch, dev, pos, edges, box):
    from paper_2105_08722_gb300._lib import NPCF
    est = NPCF(2, (3,), edges, box)
    est.accumulate(torch.from_numpy(pos).to(dev), torch.ones(len(pos), device=dev))
    counts = est.pair_counts()
    est.close()
    return counts


@pytest.mark.parametrize("box", [300.0, 0.0])
def test_noalloc_counts_equal_context_counts_on_two_calls(torch_dev, box):
    torch, dev = torch_dev
    from paper_2105_08722_gb300 import _lib
    lib = _lib.load()
    edges = np.linspace(5.0, 60.0, 9)
    nr = len(edges) - 1
    stream = torch.cuda.current_stream(dev).cuda_stream
    for call, (n, seed) in enumerate([(20000, 11), (7001, 12)]):
        pos = _catalog(n, 300.0, seed)
        want = _context_counts(torch, dev, pos, edges, box)
        tpos = torch.from_numpy(pos).to(dev)
        out = torch.full((nr,), 987654321, dtype=torch.int64, device=dev)  # must be overwritten
        st = lib.npcf_pair_counts_noalloc(ctypes.c_void_p(tpos.data_ptr()), n, nr,
                                          edges.ctypes.data, box, ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(stream))
        assert st == _lib.NPCF_OK, lib.npcf_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.uint64)
        assert want.sum() > 0
        assert np.array_equal(got, want), (call, got, want)


def test_noalloc_rejects_catalogs_beyond_its_fixed_scratch(torch_dev):
    from paper_2105_08722_gb300 import _lib
    lib = _lib.load()
    edges = np.linspace(5.0, 60.0, 9)
    st = lib.npcf_pair_counts_noalloc(None, (1 << 18) + 1, 8, edges.ctypes.data, 300.0,
                                      ctypes.c_void_p(8), None)
    assert st == _lib.NPCF_EINVAL
    assert b"exceed" in lib.npcf_last_error(None)
