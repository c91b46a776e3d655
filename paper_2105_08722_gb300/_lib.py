"""ctypes binding of libencore_gpu (include/encore_gpu.h).

Argument marshalling only: every step of the estimator runs in the CUDA library.
There is no CPU fallback; importing this module without the built library raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libencore_gpu.so")

NPCF_OK, NPCF_EINVAL, NPCF_ENOMEM, NPCF_ECUDA, NPCF_EUNSUPPORTED, NPCF_ETIMEOUT = range(6)
FP32, SPLIT_BF16 = 0, 1
_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EUNSUPPORTED", 5: "ETIMEOUT"}

# every symbol the header declares, with its ctypes signature
_vp, _i, _i64, _u, _d, _sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint,
                              ctypes.c_double, ctypes.c_size_t)
SIGNATURES = {
    "npcf_create": (_i, [ctypes.POINTER(_vp), _i, _u, _i, _vp, _d, _i, _i]),
    "npcf_accumulate": (_i, [_vp, _vp, _vp, _i64, _vp]),
    "npcf_accumulate_ex": (_i, [_vp, _vp, _vp, _vp, _i64, _vp]),
    "npcf_accumulate_host": (_i, [_vp, _vp, _vp, _i64, _vp]),
    "npcf_cache_data": (_i, [_vp, _vp, _vp, _i64, _vp]),
    "npcf_accumulate_split": (_i, [_vp, _vp, _vp, _i64, _vp]),
    "npcf_accumulate_grid": (_i, [_vp, _vp, _i, _vp]),
    "npcf_output_size": (_i, [_vp, ctypes.POINTER(_sz)]),
    "npcf_layout": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), _vp, _vp]),
    "npcf_finalize": (_i, [_vp, _vp, _sz, _i]),
    "npcf_pair_counts": (_i, [_vp, _vp]),
    "npcf_reset": (_i, [_vp]),
    "npcf_debug_alm": (_i, [_vp, _vp, _i64, _vp, _vp]),
    "npcf_set_tuning": (_i, [_vp, _i, _i]),
    "npcf_get_timings": (_i, [_vp, _vp]),
    "npcf_pair_counts_noalloc": (_i, [_vp, _i64, _i, _vp, _d, _vp, _vp]),
    "npcf_edge_correct": (_i, [_vp, _vp, _vp]),
    "npcf_accumulate_batch": (_i, [_vp, _vp, _vp, _vp, _i, _vp]),
    "npcf_accumulate_batch_ex": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _vp]),
    "npcf_finalize_batch": (_i, [_vp, _vp, _sz, _i]),
    "npcf_pair_counts_batch": (_i, [_vp, _vp, _sz]),
    "npcf_batch_info": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i64)]),
    "npcf_autotune": (_i, [_vp, _vp, _vp, _i64, _vp, _vp]),
    "npcf_gaunt": (_i, [_i, _vp, _vp, _vp, ctypes.POINTER(_d)]),
    "npcf_truncate": (_i, [_vp, _vp, _sz, _i, _vp, ctypes.POINTER(_sz)]),
    "npcf_multiplets": (_i, [_i, _i, _i, ctypes.POINTER(_i), _vp]),
    "npcf_coupling": (_i, [_i, _vp, _vp, ctypes.POINTER(_d)]),
    "npcf_probe_fp32_peak": (_i, [ctypes.POINTER(_d), ctypes.POINTER(_d)]),
    "npcf_last_error": (ctypes.c_char_p, [_vp]),
    "npcf_destroy": (None, [_vp]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library (build it first with paper_2105_08722_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libencore_gpu.so is not built (%s); run paper_2105_08722_gb300.build.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def pair_counts_noalloc(pos, edges, box: float, out, stream=None):
    """Exact per-shell pair counts into the CUDA uint64 tensor ``out`` [nr] without any
    device allocation by the library (npcf_pair_counts_noalloc)."""
    lib = load()
    e = np.ascontiguousarray(edges, dtype=np.float64)
    st = lib.npcf_pair_counts_noalloc(_ptr(pos), int(pos.shape[0]), len(e) - 1, e.ctypes.data, float(box),
                                      _ptr(out), _stream_handle(stream))
    if st != NPCF_OK:
        raise NPCFError(st, lib.npcf_last_error(None).decode())


def probe_fp32_peak() -> Tuple[float, float]:
    """Measured FP32 FMA throughput of the current device (npcf_probe_fp32_peak):
    (TFLOP/s, ms of the fastest launch)."""
    lib = load()
    t, ms = _d(), _d()
    st = lib.npcf_probe_fp32_peak(ctypes.byref(t), ctypes.byref(ms))
    if st != NPCF_OK:
        raise NPCFError(st, lib.npcf_last_error(None).decode())
    return t.value, ms.value


def gaunt(N: int, L1, L2, L3) -> float:
    """Generalized Gaunt integral G^{L1 L2 L3} as the library's edge correction uses it
    (closed forms of App. A; host-only, npcf_gaunt)."""
    lib = load()
    a, b, c = (np.ascontiguousarray(x, dtype=np.int32) for x in (L1, L2, L3))
    out = ctypes.c_double()
    st = lib.npcf_gaunt(int(N), a.ctypes.data, b.ctypes.data, c.ctypes.data, ctypes.byref(out))
    if st != NPCF_OK:
        raise NPCFError(st, "npcf_gaunt: bad arguments")
    return out.value


def multiplets(N: int, lmax: int, allparity: bool = False) -> np.ndarray:
    """Multiplets of order N (npcf_multiplets), one row each."""
    lib = load()
    n = _i()
    st = lib.npcf_multiplets(int(N), int(lmax), int(bool(allparity)), ctypes.byref(n), None)
    if st != NPCF_OK:
        raise NPCFError(st, "npcf_multiplets: bad arguments")
    width = {3: 2, 4: 3, 5: 5, 6: 7}[int(N)]
    out = np.zeros(n.value * width, dtype=np.int32)
    lib.npcf_multiplets(int(N), int(lmax), int(bool(allparity)), ctypes.byref(n), out.ctypes.data)
    return out.reshape(n.value, width)


def coupling(N: int, L, M) -> float:
    """C^L_M of Eq. basis-coupling (npcf_coupling)."""
    La = np.ascontiguousarray(L, dtype=np.int32)
    Ma = np.ascontiguousarray(M, dtype=np.int32)
    out = _d()
    st = load().npcf_coupling(int(N), La.ctypes.data, Ma.ctypes.data, ctypes.byref(out))
    if st != NPCF_OK:
        raise NPCFError(st, "npcf_coupling: bad arguments")
    return out.value


class NPCFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class NPCF:
    """One estimator context: lmax, orders (subset of {3, 4, 5}), radial edges, box."""

    def __init__(self, lmax: int, orders: Sequence[int], edges, box: float = 0.0,
                 precision: int = FP32, allparity: bool = False):
        self._lib = load()
        self.lmax = int(lmax)
        self.orders = tuple(sorted(int(o) for o in orders))
        self.edges = np.ascontiguousarray(edges, dtype=np.float64)
        self.nr = len(self.edges) - 1
        self.box = float(box)
        mask = 0
        for o in self.orders:
            mask |= 1 << o
        h = _vp()
        st = self._lib.npcf_create(ctypes.byref(h), self.lmax, mask, self.nr, self.edges.ctypes.data,
                                   self.box, int(precision), int(bool(allparity)))
        if st != NPCF_OK:
            raise NPCFError(st, self._lib.npcf_last_error(None).decode())
        self._h = h
        n = _sz()
        self._check(self._lib.npcf_output_size(self._h, ctypes.byref(n)))
        self.size = n.value

    def _check(self, st: int):
        if st != NPCF_OK:
            raise NPCFError(st, self._lib.npcf_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.npcf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def accumulate(self, pos, w, wprim=None, stream=None):
        """pos: CUDA float32 [n, 3]; w, wprim: CUDA float32 [n] (torch tensors)."""
        n = int(pos.shape[0])
        if wprim is None:
            self._check(self._lib.npcf_accumulate(self._h, _ptr(pos), _ptr(w), n, _stream_handle(stream)))
        else:
            self._check(self._lib.npcf_accumulate_ex(self._h, _ptr(pos), _ptr(w), _ptr(wprim), n,
                                                     _stream_handle(stream)))

    def cache_data(self, pos, w, stream=None):
        """Keep the data's harmonics for later random splits (npcf_cache_data); pos [n, 3]
        and w [n] CUDA float32 tensors."""
        self._check(self._lib.npcf_cache_data(self._h, _ptr(pos), _ptr(w), int(pos.shape[0]),
                                              _stream_handle(stream)))

    def accumulate_split(self, pos, w, stream=None):
        """Accumulate the cached data followed by these randoms (npcf_accumulate_split)."""
        n = int(pos.shape[0])
        self._check(self._lib.npcf_accumulate_split(self._h, _ptr(pos) if n else None, _ptr(w) if n else None, n,
                                                    _stream_handle(stream)))

    def accumulate_grid(self, delta, stream=None):
        """A density field on a periodic n^3 mesh over the box (npcf_accumulate_grid):
        delta, CUDA float32 tensor [n, n, n] indexed [z, y, x] (x fastest in memory)."""
        n = int(delta.shape[-1])
        self._check(self._lib.npcf_accumulate_grid(self._h, _ptr(delta), n, _stream_handle(stream)))

    def accumulate_host(self, pos: np.ndarray, w: np.ndarray, stream=None):
        pos = np.ascontiguousarray(pos, dtype=np.float32)
        w = np.ascontiguousarray(w, dtype=np.float32)
        self._check(self._lib.npcf_accumulate_host(self._h, pos.ctypes.data, w.ctypes.data, len(pos),
                                                   _stream_handle(stream)))

    def finalize(self, normalize: bool = False) -> np.ndarray:
        out = np.zeros(self.size, dtype=np.float64)
        self._check(self._lib.npcf_finalize(self._h, out.ctypes.data, self.size, int(normalize)))
        return out

    def accumulate_batch(self, pos, w, offsets, wprim=None, stream=None):
        """Co-add a batch of catalogs (npcf_accumulate_batch[_ex]): pos [n, 3] and w [n]
        CUDA tensors, catalog k = rows offsets[k] .. offsets[k+1]-1; wprim (optional, [n])
        separate primary weights."""
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        if wprim is None:
            st = self._lib.npcf_accumulate_batch(self._h, _ptr(pos), _ptr(w), off.ctypes.data, len(off) - 1,
                                                 _stream_handle(stream))
        else:
            st = self._lib.npcf_accumulate_batch_ex(self._h, _ptr(pos), _ptr(w), _ptr(wprim), off.ctypes.data,
                                                    len(off) - 1, _stream_handle(stream))
        self._check(st)

    def autotune(self, pos, w, stream=None) -> Dict[str, int]:
        """Pick the fastest pair-kernel and contraction settings for this catalog
        (npcf_autotune); the accumulators are left empty."""
        chosen = np.zeros(4, dtype=np.int32)
        self._check(self._lib.npcf_autotune(self._h, _ptr(pos), _ptr(w), int(pos.shape[0]),
                                            _stream_handle(stream), chosen.ctypes.data))
        return {"cells_per_rmax": int(chosen[0]), "pair_chunk": int(chosen[1]), "pair_cap": int(chosen[2]),
                "chunk": int(chosen[3])}

    def batch_info(self) -> Tuple[int, int]:
        k, g = ctypes.c_int(), ctypes.c_int64()
        self._check(self._lib.npcf_batch_info(self._h, ctypes.byref(k), ctypes.byref(g)))
        return k.value, g.value

    def finalize_batch(self, normalize: bool = False) -> np.ndarray:
        k = max(self.batch_info()[0], 1)
        out = np.zeros((k, self.size), dtype=np.float64)
        self._check(self._lib.npcf_finalize_batch(self._h, out.ctypes.data, out.size, int(normalize)))
        return out

    def pair_counts_batch(self) -> np.ndarray:
        k = max(self.batch_info()[0], 1)
        out = np.zeros((k, self.nr), dtype=np.uint64)
        self._check(self._lib.npcf_pair_counts_batch(self._h, out.ctypes.data, out.size))
        return out

    def edge_correct(self, randoms: "NPCF") -> np.ndarray:
        """Edge-corrected multiplets (npcf_edge_correct): this context holds the
        data-minus-randoms sums, ``randoms`` the randoms-only sums."""
        out = np.zeros(self.size, dtype=np.float64)
        self._check(self._lib.npcf_edge_correct(self._h, randoms._h, out.ctypes.data))
        return out

    def truncate(self, flat: np.ndarray, lmax_out: int) -> np.ndarray:
        """This context's output (finalize, one catalog of finalize_batch or edge_correct)
        cut to the multiplets of an lmax_out context (npcf_truncate)."""
        flat = np.ascontiguousarray(flat, dtype=np.float64)
        n = _sz()
        self._check(self._lib.npcf_truncate(self._h, None, flat.size, int(lmax_out), None, ctypes.byref(n)))
        out = np.zeros(n.value, dtype=np.float64)
        self._check(self._lib.npcf_truncate(self._h, flat.ctypes.data, flat.size, int(lmax_out),
                                            out.ctypes.data, ctypes.byref(n)))
        return out

    def pair_counts(self) -> np.ndarray:
        out = np.zeros(self.nr, dtype=np.uint64)
        self._check(self._lib.npcf_pair_counts(self._h, out.ctypes.data))
        return out

    def reset(self):
        self._check(self._lib.npcf_reset(self._h))

    def layout(self, order: int) -> Tuple[np.ndarray, np.ndarray]:
        nl, nb = _i(), _i()
        self._check(self._lib.npcf_layout(self._h, order, ctypes.byref(nl), ctypes.byref(nb), None, None))
        width = {3: 2, 4: 3, 5: 5, 6: 7}[order]
        lam = np.zeros(nl.value * width, dtype=np.int32)
        bins = np.zeros(nb.value * (order - 1), dtype=np.int32)
        self._check(self._lib.npcf_layout(self._h, order, ctypes.byref(nl), ctypes.byref(nb),
                                          lam.ctypes.data, bins.ctypes.data))
        return lam.reshape(nl.value, width), bins.reshape(nb.value, order - 1)

    def split(self, flat: np.ndarray) -> Dict[int, np.ndarray]:
        out, off = {}, 0
        for o in self.orders:
            lam, bins = self.layout(o)
            size = len(lam) * len(bins)
            out[o] = flat[off:off + size].reshape(len(lam), len(bins))
            off += size
        return out

    def debug_alm(self, idx) -> Tuple[np.ndarray, np.ndarray]:
        """(a [k, nr, nlm] complex64 for m >= 0, counts [k, nr]) of the last accumulate call."""
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        nlm = (self.lmax + 1) * (self.lmax + 2) // 2
        buf = np.zeros((len(idx), self.nr, nlm, 2), dtype=np.float32)
        cnt = np.zeros((len(idx), self.nr), dtype=np.uint32)
        self._check(self._lib.npcf_debug_alm(self._h, idx.ctypes.data, len(idx), buf.ctypes.data,
                                             cnt.ctypes.data))
        return buf[..., 0] + 1j * buf[..., 1], cnt

    def set_tuning(self, key: int, value: int):
        self._check(self._lib.npcf_set_tuning(self._h, key, value))

    def timings(self) -> np.ndarray:
        out = np.zeros(4, dtype=np.float32)
        self._check(self._lib.npcf_get_timings(self._h, out.ctypes.data))
        return out
