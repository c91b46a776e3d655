"""Plain FP64 CPU oracle for the isotropic NPCF estimator (arXiv:2105.08722).

TEST INFRASTRUCTURE. Only tests/, ``__graft_entry__.smoke()`` and bench.py's
``cpu_baseline`` / ``--impl reference`` leg may import this package. The GPU
library (``paper_2105_08722_gb300``) never imports it and shares no code with it.

Everything here is a thin ctypes layer over ``encore_oracle.c``; the arithmetic
and the citations live there.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "encore_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libencore_oracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FP contraction). Returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)
            and os.path.getmtime(_LIB) >= os.path.getmtime(os.path.join(_HERE, "encore_oracle.h"))):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        c_int, c_double, c_i64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64
        vp = ctypes.c_void_p
        L.orc_wigner3j.restype = c_double
        L.orc_wigner3j.argtypes = [c_int] * 6
        L.orc_ylm.restype = None
        L.orc_ylm.argtypes = [c_int, c_double, c_double, c_double, vp, vp]
        L.orc_multiplets.restype = c_int
        L.orc_multiplets.argtypes = [c_int, c_int, c_int, vp]
        L.orc_multiplets_cap.restype = c_int
        L.orc_multiplets_cap.argtypes = [c_int, c_int, c_int, c_int, vp]
        L.orc_bins.restype = c_int
        L.orc_bins.argtypes = [c_int, c_int, vp]
        L.orc_coupling.restype = c_double
        L.orc_coupling.argtypes = [c_int, vp, vp]
        L.orc_count_terms.restype = c_i64
        L.orc_count_terms.argtypes = [c_int, c_int, c_int]
        L.orc_shell.restype = c_int
        L.orc_shell.argtypes = [vp, vp, c_double, vp, c_int]
        L.orc_pair_counts.restype = c_int
        L.orc_pair_counts.argtypes = [c_i64, vp, vp, c_i64, c_int, vp, c_double, c_int, vp]
        L.orc_alm.restype = c_int
        L.orc_alm.argtypes = [c_i64, vp, vp, vp, c_i64, c_int, c_int, vp, c_double, vp, vp, vp]
        L.orc_npcf.restype = c_int
        L.orc_npcf.argtypes = [c_i64, vp, vp, vp, vp, c_i64, c_int, c_int, c_int, vp, c_double,
                               c_int, c_int, vp, vp, vp]
        L.orc_gaunt.restype = c_double
        L.orc_gaunt.argtypes = [c_int, vp, vp, vp]
        L.orc_edge_correct.restype = c_int
        L.orc_edge_correct.argtypes = [c_int, c_int, c_int, c_int, vp, vp, vp]
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def wigner3j(j1, j2, j3, m1, m2, m3) -> float:
    return lib().orc_wigner3j(j1, j2, j3, m1, m2, m3)


def ylm(lmax: int, v) -> np.ndarray:
    """Complex Y_lm for l <= lmax at direction v, index l*l + l + m."""
    n = (lmax + 1) ** 2
    re = np.zeros(n)
    im = np.zeros(n)
    lib().orc_ylm(lmax, float(v[0]), float(v[1]), float(v[2]), _p(re), _p(im))
    return re + 1j * im


WIDTH = {3: 2, 4: 3, 5: 5, 6: 7}   # ints per multiplet, intermediates included


def multiplets(N: int, lmax: int, allparity: bool = False) -> np.ndarray:
    n = lib().orc_multiplets(N, lmax, int(allparity), None)
    width = WIDTH[N]
    out = np.zeros(n * width, dtype=np.int32)
    lib().orc_multiplets(N, lmax, int(allparity), _p(out))
    return out.reshape(n, width)


def multiplets_cap(N: int, lmax: int, icap: int, allparity: bool = False) -> np.ndarray:
    """Multiplets whose intermediate l's (l12, l123) are at most icap (2 lmax is their
    natural range and gives multiplets())."""
    n = lib().orc_multiplets_cap(N, lmax, icap, int(allparity), None)
    width = WIDTH[N]
    out = np.zeros(n * width, dtype=np.int32)
    lib().orc_multiplets_cap(N, lmax, icap, int(allparity), _p(out))
    return out.reshape(n, width)


def bins(N: int, nr: int) -> np.ndarray:
    n = lib().orc_bins(N, nr, None)
    out = np.zeros(n * (N - 1), dtype=np.int32)
    lib().orc_bins(N, nr, _p(out))
    return out.reshape(n, N - 1)


def coupling(N: int, L: Sequence[int], M: Sequence[int]) -> float:
    La = np.ascontiguousarray(L, dtype=np.int32)
    Ma = np.ascontiguousarray(M, dtype=np.int32)
    return lib().orc_coupling(N, _p(La), _p(Ma))


def count_terms(N: int, lmax: int, allparity: bool = False) -> int:
    return int(lib().orc_count_terms(N, lmax, int(allparity)))


def _f32pos(pos) -> np.ndarray:
    return np.ascontiguousarray(pos, dtype=np.float32).reshape(-1, 3)


def shell(pi, pj, edges, box: float = 0.0) -> int:
    e = np.asarray(edges, dtype=np.float64)
    e2 = np.array([np.float32(x * x) for x in e], dtype=np.float32)
    a = np.ascontiguousarray(pi, dtype=np.float32)
    b = np.ascontiguousarray(pj, dtype=np.float32)
    return lib().orc_shell(_p(a), _p(b), float(box), _p(e2), len(e) - 1)


def pair_counts(pos, edges, box: float = 0.0, prim=None, nthreads: int = 0) -> np.ndarray:
    pos = _f32pos(pos)
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    nr = len(edges) - 1
    out = np.zeros(nr, dtype=np.uint64)
    pr = None if prim is None else np.ascontiguousarray(prim, dtype=np.int64)
    lib().orc_pair_counts(len(pos), _p(pos), _p(pr), 0 if pr is None else len(pr), nr,
                          _p(edges), float(box), nthreads, _p(out))
    return out


def alm(pos, w, prim, lmax: int, edges, box: float = 0.0):
    """(a [n_prim, nr, (lmax+1)^2] complex, counts [n_prim, nr]) for the given primaries."""
    pos = _f32pos(pos)
    w = np.ascontiguousarray(w, dtype=np.float32)
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    pr = np.ascontiguousarray(prim, dtype=np.int64)
    nr = len(edges) - 1
    nlm = (lmax + 1) ** 2
    re = np.zeros((len(pr), nr, nlm))
    im = np.zeros((len(pr), nr, nlm))
    cnt = np.zeros((len(pr), nr), dtype=np.uint32)
    lib().orc_alm(len(pos), _p(pos), _p(w), _p(pr), len(pr), lmax, nr, _p(edges), float(box),
                  _p(re), _p(im), _p(cnt))
    return re + 1j * im, cnt


def layout(orders: Sequence[int], lmax: int, nr: int, allparity: bool = False):
    """[(N, multiplets, bins)] in output order."""
    return [(N, multiplets(N, lmax, allparity), bins(N, nr)) for N in sorted(orders)]


def npcf(pos, w, orders: Sequence[int], lmax: int, edges, box: float = 0.0,
         allparity: bool = False, wprim=None, prim=None, nthreads: int = 0,
         return_resid: bool = False):
    """Raw zeta (flat, orders ascending, [L][B] each) and per-shell pair counts."""
    pos = _f32pos(pos)
    w = np.ascontiguousarray(w, dtype=np.float32)
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    nr = len(edges) - 1
    mask = 0
    total = 0
    for N in orders:
        mask |= 1 << N
    for N, lam, bb in layout(orders, lmax, nr, allparity):
        total += len(lam) * len(bb)
    zeta = np.zeros(total)
    resid = np.zeros(total)
    counts = np.zeros(nr, dtype=np.uint64)
    wp = None if wprim is None else np.ascontiguousarray(wprim, dtype=np.float32)
    pr = None if prim is None else np.ascontiguousarray(prim, dtype=np.int64)
    rc = lib().orc_npcf(len(pos), _p(pos), _p(w), _p(wp), _p(pr), 0 if pr is None else len(pr),
                        mask, lmax, nr, _p(edges), float(box), int(allparity), nthreads,
                        _p(zeta), _p(resid), _p(counts))
    if rc != 0:
        raise RuntimeError("orc_npcf failed: %d" % rc)
    if return_resid:
        return zeta, counts, resid
    return zeta, counts


def split_orders(flat: np.ndarray, orders: Sequence[int], lmax: int, nr: int,
                 allparity: bool = False) -> dict:
    """Split a flat output into {N: array[n_multiplets, n_bins]}."""
    out = {}
    off = 0
    for N, lam, bb in layout(orders, lmax, nr, allparity):
        size = len(lam) * len(bb)
        out[N] = flat[off:off + size].reshape(len(lam), len(bb))
        off += size
    return out


def gaunt(N: int, L1, L2, L3) -> float:
    a = np.ascontiguousarray(L1, dtype=np.int32)
    b = np.ascontiguousarray(L2, dtype=np.int32)
    c = np.ascontiguousarray(L3, dtype=np.int32)
    return lib().orc_gaunt(N, _p(a), _p(b), _p(c))


def edge_correct(N: int, lmax: int, nr: int, nraw: np.ndarray, rraw: np.ndarray) -> np.ndarray:
    """Edge-corrected zeta [L][B] from raw N and R multiplets of one order (parity-even)."""
    nraw = np.ascontiguousarray(nraw, dtype=np.float64)
    rraw = np.ascontiguousarray(rraw, dtype=np.float64)
    out = np.zeros_like(nraw)
    rc = lib().orc_edge_correct(N, lmax, nr, 0, _p(nraw), _p(rraw), _p(out))
    if rc != 0:
        raise RuntimeError("orc_edge_correct failed: %d" % rc)
    return out
