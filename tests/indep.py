"""Library-based, independently written references used to pin the oracle.

Nothing here calls the oracle: spherical harmonics come from scipy
(``sph_harm_y``), 3-j / 9-j symbols from sympy, the neighbour rule is
re-implemented in numpy float32, and the brute-force NPCF evaluates the basis
function P_L for every tuple of secondaries (the brute-force estimator of
Sec. 5.2) instead of factorising through a_lm.
"""
from __future__ import annotations

import itertools
import math
from functools import lru_cache

import numpy as np
from scipy.special import sph_harm_y


def ylm_scipy(l: int, m: int, v: np.ndarray) -> np.ndarray:
    """Y_lm at unit vectors v [..., 3] (Condon-Shortley, orthonormal)."""
    v = np.asarray(v, dtype=np.float64)
    r = np.linalg.norm(v, axis=-1)
    theta = np.arccos(np.clip(v[..., 2] / r, -1.0, 1.0))
    phi = np.arctan2(v[..., 1], v[..., 0])
    return sph_harm_y(l, m, theta, phi)


@lru_cache(maxsize=None)
def w3j(j1, j2, j3, m1, m2, m3) -> float:
    from sympy.physics.wigner import wigner_3j
    return float(wigner_3j(j1, j2, j3, m1, m2, m3))


@lru_cache(maxsize=None)
def w9j(*a) -> float:
    from sympy.physics.wigner import wigner_9j
    return float(wigner_9j(*a, prec=40))


def coupling_sympy(N: int, L, M) -> float:
    """C^L_M from Eq. (N=3-coeff), Eq. (N=4-coeff) and Eq. (basis-coupling) at N=5, 6."""
    if N == 3:
        l = L[0]
        if L[0] != L[1] or M[0] != -M[1] or abs(M[0]) > l:
            return 0.0
        return (-1) ** (l - M[0]) / math.sqrt(2 * l + 1)
    if N == 4:
        return (-1) ** sum(L) * w3j(L[0], L[1], L[2], M[0], M[1], M[2])
    if N == 5:
        l1, l2, l12, l3, l4 = L
        m12 = M[0] + M[1]
        if abs(m12) > l12:
            return 0.0
        return ((-1) ** (l1 + l2 + l3 + l4) * math.sqrt(2 * l12 + 1) * (-1) ** (l12 - m12)
                * w3j(l1, l2, l12, M[0], M[1], -m12) * w3j(l12, l3, l4, m12, M[2], M[3]))
    # N = 6: two intermediates, the sums over m12 and m123 fixed by the 3-j symbols
    l1, l2, l12, l3, l123, l4, l5 = L
    m12 = M[0] + M[1]
    m123 = m12 + M[2]
    if abs(m12) > l12 or abs(m123) > l123:
        return 0.0
    return ((-1) ** (l1 + l2 + l3 + l4 + l5) * math.sqrt((2 * l12 + 1) * (2 * l123 + 1))
            * (-1) ** (l12 - m12 + l123 - m123)
            * w3j(l1, l2, l12, M[0], M[1], -m12) * w3j(l12, l3, l123, m12, M[2], -m123)
            * w3j(l123, l4, l5, m123, M[3], M[4]))


def principal(N, L):
    if N in (3, 4):
        return list(L)
    if N == 5:
        return [L[0], L[1], L[3], L[4]]
    return [L[0], L[1], L[3], L[5], L[6]]


def basis_terms(N, L):
    """[(M, C^L_M)] over the full M range with C != 0."""
    ell = principal(N, L)
    out = []
    for M in itertools.product(*[range(-l, l + 1) for l in ell[:-1]]):
        mlast = -sum(M)
        if abs(mlast) > ell[-1]:
            continue
        Mf = tuple(M) + (mlast,)
        c = coupling_sympy(N, L, Mf)
        if abs(c) > 1e-14:
            out.append((Mf, c))
    return out


def basis_function(N, L, dirs) -> np.ndarray:
    """P_L(r1, ..., r_{N-1}) by Eq. (basis-def); dirs is a list of [..., 3] arrays that
    broadcast against each other."""
    ell = principal(N, L)
    total = 0.0
    for M, c in basis_terms(N, L):
        prod = c
        for k in range(N - 1):
            prod = prod * ylm_scipy(ell[k], M[k], dirs[k])
        total = total + prod
    return total


def shells_f32(pos: np.ndarray, i: int, edges, box: float = 0.0):
    """Neighbour shells of primary i by the float32 rule; returns (shell[n], d[n,3] float32)."""
    pos = np.asarray(pos, dtype=np.float32)
    d = (pos - pos[i]).astype(np.float32)
    if box > 0:
        L = np.float32(box)
        h = np.float32(0.5 * box)
        d = np.where(d > h, d - L, np.where(d < -h, d + L, d)).astype(np.float32)
    r2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]).astype(np.float32)
    r2 = (r2 + d[:, 2] * d[:, 2]).astype(np.float32)
    e2 = np.array([np.float32(e * e) for e in edges], dtype=np.float32)
    ok = (r2 > 0) & (r2 >= e2[0]) & (r2 < e2[-1])
    b = np.searchsorted(e2, r2, side="right") - 1
    b = np.where(ok, b, -1)
    return b, d


def brute_force_npcf(pos, w, N, lmax, edges, multiplets, bins, box=0.0):
    """sum_i w_i sum_{tuples} prod w_j P_L^*(unit vectors), one P per tuple (Sec. 5.2)."""
    pos = np.asarray(pos, dtype=np.float32)
    w = np.asarray(w, dtype=np.float64)
    out = np.zeros((len(multiplets), len(bins)), dtype=np.complex128)
    for i in range(len(pos)):
        b, d = shells_f32(pos, i, edges, box)
        dd = d.astype(np.float64)
        u = dd / np.linalg.norm(np.where(b[:, None] >= 0, dd, 1.0), axis=1)[:, None]
        members = [np.nonzero(b == s)[0] for s in range(len(edges) - 1)]
        for bi, B in enumerate(bins):
            sets = [members[s] for s in B]
            if any(len(s) == 0 for s in sets):
                continue
            # broadcast grid of tuples (j1, ..., j_{N-1})
            dirs, wts = [], 1.0
            for k, s in enumerate(sets):
                shape = [1] * (N - 1)
                shape[k] = len(s)
                dirs.append(u[s].reshape(shape + [3]))
                wts = wts * w[s].reshape(shape)
            for a, L in enumerate(multiplets):
                P = basis_function(N, tuple(int(x) for x in L), dirs)
                out[a, bi] += w[i] * np.sum(np.conj(P) * wts)
    return out
