"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check compares the oracle with something other than itself: numbers the
paper prints (tests/golden/), closed forms, library routines (scipy spherical
harmonics, sympy 3-j / 9-j symbols), invariances, and brute-force tuple sums.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
import indep

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
FOURPI = 4.0 * math.pi


def _golden_rows(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("|")[0].strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


# ---------------------------------------------------------------- enumerations

def test_printed_dimension_counts():
    for q, N, lmax, ap, val in _golden_rows("enumeration_counts.txt"):
        N, val = int(N), int(val)
        if q == "multiplets":
            assert len(oracle.multiplets(N, int(lmax), bool(int(ap)))) == val, (q, N, lmax, ap)
        elif q == "terms":
            assert oracle.count_terms(N, int(lmax), bool(int(ap))) == val, (q, N, lmax, ap)
        elif q == "components":
            assert len(oracle.multiplets(N, int(lmax))) * len(oracle.bins(N, 10)) == val
        elif q == "bins":
            assert len(oracle.bins(N, 10)) == val
        elif q == "multiplets_icap":
            lm = int(lmax)
            assert len(oracle.multiplets_cap(N, lm, lm, bool(int(ap)))) == val, (q, N, lmax)


def test_bins_are_strictly_ordered_tuples():
    for N, nr in [(3, 10), (4, 10), (5, 8)]:
        b = oracle.bins(N, nr)
        assert len(b) == math.comb(nr, N - 1)
        assert np.all(np.diff(b, axis=1) > 0)
        assert len({tuple(x) for x in b}) == len(b)
        assert [tuple(x) for x in b] == sorted(tuple(x) for x in b)


def test_multiplets_triangle_and_parity():
    for L in oracle.multiplets(4, 5, True):
        l1, l2, l3 = L
        assert abs(l1 - l2) <= l3 <= l1 + l2 and max(L) <= 5
    for L in oracle.multiplets(5, 4, False):
        l1, l2, l12, l3, l4 = L
        assert abs(l1 - l2) <= l12 <= l1 + l2 and abs(l12 - l3) <= l4 <= l12 + l3
        assert (l1 + l2 + l3 + l4) % 2 == 0
    lam6 = oracle.multiplets(6, 3, False)
    for L in lam6:
        l1, l2, l12, l3, l123, l4, l5 = L
        assert abs(l1 - l2) <= l12 <= l1 + l2 and abs(l12 - l3) <= l123 <= l12 + l3
        assert abs(l123 - l4) <= l5 <= l123 + l4 and max(l1, l2, l3, l4, l5) <= 3
        assert (l1 + l2 + l3 + l4 + l5) % 2 == 0
    # the natural range of the intermediates is 2 lmax: a cap there changes nothing, and
    # every capped multiplet is one of the uncapped ones
    assert np.array_equal(oracle.multiplets_cap(6, 3, 6), lam6)
    capped = {tuple(x) for x in oracle.multiplets_cap(6, 3, 3)}
    assert capped <= {tuple(x) for x in lam6} and all(max(L[2], L[4]) <= 3 for L in capped)


# ---------------------------------------------------------------- 3-j symbols

def test_wigner3j_matches_sympy():
    pytest.importorskip("sympy")
    for j1, j2, j3 in itertools.product(range(6), repeat=3):
        if not abs(j1 - j2) <= j3 <= j1 + j2:
            continue
        for m1 in range(-j1, j1 + 1):
            for m2 in range(-j2, j2 + 1):
                m3 = -m1 - m2
                if abs(m3) > j3:
                    continue
                assert oracle.wigner3j(j1, j2, j3, m1, m2, m3) == pytest.approx(
                    indep.w3j(j1, j2, j3, m1, m2, m3), abs=1e-14)


def test_wigner3j_orthogonality():
    # sum_{m1 m2} (j1 j2 j3; m1 m2 m3)(j1 j2 j3'; m1 m2 m3') = delta delta / (2 j3 + 1)
    for j1, j2 in [(2, 3), (5, 4), (7, 7)]:
        for j3 in range(abs(j1 - j2), j1 + j2 + 1):
            for j3p in range(abs(j1 - j2), j1 + j2 + 1):
                for m3 in range(-min(j3, j3p), min(j3, j3p) + 1):
                    s = sum(oracle.wigner3j(j1, j2, j3, m1, -m1 - m3, m3) *
                            oracle.wigner3j(j1, j2, j3p, m1, -m1 - m3, m3)
                            for m1 in range(-j1, j1 + 1) if abs(m1 + m3) <= j2)
                    want = 1.0 / (2 * j3 + 1) if j3 == j3p else 0.0
                    assert s == pytest.approx(want, abs=1e-13)


def test_wigner3j_special_value():
    # (l l 0; m -m 0) = (-1)^{l-m} / sqrt(2l+1)  (DLMF 34.3.1)
    for l in range(11):
        for m in range(-l, l + 1):
            assert oracle.wigner3j(l, l, 0, m, -m, 0) == pytest.approx(
                (-1) ** (l - m) / math.sqrt(2 * l + 1), abs=1e-15)


# ---------------------------------------------------------------- spherical harmonics

def _dirs(n, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1)[:, None]


def test_ylm_closed_forms():
    for x, y, z in _dirs(20, 1):
        Y = oracle.ylm(2, (x, y, z))
        assert Y[0] == pytest.approx(1 / math.sqrt(FOURPI), abs=1e-15)
        assert Y[2] == pytest.approx(math.sqrt(3 / FOURPI) * z, abs=1e-15)             # Y_10
        assert Y[3] == pytest.approx(-math.sqrt(3 / (2 * FOURPI)) * (x + 1j * y), abs=1e-15)  # Y_11
        # Y_{2,-1} = sqrt(15/(8 pi)) (x - i y) z  (the example in Sec. 4.1.1)
        assert Y[5] == pytest.approx(math.sqrt(15 / (8 * math.pi)) * (x - 1j * y) * z, abs=1e-14)
        assert Y[6] == pytest.approx(math.sqrt(5 / (16 * math.pi)) * (3 * z * z - 1), abs=1e-14)


def test_ylm_matches_scipy():
    for v in _dirs(30, 2):
        Y = oracle.ylm(10, v)
        for l in range(11):
            for m in range(-l, l + 1):
                assert Y[l * l + l + m] == pytest.approx(complex(indep.ylm_scipy(l, m, v)), abs=1e-12)


def test_ylm_addition_theorem():
    from scipy.special import eval_legendre
    d = _dirs(10, 3)
    for u, v in zip(d[:5], d[5:]):
        Yu, Yv = oracle.ylm(8, u), oracle.ylm(8, v)
        for l in range(9):
            s = sum(Yu[l * l + l + m] * np.conj(Yv[l * l + l + m]) for m in range(-l, l + 1))
            assert s == pytest.approx((2 * l + 1) / FOURPI * eval_legendre(l, float(u @ v)), abs=1e-13)


def test_ylm_orthonormal_by_quadrature():
    lmax = 5
    xg, wg = np.polynomial.legendre.leggauss(16)
    nphi = 24
    phis = 2 * math.pi * np.arange(nphi) / nphi
    gram = np.zeros(((lmax + 1) ** 2,) * 2, dtype=complex)
    for ct, wt in zip(xg, wg):
        st = math.sqrt(1 - ct * ct)
        for ph in phis:
            Y = oracle.ylm(lmax, (st * math.cos(ph), st * math.sin(ph), ct))
            gram += wt * (2 * math.pi / nphi) * np.outer(Y, np.conj(Y))
    assert np.allclose(gram, np.eye(len(gram)), atol=1e-12)


# ---------------------------------------------------------------- couplings / basis

def test_coupling_orthonormality():
    # Eq. (basis-orthogonality) with orthonormal Y's: sum_M C^L_M C^L'_M = delta_{LL'}.
    # For N=5 and 6 this fixes the sqrt(2 l12 + 1) (sqrt(2 l123 + 1)) factors of
    # Eq. (basis-coupling); for N=6 it also separates multiplets that differ only in l123.
    for N, lmax in [(3, 6), (4, 3), (5, 2), (6, 1)]:
        lam = oracle.multiplets(N, lmax, True)
        ell = [indep.principal(N, L) for L in lam]
        for a, La in enumerate(lam):
            for b, Lb in enumerate(lam):
                if ell[a] != ell[b]:
                    continue
                s = 0.0
                for M in itertools.product(*[range(-l, l + 1) for l in ell[a]]):
                    if sum(M) != 0:
                        continue
                    s += oracle.coupling(N, La, M) * oracle.coupling(N, Lb, M)
                assert s == pytest.approx(1.0 if a == b else 0.0, abs=1e-13), (N, La, Lb)


def test_coupling_matches_sympy_definition():
    pytest.importorskip("sympy")
    for N, lmax in [(3, 4), (4, 3), (5, 2), (6, 1)]:
        for L in oracle.multiplets(N, lmax, True):
            for M, c in indep.basis_terms(N, tuple(int(x) for x in L)):
                assert oracle.coupling(N, L, M) == pytest.approx(c, abs=1e-14)


def test_coupling_M_inversion():
    # Eq. (basis-coupling-M-inversion): C^L_{-M} = E(L) C^L_M
    for N, lmax in [(4, 4), (5, 3), (6, 1)]:
        for L in oracle.multiplets(N, lmax, True):
            ell = indep.principal(N, L)
            E = (-1) ** sum(ell)
            for M in itertools.product(*[range(-l, l + 1) for l in ell]):
                if sum(M) != 0:
                    continue
                assert oracle.coupling(N, L, [-m for m in M]) == pytest.approx(
                    E * oracle.coupling(N, L, M), abs=1e-15)


def test_n5_coupling_is_n6_with_l5_zero():
    # Eq. (basis-coupling): with l5 = 0 the last 3-j symbol forces l123 = l4, m123 = -m4 and
    # equals (-1)^{l4+m4} / sqrt(2 l4 + 1), which cancels the sqrt(2 l123 + 1) factor and
    # the (-1)^{l123 - m123} phase: the N=6 coefficient is the N=5 one
    for L in oracle.multiplets(5, 2, True):
        l1, l2, l12, l3, l4 = (int(x) for x in L)
        L6 = [l1, l2, l12, l3, l4, l4, 0]
        for M in itertools.product(*[range(-l, l + 1) for l in (l1, l2, l3)]):
            m4 = -sum(M)
            if abs(m4) > l4:
                continue
            assert oracle.coupling(6, L6, list(M) + [m4, 0]) == pytest.approx(
                oracle.coupling(5, L, list(M) + [m4]), abs=1e-14)


def test_n3_coupling_is_n4_with_l3_zero():
    # Eq. (N=3-coeff) equals Eq. (N=4-coeff) at l3 = 0
    for l in range(8):
        for m in range(-l, l + 1):
            assert oracle.coupling(3, [l, l], [m, -m]) == pytest.approx(
                oracle.coupling(4, [l, l, 0], [m, -m, 0]), abs=1e-15)


def _oracle_basis(N, L, dirs):
    """P_L at one configuration from the oracle's own Y and C (Eq. basis-def)."""
    ell = indep.principal(N, L)
    lmax = max(ell)
    Ys = [oracle.ylm(lmax, d) for d in dirs]
    tot = 0.0
    for M in itertools.product(*[range(-l, l + 1) for l in ell]):
        if sum(M) != 0:
            continue
        c = oracle.coupling(N, L, M)
        p = c
        for k, (l, m) in enumerate(zip(ell, M)):
            p = p * Ys[k][l * l + l + m]
        tot += p
    return tot


def test_basis_p110_printed_closed_form():
    rows = _golden_rows("basis_p110.txt")
    N, l1, l2, l3, coef = rows[0]
    d = _dirs(9, 4)
    for k in range(3):
        r1, r2, r3 = d[3 * k], d[3 * k + 1], d[3 * k + 2]
        P = _oracle_basis(int(N), (int(l1), int(l2), int(l3)), [r1, r2, r3])
        assert P == pytest.approx(float(coef) * float(r1 @ r2), abs=1e-15)


def test_basis_zero_multiplet_constant():
    # Eq. (basis-zero-ell): P_0 = (4 pi)^{-(N-1)/2}
    d = _dirs(4, 5)
    assert _oracle_basis(3, (0, 0), d[:2]) == pytest.approx(FOURPI ** -1.0)
    assert _oracle_basis(4, (0, 0, 0), d[:3]) == pytest.approx(FOURPI ** -1.5)
    assert _oracle_basis(5, (0, 0, 0, 0, 0), d[:4]) == pytest.approx(FOURPI ** -2.0)


def test_basis_rotation_invariance_and_conjugation():
    from scipy.spatial.transform import Rotation
    R = Rotation.random(random_state=6).as_matrix()
    d = _dirs(4, 7)
    for N, lmax in [(4, 3), (5, 2)]:
        for L in oracle.multiplets(N, lmax, True)[::3]:
            k = N - 1
            P = _oracle_basis(N, L, d[:k])
            PR = _oracle_basis(N, L, [R @ x for x in d[:k]])
            assert PR == pytest.approx(P, abs=1e-13)             # Eq. (basis-rotation)
            E = (-1) ** sum(indep.principal(N, L))
            assert np.conj(P) == pytest.approx(E * P, abs=1e-13)  # Eq. (basis-conjugation)


# ---------------------------------------------------------------- neighbour rule

def test_shell_rule_edges_and_wrap():
    edges = [0.0, 1.0, 2.0, 3.0]
    o = np.zeros(3, np.float32)
    assert oracle.shell(o, [0.5, 0, 0], edges) == 0
    assert oracle.shell(o, [1.0, 0, 0], edges) == 1         # lower edge belongs to the shell
    assert oracle.shell(o, [3.0, 0, 0], edges) == -1        # upper edge of the last shell excluded
    assert oracle.shell(o, [0, 0, 0], edges) == -1          # coincident point
    assert oracle.shell([0.5, 0, 0], [9.8, 0, 0], edges, box=10.0) == 0   # wraps to -0.7
    assert oracle.shell([9.9, 0, 0], [0.2, 0, 0], edges, box=10.0) == 0   # wraps to +0.3
    assert oracle.shell([0.0, 0, 0], [5.0, 0, 0], [0, 6.0], box=10.0) == 0  # exactly L/2 not wrapped


def test_pair_counts_match_numpy_float32_rule():
    rng = np.random.default_rng(8)
    pos = rng.uniform(0, 100, size=(400, 3)).astype(np.float32)
    edges = np.linspace(3.0, 30.0, 8)
    for box in (0.0, 100.0):
        want = np.zeros(7, np.uint64)
        for i in range(len(pos)):
            b, _ = indep.shells_f32(pos, i, edges, box)
            want += np.bincount(b[b >= 0], minlength=7).astype(np.uint64)
        got = oracle.pair_counts(pos, edges, box)
        assert np.array_equal(got, want)


# ---------------------------------------------------------------- a_lm

def test_alm_matches_scipy_and_conjugation():
    rng = np.random.default_rng(9)
    pos = rng.uniform(0, 60, size=(300, 3)).astype(np.float32)
    w = rng.uniform(0.5, 1.5, size=300).astype(np.float32)
    edges = np.linspace(2.0, 20.0, 5)
    lmax = 4
    prim = np.array([0, 17, 123])
    a, cnt = oracle.alm(pos, w, prim, lmax, edges, box=60.0)
    for q, i in enumerate(prim):
        b, d = indep.shells_f32(pos, i, edges, 60.0)
        for s in range(4):
            sel = b == s
            assert cnt[q, s] == sel.sum()
            u = d[sel].astype(np.float64)
            for l in range(lmax + 1):
                for m in range(-l, l + 1):
                    want = np.sum(w[sel] * indep.ylm_scipy(l, m, u)) if sel.any() else 0
                    assert a[q, s, l * l + l + m] == pytest.approx(complex(want), abs=1e-11)
                    # a_{l,-m} = (-1)^m conj(a_{lm})  (Sec. 4.1.1, App. B)
                    assert a[q, s, l * l + l - m] == pytest.approx(
                        (-1) ** m * np.conj(a[q, s, l * l + l + m]), abs=1e-12)


# ---------------------------------------------------------------- NPCF estimator

def _small_catalog(n, side, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, side, size=(n, 3)).astype(np.float32), \
        rng.uniform(0.5, 1.5, size=n).astype(np.float32)


def test_npcf3_equals_legendre_form():
    # Eq. (N=3-basis): P_l = sqrt(2l+1)/(4 pi) (-1)^l L_l(r1 . r2); brute force over pairs
    from scipy.special import eval_legendre
    pos, w = _small_catalog(250, 50.0, 10)
    edges = np.linspace(2.0, 14.0, 5)
    lmax, box = 6, 50.0
    z, cnt = oracle.npcf(pos, w, (3,), lmax, edges, box)
    z = z.reshape(lmax + 1, -1)
    bins = oracle.bins(3, 4)
    want = np.zeros_like(z)
    for i in range(len(pos)):
        b, d = indep.shells_f32(pos, i, edges, box)
        u = d.astype(np.float64)
        u[b >= 0] /= np.linalg.norm(u[b >= 0], axis=1)[:, None]
        for bi, (b1, b2) in enumerate(bins):
            s1, s2 = np.nonzero(b == b1)[0], np.nonzero(b == b2)[0]
            if len(s1) == 0 or len(s2) == 0:
                continue
            mu = u[s1] @ u[s2].T
            ww = np.outer(w[s1].astype(np.float64), w[s2].astype(np.float64))
            for l in range(lmax + 1):
                P = math.sqrt(2 * l + 1) / FOURPI * (-1) ** l * eval_legendre(l, mu)
                want[l, bi] += float(w[i]) * np.sum(ww * P)
    scale = np.sqrt(np.mean(want ** 2))
    assert np.max(np.abs(z - want)) <= 1e-12 * scale


def test_npcf4_brute_force_tuples_all_parity():
    pytest.importorskip("sympy")
    pos, w = _small_catalog(70, 40.0, 11)
    edges = np.array([3.0, 7.0, 10.0, 13.0, 16.0])
    lmax = 2
    lam = oracle.multiplets(4, lmax, True)
    bins = oracle.bins(4, 4)
    z, _, resid = oracle.npcf(pos, w, (4,), lmax, edges, 0.0, allparity=True, return_resid=True)
    z = z.reshape(len(lam), len(bins))
    bf = indep.brute_force_npcf(pos, w, 4, lmax, edges, lam, bins)
    odd = np.array([sum(L) % 2 for L in lam], bool)
    want = np.where(odd[:, None], bf.imag, bf.real)
    other = np.where(odd[:, None], bf.real, bf.imag)
    scale = np.sqrt(np.mean(want ** 2))
    assert scale > 0
    assert np.max(np.abs(z - want)) <= 1e-12 * scale
    assert np.max(np.abs(other)) <= 1e-12 * scale
    assert np.max(np.abs(resid)) <= 1e-12 * scale


def test_npcf5_brute_force_tuples():
    pytest.importorskip("sympy")
    pos, w = _small_catalog(40, 30.0, 12)
    edges = np.array([3.0, 6.0, 9.0, 12.0, 15.0])
    lmax = 1
    lam = oracle.multiplets(5, lmax, True)
    bins = oracle.bins(5, 4)
    z, _ = oracle.npcf(pos, w, (5,), lmax, edges, 0.0, allparity=True)
    z = z.reshape(len(lam), len(bins))
    bf = indep.brute_force_npcf(pos, w, 5, lmax, edges, lam, bins)
    odd = np.array([(L[0] + L[1] + L[3] + L[4]) % 2 for L in lam], bool)
    want = np.where(odd[:, None], bf.imag, bf.real)
    scale = np.sqrt(np.mean(want ** 2))
    assert scale > 0
    assert np.max(np.abs(z - want)) <= 1e-12 * scale


def test_npcf6_brute_force_tuples():
    # Sec. 5.2 brute force for the 6PCF: every 5-tuple of secondaries in distinct shells,
    # P_L from scipy Y's and sympy 3-j symbols (all parities, lmax 1)
    pytest.importorskip("sympy")
    pos, w = _small_catalog(36, 30.0, 19)
    edges = np.array([2.0, 5.0, 8.0, 11.0, 14.0, 17.0])
    lmax = 1
    lam = oracle.multiplets(6, lmax, True)
    bins = oracle.bins(6, 5)
    z, _ = oracle.npcf(pos, w, (6,), lmax, edges, 0.0, allparity=True)
    z = z.reshape(len(lam), len(bins))
    bf = indep.brute_force_npcf(pos, w, 6, lmax, edges, lam, bins)
    odd = np.array([(L[0] + L[1] + L[3] + L[5] + L[6]) % 2 for L in lam], bool)
    want = np.where(odd[:, None], bf.imag, bf.real)
    scale = np.sqrt(np.mean(want ** 2))
    assert scale > 0
    assert np.max(np.abs(z - want)) <= 1e-12 * scale


def _pair_weights(pos, w, edges, box):
    """W_b(i) = sum of secondary weights of i in shell b (a weighted pair count)."""
    nr = len(edges) - 1
    W = np.zeros((len(pos), nr))
    for i in range(len(pos)):
        b, _ = indep.shells_f32(pos, i, edges, box)
        for s in range(nr):
            W[i, s] = w[b == s].astype(np.float64).sum()
    return W


def test_l0_multiplets_are_pair_count_products():
    # Eq. (basis-zero-ell): the L = 0 multiplet is (4 pi)^{-(N-1)/2} sum_i w_i prod_k W_{b_k}(i)
    pos, w = _small_catalog(300, 60.0, 13)
    edges = np.linspace(4.0, 20.0, 6)
    box = 60.0
    W = _pair_weights(pos, w, edges, box)
    z, _ = oracle.npcf(pos, w, (3, 4, 5, 6), 2, edges, box)
    parts = oracle.split_orders(z, (3, 4, 5, 6), 2, 5)
    for N in (3, 4, 5, 6):
        want = np.array([np.sum(w.astype(np.float64) * np.prod(W[:, list(B)], axis=1))
                         for B in oracle.bins(N, 5)]) * FOURPI ** (-(N - 1) / 2)
        assert np.allclose(parts[N][0], want, rtol=1e-12, atol=0)


def test_cross_order_identity_0ll():
    # C^{0 l l}_{0,m,-m} (Eq. N=4-coeff) equals the N=3 coefficient, so
    # zeta4_{0 l l}(b1,b2,b3) = (4 pi)^{-1/2} sum_i w_i W_{b1}(i) h_l(b2,b3; i)
    pos, w = _small_catalog(120, 50.0, 14)
    edges = np.linspace(3.0, 18.0, 5)
    box, lmax = 50.0, 3
    W = _pair_weights(pos, w, edges, box)
    lam4 = [tuple(L) for L in oracle.multiplets(4, lmax)]
    b3 = [tuple(B) for B in oracle.bins(3, 4)]
    b4 = [tuple(B) for B in oracle.bins(4, 4)]
    z4, _ = oracle.npcf(pos, w, (4,), lmax, edges, box)
    z4 = z4.reshape(len(lam4), len(b4))
    want = np.zeros((lmax + 1, len(b4)))
    for i in range(len(pos)):
        # h_l(b2, b3; i): the 3PCF contribution of primary i with unit primary weight
        wp = np.zeros(len(pos), np.float32)
        wp[i] = 1.0
        h, _ = oracle.npcf(pos, w, (3,), lmax, edges, box, wprim=wp, prim=[i])
        h = h.reshape(lmax + 1, len(b3))
        for bi, (x1, x2, x3) in enumerate(b4):
            want[:, bi] += float(w[i]) * W[i, x1] * h[:, b3.index((x2, x3))]
    want *= FOURPI ** -0.5
    for l in range(lmax + 1):
        assert np.allclose(z4[lam4.index((0, l, l))], want[l], rtol=1e-11, atol=1e-12)


def _edges_avoiding(pos, lo, hi, nr, gap=2e-4):
    """Shell edges placed away from every pair distance, so float32 rounding of a
    rotated catalog cannot move a pair across an edge."""
    d = np.sqrt(((pos[:, None, :].astype(np.float64) - pos[None, :, :]) ** 2).sum(-1))
    dist = np.sort(d[np.triu_indices(len(pos), 1)])
    edges = []
    for t in np.linspace(lo, hi, nr + 1):
        k = np.searchsorted(dist, t)
        cands = []
        for j in range(max(k - 200, 1), min(k + 200, len(dist))):
            if dist[j] - dist[j - 1] > 2 * gap:
                cands.append(0.5 * (dist[j] + dist[j - 1]))
        edges.append(min(cands, key=lambda c: abs(c - t)))
    return np.array(edges)


def test_rotation_invariance_non_periodic():
    from scipy.spatial.transform import Rotation
    pos, w = _small_catalog(150, 40.0, 15)
    pos = pos - 20.0
    edges4 = _edges_avoiding(pos, 4.0, 16.0, 4)
    edges5 = _edges_avoiding(pos, 4.0, 18.0, 5)   # the 6PCF needs five shells
    R = Rotation.random(random_state=16).as_matrix()
    rpos = (pos.astype(np.float64) @ R.T).astype(np.float32)
    for orders, lmax, edges in [((3, 4), 3, edges4), ((5,), 2, edges4), ((6,), 1, edges5)]:
        z, c = oracle.npcf(pos, w, orders, lmax, edges, 0.0, allparity=True)
        zr, cr = oracle.npcf(rpos, w, orders, lmax, edges, 0.0, allparity=True)
        assert np.array_equal(c, cr)
        # rotated float32 positions are rounded (~1e-7 relative), which moves each unit
        # vector by ~1e-7; a wrong sign or index would move zeta by O(1) of its RMS
        scale = np.sqrt(np.mean(z ** 2))
        assert np.max(np.abs(z - zr)) <= 1e-6 * scale


def test_reflection_multiplies_by_parity():
    # Sec. 3.1: under x -> -x (parity) zeta_L picks up E(L); negation is exact in float32.
    pos, w = _small_catalog(150, 40.0, 17)
    pos = pos - np.float32(20.0)
    edges = np.linspace(4.0, 16.0, 5)
    lmax = 3
    z, _ = oracle.npcf(pos, w, (4,), lmax, edges, 0.0, allparity=True)
    zr, _ = oracle.npcf(-pos, w, (4,), lmax, edges, 0.0, allparity=True)
    lam = oracle.multiplets(4, lmax, True)
    E = np.array([(-1) ** sum(L) for L in lam], float)
    z, zr = z.reshape(len(lam), -1), zr.reshape(len(lam), -1)
    scale = np.sqrt(np.mean(z ** 2))
    assert np.max(np.abs(zr - E[:, None] * z)) <= 1e-12 * scale
    assert np.max(np.abs(z[E < 0])) > 1e-6 * scale   # odd multiplets are not trivially zero


def test_primary_subset_and_weights_are_additive():
    pos, w = _small_catalog(200, 50.0, 18)
    edges = np.linspace(3.0, 15.0, 5)
    full, _ = oracle.npcf(pos, w, (3, 4), 2, edges, 50.0)
    a, _ = oracle.npcf(pos, w, (3, 4), 2, edges, 50.0, prim=np.arange(0, 90))
    b, _ = oracle.npcf(pos, w, (3, 4), 2, edges, 50.0, prim=np.arange(90, 200))
    assert np.allclose(a + b, full, rtol=1e-12, atol=1e-12 * np.abs(full).max())
    wp = w.copy()
    wp[100:] = 0
    c, _ = oracle.npcf(pos, w, (3, 4), 2, edges, 50.0, wprim=wp)
    d, _ = oracle.npcf(pos, w, (3, 4), 2, edges, 50.0, prim=np.arange(100))
    assert np.allclose(c, d, rtol=1e-12, atol=1e-12 * np.abs(full).max())


# ---------------------------------------------------------------- generalised Gaunt / edge correction

def test_gaunt_n3_appendix_form():
    # App. A, N=3: G = (4 pi)^-1 sqrt((2l+1)(2l'+1)(2l''+1)) (l l' l''; 0 0 0)^2
    for l, lp, lpp in itertools.product(range(4), repeat=3):
        want = math.sqrt((2 * l + 1) * (2 * lp + 1) * (2 * lpp + 1)) / FOURPI * \
            oracle.wigner3j(l, lp, lpp, 0, 0, 0) ** 2
        assert oracle.gaunt(3, [l, l], [lp, lp], [lpp, lpp]) == pytest.approx(want, abs=1e-14)


def _gaunt_appendix(N, L, Lp, Lpp):
    """App. A closed forms with sympy 3-j and 9-j symbols."""
    ell, ellp, ellpp = (indep.principal(N, x) for x in (L, Lp, Lpp))
    pref = 1.0
    for a, b, c in zip(ell, ellp, ellpp):
        pref *= math.sqrt((2 * a + 1) * (2 * b + 1) * (2 * c + 1)) * indep.w3j(a, b, c, 0, 0, 0)
    if N == 4:
        return FOURPI ** -1.5 * pref * indep.w9j(L[0], Lp[0], Lpp[0], L[1], Lp[1], Lpp[1],
                                                 L[2], Lp[2], Lpp[2])
    l12, l12p, l12pp = L[2], Lp[2], Lpp[2]
    pref *= math.sqrt((2 * l12 + 1) * (2 * l12p + 1) * (2 * l12pp + 1))
    return FOURPI ** -2 * pref * \
        indep.w9j(L[0], L[1], l12, Lp[0], Lp[1], l12p, Lpp[0], Lpp[1], l12pp) * \
        indep.w9j(l12, L[3], L[4], l12p, Lp[3], Lp[4], l12pp, Lpp[3], Lpp[4])


def test_gaunt_n4_n5_appendix_9j_forms():
    pytest.importorskip("sympy")
    rng = np.random.default_rng(19)
    for N, lmax, ntrip in [(4, 2, 150), (5, 1, 150)]:
        lam = oracle.multiplets(N, lmax, False)
        for _ in range(ntrip):
            a, b, c = (lam[k] for k in rng.integers(0, len(lam), 3))
            got = oracle.gaunt(N, a, b, c)
            want = _gaunt_appendix(N, a, b, c)
            assert got == pytest.approx(want, abs=1e-13), (N, a, b, c)


def test_gaunt_with_zero_multiplet():
    # From Eqs. (basis-orthogonality), (basis-zero-ell): G^{L 0 L''} = (4pi)^{-(N-1)/2} E(L'') delta
    for N, lmax in [(3, 3), (4, 2), (5, 1)]:
        lam = oracle.multiplets(N, lmax, True)
        zero = lam[0]
        for a in lam:
            for c in lam:
                E = (-1) ** sum(indep.principal(N, c))
                want = FOURPI ** (-(N - 1) / 2) * E if tuple(a) == tuple(c) else 0.0
                assert oracle.gaunt(N, a, zero, c) == pytest.approx(want, abs=1e-14)


def test_edge_correction_uniform_window_is_diagonal():
    # Eq. (R-periodic-form): R_L = R_0 delta_{L0} gives M = (4pi)^{-(N-1)/2} I
    N, lmax, nr = 4, 2, 4
    nl, nb = len(oracle.multiplets(N, lmax)), len(oracle.bins(N, nr))
    rng = np.random.default_rng(20)
    nraw = rng.normal(size=(nl, nb))
    rraw = np.zeros((nl, nb))
    rraw[0] = rng.uniform(1, 2, size=nb)
    z = oracle.edge_correct(N, lmax, nr, nraw, rraw)
    assert np.allclose(z, nraw / rraw[0] * FOURPI ** 1.5, rtol=1e-13)


def test_edge_correction_recovers_injected_zeta():
    # Build N_{L''}/R_0 = sum_L zeta_L M_{L L''} from the App. A closed form of G and a
    # random near-uniform window; the oracle's solve must give zeta back (Eq. edge-corrected-NPCF).
    pytest.importorskip("sympy")
    N, lmax, nr = 4, 2, 3
    lam = oracle.multiplets(N, lmax)
    nl, nb = len(lam), len(oracle.bins(N, nr))
    G = np.array([[[_gaunt_appendix(N, a, b, c) for c in lam] for b in lam] for a in lam])
    rng = np.random.default_rng(21)
    zeta = rng.normal(size=(nl, nb))
    rraw = rng.normal(scale=0.1, size=(nl, nb))
    rraw[0] = rng.uniform(1, 2, size=nb)
    nraw = np.zeros((nl, nb))
    for bb in range(nb):
        f = rraw[:, bb] / rraw[0, bb]
        M = np.einsum("b,abc->ac", f, G)       # M_{L L''} = sum_L' f_L' G^{L L' L''}
        nraw[:, bb] = (zeta[:, bb] @ M) * rraw[0, bb]
    z = oracle.edge_correct(N, lmax, nr, nraw, rraw)
    assert np.allclose(z, zeta, rtol=1e-10, atol=1e-10)
