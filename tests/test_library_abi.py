"""The C-ABI library builds for sm_103a, loads, and exports every declared symbol.

No compute call is made here (no GPU): only symbol resolution and the argument checks
that npcf_create performs before touching the device.
"""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(npcf_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2105_08722_gb300 import build
    from paper_2105_08722_gb300 import _lib
    build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_symbols()
    assert len(names) >= 14
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_2105_08722_gb300 import _lib
    assert _declared_symbols() == set(_lib.SIGNATURES)


def test_create_rejects_bad_arguments_before_touching_the_device(lib):
    from paper_2105_08722_gb300._lib import NPCF, NPCFError, NPCF_EINVAL, NPCF_EUNSUPPORTED
    edges = np.linspace(1.0, 10.0, 4)
    with pytest.raises(NPCFError) as e:
        NPCF(11, (3,), edges)                       # lmax too large
    assert e.value.status == NPCF_EINVAL
    with pytest.raises(NPCFError) as e:
        NPCF(3, (3,), [1.0, 0.5, 2.0])              # edges not increasing
    assert e.value.status == NPCF_EINVAL
    with pytest.raises(NPCFError) as e:
        NPCF(3, (3,), edges, box=20.0)              # periodic box must exceed 3 r_max
    assert e.value.status == NPCF_EINVAL
    with pytest.raises(NPCFError) as e:
        NPCF(3, (7,), edges)                        # unsupported order
    assert e.value.status == NPCF_EINVAL
    with pytest.raises(NPCFError) as e:
        NPCF(3, (3,), np.linspace(1, 2, 18))        # more than 16 shells
    assert e.value.status == NPCF_EINVAL
    h = ctypes.c_void_p()
    assert lib.npcf_create(None, 3, 8, 3, edges.ctypes.data, 0.0, 0, 0) == NPCF_EINVAL
    assert lib.npcf_create(ctypes.byref(h), 3, 8, 3, None, 0.0, 0, 0) == NPCF_EINVAL
    assert h.value is None
    assert b"edges" in lib.npcf_last_error(None)


@pytest.mark.parametrize("N,lmax", [(3, 6), (4, 2), (5, 1)])
def test_library_gaunt_closed_forms_match_the_oracle_definition(lib, N, lmax):
    # npcf_gaunt evaluates the App. A closed forms (3-j and 9-j symbols, host code of
    # the library); the oracle integrates Eq. (generalized-gaunt-def) through its dense
    # coupling coefficients. Every triple of multiplets at small lmax.
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import oracle
    from paper_2105_08722_gb300 import _lib
    oracle.build()
    width = {3: 2, 4: 3, 5: 5}[N]
    lam = np.asarray(oracle.multiplets(N, lmax, False)).reshape(-1, width)
    nonzero = 0
    for a in lam:
        for b in lam:
            for c in lam:
                got = _lib.gaunt(N, a, b, c)
                want = oracle.gaunt(N, a, b, c)
                assert got == pytest.approx(want, abs=1e-13), (a, b, c)
                nonzero += abs(want) > 1e-12
    assert nonzero > len(lam)


def test_gaunt_rejects_bad_order(lib):
    from paper_2105_08722_gb300 import _lib
    with pytest.raises(_lib.NPCFError):
        _lib.gaunt(6, [0] * 5, [0] * 5, [0] * 5)


@pytest.mark.parametrize("N,lmax", [(3, 4), (4, 3), (5, 2), (6, 1), (6, 2)])
def test_library_multiplets_and_couplings_match_the_oracle(lib, N, lmax):
    # the library's host tables (npcf_multiplets, npcf_coupling) against the oracle's own
    # enumeration and Eq. (basis-coupling), written separately; the 6PCF tables are the
    # first piece of its GPU path
    import itertools
    import oracle
    from paper_2105_08722_gb300 import _lib
    oracle.build()
    for ap in (False, True):
        got = _lib.multiplets(N, lmax, ap)
        assert np.array_equal(got, oracle.multiplets(N, lmax, ap)), (N, lmax, ap)
    principal = {3: [0, 1], 4: [0, 1, 2], 5: [0, 1, 3, 4], 6: [0, 1, 3, 5, 6]}[N]
    for L in _lib.multiplets(N, lmax, True):
        ell = [int(L[i]) for i in principal]
        for M in itertools.product(*[range(-l, l + 1) for l in ell[:-1]]):
            M = list(M) + [-sum(M)]
            if abs(M[-1]) > ell[-1]:
                continue
            assert _lib.coupling(N, L, M) == pytest.approx(oracle.coupling(N, L, M), abs=1e-14), (L, M)


def test_multiplets_and_coupling_reject_bad_arguments(lib):
    from paper_2105_08722_gb300 import _lib
    with pytest.raises(_lib.NPCFError):
        _lib.multiplets(7, 2)
    with pytest.raises(_lib.NPCFError):
        _lib.multiplets(4, 11)
    with pytest.raises(_lib.NPCFError):
        _lib.coupling(2, [0, 0], [0, 0])
    with pytest.raises(_lib.NPCFError):
        _lib.coupling(4, [1, -1, 0], [0, 0, 0])
