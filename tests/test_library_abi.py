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
        NPCF(3, (6,), edges)                        # unsupported order
    assert e.value.status == NPCF_EINVAL
    with pytest.raises(NPCFError) as e:
        NPCF(3, (3,), np.linspace(1, 2, 18))        # more than 16 shells
    assert e.value.status == NPCF_EINVAL
    h = ctypes.c_void_p()
    assert lib.npcf_create(None, 3, 8, 3, edges.ctypes.data, 0.0, 0, 0) == NPCF_EINVAL
    assert lib.npcf_create(ctypes.byref(h), 3, 8, 3, None, 0.0, 0, 0) == NPCF_EINVAL
    assert h.value is None
    assert b"edges" in lib.npcf_last_error(None)
