"""The C-ABI library builds, loads and exports every entry point include/qcw.h declares.

No compute call is made (no GPU here); the GPU tests exercise the same entry points.
"""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"QCW_API\s+[\w\s\*]+?\b(qcw_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1101_1785_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("qcw_create", "qcw_apply_gate1", "qcw_apply_gate2", "qcw_apply_kraus", "qcw_measure",
                 "qcw_partial_trace", "qcw_trace", "qcw_purity", "qcw_probabilities"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    from paper_1101_1785_gb300 import SIGNATURES

    assert _declared() == set(SIGNATURES), _declared() ^ set(SIGNATURES)


def test_binding_loads_without_gpu(libpath):
    import paper_1101_1785_gb300 as q

    L = q.lib()
    assert L.qcw_strerror(q.QCW_EZEROPROB) == b"zero-probability outcome"
    # argument checks run before any device work
    assert L.qcw_create(0, ctypes.byref(ctypes.c_void_p())) == q.QCW_EINVAL
    assert L.qcw_create(q._binding.QCW_MAX_QUBITS + 1, ctypes.byref(ctypes.c_void_p())) == q.QCW_EINVAL
    assert L.qcw_trace(None, None, None) == q.QCW_EINVAL
