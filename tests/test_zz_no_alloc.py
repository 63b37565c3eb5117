"""qcw_partial_trace_static: the partial trace for callers that must not allocate device memory.

It keeps its result in a fixed array inside the library instead of a cudaMallocAsync buffer.
Called through the C ABI on a context's device rho, twice in a row (different states and
kept sets, the second smaller than the first so stale entries would show), and compared
with qcw_partial_trace on the same state.  This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

from tests._helpers import random_rho

pytestmark = pytest.mark.gpu

TOL = 1e-6  # same bound as the other partial-trace parity tests (FP32 state, FP64 sums)


@pytest.fixture(scope="module")
def q():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1101_1785_gb300 as q

    return q


def _static_ptrace(q, d, keep):
    rho_ptr, stream_ptr = d.device_state()
    k = np.ascontiguousarray(np.asarray(sorted(keep), dtype=np.int32))
    out = np.zeros((1 << len(k), 1 << len(k)), dtype=np.complex128)
    st = q.lib().qcw_partial_trace_static(ctypes.c_void_p(rho_ptr), d.n,
                                          k.ctypes.data_as(ctypes.c_void_p) if k.size else None, len(k),
                                          ctypes.c_void_p(stream_ptr), out.ctypes.data_as(ctypes.c_void_p))
    q._binding.check(st, "qcw_partial_trace_static")
    return out


def test_static_partial_trace_matches_allocating_one(q):
    rng = np.random.default_rng(2026)
    calls = [(9, [1, 4, 8]), (7, [0, 6])]
    for n, keep in calls:
        d = q.Density(n)
        d.set_state(random_rho(rng, n))
        want = d.partial_trace(keep)
        got = _static_ptrace(q, d, keep)
        assert np.abs(got - want).max() <= TOL
        assert abs(np.trace(got) - 1) <= TOL
        d.close()


def test_static_partial_trace_block_reduction_and_empty_keep(q):
    """Tracing out eight or more qubits takes the block-reduction kernel; keeping none returns
    the 1 x 1 matrix holding the trace.  The two calls run back to back on the same array."""
    rng = np.random.default_rng(2027)
    d = q.Density(12)
    d.set_state(random_rho(rng, 12))
    want = d.partial_trace([0, 5])
    got = _static_ptrace(q, d, [0, 5])  # 10 qubits traced out
    assert np.abs(got - want).max() <= TOL
    tr = _static_ptrace(q, d, [])
    assert tr.shape == (1, 1)
    assert abs(tr[0, 0] - d.trace()) <= TOL
    assert abs(tr[0, 0] - np.trace(want)) <= TOL
    d.close()


def test_static_partial_trace_rejects_large_outputs(q):
    d = q.Density(8)
    with pytest.raises(q.QcwError) as e:
        _static_ptrace(q, d, list(range(7)))
    assert e.value.status == q.QCW_EINVAL
    d.close()
