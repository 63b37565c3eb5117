"""GPU parity at the depth the benchmark runs, against the complex128 CPU oracle.

* The benchmark's 1000-gate circuit (kinds uniform over H, X, Z, S, T, CNOT, Haar SU(2);
  AD(0.01) + PD(0.02) on every touched qubit, Eq. rhoE2) at 11 qubits, where the oracle
  replays it in minutes: every kernel variant runs it in the benchmark's launch configuration
  (100-gate chunks, an asynchronous checkpoint after each, then probabilities, the u-driven
  measurement of qubit 0 and a partial trace), and the whole final state, every checkpoint,
  the outcome and the post-measurement state are compared with the oracle.
* The 500-gate, 12-qubit depolarising circuit at full depth on the plain path (one launch per
  gate and per channel) and on the fused path, against the oracle's readouts stored by
  tests/golden/make_deep_goldens.py (the oracle needs too long for a test there).
* Caller-owned memory and stream (qcw_create_from_ptr through Density.from_tensor).

Tolerances as everywhere: max |delta rho| <= 1e-5 and |tr rho - 1| <= 1e-6 for the FP32 state
against the FP64 oracle; FP64-summed readouts (purity, probabilities, partial traces) within
1e-6; measurement outcomes identical.
"""

import numpy as np
import pytest

import oracle
import workloads as wl
from tests._helpers import read_golden

pytestmark = pytest.mark.gpu

ATOL = 1e-5
TRACE_TOL = 1e-6
READ_TOL = 1e-6
# Purity after 1000+ operations: each operation's FP32 transfer coefficients (e.g. the
# depolarising factor 1 - 4p/3) carry a relative rounding of up to 6e-8 that repeats with every
# application, so the Pauli components of rho drift by ~1e-6 relative and the purity (quadratic)
# by twice that times its value; the bound is the element tolerance.
DEEP_PURITY_TOL = ATOL
CHUNK = 100
U_MEASURE = 0.37


@pytest.fixture(scope="module")
def q():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1101_1785_gb300 as q

    return q


def _chunks(c):
    bounds = list(range(0, c.n_gates + 1, CHUNK))
    pre = [len(c.gate_prefix(g).ops) for g in bounds]
    return [c.ops[pre[i]:pre[i + 1]] for i in range(len(pre) - 1)]


@pytest.fixture(scope="module")
def deep11():
    """Oracle replay of the 1000-gate benchmark circuit at 11 qubits: readouts after every
    100 gates, the final state, the measurement of qubit 0 and the post-measurement state."""
    c = wl.config3_circuit(n=11)
    rho = oracle.initial_state(c)
    ckpts = []
    for part in _chunks(c):
        for op in part:
            oracle.apply_op(rho, op)
        ckpts.append((oracle.trace(rho), oracle.purity(rho), oracle.probabilities(rho)))
    final = rho.copy()
    m, pm = oracle.measure(rho, 0, -1, U_MEASURE)
    return c, ckpts, final, (m, pm), rho


def _bench_like(q, d, c):
    """The benchmark's sequence of calls: packed 100-gate chunks with a checkpoint after each."""
    tickets = []
    for part in _chunks(c):
        d.apply_packed(q.PackedOps(part))
        tickets.append(d.checkpoint())
    return [d.checkpoint_read(t) for t in tickets]


VARIANTS = {
    "ws_auto_width": ("fused", 0, 0),  # the benchmark's configuration
    "ws_width5": ("fused", 3, 5),
    "ws_width4": ("fused", 3, 4),
    "tc_width5": ("fused", 4, 5),
    "plain": ("plain", 0, 0),
}


@pytest.mark.parametrize("variant", list(VARIANTS))
def test_benchmark_circuit_full_depth_n11(q, deep11, variant):
    c, ckpts, final, (m_ref, p_ref), post = deep11
    mode, kernel, k = VARIANTS[variant]
    d = q.Density(c.n)
    if mode == "fused":
        d.set_mode(q.QCW_MODE_FUSED, k)
        d.set_fused_kernel(kernel)
    got_ck = _bench_like(q, d, c)
    for (tr, pu, pr), (gtr, gpu, gpr) in zip(ckpts, got_ck):
        assert abs(gtr - tr.real) <= TRACE_TOL
        assert abs(gpu - pu) <= DEEP_PURITY_TOL
        assert np.abs(gpr - pr).max() <= READ_TOL
    np.testing.assert_allclose(d.probabilities(), oracle.probabilities(final), atol=READ_TOL, rtol=0)
    got = d.get_state()
    err = np.abs(got - final).max()
    tr_err = abs(d.trace() - 1)
    print(f"{variant}: max|d rho| {err:.3e}, |tr - 1| {tr_err:.3e}, "
          f"max |d purity| {max(abs(g[1] - w[1]) for g, w in zip(got_ck, ckpts)):.3e}")
    assert err <= ATOL, err
    assert tr_err <= TRACE_TOL
    # the draw is far enough from p_0 that FP32 drift cannot flip the outcome
    p0 = oracle.probabilities(final)
    assert abs(U_MEASURE - (1 - p0[0])) > 1e-4
    m, p = d.measure(0, -1, U_MEASURE)
    assert m == m_ref and abs(p - p_ref) <= READ_TOL
    np.testing.assert_allclose(d.partial_trace([0, 1]), oracle.partial_trace(post, [0, 1]), atol=READ_TOL, rtol=0)
    assert np.abs(d.get_state() - post).max() <= ATOL
    d.close()


def _golden(name):
    rows = read_golden(name)
    g = {"elem": [], "ptrace": {}}
    for key, vals in rows:
        if key == "elem":
            g["elem"].append(vals)
        elif key == "ptrace":
            z = np.array(vals[2:], dtype=np.float64)
            g["ptrace"][(int(vals[0]), int(vals[1]))] = (z[0::2] + 1j * z[1::2]).reshape(4, 4)
        else:
            g[key] = vals
    return g


def _check_golden_readouts(d, g, n):
    tr_re, tr_im, pur = g["final"][0], g["final"][1], g["final"][2]
    p1 = np.array(g["final"][3:])
    tr = d.trace()
    assert abs(tr.real - tr_re) <= TRACE_TOL and abs(tr.imag - tr_im) <= TRACE_TOL
    assert abs(d.purity() - pur) <= DEEP_PURITY_TOL
    assert np.abs(d.probabilities() - p1).max() <= READ_TOL
    for keep, want in g["ptrace"].items():
        assert np.abs(d.partial_trace(list(keep)) - want).max() <= READ_TOL, keep


def _device_view(d):
    """The context's rho as a (2^n, 2 * 2^n) float32 torch view of its device buffer (Re and Im
    interleaved), completed and ordered on the context's stream.  Valid while the context lives."""
    import torch

    ptr, sp = d.device_state()
    torch.cuda.ExternalStream(sp).synchronize()
    dim = 1 << d.n

    class _Buf:
        pass

    buf = _Buf()
    buf.__cuda_array_interface__ = {"shape": (dim, 2 * dim), "typestr": "<f4", "data": (ptr, False),
                                    "version": 2}
    return torch.as_tensor(buf, device="cuda")


def _golden_element_error(d, g):
    """max |delta rho| over the golden file's sampled elements (row, column, Re, Im)."""
    import torch

    e = np.array(g["elem"], dtype=np.float64)
    view = _device_view(d)
    r = torch.as_tensor(e[:, 0].astype(np.int64), device="cuda")
    c2 = torch.as_tensor(2 * e[:, 1].astype(np.int64), device="cuda")
    re = view[r, c2].double().cpu().numpy()
    im = view[r, c2 + 1].double().cpu().numpy()
    return np.abs((re + 1j * im) - (e[:, 2] + 1j * e[:, 3])).max()


@pytest.mark.parametrize("mode", ["plain", "fused"])
def test_config2_full_depth_n12_against_stored_oracle(q, mode):
    c = wl.config2_circuit()
    g = _golden("config2_n12.txt")
    assert g["n"] == [c.n] and g["gates"] == [c.n_gates] and g["channels"] == [c.n_channels]
    d = q.Density(c.n)
    if mode == "fused":
        d.set_mode(q.QCW_MODE_FUSED, 0)
    d.set_state(c.rho0)
    for part in _chunks(c):
        d.apply_packed(q.PackedOps(part))
    _check_golden_readouts(d, g, c.n)
    err = _golden_element_error(d, g)
    print(f"config2 {mode}: max|d rho| over {len(g['elem'])} sampled elements {err:.3e}, "
          f"|tr - 1| {abs(d.trace() - 1):.3e}")
    assert err <= ATOL
    assert abs(d.trace() - 1) <= TRACE_TOL
    d.close()


@pytest.mark.parametrize("mode,kernel,k", [("plain", 0, 0), ("fused", 3, 5), ("fused", 4, 4)])
def test_torch_owned_memory_and_stream(q, mode, kernel, k):
    """rho lives in a torch tensor and the work runs on a torch stream (qcw_create_from_ptr via
    Density.from_tensor).  The evolved state is in the tensor, ordered on that stream, and the
    context never frees the tensor's memory."""
    import torch

    n = 11
    c = wl.random_circuit(n, 40, 5150 + k, "mixed", "adpd")
    want = oracle.run_circuit(c)
    # the borrowed rho is the head of a 1 GiB torch allocation, so that a wrongful cudaFree
    # of it would show as a gigabyte of newly free device memory
    backing = torch.zeros(1 << 27, dtype=torch.complex64, device="cuda")
    t = backing[: 4 ** n]
    t[0] = 1.0
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    d = q.Density.from_tensor(t, s)
    ptr, sp = d.device_state()
    assert ptr == t.data_ptr() == backing.data_ptr()
    assert sp == s.cuda_stream
    if mode == "fused":
        d.set_mode(q.QCW_MODE_FUSED, k)
        d.set_fused_kernel(kernel)
    for op in c.ops:
        d.apply_op(op)
    d.device_state()  # flush and complete the matrix on the stream, without waiting
    with torch.cuda.stream(s):
        snap = t.clone()  # ordered after the library's work by the stream alone
    s.synchronize()
    got = snap.view(1 << n, 1 << n).cpu().numpy().astype(np.complex128)
    assert np.abs(got - want).max() <= ATOL
    assert abs(d.trace() - 1) <= TRACE_TOL
    torch.cuda.synchronize()
    free_before, _ = torch.cuda.mem_get_info()
    d.close()
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after - free_before < (256 << 20)  # the library released only its own scratch
    # the tensor and the stream remain the caller's and stay usable
    with torch.cuda.stream(s):
        t.mul_(2.0)
    s.synchronize()
    back = t.view(1 << n, 1 << n).cpu().numpy().astype(np.complex128)
    assert np.abs(back - 2 * want).max() <= 2 * ATOL
    del t, backing, snap


@pytest.mark.parametrize("mode,kernel,k", [("fused", 0, 0), ("fused", 4, 5), ("plain", 0, 0)])
def test_benchmark_circuit_full_depth_n14_against_stored_oracle(q, mode, kernel, k):
    """The 14-qubit benchmark circuit itself, all 1000 gates, in the benchmark's launch
    configuration (the default kernel at the autotuned width), on the tensor-core variant and on
    the plain path (one launch per gate and per channel, 3296 launches), against the complex128
    oracle's readouts stored by tests/golden/make_deep_goldens.py: every
    100-gate checkpoint (trace, purity, probabilities), 1024 sampled elements of the final state,
    two partial traces, the u-driven measurement of qubit 0 and the post-measurement state."""
    import os

    from tests._helpers import GOLDEN

    if not os.path.exists(os.path.join(GOLDEN, "config3_n14.txt")):
        pytest.skip("stored oracle readouts of the 14-qubit circuit not generated yet")
    c = wl.config3_circuit()
    g = _golden("config3_n14.txt")
    assert g["n"] == [c.n] and g["gates"] == [c.n_gates] and g["channels"] == [c.n_channels]
    ck_want = [row for key, row in read_golden("config3_n14.txt") if key == "ckpt"]
    d = q.Density(c.n)
    if mode == "fused":
        d.set_mode(q.QCW_MODE_FUSED, k)
        d.set_fused_kernel(kernel)
    ck = _bench_like(q, d, c)
    assert len(ck) == len(ck_want) == 10
    for (gtr, gpu, gpr), w in zip(ck, ck_want):
        assert abs(gtr.real - w[1]) <= TRACE_TOL and abs(gtr - 1) <= TRACE_TOL
        assert abs(gpu - w[3]) <= DEEP_PURITY_TOL
        assert np.abs(gpr - np.asarray(w[4:])).max() <= READ_TOL
    err = _golden_element_error(d, g)
    assert err <= ATOL
    for keep, want in g["ptrace"].items():
        assert np.abs(d.partial_trace(list(keep)) - want).max() <= READ_TOL, keep
    qubit, u, m_ref, p_ref = g["measure"]
    m, p = d.measure(int(qubit), -1, u)
    assert m == int(m_ref) and abs(p - p_ref) <= READ_TOL
    post = [vals for key, vals in read_golden("config3_n14.txt") if key == "post_ptrace"][0]
    z = np.array(post[2:], dtype=np.float64)
    assert np.abs(d.partial_trace([0, 1]) - (z[0::2] + 1j * z[1::2]).reshape(4, 4)).max() <= READ_TOL
    assert abs(d.purity() - g["post_purity"][0]) <= DEEP_PURITY_TOL
    print(f"n14 kernel {kernel}: max|d rho| over {len(g['elem'])} sampled elements {err:.3e}")
    d.close()
