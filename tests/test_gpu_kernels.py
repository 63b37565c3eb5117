"""GPU parity of every kernel against the CPU oracle, through the C ABI.

Tolerance: max |delta rho| <= 1e-5 elementwise and |tr rho - 1| <= 1e-6 (FP32 complex
state, FP64 oracle); measurement outcomes must be identical.
"""

import numpy as np
import pytest

import oracle
import workloads as wl
from tests._helpers import haar_unitary, random_rho

pytestmark = pytest.mark.gpu

ATOL = 1e-5
TRACE_TOL = 1e-6


@pytest.fixture(scope="module")
def q():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1101_1785_gb300 as q

    return q


def _dens(q, rho, mode=None, k=0):
    d = q.Density((rho.shape[0]).bit_length() - 1)
    d.set_state(rho)
    if mode is not None:
        d.set_mode(mode, k)
    return d


def _close(got, want, atol=ATOL):
    err = np.abs(got - want).max()
    assert err <= atol, err
    return err


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7])
def test_gate1_every_target(q, n):
    rng = np.random.default_rng(100 + n)
    for t in range(n):
        u = haar_unitary(rng, 2)
        rho = random_rho(rng, n)
        d = _dens(q, rho)
        d.apply_gate1(u, t)
        _close(d.get_state(), oracle.apply_unitary(rho.copy(), u, [t]))
        d.close()


@pytest.mark.parametrize("n", [3, 6])
def test_gate1_controls(q, n):
    rng = np.random.default_rng(7)
    cases = [(0, [n - 1]), (n - 1, [0]), (1, [0, 2])] if n > 3 else [(0, [2]), (2, [0, 1]), (1, [2])]
    for t, ctrl in cases:
        u = haar_unitary(rng, 2)
        rho = random_rho(rng, n)
        d = _dens(q, rho)
        d.apply_gate1(u, t, ctrl)
        _close(d.get_state(), oracle.apply_unitary(rho.copy(), u, [t], ctrl))
        d.close()


@pytest.mark.parametrize("n", [2, 3, 5])
def test_gate2_every_ordered_pair(q, n):
    rng = np.random.default_rng(200 + n)
    for a in range(n):
        for b in range(n):
            if a == b:
                continue
            v = haar_unitary(rng, 4)
            rho = random_rho(rng, n)
            d = _dens(q, rho)
            d.apply_gate2(v, a, b)
            _close(d.get_state(), oracle.apply_unitary(rho.copy(), v, [a, b]))
            d.close()


def test_gate2_controls(q):
    rng = np.random.default_rng(9)
    n = 5
    for (a, b), ctrl in (((0, 4), [2]), ((3, 1), [4, 0]), ((4, 2), [0])):
        v = haar_unitary(rng, 4)
        rho = random_rho(rng, n)
        d = _dens(q, rho)
        d.apply_gate2(v, a, b, ctrl)
        _close(d.get_state(), oracle.apply_unitary(rho.copy(), v, [a, b], ctrl))
        d.close()


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_gate_k_dense(q, k):
    rng = np.random.default_rng(300 + k)
    n = 6
    for _ in range(2):
        qs = [int(x) for x in rng.permutation(n)[:k]]
        u = haar_unitary(rng, 1 << k)
        rho = random_rho(rng, n)
        d = _dens(q, rho)
        d.apply_gate(u, qs)
        _close(d.get_state(), oracle.apply_unitary(rho.copy(), u, qs))
        d.close()


@pytest.mark.parametrize("n", [1, 2, 4, 6])
def test_kraus_one_qubit(q, n):
    rng = np.random.default_rng(400 + n)
    sets = [wl.kraus_ad(0.13), wl.kraus_pd(0.2), wl.kraus_depolarising(0.1),
            np.stack([np.sqrt(0.3) * haar_unitary(rng, 2), np.sqrt(0.7) * haar_unitary(rng, 2)])]
    for t in range(n):
        ks = sets[t % len(sets)]
        rho = random_rho(rng, n)
        d = _dens(q, rho)
        d.apply_kraus(ks, [t])
        _close(d.get_state(), oracle.apply_kraus(rho.copy(), ks, [t]))
        d.close()


@pytest.mark.parametrize("n", [2, 3, 5])
def test_kraus_two_qubit(q, n):
    rng = np.random.default_rng(500 + n)
    for a, b in [(0, n - 1), (n - 1, 0)] + ([(1, 2)] if n > 2 else []):
        ks = np.stack([np.sqrt(w) * haar_unitary(rng, 4) for w in (0.5, 0.3, 0.2)])
        rho = random_rho(rng, n)
        d = _dens(q, rho)
        d.apply_kraus(ks, [a, b])
        _close(d.get_state(), oracle.apply_kraus(rho.copy(), ks, [a, b]))
        d.close()


@pytest.mark.parametrize("n", [1, 3, 6, 9])
def test_readouts(q, n):
    rng = np.random.default_rng(600 + n)
    rho = random_rho(rng, n)
    d = _dens(q, rho)
    tr = d.trace()
    assert abs(tr - oracle.trace(rho)) <= TRACE_TOL
    assert abs(d.purity() - oracle.purity(rho)) <= 1e-6
    np.testing.assert_allclose(d.probabilities(), oracle.probabilities(rho), atol=1e-6)
    keeps = [[0], [n - 1], list(range(n))] + ([[0, n - 1], [1, n - 2]] if n >= 4 else [])
    for keep in keeps:
        _close(d.partial_trace(keep), oracle.partial_trace(rho, keep), atol=1e-6)
    d.close()


@pytest.mark.parametrize("n", [1, 4, 7])
def test_measure(q, n):
    rng = np.random.default_rng(700 + n)
    rho = random_rho(rng, n)
    for qb in sorted({0, n // 2, n - 1}):
        for forced in (0, 1):
            d = _dens(q, rho)
            ref = rho.copy()
            m_ref, p_ref = oracle.measure(ref, qb, forced)
            m, p = d.measure(qb, forced)
            assert m == m_ref and abs(p - p_ref) <= 1e-6
            _close(d.get_state(), ref)
            assert abs(d.trace() - 1) <= TRACE_TOL
            d.close()
        # u-driven outcome, u kept 1e-4 away from p0
        p0 = 1 - oracle.probabilities(rho)[qb]
        for u in (max(p0 - 0.05, 0.0), min(p0 + 0.05, 0.9999)):
            if abs(u - p0) < 1e-4:
                continue
            d = _dens(q, rho)
            ref = rho.copy()
            m_ref, _ = oracle.measure(ref, qb, -1, u)
            m, _ = d.measure(qb, -1, u)
            assert m == m_ref
            _close(d.get_state(), ref)
            d.close()


def test_measure_zero_probability(q):
    d = q.Density(3)
    before = d.get_state()
    with pytest.raises(q.QcwError) as e:
        d.measure(1, 1)
    assert e.value.status == q.QCW_EZEROPROB
    np.testing.assert_array_equal(d.get_state(), before)
    d.close()


def test_invalid_arguments_leave_state(q):
    rng = np.random.default_rng(1)
    rho = random_rho(rng, 3)
    d = _dens(q, rho)
    before = d.get_state()
    for call in (lambda: d.apply_gate1(np.eye(2), 3),
                 lambda: d.apply_gate1(np.eye(2), 0, [0]),
                 lambda: d.apply_gate2(np.eye(4), 1, 1),
                 lambda: d.apply_gate1(np.array([[np.nan, 0], [0, 1]]), 0),
                 lambda: d.apply_kraus(np.zeros((0, 2, 2)), [0]),
                 lambda: d.partial_trace([2, 2])):
        with pytest.raises((q.QcwError, ValueError)):
            call()
    np.testing.assert_array_equal(d.get_state(), before)
    d.close()


def test_config1_plain(q):
    c = wl.config1_circuit()
    want = oracle.run_circuit(c)
    d = q.run_circuit(c)
    err = _close(d.get_state(), want)
    assert abs(d.trace() - 1) <= TRACE_TOL
    for forced in (0, 1):
        ref = want.copy()
        m_ref, p_ref = oracle.measure(ref, c.measure_qubit, forced)
        dd = q.run_circuit(c)
        m, p = dd.measure(c.measure_qubit, forced)
        assert (m, round(p, 5)) == (m_ref, round(p_ref, 5)) or abs(p - p_ref) <= 1e-6
        _close(dd.get_state(), ref)
        dd.close()
    print(f"config1 plain: max|drho| = {err:.2e}")
    d.close()


def test_determinism(q):
    c = wl.random_circuit(8, 60, 5, "mixed", "adpd")
    a = q.run_circuit(c).get_state()
    b = q.run_circuit(c).get_state()
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("mode,kernel,n", [("plain", 0, 5), ("fused", 2, 7), ("fused", 3, 9), ("fused", 4, 10)])
def test_polarization_and_correlation_match_oracle(q, mode, kernel, n):
    """Polarisation vectors and spin correlation tensors (Sec. 5.2) of a noisy circuit's state,
    on full storage (plain path, per-tile Hermitian kernel) and on the lower triangle left by
    the warp-specialised kernels, against the oracle's traces Tr[P rho]."""
    c = wl.random_circuit(n, 60, 5200 + n, "mixed", "adpd")
    rho = oracle.run_circuit(c)
    d = q.Density(n)
    if mode == "fused":
        d.set_mode(q.QCW_MODE_FUSED, 5)
        d.set_fused_kernel(kernel)
    for op in c.ops:
        d.apply_op(op)
    np.testing.assert_allclose(d.polarization(), oracle.polarization(rho), atol=1e-5, rtol=0)
    for q1, q2 in ((0, n - 1), (n - 1, 1), (2, 3)):
        np.testing.assert_allclose(d.correlation(q1, q2), oracle.correlation(rho, q1, q2), atol=1e-5, rtol=0)
    with pytest.raises(q.QcwError) as e:
        d.correlation(1, 1)
    assert e.value.status == q.QCW_EINVAL
    d.close()


def test_bell_state_polarization_and_correlation(q):
    """(|00> + |11>)/sqrt 2 on qubits 1 and 3 of four: the pair has no polarisation, the
    spectators in |0> point along +z; correlation tensor diag(1, -1, 1) between the pair, zero
    between the pair and a spectator (the product P_0 (x) P_3 = 0)."""
    d = q.Density(4)
    d.apply_gate1(wl.gate_matrix("H"), 1)
    d.apply_gate2(wl.gate_matrix("CNOT"), 1, 3)
    want = np.zeros((4, 3))
    want[0, 2] = want[2, 2] = 1.0
    np.testing.assert_allclose(d.polarization(), want, atol=1e-7, rtol=0)
    np.testing.assert_allclose(d.correlation(1, 3), np.diag([1.0, -1.0, 1.0]), atol=1e-6)
    np.testing.assert_allclose(d.correlation(0, 3), np.zeros((3, 3)), atol=1e-7)
    d.close()


@pytest.mark.parametrize("mode,kernel,n", [("plain", 0, 6), ("fused", 3, 9), ("fused", 4, 8)])
def test_entropy_and_fidelity_match_oracle(q, mode, kernel, n):
    """Subsystem entropy and fidelity (Sec. 5.2) of a noisy circuit's state: GPU partial trace,
    host eigensolver, against the oracle's reduced states and numpy's eigensolver."""
    c = wl.random_circuit(n, 60, 5300 + n, "mixed", "adpd")
    rho = oracle.run_circuit(c)
    rng = np.random.default_rng(n)
    d = q.Density(n)
    if mode == "fused":
        d.set_mode(q.QCW_MODE_FUSED, 5)
        d.set_fused_kernel(kernel)
    for op in c.ops:
        d.apply_op(op)
    for keep in ([0], [1, n - 1], [0, 2, 3]):
        assert abs(d.entropy(keep) - oracle.entropy(rho, keep)) <= 1e-5
        sigma = random_rho(rng, len(keep))
        assert abs(d.fidelity(keep, sigma) - oracle.fidelity(rho, keep, sigma)) <= 1e-5
    for bad in ([], list(range(7)), [2, 1]):
        with pytest.raises(q.QcwError) as e:
            d.entropy(bad)
        assert e.value.status == q.QCW_EINVAL
    d.close()


def test_entropy_of_a_bell_pair(q):
    """(|00> + |11>)/sqrt 2 on qubits 0 and 2 of three: each qubit of the pair 1 bit, the pair
    and the spectator 0 bits, fidelity of qubit 0 with |0><0| 1/sqrt 2."""
    d = q.Density(3)
    d.apply_gate1(wl.gate_matrix("H"), 0)
    d.apply_gate2(wl.gate_matrix("CNOT"), 0, 2)
    assert abs(d.entropy([0]) - 1) < 1e-6 and abs(d.entropy([2]) - 1) < 1e-6
    assert abs(d.entropy([0, 2])) < 1e-6 and abs(d.entropy([1])) < 1e-6
    assert abs(d.fidelity([0], np.diag([1.0, 0.0])) - 2 ** -0.5) < 1e-6
    d.close()


@pytest.mark.parametrize("mode,k", [("plain", 3), ("fused", 3), ("plain", 4)])
def test_kraus_channels_on_three_and_four_qubits(q, mode, k):
    """A random trace-preserving channel on k = 3, 4 qubits (three Kraus operators cut from a
    Haar isometry, Eq. rhoE2) between two noisy circuit halves, against the oracle; in fused
    mode the wide channel splits the queue and runs on the plain path."""
    n = 6
    rng = np.random.default_rng(40 + k)
    d_k = 1 << k
    iso = haar_unitary(rng, 3 * d_k)[:, :d_k]
    ks = np.stack([iso[d_k * j:d_k * (j + 1)] for j in range(3)])
    qubits = [int(x) for x in rng.permutation(n)[:k]]
    c = wl.random_circuit(n, 20, 4400 + k, "mixed", "adpd")
    rho0 = random_rho(rng, n)
    want = rho0.copy()
    d = q.Density(n)
    if mode == "fused":
        d.set_mode(q.QCW_MODE_FUSED, 4)
    d.set_state(rho0)
    for op in c.ops:
        d.apply_op(op)
        oracle.apply_op(want, op)
    d.apply_kraus(ks, qubits)
    oracle.apply_kraus(want, ks, qubits)
    for op in c.ops:
        d.apply_op(op)
        oracle.apply_op(want, op)
    got = d.get_state()
    assert np.abs(got - want).max() <= 1e-5
    assert abs(d.trace() - oracle.trace(want)) <= 1e-6
    d.close()


def test_validation_mode(q):
    """Off by default (a non-unitary matrix is applied as given); on, non-unitary gates, Kraus
    sets that increase the trace and states that are not Hermitian with unit trace are rejected
    with QCW_EINVAL and the state is unchanged; unitary gates, trace-preserving and trace-decreasing
    Kraus sets and proper states pass, in plain and fused mode and through qcw_apply_ops."""
    n = 3
    rng = np.random.default_rng(91)
    d = q.Density(n)
    d.apply_gate1(2.0 * np.eye(2), 0)  # not validated: accepted
    d.reset()
    for mode in (q.QCW_MODE_PLAIN, q.QCW_MODE_FUSED):
        d.set_mode(mode, 0)
        d.set_validation(True)
        rho = random_rho(rng, n)
        d.set_state(rho)
        bad = [lambda: d.apply_gate1(2.0 * np.eye(2), 0),
               lambda: d.apply_gate2(1.1 * np.eye(4), 0, 1),
               lambda: d.apply_gate(1.01 * np.eye(8), [0, 1, 2]),
               lambda: d.apply_kraus(np.stack([np.eye(2), 0.1 * np.eye(2)]), [1]),
               lambda: d.apply_op(wl.Op("gate", (2,), np.array([[[1.0, 0.0], [0.5, 1.0]]]))),
               lambda: d.set_state(rho + 1e-3 * np.triu(np.ones((8, 8)), 1)),
               lambda: d.set_state(1.01 * rho)]
        for f in bad:
            with pytest.raises(q.QcwError) as e:
                f()
            assert e.value.status == q.QCW_EINVAL
        assert np.abs(d.get_state() - rho).max() <= 1e-6
        u = haar_unitary(rng, 2)
        d.apply_gate1(u, 1)
        d.apply_kraus(wl.kraus_ad(0.1), [2])
        d.apply_kraus(np.stack([np.sqrt(0.5) * np.eye(2)]), [0])  # trace-decreasing: allowed
        want = rho.copy()
        oracle.apply_unitary(want, u, [1])
        oracle.apply_kraus(want, wl.kraus_ad(0.1), [2])
        oracle.apply_kraus(want, np.stack([np.sqrt(0.5) * np.eye(2)]), [0])
        assert np.abs(d.get_state() - want).max() <= 1e-5
        d.set_validation(False)
        d.reset()
    d.close()


def test_monomial_two_qubit_gates_are_exact_permutations(q):
    """CNOT (both orders), CZ, SWAP, iSWAP and Pauli products on the plain path move the members
    of each 16-element group with factors 1, -1, i, -i only: the result equals the oracle and
    every element is a signed / rotated copy of an input element, so the trace (a permutation of
    the diagonal) is unchanged to the last bit; a gate that is not of that form (a Haar unitary)
    and a controlled monomial take the general kernels and still match the oracle."""
    n = 5
    rng = np.random.default_rng(92)
    rho = random_rho(rng, n)
    d = q.Density(n)
    d.set_state(rho)
    want = rho.copy()
    iswap = np.array([[1, 0, 0, 0], [0, 0, 1j, 0], [0, 1j, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)
    xz = np.kron(wl.gate_matrix("X"), wl.gate_matrix("Z"))
    yy = np.kron(wl.gate_matrix("Y"), wl.gate_matrix("Y"))
    gates = [(wl.gate_matrix("CNOT"), (0, 4)), (wl.gate_matrix("CNOT"), (4, 0)), (wl.gate_matrix("CZ"), (1, 3)),
             (wl.gate_matrix("SWAP"), (2, 4)), (iswap, (3, 0)), (xz, (1, 2)), (yy, (4, 3))]
    tr0 = d.trace()
    for u, (a, b) in gates:
        d.apply_gate2(u, a, b)
        oracle.apply_unitary(want, u, [a, b])
        assert d.trace() == tr0
    got = d.get_state()
    assert np.abs(got - want).max() <= 1e-6
    vals = np.sort(np.abs(np.concatenate([got.real.ravel(), got.imag.ravel()])))
    src = np.sort(np.abs(np.concatenate([d_ for d_ in (rho.astype(np.complex64).real.ravel(),
                                                          rho.astype(np.complex64).imag.ravel())])))
    np.testing.assert_array_equal(vals.astype(np.float32), src.astype(np.float32))
    u = haar_unitary(rng, 4)
    d.apply_gate2(u, 0, 2)
    oracle.apply_unitary(want, u, [0, 2])
    d.apply_gate2(wl.gate_matrix("CNOT"), 1, 3, [4])
    oracle.apply_unitary(want, wl.gate_matrix("CNOT"), [1, 3], [4])
    assert np.abs(d.get_state() - want).max() <= 1e-5
    d.close()
