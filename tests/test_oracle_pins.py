"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test ties one oracle function to something other than itself: a worked example of
the paper (tests/golden/*), a brute-force full-space operator built entry by entry, a
library routine (numpy kron / einsum / eigvalsh), a closed form, or an invariant.
"""

import numpy as np
import pytest

import oracle
import workloads as wl
from tests._helpers import (bloch, embed, haar_unitary, kron_single, numpy_partial_trace,
                            random_rho, read_golden)

RNG = np.random.default_rng(1234)


def _zero(n):
    r = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    r[0, 0] = 1
    return r


# ---------------------------------------------------------------- index convention
def test_h_on_qubit1_of_000_golden():
    """Sec. 4.1 worked example: Op1[H,1,|000>] -> C_0 = C_4 = 1/sqrt(2) (stride 4)."""
    rows = read_golden("h_qubit1_000.txt")
    n = dict((k, v) for k, v in rows if k == "n")["n"][0]
    _, (name, q) = next(r for r in rows if r[0] == "gate")
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1
    oracle.apply_vec(psi, wl.gate_matrix(name), [q])
    want = np.zeros(1 << n, dtype=np.complex128)
    for k, v in rows:
        if k == "amp":
            want[v[0]] = v[1] + 1j * v[2]
    np.testing.assert_allclose(psi, want, atol=1e-15)
    # same example on the density matrix: rho = |psi><psi|
    rho = _zero(n)
    oracle.apply_unitary(rho, wl.gate_matrix(name), [q])
    np.testing.assert_allclose(rho, np.outer(want, want.conj()), atol=1e-15)


# ---------------------------------------------------------------- brute force sweeps
@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_single_qubit_sweep_matches_kron(n):
    """Eq. resmat1 on rows and conj on columns == dense (I (x) U (x) I) rho (...)^dagger."""
    for q in range(n):
        u = wl.haar_su2(RNG) if q % 2 else haar_unitary(RNG, 2)
        rho = random_rho(RNG, n)
        full = kron_single(u, q, n)
        want = full @ rho @ full.conj().T
        got = oracle.apply_unitary(rho.copy(), u, [q])
        np.testing.assert_allclose(got, want, atol=1e-14)
        # the entry-by-entry embedding agrees with the kron construction
        np.testing.assert_allclose(embed(u, [q], n), full, atol=0)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_two_qubit_sweep_matches_embedding(n):
    """Eq. resmat2 with index 2*q(is1) + q(is2), every ordered pair incl. reversed ones."""
    for a in range(n):
        for b in range(n):
            if a == b:
                continue
            v = haar_unitary(RNG, 4)
            rho = random_rho(RNG, n)
            full = embed(v, [a, b], n)
            want = full @ rho @ full.conj().T
            got = oracle.apply_unitary(rho.copy(), v, [a, b])
            np.testing.assert_allclose(got, want, atol=1e-14)


def test_cnot_order_convention():
    """CNOT with (is1, is2) = (control, target): |10> -> |11>, |01> -> |01>."""
    cn = wl.gate_matrix("CNOT")
    for ctrl, tgt in ((0, 1), (1, 0)):
        psi = np.zeros(4, dtype=np.complex128)
        psi[2 if ctrl == 0 else 1] = 1  # control qubit set to 1
        oracle.apply_vec(psi, cn, [ctrl, tgt])
        assert abs(psi[3]) == 1.0


@pytest.mark.parametrize("k", [3, 4])
def test_k_qubit_sweep_matches_embedding(k):
    """Octets (Sec. 3.3) and their k = 4 analogue against the entry-by-entry operator."""
    n = 5
    qs = [int(x) for x in RNG.permutation(n)[:k]]
    u = haar_unitary(RNG, 1 << k)
    rho = random_rho(RNG, n)
    full = embed(u, qs, n)
    got = oracle.apply_unitary(rho.copy(), u, qs)
    np.testing.assert_allclose(got, full @ rho @ full.conj().T, atol=1e-13)


def test_controlled_gates_match_embedding():
    n = 4
    for tgt, ctrls in ((3, [0]), (0, [2, 3]), (1, [3]), (2, [0, 1, 3])):
        u = haar_unitary(RNG, 2)
        rho = random_rho(RNG, n)
        full = embed(u, [tgt], n, ctrls)
        got = oracle.apply_unitary(rho.copy(), u, [tgt], ctrls)
        np.testing.assert_allclose(got, full @ rho @ full.conj().T, atol=1e-14)
    v = haar_unitary(RNG, 4)
    rho = random_rho(RNG, n)
    full = embed(v, [3, 1], n, [0])
    got = oracle.apply_unitary(rho.copy(), v, [3, 1], [0])
    np.testing.assert_allclose(got, full @ rho @ full.conj().T, atol=1e-14)


def test_kraus_matches_dense_sum():
    """Eq. rhoE2 against sum_k K_full rho K_full^dagger (dense), 1- and 2-qubit sets."""
    n = 3
    for qs, ks in (([1], wl.kraus_ad(0.3)), ([2], wl.kraus_depolarising(0.2)),
                   ([2, 0], np.stack([np.sqrt(0.5) * haar_unitary(RNG, 4) for _ in range(2)]))):
        rho = random_rho(RNG, n)
        want = sum(embed(k, qs, n) @ rho @ embed(k, qs, n).conj().T for k in ks)
        got = oracle.apply_kraus(rho.copy(), ks, qs)
        np.testing.assert_allclose(got, want, atol=1e-14)


def test_planted_mistakes_are_caught():
    """A transposed or unconjugated operand fails the brute-force pin (pin sensitivity)."""
    n = 3
    u = haar_unitary(RNG, 4)
    rho = random_rho(RNG, n)
    full = embed(u, [0, 2], n)
    want = full @ rho @ full.conj().T
    for bad in (u.T, u.conj(), u.conj().T):
        got = oracle.apply_unitary(rho.copy(), bad, [0, 2])
        assert np.abs(got - want).max() > 1e-3
    got = oracle.apply_unitary(rho.copy(), u, [2, 0])  # swapped qubit order
    assert np.abs(got - want).max() > 1e-3


# ---------------------------------------------------------------- worked circuits
def test_bell_and_inverse_golden():
    rows = read_golden("bell.txt")
    rho = _zero(2)
    oracle.apply_unitary(rho, wl.gate_matrix("H"), [0])
    oracle.apply_unitary(rho, wl.gate_matrix("CNOT"), [0, 1])
    want = np.zeros((4, 4), dtype=np.complex128)
    for k, v in rows:
        if k == "rho":
            want[v[0], v[1]] = v[2] + 1j * v[3]
    np.testing.assert_allclose(rho, want, atol=1e-15)
    oracle.apply_unitary(rho, wl.gate_matrix("CNOT"), [0, 1])
    oracle.apply_unitary(rho, wl.gate_matrix("H"), [0])
    np.testing.assert_allclose(rho, _zero(2), atol=1e-15)


def test_ghz5_golden():
    rows = read_golden("ghz5.txt")
    rho = _zero(5)
    oracle.apply_unitary(rho, wl.gate_matrix("H"), [0])
    for t in (1, 2, 3, 4):
        oracle.apply_unitary(rho, wl.gate_matrix("CNOT"), [0, t])
    want = np.zeros((32, 32), dtype=np.complex128)
    for k, v in rows:
        if k == "rho":
            want[v[0], v[1]] = v[2] + 1j * v[3]
    np.testing.assert_allclose(rho, want, atol=1e-15)


def test_mv1_noiseless_fidelity_golden():
    """F(rho, |0><0|) = sqrt(<0|rho|0>) for pure rho_0: 1 -> 1/sqrt(2) -> 1."""
    steps = [v[1] for k, v in read_golden("mv1_fidelity.txt") if k == "step"]
    rho = _zero(1)
    got = [np.sqrt(rho[0, 0].real)]
    for _ in range(2):
        oracle.apply_unitary(rho, wl.gate_matrix("H"), [0])
        got.append(np.sqrt(rho[0, 0].real))
    np.testing.assert_allclose(got, steps, atol=1e-15)


# ---------------------------------------------------------------- channels: closed forms
@pytest.mark.parametrize("m", [1, 5, 17])
def test_amplitude_damping_closed_form(m):
    g = 0.07
    n, q = 3, 1
    rho = _zero(n)
    oracle.apply_unitary(rho, wl.gate_matrix("H"), [q])  # |0+0>
    for _ in range(m):
        oracle.apply_kraus(rho, wl.kraus_ad(g), [q])
    r1 = oracle.partial_trace(rho, [q])
    np.testing.assert_allclose(r1[0, 1], 0.5 * (1 - g) ** (m / 2), atol=1e-15)
    np.testing.assert_allclose(r1[1, 1], 0.5 * (1 - g) ** m, atol=1e-15)
    np.testing.assert_allclose(rho[0b010, 0b000], 0.5 * (1 - g) ** (m / 2), atol=1e-15)


@pytest.mark.parametrize("m", [1, 4, 11])
def test_phase_damping_closed_form(m):
    lam = 0.13
    rho = _zero(2)
    oracle.apply_unitary(rho, wl.gate_matrix("H"), [1])
    for _ in range(m):
        oracle.apply_kraus(rho, wl.kraus_pd(lam), [1])
    np.testing.assert_allclose(rho[0, 1], 0.5 * (1 - lam) ** (m / 2), atol=1e-15)
    np.testing.assert_allclose(rho[1, 1], 0.5, atol=1e-15)


@pytest.mark.parametrize("m", [1, 3, 9])
def test_depolarising_bloch_shrink(m):
    p = 0.05
    rng = np.random.default_rng(m)
    rho = random_rho(rng, 1, rank=1)
    b0 = bloch(rho)
    for _ in range(m):
        oracle.apply_kraus(rho, wl.kraus_depolarising(p), [0])
    np.testing.assert_allclose(bloch(rho), b0 * (1 - 4 * p / 3) ** m, atol=1e-14)


def test_multiverse_ensemble_equals_kraus():
    """Eq. rhoE1 == Eq. rhoE2: explicit statevector ensemble vs the Kraus sum."""
    n, p, eps = 3, 0.8, 0.2
    rng = np.random.default_rng(7)
    psi = wl.haar_state(rng, n)
    qs = [2, 0]
    omegas = [haar_unitary(rng, 4) for _ in range(4)]
    # ensemble: path 0 untouched (weight p), path j hit by Omega_j (weight eps / n_p)
    ens = p * np.outer(psi, psi.conj())
    for om in omegas:
        phi = psi.copy()
        oracle.apply_vec(phi, om, qs)
        ens += eps / len(omegas) * np.outer(phi, phi.conj())
    rho = np.outer(psi, psi.conj())
    oracle.apply_kraus(rho, wl.kraus_pauli_multiverse(p, eps, omegas), qs)
    np.testing.assert_allclose(rho, ens, atol=1e-15)
    assert abs(oracle.trace(rho) - 1) < 1e-14  # trace preserved (Sec. 5.2.1)


def test_classical_limit_golden():
    """Repeated XYZ multiverse noise (p = .8, eps = .2) -> I/2^n (Eq. rhoE3)."""
    g = dict(read_golden("classical_limit.txt"))
    n = g["n"][0]
    rng = np.random.default_rng(3)
    rho = random_rho(rng, n, rank=1)
    xyz = [wl.gate_matrix(s) for s in ("X", "Y", "Z")]
    ks = wl.kraus_pauli_multiverse(0.8, 0.2, xyz)
    for _ in range(400):
        for q in range(n):
            oracle.apply_kraus(rho, ks, [q])
    ev = np.linalg.eigvalsh(rho)
    np.testing.assert_allclose(ev, g["eigenvalue"][0], atol=1e-9)
    np.testing.assert_allclose(oracle.purity(rho), g["purity"][0], atol=1e-9)
    ent = -sum(x * np.log2(x) for x in ev)
    np.testing.assert_allclose(ent, g["entropy_bits"][0], atol=1e-8)
    np.testing.assert_allclose(oracle.entropy(rho, list(range(n))), g["entropy_bits"][0], atol=1e-8)
    assert np.abs(rho - np.diag(np.diag(rho))).max() < 1e-9


# ---------------------------------------------------------------- invariants on circuits
def test_noisy_circuit_invariants():
    c = wl.config1_circuit()
    rho = oracle.initial_state(c)
    for op in c.ops:
        oracle.apply_op(rho, op)
        assert abs(oracle.trace(rho) - 1) < 1e-13
    np.testing.assert_allclose(rho, rho.conj().T, atol=1e-15)
    assert np.linalg.eigvalsh(rho).min() > -1e-12
    assert oracle.purity(rho) < 1.0


def test_noiseless_circuit_stays_pure():
    c = wl.random_circuit(5, 60, 99, "mixed", "none")
    rho = oracle.run_circuit(c)
    assert abs(oracle.purity(rho) - 1) < 1e-12
    assert abs(oracle.trace(rho) - 1) < 1e-13
    # equals the state-vector run of the same gates (Op1/Op2 on psi)
    psi = np.zeros(32, dtype=np.complex128)
    psi[0] = 1
    for op in c.ops:
        oracle.apply_vec(psi, op.mats[0], op.qubits)
    np.testing.assert_allclose(rho, np.outer(psi, psi.conj()), atol=1e-13)


# ---------------------------------------------------------------- readouts
def test_purity_trace_probabilities_against_numpy():
    rng = np.random.default_rng(11)
    n = 4
    rho = random_rho(rng, n)
    assert abs(oracle.purity(rho) - np.trace(rho @ rho).real) < 1e-14
    assert abs(oracle.purity(rho) - (np.linalg.eigvalsh(rho) ** 2).sum()) < 1e-14
    assert abs(oracle.trace(rho) - np.trace(rho)) < 1e-14
    diag = np.diag(rho).real.reshape([2] * n)
    for q in range(n):
        want = np.take(diag, 1, axis=q).sum()
        assert abs(oracle.probabilities(rho)[q] - want) < 1e-14


def test_measure_bell_and_support():
    rho = _zero(2)
    oracle.apply_unitary(rho, wl.gate_matrix("H"), [0])
    oracle.apply_unitary(rho, wl.gate_matrix("CNOT"), [0, 1])
    for forced, corner in ((0, 0), (1, 3)):
        r = rho.copy()
        m, p = oracle.measure(r, 0, forced)
        assert m == forced and abs(p - 0.5) < 1e-15
        want = np.zeros((4, 4))
        want[corner, corner] = 1
        np.testing.assert_allclose(r, want, atol=1e-15)
    r = rho.copy()
    assert oracle.measure(r, 1, -1, 0.4999)[0] == 0
    r = rho.copy()
    assert oracle.measure(r, 1, -1, 0.5001)[0] == 1
    # random state: p0 + p1 = tr, post-state has unit trace and lives on bit q = m
    rng = np.random.default_rng(5)
    n = 4
    rho = random_rho(rng, n)
    for q in range(n):
        for forced in (0, 1):
            r = rho.copy()
            m, p = oracle.measure(r, q, forced)
            m2, p2 = oracle.measure(rho.copy(), q, 1 - forced)
            assert abs(p + p2 - 1) < 1e-14
            assert abs(oracle.trace(r) - 1) < 1e-14
            w = 1 << (n - 1 - q)
            bad = [i for i in range(1 << n) if bool(i & w) != bool(m)]
            assert np.abs(r[bad, :]).max() == 0 and np.abs(r[:, bad]).max() == 0
            good = [i for i in range(1 << n) if bool(i & w) == bool(m)]
            np.testing.assert_allclose(r[np.ix_(good, good)], rho[np.ix_(good, good)] / p, atol=1e-15)


def test_measure_zero_probability_leaves_state():
    rho = _zero(3)
    before = rho.copy()
    with pytest.raises(oracle.OracleError) as e:
        oracle.measure(rho, 1, 1)
    assert e.value.code == oracle.ORC_EZEROPROB
    np.testing.assert_array_equal(rho, before)


def test_partial_trace_pins():
    rng = np.random.default_rng(21)
    # product state: rho_A (x) rho_B with A = qubits {0, 2}, B = {1}
    ra, rb = random_rho(rng, 2), random_rho(rng, 1)
    full = np.kron(ra, rb)  # order (a0, a1, b) -> qubits 0,1 from A, 2 from B
    np.testing.assert_allclose(oracle.partial_trace(full, [0, 1]), ra, atol=1e-15)
    np.testing.assert_allclose(oracle.partial_trace(full, [2]), rb, atol=1e-15)
    # Bell pair -> I/2 on either qubit
    rho = _zero(2)
    oracle.apply_unitary(rho, wl.gate_matrix("H"), [0])
    oracle.apply_unitary(rho, wl.gate_matrix("CNOT"), [0, 1])
    for q in (0, 1):
        np.testing.assert_allclose(oracle.partial_trace(rho, [q]), np.eye(2) / 2, atol=1e-15)
    # random state, non-contiguous kept sets, against numpy.einsum
    n = 5
    rho = random_rho(rng, n)
    for keep in ([0], [4], [1, 3], [0, 2, 4], [0, 1, 2, 3, 4], []):
        got = oracle.partial_trace(rho, keep)
        np.testing.assert_allclose(got, numpy_partial_trace(rho, keep, n), atol=1e-14)
        assert abs(np.trace(got) - np.trace(rho)) < 1e-14


def test_invalid_inputs():
    rho = _zero(2)
    with pytest.raises(oracle.OracleError):
        oracle.apply_unitary(rho, np.eye(2), [2])
    with pytest.raises(oracle.OracleError):
        oracle.apply_unitary(rho, np.eye(4), [1, 1])
    with pytest.raises(oracle.OracleError):
        oracle.apply_kraus(rho, np.zeros((0, 2, 2)), [0])


def _sigma(i):
    return [np.eye(2), np.array([[0, 1], [1, 0]]), np.array([[0, -1j], [1j, 0]]),
            np.array([[1, 0], [0, -1]])][i]


def test_polarization_of_the_axis_states():
    """|0>, |1>, |+> = H|0> and |+i> = S H|0> point along +z, -z, +x and +y (Sec. 5.2's
    one-qubit form rho = (1 + P . sigma) / 2); the Y sign is fixed by |+i>."""
    cases = [((), (0, 0, 1)), (("X",), (0, 0, -1)), (("H",), (1, 0, 0)), (("H", "S"), (0, 1, 0))]
    for gates, want in cases:
        rho = _zero(1)
        for g in gates:
            oracle.apply_unitary(rho, wl.gate_matrix(g), [0])
        np.testing.assert_allclose(oracle.polarization(rho)[0], want, atol=1e-15)


def test_polarization_and_correlation_recover_the_pauli_form():
    """rho = (1 + P1 . sigma x 1 + P2 . 1 x sigma + sum_ij C_ij sigma_i x sigma_j) / 4 with
    random real coefficients: the traces return P1, P2 and C (the two-qubit form of Sec. 5.2);
    a one-qubit rho = (1 + P . sigma) / 2 returns P."""
    rng = np.random.default_rng(31)
    p = rng.uniform(-0.5, 0.5, 3)
    rho1 = (np.eye(2) + sum(p[i] * _sigma(i + 1) for i in range(3))) / 2
    np.testing.assert_allclose(oracle.polarization(rho1.astype(np.complex128))[0], p, atol=1e-15)
    p1, p2 = rng.uniform(-0.3, 0.3, 3), rng.uniform(-0.3, 0.3, 3)
    c = rng.uniform(-0.3, 0.3, (3, 3))
    rho = np.eye(4, dtype=np.complex128)
    for i in range(3):
        rho += p1[i] * np.kron(_sigma(i + 1), np.eye(2)) + p2[i] * np.kron(np.eye(2), _sigma(i + 1))
        for j in range(3):
            rho += c[i, j] * np.kron(_sigma(i + 1), _sigma(j + 1))
    rho /= 4
    pol = oracle.polarization(rho)
    np.testing.assert_allclose(pol[0], p1, atol=1e-15)
    np.testing.assert_allclose(pol[1], p2, atol=1e-15)
    np.testing.assert_allclose(oracle.correlation(rho, 0, 1), c, atol=1e-15)
    np.testing.assert_allclose(oracle.correlation(rho, 1, 0), c.T, atol=1e-15)


def test_bell_state_correlations():
    """(|00> + |11>)/sqrt 2: no polarisation, correlation tensor diag(1, -1, 1)."""
    rho = _zero(2)
    oracle.apply_unitary(rho, wl.gate_matrix("H"), [0])
    oracle.apply_unitary(rho, wl.gate_matrix("CNOT"), [0, 1])
    np.testing.assert_allclose(oracle.polarization(rho), np.zeros((2, 3)), atol=1e-15)
    np.testing.assert_allclose(oracle.correlation(rho, 0, 1), np.diag([1.0, -1.0, 1.0]), atol=1e-15)


def test_polarization_of_a_product_state():
    """rho_a (x) rho_b (x) rho_c: each qubit's vector is its factor's (numpy Bloch vector), and
    the correlation of qubits 0 and 2 is the outer product of theirs."""
    rng = np.random.default_rng(32)
    f = [random_rho(rng, 1) for _ in range(3)]
    rho = np.kron(np.kron(f[0], f[1]), f[2]).astype(np.complex128)
    pol = oracle.polarization(rho)
    for q in range(3):
        np.testing.assert_allclose(pol[q], bloch(f[q]), atol=1e-14)
    np.testing.assert_allclose(oracle.correlation(rho, 0, 2), np.outer(bloch(f[0]), bloch(f[2])), atol=1e-14)


def test_entropy_and_fidelity_of_entangled_states():
    """Bell pair: the whole state is pure (0 bits), each qubit maximally mixed (1 bit), whose
    fidelity with |0><0| is 1/sqrt 2 and with I/2 is 1; GHZ on five qubits: any two qubits
    carry 1 bit; a product of pure states has 0 bits everywhere."""
    rho = _zero(2)
    oracle.apply_unitary(rho, wl.gate_matrix("H"), [0])
    oracle.apply_unitary(rho, wl.gate_matrix("CNOT"), [0, 1])
    assert abs(oracle.entropy(rho, [0, 1])) < 1e-12
    assert abs(oracle.entropy(rho, [0]) - 1) < 1e-12 and abs(oracle.entropy(rho, [1]) - 1) < 1e-12
    assert abs(oracle.fidelity(rho, [1], np.diag([1.0, 0.0])) - 2 ** -0.5) < 1e-12
    assert abs(oracle.fidelity(rho, [0], np.eye(2) / 2) - 1) < 1e-12
    ghz = _zero(5)
    oracle.apply_unitary(ghz, wl.gate_matrix("H"), [0])
    for q in range(1, 5):
        oracle.apply_unitary(ghz, wl.gate_matrix("CNOT"), [0, q])
    assert abs(oracle.entropy(ghz, [1, 3]) - 1) < 1e-12
    prod = _zero(3)
    oracle.apply_unitary(prod, wl.gate_matrix("H"), [1])
    for keep in ([0], [1], [0, 2], [0, 1, 2]):
        assert abs(oracle.entropy(prod, keep)) < 1e-12


def test_fidelity_of_a_state_with_itself_and_commuting_states():
    """F(rho_A, rho_A) = 1 for a mixed reduced state; diagonal (commuting) states give
    sum_i sqrt(p_i q_i)."""
    rng = np.random.default_rng(33)
    rho = random_rho(rng, 4)
    ra = oracle.partial_trace(rho, [1, 3])
    assert abs(oracle.fidelity(rho, [1, 3], ra) - 1) < 1e-10
    p, q = rng.dirichlet(np.ones(4)), rng.dirichlet(np.ones(4))
    d = np.diag(p).astype(np.complex128)
    assert abs(oracle.fidelity(d, [0, 1], np.diag(q)) - np.sum(np.sqrt(p * q))) < 1e-12


# ----------------------------------------------------------------------------- noise experiments
def _oracle_mv(exp):
    """The oracle replaying one of the paper's noise experiments (Sec. 5.3-5.4): per step the
    Kraus form of Eq. rhoE4's average on the whole register, then the step's algorithm gates."""
    rho = exp.rho0()
    allq = list(range(exp.n))
    states = [rho.copy()]
    prev = oracle.set_threads(0)
    oracle.set_threads(1)  # a few-qubit state: one thread
    try:
        for s in range(1, exp.nsteps + 1):
            oracle.apply_kraus(rho, exp.kraus(s), allq)
            for u, qs in exp.gates(s):
                oracle.apply_unitary(rho, u, qs)
            states.append(rho.copy())
    finally:
        oracle.set_threads(prev)
    return states


def test_mv1_noiseless_fidelity_path():
    """MV1 without noise (caption of the MV1 figure): the fidelity with |0> is 1, drops to 1/sqrt 2
    after the Hadamard of step 1, stays there, and returns to 1 after the Hadamard of step 3; the
    state stays pure."""
    exp = wl.mv_experiment("MV1", "none", nsteps=6)
    states = _oracle_mv(exp)
    f = [oracle.fidelity(r, [0], exp.rho0()) for r in states]
    np.testing.assert_allclose(f, [1, 2 ** -0.5, 2 ** -0.5, 1, 1, 1, 1], atol=1e-12)
    assert all(abs(oracle.purity(r) - 1) < 1e-12 for r in states)


def test_mv2_noiseless_bell_and_return():
    """MV2 without noise (Sec. 5.3): after CNOT_12 H_1 the state is the Bell state, corners 1/2
    (golden bell.txt gives the same); the fidelity with |00> is 1/sqrt 2 from step 1 to 3 and
    1 again after the inverse Bell operator of steps 3-4."""
    exp = wl.mv_experiment("MV2", "none", nsteps=6)
    states = _oracle_mv(exp)
    bell = states[2]
    for r, c in ((0, 0), (0, 3), (3, 0), (3, 3)):
        assert abs(bell[r, c] - 0.5) < 1e-12
    assert abs(np.abs(bell).sum() - 2.0) < 1e-12
    f = [oracle.fidelity(r, [0, 1], exp.rho0()) for r in states]
    np.testing.assert_allclose(f, [1, 2 ** -0.5, 2 ** -0.5, 2 ** -0.5, 1, 1, 1], atol=1e-12)


def test_mvn_noiseless_ghz_corners():
    """MVn without noise (Sec. 5.4): after H_1 and CNOT_12 .. CNOT_15 the five qubits are in the GHZ
    state: the four corners of rho are 1/2 and everything else 0."""
    exp = wl.mv_experiment("MVn", "none", nsteps=6)
    rho = _oracle_mv(exp)[5]
    want = np.zeros((32, 32))
    for r, c in ((0, 0), (0, 31), (31, 0), (31, 31)):
        want[r, c] = 0.5
    np.testing.assert_allclose(rho, want, atol=1e-12)


def test_mv2_long_noise_classical_limit():
    """Sec. 5.2.3: continued noise drives rho to the classical form, all eigenvalues 1/2^n_q
    (1/4 for MV2), entropy n_q bits, purity 1/4."""
    exp = wl.mv_experiment("MV2", "xyz", nsteps=300)
    rho = _oracle_mv(exp)[-1]
    w = np.linalg.eigvalsh(rho)
    np.testing.assert_allclose(w, 0.25, atol=1e-4)
    assert abs(oracle.entropy(rho, [0, 1]) - 2) < 1e-4
    assert abs(oracle.purity(rho) - 0.25) < 1e-4


@pytest.mark.parametrize("name", ["MV1", "MV2", "MVn"])
def test_mv_noise_step_is_the_pauli_average(name):
    """One noise step of Eq. rhoE4 on a random state, by the oracle's Kraus sum, against the
    definition: p rho + sum over the noise paths of (eps p_s / n_p) P rho P, each P a Pauli
    string written out by Kronecker products (numpy), with Z-only noise leaving the diagonal as
    it was (Z strings commute with the computational-basis projectors)."""
    rng = np.random.default_rng(55)
    for noise in ("xyz", "yz", "z"):
        exp = wl.mv_experiment(name, noise, nsteps=3)
        rho = random_rho(rng, exp.n)
        got = oracle.apply_kraus(rho.copy(), exp.kraus(2), list(range(exp.n)))
        want = np.zeros_like(rho)
        for w, hits in exp.noise_terms(2):
            P = np.ones((1, 1))
            for q in range(exp.n):
                a = dict(hits).get(q, 0)
                P = np.kron(P, (np.eye(2), wl.gate_matrix("X"), wl.gate_matrix("Y"), wl.gate_matrix("Z"))[a])
            want += w * P @ rho @ P.conj().T
        np.testing.assert_allclose(got, want, atol=1e-14)
        if noise == "z":
            np.testing.assert_allclose(np.diag(got), np.diag(rho), atol=1e-15)
