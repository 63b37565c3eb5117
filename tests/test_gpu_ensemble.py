"""GPU parity of the multiverse ensemble (Sec. 5.2.1, Eq. rhoE1) against the oracle: the
ensemble's state vectors follow the oracle's Op1 / Op2 sweeps, and an ensemble that enumerates
every branch of its noise steps reproduces the Kraus-sum evolution of the density matrix
(Eq. rhoE2)."""

import itertools

import numpy as np
import pytest

import oracle
import workloads as wl
from tests._helpers import haar_unitary

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1101_1785_gb300 as q

    return q


def _random_vectors(rng, nvec, n):
    psi = rng.normal(size=(nvec, 1 << n)) + 1j * rng.normal(size=(nvec, 1 << n))
    return psi / np.linalg.norm(psi, axis=1, keepdims=True)


def test_ensemble_gates_match_oracle_statevectors(q):
    n, nvec = 5, 7
    rng = np.random.default_rng(61)
    psi = _random_vectors(rng, nvec, n)
    e = q.Ensemble(n, nvec)
    e.set(psi)
    want = psi.copy()
    for step in range(30):
        if step % 3 == 2:
            a, b = [int(x) for x in rng.permutation(n)[:2]]
            u = haar_unitary(rng, 4)
            e.apply_gate2(u, a, b)
            for v in range(nvec):
                oracle.apply_vec(want[v], u, [a, b])
        else:
            t = int(rng.integers(n))
            u = haar_unitary(rng, 2)
            e.apply_gate1(u, t)
            for v in range(nvec):
                oracle.apply_vec(want[v], u, [t])
    assert np.abs(e.get() - want).max() <= 1e-5
    e.close()


def test_enumerated_multiverse_equals_kraus_sum(q):
    """Two noise steps of Eq. rhoE1's form (Omega = sqrt(p) I, sqrt((1 - p)/3) X, Y, Z) between
    gates: 16 universes, one per branch pair, weight 1 each (the sqrt(p_k) sit in the
    operators).  Their density matrix equals the oracle's Kraus evolution, and so do its trace,
    purity and polarisation readouts."""
    n, p = 3, 0.9
    rng = np.random.default_rng(62)
    xyz = [wl.gate_matrix(s) for s in ("X", "Y", "Z")]
    omegas = np.stack([np.sqrt(p) * np.eye(2)] + [np.sqrt((1 - p) / 3) * m for m in xyz])
    gates = [("u1", haar_unitary(rng, 2), (0,)), ("noise", None, (1,)), ("u2", wl.gate_matrix("CNOT"), (0, 1)),
             ("u1", haar_unitary(rng, 2), (2,)), ("noise", None, (0,)), ("u2", haar_unitary(rng, 4), (2, 1))]
    psi0 = _random_vectors(rng, 1, n)[0]
    branches = list(itertools.product(range(4), repeat=2))
    e = q.Ensemble(n, len(branches))
    e.set(np.tile(psi0, (len(branches), 1)))
    rho = np.outer(psi0, psi0.conj())
    step = 0
    for kind, u, qs in gates:
        if kind == "u1":
            e.apply_gate1(u, qs[0])
            oracle.apply_unitary(rho, u, list(qs))
        elif kind == "u2":
            e.apply_gate2(u, qs[0], qs[1])
            oracle.apply_unitary(rho, u, list(qs))
        else:
            e.apply_noise1(omegas, qs[0], [b[step] for b in branches])
            oracle.apply_kraus(rho, omegas, list(qs))
            step += 1
    d = q.Density(n)
    e.density(np.ones(len(branches)), d)
    assert np.abs(d.get_state() - rho).max() <= 1e-5
    assert abs(d.trace() - oracle.trace(rho)) <= 1e-6
    assert abs(d.purity() - oracle.purity(rho)) <= 1e-5
    np.testing.assert_allclose(d.polarization(), oracle.polarization(rho), atol=1e-5, rtol=0)
    d.close()
    e.close()


def test_density_weights_and_validation(q):
    """One-hot weights give |psi_v><psi_v|; a noise choice out of range and a qubit-count
    mismatch are rejected."""
    n, nvec = 4, 3
    rng = np.random.default_rng(63)
    psi = _random_vectors(rng, nvec, n)
    e = q.Ensemble(n, nvec)
    e.set(psi)
    d = q.Density(n)
    e.density([0.0, 1.0, 0.0], d)
    assert np.abs(d.get_state() - np.outer(psi[1], psi[1].conj())).max() <= 1e-6
    with pytest.raises(q.QcwError) as err:
        e.apply_noise1(np.stack([np.eye(2)]), 0, [0, 1, 0])
    assert err.value.status == q.QCW_EINVAL
    d3 = q.Density(3)
    with pytest.raises(q.QcwError) as err:
        e.density(np.ones(nvec), d3)
    assert err.value.status == q.QCW_EINVAL
    d.close()
    d3.close()
    e.close()


@pytest.mark.parametrize("n,nvec", [(5, 9), (6, 16), (7, 64), (8, 37), (9, 3), (10, 130), (11, 64)])
def test_density_of_host_vectors_against_the_definition(q, n, nvec):
    """rho = sum_v w_v |psi_v><psi_v| (Eq. rhoE1's ensemble average) of vectors and weights drawn
    on the host, against the definition in numpy: below 64 amplitudes one thread per element, at 64
    and 128 the tiled FP32 kernel, from 256 on the tensor-core kernel (3xTF32) for the tiles below
    the 128 x 128 diagonal blocks and their mirrors, the FP32 kernel for the diagonal blocks
    (partial last rounds of four vectors for nvec = 37, 3 and 130)."""
    rng = np.random.default_rng(64 + n)
    psi = _random_vectors(rng, nvec, n)
    w = rng.uniform(0.1, 1.0, nvec)
    w /= w.sum()
    want = np.einsum("v,vr,vc->rc", w, psi, psi.conj())
    e = q.Ensemble(n, nvec)
    e.set(psi)
    d = q.Density(n)
    e.density(w, d)
    got = d.get_state()
    assert np.abs(got - want).max() <= 1e-6
    assert np.abs(got - got.conj().T).max() <= 1e-7
    assert abs(d.trace() - 1) <= 1e-6
    d.close()
    e.close()


def test_density_at_the_largest_register(q):
    """17 qubits (rho = 2^34 complex64 = 128 GiB, element offsets beyond 32 bits): rho = sum_v w_v
    |psi_v><psi_v| of 16 vectors drawn on the host, at seeded elements on, below and above the
    diagonal, against the definition (within 1e-5 of the largest element; the amplitudes are FP32
    on the device), Hermitian at the mirrored positions, trace 1."""
    import torch

    from paper_1101_1785_gb300._binding import QCW_MAX_QUBITS
    from tests._helpers import gather_elements

    n, nvec = QCW_MAX_QUBITS, 16
    free, _ = torch.cuda.mem_get_info()
    if free < (8 << (2 * n)) + (16 << 30):
        pytest.skip(f"needs {(8 << (2 * n)) >> 30} GiB of free device memory and some headroom")
    rng = np.random.default_rng(1717)
    psi = _random_vectors(rng, nvec, n)
    w = rng.uniform(0.1, 1.0, nvec)
    w /= w.sum()
    e = q.Ensemble(n, nvec)
    e.set(psi)
    d = q.Density(n)
    e.density(w, d)
    dim = 1 << n
    diag = rng.integers(0, dim, 512)
    rows = np.concatenate([diag, rng.integers(0, dim, 4096)])
    cols = np.concatenate([diag, rng.integers(0, dim, 4096)])
    want = np.einsum("v,vi,vi->i", w, psi[:, rows], psi[:, cols].conj())
    got = gather_elements(d, rows, cols)
    assert np.abs(got - want).max() <= 1e-5 * np.abs(want).max()
    # off the 64 x 64 diagonal tiles each mirror is written as the exact conjugate; inside them
    # (the sampled diagonal) both triangles are computed, equal to rounding
    assert np.abs(gather_elements(d, cols, rows) - got.conj()).max() <= 1e-5 * np.abs(want).max()
    assert abs(d.trace() - 1) <= 1e-6
    d.close()
    e.close()
