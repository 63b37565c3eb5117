"""CPU tests of the library's host spectral functions (eigenvalues of Hermitian matrices, von
Neumann entropy, fidelity), which turn the GPU's reduced density matrices into the entropy and
fidelity observables of Sec. 5.2.  Compiled from the library source with a test shim; checked
against numpy's eigensolver and closed forms."""

import ctypes
import os
import subprocess

import numpy as np
import pytest

from tests._helpers import haar_unitary, random_rho

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1101_1785_gb300", "csrc")
SHIM = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cpp", "hermitian_shim.cpp")


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("herm") / "libherm_shim.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", CSRC, "-o", out, SHIM,
                           os.path.join(CSRC, "hermitian.cpp")])
    L = ctypes.CDLL(out)
    L.shim_entropy_bits.restype = ctypes.c_double
    L.shim_fidelity.restype = ctypes.c_double
    return L


P = ctypes.c_void_p


def _p(a):
    return a.ctypes.data_as(P)


def _eig(lib, a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    n = a.shape[0]
    w = np.zeros(n)
    v = np.zeros((n, n), dtype=np.complex128)
    lib.shim_herm_eig(_p(a), n, _p(w), _p(v))
    return w, v


def _random_hermitian(rng, n):
    x = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    return (x + x.conj().T) / 2


@pytest.mark.parametrize("n", [1, 2, 3, 8, 17, 64])
def test_eigen_decomposition_matches_numpy(lib, n):
    rng = np.random.default_rng(n)
    a = _random_hermitian(rng, n)
    w, v = _eig(lib, a)
    np.testing.assert_allclose(w, np.linalg.eigvalsh(a), atol=1e-12 * np.linalg.norm(a))
    np.testing.assert_allclose(v.conj().T @ v, np.eye(n), atol=1e-12)
    np.testing.assert_allclose(v @ np.diag(w) @ v.conj().T, a, atol=1e-12 * np.linalg.norm(a))


def test_degenerate_and_diagonal_spectra(lib):
    """Repeated eigenvalues (a unitary conjugate of diag(1, 1, 1, 2)) and an already diagonal
    matrix (no rotation needed)."""
    rng = np.random.default_rng(5)
    u = haar_unitary(rng, 4)
    w, _ = _eig(lib, u @ np.diag([1.0, 1.0, 1.0, 2.0]) @ u.conj().T)
    np.testing.assert_allclose(w, [1, 1, 1, 2], atol=1e-13)
    w, v = _eig(lib, np.diag([3.0, -1.0, 2.0]))
    np.testing.assert_allclose(w, [-1, 2, 3], atol=0)
    np.testing.assert_allclose(np.abs(v), np.eye(3)[:, [1, 2, 0]], atol=0)


def test_entropy(lib):
    """Pure state 0 bits, maximally mixed k qubits k bits, a random state's spectrum
    -sum w log2 w."""
    for k in (1, 2, 3):
        w = np.full(1 << k, 1.0 / (1 << k))
        assert abs(lib.shim_entropy_bits(_p(w), len(w)) - k) < 1e-14
    w = np.array([0.0, 0.0, 1.0, -1e-17])
    assert lib.shim_entropy_bits(_p(w), 4) == 0.0
    rng = np.random.default_rng(7)
    rho = random_rho(rng, 3)
    w, _ = _eig(lib, rho)
    ev = np.linalg.eigvalsh(rho)
    assert abs(lib.shim_entropy_bits(_p(w), 8) + sum(x * np.log2(x) for x in ev if x > 1e-15)) < 1e-12


def _fid(lib, rho, sigma):
    rho = np.ascontiguousarray(rho, dtype=np.complex128)
    sigma = np.ascontiguousarray(sigma, dtype=np.complex128)
    return lib.shim_fidelity(_p(rho), _p(sigma), rho.shape[0])


def test_fidelity_closed_forms(lib):
    """F(rho, rho) = 1; commuting states sum_i sqrt(p_i q_i); pure states |<psi|phi>|;
    orthogonal pure states 0; symmetric in its arguments."""
    rng = np.random.default_rng(8)
    rho = random_rho(rng, 3)
    assert abs(_fid(lib, rho, rho) - 1) < 1e-12
    p, q = rng.dirichlet(np.ones(8)), rng.dirichlet(np.ones(8))
    assert abs(_fid(lib, np.diag(p), np.diag(q)) - np.sum(np.sqrt(p * q))) < 1e-13
    psi, phi = haar_unitary(rng, 8)[:, 0], haar_unitary(rng, 8)[:, 0]
    assert abs(_fid(lib, np.outer(psi, psi.conj()), np.outer(phi, phi.conj())) - abs(np.vdot(psi, phi))) < 1e-7
    e0, e1 = np.eye(4)[0], np.eye(4)[1]
    assert abs(_fid(lib, np.outer(e0, e0), np.outer(e1, e1))) < 1e-15
    sigma = random_rho(rng, 3)
    assert abs(_fid(lib, rho, sigma) - _fid(lib, sigma, rho)) < 1e-10


def test_fidelity_matches_the_matrix_square_root_definition(lib):
    """Tr sqrt(sqrt(sigma) rho sqrt(sigma)) with numpy's eigh for the square roots."""
    rng = np.random.default_rng(9)
    for n in (1, 2, 4):
        rho, sigma = random_rho(rng, n), random_rho(rng, n)
        mu, v = np.linalg.eigh(sigma)
        s = v @ np.diag(np.sqrt(np.clip(mu, 0, None))) @ v.conj().T
        want = np.sum(np.sqrt(np.clip(np.linalg.eigvalsh(s @ rho @ s), 0, None)))
        assert abs(_fid(lib, rho, sigma) - want) < 1e-10
