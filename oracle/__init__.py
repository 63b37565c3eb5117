"""CPU oracle for the QCWAVE density-matrix path: TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference
legs may import this package.  The product library never loads it and shares no code
with it.  The arithmetic lives in ``qcw_oracle.c`` (plain complex128 loops following the
paper's pair / quartet sweeps, Sec. 3, and its Kraus form, Eq. rhoE2); this module marshals
numpy arrays into that library and replays circuits op by op.  The spectral observables
(entropy, fidelity) take numpy's Hermitian eigensolver as a library step on the C partial
trace.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qcw_oracle.c")
_HDR = os.path.join(_HERE, "qcw_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_EZEROPROB = 0, -1, -2, -3


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with code {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp) into oracle/_build/liborc.so."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            lib.orc_apply_unitary.argtypes = [P, I, P, P, I, P, I]
            lib.orc_apply_kraus.argtypes = [P, I, P, I, P, I]
            lib.orc_apply_vec.argtypes = [P, I, P, P, I, P, I]
            lib.orc_trace.argtypes = [P, I, P, P]
            lib.orc_trace.restype = None
            lib.orc_purity.argtypes = [P, I]
            lib.orc_purity.restype = D
            lib.orc_probabilities.argtypes = [P, I, P]
            lib.orc_probabilities.restype = None
            lib.orc_measure.argtypes = [P, I, I, I, D, P, P]
            lib.orc_partial_trace.argtypes = [P, I, P, I, P]
            lib.orc_pauli_expectation.argtypes = [P, I, P, P, I, P]
            lib.orc_set_threads.argtypes = [I]
            for f in ("orc_apply_unitary", "orc_apply_kraus", "orc_apply_vec", "orc_measure",
                      "orc_partial_trace", "orc_pauli_expectation", "orc_set_threads"):
                getattr(lib, f).restype = I
            _lib = lib
    return _lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ints(xs) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(list(xs), dtype=np.int32))


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None and a.size else None


def _check(code: int, what: str):
    if code != ORC_OK:
        raise OracleError(code, what)


def set_threads(n: int = 0) -> int:
    """Set the OpenMP thread count (0 = leave as is); returns the count in use."""
    return int(_load().orc_set_threads(int(n)))


def nqubits_of(rho: np.ndarray) -> int:
    d = rho.shape[0]
    n = d.bit_length() - 1
    assert rho.shape == (d, d) and (1 << n) == d
    return n


def apply_unitary(rho: np.ndarray, u: np.ndarray, qubits, controls=()) -> np.ndarray:
    """rho <- U rho U^dagger in place (U acts on ``qubits`` in paper order; controls all 1)."""
    n = nqubits_of(rho)
    u = _c128(u)
    q, c = _ints(qubits), _ints(controls)
    _check(_load().orc_apply_unitary(_ptr(rho), n, _ptr(u), _ptr(q), len(q), _ptr(c), len(c)),
           "apply_unitary")
    return rho


def apply_kraus(rho: np.ndarray, kraus: np.ndarray, qubits) -> np.ndarray:
    """rho <- sum_k K_k rho K_k^dagger in place (Eq. rhoE2)."""
    n = nqubits_of(rho)
    ks = _c128(kraus)
    q = _ints(qubits)
    _check(_load().orc_apply_kraus(_ptr(rho), n, _ptr(ks), ks.shape[0], _ptr(q), len(q)),
           "apply_kraus")
    return rho


def apply_vec(psi: np.ndarray, u: np.ndarray, qubits, controls=()) -> np.ndarray:
    """Op1 / Op2 / Op3 on a state vector in place (Sec. 3)."""
    n = psi.shape[0].bit_length() - 1
    u = _c128(u)
    q, c = _ints(qubits), _ints(controls)
    _check(_load().orc_apply_vec(_ptr(psi), n, _ptr(u), _ptr(q), len(q), _ptr(c), len(c)),
           "apply_vec")
    return psi


def trace(rho: np.ndarray) -> complex:
    re, im = ctypes.c_double(), ctypes.c_double()
    _load().orc_trace(_ptr(rho), nqubits_of(rho), ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def purity(rho: np.ndarray) -> float:
    return float(_load().orc_purity(_ptr(rho), nqubits_of(rho)))


def probabilities(rho: np.ndarray) -> np.ndarray:
    n = nqubits_of(rho)
    out = np.zeros(n, dtype=np.float64)
    _load().orc_probabilities(_ptr(rho), n, _ptr(out))
    return out


def measure(rho: np.ndarray, qubit: int, forced: int = -1, u: float = 0.0):
    """Projective measurement in place; returns (outcome, p_outcome)."""
    oc, pr = ctypes.c_int(), ctypes.c_double()
    _check(_load().orc_measure(_ptr(rho), nqubits_of(rho), int(qubit), int(forced), float(u),
                               ctypes.byref(oc), ctypes.byref(pr)), "measure")
    return int(oc.value), float(pr.value)


def partial_trace(rho: np.ndarray, keep) -> np.ndarray:
    keep = _ints(sorted(keep))
    out = np.zeros((1 << len(keep), 1 << len(keep)), dtype=np.complex128)
    _check(_load().orc_partial_trace(_ptr(rho), nqubits_of(rho), _ptr(keep), len(keep), _ptr(out)),
           "partial_trace")
    return out


def pauli_expectation(rho: np.ndarray, qubits, paulis) -> complex:
    """Tr[P rho], P the Pauli string sigma_{paulis[j]} on qubits[j] (1 = X, 2 = Y, 3 = Z)."""
    q, p = _ints(qubits), _ints(paulis)
    out = np.zeros(2, dtype=np.float64)
    _check(_load().orc_pauli_expectation(_ptr(rho), nqubits_of(rho), _ptr(q), _ptr(p), len(q), _ptr(out)),
           "pauli_expectation")
    return complex(out[0], out[1])


def polarization(rho: np.ndarray) -> np.ndarray:
    """Polarisation vectors P_q = Tr[sigma^(q) rho] (Sec. 5.2), shape (n, 3)."""
    n = nqubits_of(rho)
    return np.array([[pauli_expectation(rho, [q], [i]).real for i in (1, 2, 3)] for q in range(n)])


def correlation(rho: np.ndarray, q1: int, q2: int) -> np.ndarray:
    """Spin correlation tensor C_ij = Tr[sigma_i^(q1) sigma_j^(q2) rho] (Sec. 5.2), shape (3, 3)."""
    return np.array([[pauli_expectation(rho, [q1, q2], [i, j]).real for j in (1, 2, 3)] for i in (1, 2, 3)])


def entropy(rho: np.ndarray, keep) -> float:
    """von Neumann entropy S = -Tr[rho_A log2 rho_A] of the reduced state of `keep`, in bits
    (Sec. 5.2: S tends to n_q in the classical limit, hence base 2)."""
    w = np.linalg.eigvalsh(partial_trace(rho, keep))
    w = w[w > 1e-15]
    return float(-(w * np.log2(w)).sum())


def fidelity(rho: np.ndarray, keep, sigma: np.ndarray) -> float:
    """F = Tr sqrt(sqrt(sigma) rho_A sqrt(sigma)) (Sec. 5.2) of the reduced state of `keep`
    against the caller's sigma."""
    ra = partial_trace(rho, keep)
    mu, v = np.linalg.eigh(np.asarray(sigma, dtype=np.complex128))
    s = v @ np.diag(np.sqrt(np.clip(mu, 0, None))) @ v.conj().T
    return float(np.sqrt(np.clip(np.linalg.eigvalsh(s @ ra @ s), 0, None)).sum())


def initial_state(circuit) -> np.ndarray:
    if circuit.init == "matrix":
        return _c128(circuit.rho0).copy()
    rho = np.zeros((1 << circuit.n, 1 << circuit.n), dtype=np.complex128)
    rho[0, 0] = 1.0
    return rho


def apply_op(rho: np.ndarray, op) -> np.ndarray:
    if op.kind == "gate":
        return apply_unitary(rho, op.mats[0], op.qubits)
    return apply_kraus(rho, op.mats, op.qubits)


def run_circuit(circuit, rho: np.ndarray | None = None, ops=None) -> np.ndarray:
    """Replay ``circuit`` (or the given op list) on a fresh or supplied state."""
    rho = initial_state(circuit) if rho is None else rho
    for op in (circuit.ops if ops is None else ops):
        apply_op(rho, op)
    return rho
