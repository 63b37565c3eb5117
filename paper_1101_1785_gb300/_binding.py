"""ctypes binding of libqcw.so: argument marshalling only.

Every function of include/qcw.h is reachable under its C name through ``lib()``; the
``Density`` class wraps one context and converts numpy arrays to the pointers and sizes
the C ABI expects.  No computation happens here: each call goes to the CUDA library, and
loading fails loudly when the library has not been built.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqcw.so")

QCW_OK, QCW_EINVAL, QCW_ENOMEM, QCW_ECUDA, QCW_EZEROPROB, QCW_ETIMEOUT, QCW_ENOTSUP = range(7)
QCW_MODE_PLAIN, QCW_MODE_FUSED = 0, 1
QCW_MAX_QUBITS = 17
QCW_MAX_KRAUS = 64

_lock = threading.Lock()
_lib = None

P = ctypes.c_void_p
I = ctypes.c_int
D = ctypes.c_double
LL = ctypes.c_longlong
PP = ctypes.POINTER(ctypes.c_void_p)
PD = ctypes.POINTER(ctypes.c_double)
PI = ctypes.POINTER(ctypes.c_int)
PLL = ctypes.POINTER(ctypes.c_longlong)

# name -> (restype, argtypes) for every declaration of include/qcw.h
SIGNATURES = {
    "qcw_create": (I, [I, PP]),
    "qcw_create_from_ptr": (I, [I, P, P, PP]),
    "qcw_destroy": (I, [P]),
    "qcw_set_mode": (I, [P, I, I]),
    "qcw_set_validation": (I, [P, I]),
    "qcw_set_fused_kernel": (I, [P, I]),
    "qcw_set_fused_wait_limit": (I, [P, ctypes.c_uint, I]),
    "qcw_get_device_state": (I, [P, PP, PP]),
    "qcw_nqubits": (I, [P]),
    "qcw_reset": (I, [P]),
    "qcw_set_state": (I, [P, P]),
    "qcw_set_state_c64": (I, [P, P]),
    "qcw_get_state": (I, [P, P]),
    "qcw_apply_gate1": (I, [P, P, I, P, I]),
    "qcw_apply_gate2": (I, [P, P, I, I, P, I]),
    "qcw_apply_gate": (I, [P, P, P, I]),
    "qcw_apply_kraus": (I, [P, P, I, P, I]),
    "qcw_apply_ops": (I, [P, P, I, P]),
    "qcw_flush": (I, [P]),
    "qcw_sync": (I, [P]),
    "qcw_trace": (I, [P, PD, PD]),
    "qcw_purity": (I, [P, PD]),
    "qcw_probabilities": (I, [P, P]),
    "qcw_polarization": (I, [P, P]),
    "qcw_correlation": (I, [P, I, I, P]),
    "qcw_entropy": (I, [P, P, I, PD]),
    "qcw_eigenvalues": (I, [P, P, I, P]),
    "qcw_fidelity": (I, [P, P, I, P, PD]),
    "qcw_ensemble_create": (I, [I, I, PP]),
    "qcw_ensemble_destroy": (I, [P]),
    "qcw_ensemble_set": (I, [P, P]),
    "qcw_ensemble_get": (I, [P, P]),
    "qcw_ensemble_apply_gate1": (I, [P, P, I]),
    "qcw_ensemble_apply_gate2": (I, [P, P, I, I]),
    "qcw_ensemble_apply_noise1": (I, [P, P, I, I, P]),
    "qcw_ensemble_density": (I, [P, P, P]),
    "qcw_checkpoint": (I, [P, PLL]),
    "qcw_checkpoint_read": (I, [P, LL, P]),
    "qcw_measure": (I, [P, I, I, D, PI, PD]),
    "qcw_partial_trace": (I, [P, P, I, P]),
    "qcw_partial_trace_static": (I, [P, I, P, I, P, P]),
    "qcw_batch_create": (I, [I, P, P, P, P, I, P, PP]),
    "qcw_batch_run": (I, [P]),
    "qcw_batch_wait": (I, [P, D]),
    "qcw_batch_results": (I, [P, P, P, P]),
    "qcw_batch_get_state": (I, [P, I, P]),
    "qcw_batch_info": (I, [P, PLL, PLL, PLL, PD]),
    "qcw_batch_set_wait_limit": (I, [P, LL, I]),
    "qcw_batch_destroy": (I, [P]),
    "qcw_server_create": (I, [ctypes.c_size_t, I, I, P, PP]),
    "qcw_server_submit": (I, [P, I, P, I, P, PLL]),
    "qcw_server_step": (I, [P, PI]),
    "qcw_server_drain": (I, [P, D]),
    "qcw_server_poll": (I, [P, P, I, PI]),
    "qcw_server_stats": (I, [P, PLL, PLL, PLL, PLL]),
    "qcw_server_set_limits": (I, [P, D, LL, I]),
    "qcw_server_destroy": (I, [P]),
    "qcw_last_error": (ctypes.c_char_p, []),
    "qcw_strerror": (ctypes.c_char_p, [I]),
    "qcw_stats": (I, [P, PLL, PLL, PD, PLL]),
    "qcw_stats_reset": (I, [P]),
    "qcw_enable_pass_timing": (I, [P, I]),
}


class QcwOp(ctypes.Structure):
    """Mirror of qcw_op (include/qcw.h)."""

    _fields_ = [("kind", ctypes.c_int), ("k", ctypes.c_int), ("qubits", ctypes.c_int * 5),
                ("nkraus", ctypes.c_int), ("offset", ctypes.c_longlong)]


QCW_OP_GATE, QCW_OP_KRAUS = 0, 1


class PackedOps:
    """A circuit's op list packed once into the qcw_op array + matrix buffer of qcw_apply_ops."""

    def __init__(self, ops):
        ops = list(ops)
        self.n_ops = len(ops)
        self.descs = (QcwOp * max(1, len(ops)))()
        mats = []
        off = 0
        for i, op in enumerate(ops):
            d = self.descs[i]
            d.kind = QCW_OP_GATE if op.kind == "gate" else QCW_OP_KRAUS
            d.k = len(op.qubits)
            for j, qb in enumerate(op.qubits):
                d.qubits[j] = int(qb)
            m = np.ascontiguousarray(np.asarray(op.mats if op.kind != "gate" else op.mats[0], dtype=np.complex128))
            d.nkraus = int(op.mats.shape[0]) if op.kind != "gate" else 1
            d.offset = off
            mats.append(m.reshape(-1))
            off += 2 * m.size
        self.matrices = np.ascontiguousarray(np.concatenate(mats) if mats else np.zeros(1, np.complex128))

    @property
    def nbytes(self) -> int:
        return ctypes.sizeof(QcwOp) * self.n_ops + self.matrices.nbytes


class QcwError(RuntimeError):
    def __init__(self, status: int, what: str, msg: str):
        super().__init__(f"{what}: status {status} ({msg})")
        self.status = status


def lib(path: str | None = None):
    """Load libqcw.so once (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"qcw CUDA library missing at {p}: run __graft_entry__.build()")
            L = ctypes.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def check(status: int, what: str):
    if status != QCW_OK:
        L = lib()
        raise QcwError(status, what, L.qcw_last_error().decode() or L.qcw_strerror(status).decode())


def _mat(u, dim: int) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(u, dtype=np.complex128))
    if a.size != dim:
        raise ValueError(f"expected {dim} complex entries, got {a.size}")
    return a


def _ints(xs) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(list(xs), dtype=np.int32))


def _p(a: np.ndarray):
    return a.ctypes.data_as(P) if a is not None and a.size else None


class Ensemble:
    """Multiverse ensemble: nvec device state vectors of n qubits (qcw_ensemble_*)."""

    def __init__(self, n: int, nvec: int):
        h = P()
        check(lib().qcw_ensemble_create(int(n), int(nvec), ctypes.byref(h)), "qcw_ensemble_create")
        self.h, self.n, self.nvec = h, int(n), int(nvec)

    def set(self, psi):
        a = np.ascontiguousarray(psi, dtype=np.complex128).reshape(self.nvec, 1 << self.n)
        check(lib().qcw_ensemble_set(self.h, _p(a)), "qcw_ensemble_set")

    def get(self) -> np.ndarray:
        out = np.zeros((self.nvec, 1 << self.n), dtype=np.complex128)
        check(lib().qcw_ensemble_get(self.h, _p(out)), "qcw_ensemble_get")
        return out

    def apply_gate1(self, u, target: int):
        a = np.ascontiguousarray(u, dtype=np.complex128)
        check(lib().qcw_ensemble_apply_gate1(self.h, _p(a), int(target)), "qcw_ensemble_apply_gate1")

    def apply_gate2(self, u, q1: int, q2: int):
        a = np.ascontiguousarray(u, dtype=np.complex128)
        check(lib().qcw_ensemble_apply_gate2(self.h, _p(a), int(q1), int(q2)), "qcw_ensemble_apply_gate2")

    def apply_noise1(self, omegas, target: int, choice):
        om = np.ascontiguousarray(omegas, dtype=np.complex128)
        ch = np.ascontiguousarray(choice, dtype=np.int32)
        check(lib().qcw_ensemble_apply_noise1(self.h, _p(om), om.shape[0], int(target), _p(ch)),
              "qcw_ensemble_apply_noise1")

    def density(self, weights, d: "Density"):
        w = np.ascontiguousarray(weights, dtype=np.float64)
        check(lib().qcw_ensemble_density(self.h, _p(w), d.h), "qcw_ensemble_density")

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().qcw_ensemble_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Density:
    """One qcw context: a device density matrix of n qubits and its stream."""

    def __init__(self, n: int, dev_ptr: int | None = None, stream: int | None = None):
        L = lib()
        h = P()
        if dev_ptr is None:
            check(L.qcw_create(int(n), ctypes.byref(h)), "qcw_create")
        else:
            check(L.qcw_create_from_ptr(int(n), P(dev_ptr), P(stream or 0), ctypes.byref(h)), "qcw_create_from_ptr")
        self.h = h
        self.n = int(n)

    @classmethod
    def from_tensor(cls, t, stream=None) -> "Density":
        """Borrow a torch tensor of 4^n complex64 values (and a torch.cuda.Stream)."""
        n = (int(t.numel()).bit_length() - 1) // 2
        sp = 0 if stream is None else int(stream.cuda_stream)
        return cls(n, t.data_ptr(), sp)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().qcw_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------- configuration / state
    def set_mode(self, mode: int, fuse_k: int = 0):
        check(lib().qcw_set_mode(self.h, int(mode), int(fuse_k)), "qcw_set_mode")

    def set_validation(self, on: bool = True):
        """Check unitarity, Kraus trace and Hermitian states on every call (QCW_EINVAL if not)."""
        check(lib().qcw_set_validation(self.h, int(bool(on))), "qcw_set_validation")

    def set_fused_kernel(self, which: int):
        """0 = auto (warp-specialised Hermitian from 6 qubits), 1 = one CTA per tile (no symmetry
        assumed), 2 = Hermitian, one CTA per tile pair, 3 = warp-specialised Hermitian (FP32 CUDA
        cores), 4 = 3 with its two-qubit phases on the tensor cores (tcgen05, 3xTF32)."""
        check(lib().qcw_set_fused_kernel(self.h, int(which)), "qcw_set_fused_kernel")

    def set_fused_wait_limit(self, polls: int, stall_tile: int = -1):
        """Poll limit of the fused kernel's in-kernel waits (0 = default) and an optional tile
        whose load the first CTA skips, so that the wait runs out."""
        check(lib().qcw_set_fused_wait_limit(self.h, int(polls), int(stall_tile)), "qcw_set_fused_wait_limit")

    def device_state(self):
        r, s = P(), P()
        check(lib().qcw_get_device_state(self.h, ctypes.byref(r), ctypes.byref(s)), "qcw_get_device_state")
        return r.value, s.value

    def reset(self):
        check(lib().qcw_reset(self.h), "qcw_reset")

    def set_state(self, rho: np.ndarray):
        a = np.ascontiguousarray(rho, dtype=np.complex128)
        assert a.shape == (1 << self.n, 1 << self.n)
        check(lib().qcw_set_state(self.h, _p(a)), "qcw_set_state")

    def set_state_c64(self, host_ptr: int):
        """Upload from a host buffer of 4^n complex64 (e.g. a pinned torch tensor's data_ptr)."""
        check(lib().qcw_set_state_c64(self.h, P(host_ptr)), "qcw_set_state_c64")

    def get_state(self) -> np.ndarray:
        out = np.empty((1 << self.n, 1 << self.n), dtype=np.complex128)
        check(lib().qcw_get_state(self.h, _p(out)), "qcw_get_state")
        return out

    # ---------------------------------------------------------------- evolution
    def apply_gate1(self, u, target: int, controls=()):
        m = _mat(u, 4)
        c = _ints(controls)
        check(lib().qcw_apply_gate1(self.h, _p(m), int(target), _p(c), len(c)), "qcw_apply_gate1")

    def apply_gate2(self, u, q1: int, q2: int, controls=()):
        m = _mat(u, 16)
        c = _ints(controls)
        check(lib().qcw_apply_gate2(self.h, _p(m), int(q1), int(q2), _p(c), len(c)), "qcw_apply_gate2")

    def apply_gate(self, u, qubits):
        q = _ints(qubits)
        m = _mat(u, 1 << (2 * len(q)))
        check(lib().qcw_apply_gate(self.h, _p(m), _p(q), len(q)), "qcw_apply_gate")

    def apply_kraus(self, kraus, qubits):
        q = _ints(qubits)
        ks = np.ascontiguousarray(np.asarray(kraus, dtype=np.complex128))
        nk = ks.shape[0] if ks.ndim == 3 else 1
        if ks.size != nk << (2 * len(q)):
            raise ValueError("Kraus array has the wrong size")
        check(lib().qcw_apply_kraus(self.h, _p(ks), nk, _p(q), len(q)), "qcw_apply_kraus")

    def apply_op(self, op):
        """Apply one workloads.Op (gate or Kraus channel)."""
        if op.kind == "gate":
            if op.k == 1:
                self.apply_gate1(op.mats[0], op.qubits[0])
            elif op.k == 2:
                self.apply_gate2(op.mats[0], op.qubits[0], op.qubits[1])
            else:
                self.apply_gate(op.mats[0], op.qubits)
        else:
            self.apply_kraus(op.mats, op.qubits)

    def apply_packed(self, packed: "PackedOps"):
        """Apply a PackedOps list in one C call (qcw_apply_ops)."""
        check(lib().qcw_apply_ops(self.h, ctypes.cast(packed.descs, P), packed.n_ops,
                                  packed.matrices.ctypes.data_as(P)), "qcw_apply_ops")

    def flush(self):
        check(lib().qcw_flush(self.h), "qcw_flush")

    def sync(self):
        check(lib().qcw_sync(self.h), "qcw_sync")

    # ---------------------------------------------------------------- readouts
    def trace(self) -> complex:
        re, im = D(), D()
        check(lib().qcw_trace(self.h, ctypes.byref(re), ctypes.byref(im)), "qcw_trace")
        return complex(re.value, im.value)

    def purity(self) -> float:
        v = D()
        check(lib().qcw_purity(self.h, ctypes.byref(v)), "qcw_purity")
        return v.value

    def probabilities(self) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.float64)
        check(lib().qcw_probabilities(self.h, _p(out)), "qcw_probabilities")
        return out

    def polarization(self) -> np.ndarray:
        """Polarisation vectors Tr[sigma^(q) rho], shape (n, 3) (x, y, z per qubit)."""
        out = np.zeros(3 * self.n, dtype=np.float64)
        check(lib().qcw_polarization(self.h, _p(out)), "qcw_polarization")
        return out.reshape(self.n, 3)

    def correlation(self, q1: int, q2: int) -> np.ndarray:
        """Spin correlation tensor Tr[sigma_i^(q1) sigma_j^(q2) rho], shape (3, 3)."""
        out = np.zeros(9, dtype=np.float64)
        check(lib().qcw_correlation(self.h, int(q1), int(q2), _p(out)), "qcw_correlation")
        return out.reshape(3, 3)

    def entropy(self, keep) -> float:
        """von Neumann entropy (bits) of the reduced state of the kept qubits (1..6, ascending)."""
        k = np.ascontiguousarray(keep, dtype=np.int32)
        v = D()
        check(lib().qcw_entropy(self.h, _p(k), len(k), ctypes.byref(v)), "qcw_entropy")
        return v.value

    def eigenvalues(self, keep) -> np.ndarray:
        """Eigenvalues (ascending) of the reduced state of the kept qubits."""
        k = _ints(sorted(keep))
        out = np.zeros(1 << len(k), dtype=np.float64)
        check(lib().qcw_eigenvalues(self.h, _p(k), len(k), _p(out)), "qcw_eigenvalues")
        return out

    def fidelity(self, keep, sigma) -> float:
        """Tr sqrt(sqrt(sigma) rho_A sqrt(sigma)) of the reduced state of `keep` with sigma."""
        k = np.ascontiguousarray(keep, dtype=np.int32)
        s = np.ascontiguousarray(sigma, dtype=np.complex128)
        v = D()
        check(lib().qcw_fidelity(self.h, _p(k), len(k), _p(s), ctypes.byref(v)), "qcw_fidelity")
        return v.value

    def checkpoint(self) -> int:
        """Enqueue the trace / purity / probability reductions of the current rho (flushes queued
        work, does not wait); returns the ticket for checkpoint_read."""
        t = LL()
        check(lib().qcw_checkpoint(self.h, ctypes.byref(t)), "qcw_checkpoint")
        return t.value

    def checkpoint_read(self, ticket: int):
        """(trace, purity, probabilities) of checkpoint `ticket` (waits for it)."""
        out = np.zeros(self.n + 3, dtype=np.float64)
        check(lib().qcw_checkpoint_read(self.h, int(ticket), _p(out)), "qcw_checkpoint_read")
        return complex(out[0], out[1]), float(out[2 + self.n]), out[2:2 + self.n].copy()

    def measure(self, qubit: int, forced: int = -1, u: float = 0.0):
        oc, pr = I(), D()
        check(lib().qcw_measure(self.h, int(qubit), int(forced), float(u), ctypes.byref(oc), ctypes.byref(pr)),
              "qcw_measure")
        return oc.value, pr.value

    def partial_trace(self, keep) -> np.ndarray:
        k = _ints(sorted(keep))
        out = np.zeros((1 << len(k), 1 << len(k)), dtype=np.complex128)
        check(lib().qcw_partial_trace(self.h, _p(k), len(k), _p(out)), "qcw_partial_trace")
        return out

    # ---------------------------------------------------------------- diagnostics
    def enable_pass_timing(self, on: bool = True):
        check(lib().qcw_enable_pass_timing(self.h, int(bool(on))), "qcw_enable_pass_timing")

    def stats(self) -> dict:
        la, ps, ts = LL(), LL(), LL()
        ms = D()
        check(lib().qcw_stats(self.h, ctypes.byref(la), ctypes.byref(ps), ctypes.byref(ms), ctypes.byref(ts)),
              "qcw_stats")
        return {"launches": la.value, "fused_passes": ps.value, "fused_pass_ms": ms.value, "timed_passes": ts.value}

    def stats_reset(self):
        check(lib().qcw_stats_reset(self.h), "qcw_stats_reset")


def run_circuit(circuit, dens: Density | None = None, ops=None) -> Density:
    """Apply a workloads.Circuit through the C ABI (initial state uploaded when given)."""
    d = dens or Density(circuit.n)
    if circuit.init == "matrix":
        d.set_state(circuit.rho0)
    else:
        d.reset()
    for op in (circuit.ops if ops is None else ops):
        d.apply_op(op)
    return d


class QcwResult(ctypes.Structure):
    """Mirror of qcw_result (include/qcw.h)."""

    _fields_ = [("id", ctypes.c_longlong), ("nqubits", ctypes.c_int), ("status", ctypes.c_int),
                ("trace", ctypes.c_double), ("purity", ctypes.c_double), ("p1", ctypes.c_double * QCW_MAX_QUBITS),
                ("t_submit", ctypes.c_double), ("t_done", ctypes.c_double)]


class Batch:
    """qcw_batch_*: many circuits (workloads.Circuit, starting from |0..0>) in one graph launch."""

    def __init__(self, circuits, fuse_k: int = 0, stream: int = 0):
        circuits = list(circuits)
        packs = [PackedOps(c.ops) for c in circuits]
        nq = np.asarray([c.n for c in circuits], dtype=np.int32)
        begin = np.zeros(len(circuits) + 1, dtype=np.int64)
        total = sum(p.n_ops for p in packs)
        descs = (QcwOp * max(1, total))()
        mats = []
        k = 0
        moff = 0
        for j, p in enumerate(packs):
            begin[j] = k
            for i in range(p.n_ops):
                descs[k] = p.descs[i]
                descs[k].offset = p.descs[i].offset + moff
                k += 1
            mats.append(p.matrices)
            moff += 2 * p.matrices.size
        begin[len(circuits)] = k
        self.matrices = np.ascontiguousarray(np.concatenate(mats))
        self.nqubits = nq
        h = P()
        check(lib().qcw_batch_create(len(circuits), nq.ctypes.data_as(P), begin.ctypes.data_as(P),
                                     ctypes.cast(descs, P), self.matrices.ctypes.data_as(P), int(fuse_k),
                                     P(stream), ctypes.byref(h)), "qcw_batch_create")
        self.h = h

    def run(self):
        check(lib().qcw_batch_run(self.h), "qcw_batch_run")

    def wait(self, timeout_s: float = -1.0):
        check(lib().qcw_batch_wait(self.h, float(timeout_s)), "qcw_batch_wait")

    def results(self):
        """(list of per-circuit p1 arrays, purity array, trace array)."""
        p1 = np.zeros(int(self.nqubits.sum()), dtype=np.float64)
        pur = np.zeros(len(self.nqubits), dtype=np.float64)
        tr = np.zeros(len(self.nqubits), dtype=np.float64)
        check(lib().qcw_batch_results(self.h, _p(p1), _p(pur), _p(tr)), "qcw_batch_results")
        out, o = [], 0
        for n in self.nqubits:
            out.append(p1[o:o + n].copy())
            o += n
        return out, pur, tr

    def get_state(self, j: int) -> np.ndarray:
        n = int(self.nqubits[j])
        out = np.empty((1 << n, 1 << n), dtype=np.complex128)
        check(lib().qcw_batch_get_state(self.h, int(j), _p(out)), "qcw_batch_get_state")
        return out

    def info(self) -> dict:
        it, ps, ph = LL(), LL(), LL()
        md = D()
        check(lib().qcw_batch_info(self.h, ctypes.byref(it), ctypes.byref(ps), ctypes.byref(ph), ctypes.byref(md)),
              "qcw_batch_info")
        return {"items": it.value, "passes": ps.value, "phases": ph.value, "modeled_sm_s": md.value}

    def set_wait_limit(self, polls: int, stall_item: int = -1):
        check(lib().qcw_batch_set_wait_limit(self.h, int(polls), int(stall_item)), "qcw_batch_set_wait_limit")

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().qcw_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """qcw_server_*: continuous batching of circuit requests."""

    def __init__(self, budget_bytes: int, max_live: int = 4096, passes_per_step: int = 4, stream: int = 0):
        h = P()
        check(lib().qcw_server_create(int(budget_bytes), int(max_live), int(passes_per_step), P(stream),
                                      ctypes.byref(h)), "qcw_server_create")
        self.h = h
        self._buf = (QcwResult * 256)()

    def submit(self, circuit, packed: "PackedOps | None" = None) -> int:
        """Queue a workloads.Circuit (optionally with its op list packed in advance)."""
        p = packed or PackedOps(circuit.ops)
        rid = LL()
        check(lib().qcw_server_submit(self.h, int(circuit.n), ctypes.cast(p.descs, P), p.n_ops,
                                      p.matrices.ctypes.data_as(P), ctypes.byref(rid)), "qcw_server_submit")
        return rid.value

    def step(self) -> int:
        k = I()
        check(lib().qcw_server_step(self.h, ctypes.byref(k)), "qcw_server_step")
        return k.value

    def drain(self, timeout_s: float = -1.0):
        check(lib().qcw_server_drain(self.h, float(timeout_s)), "qcw_server_drain")

    def poll(self):
        """Finished results as dicts (id, n, status, trace, purity, p1, t_submit, t_done)."""
        out = []
        while True:
            c = I()
            check(lib().qcw_server_poll(self.h, ctypes.cast(self._buf, P), len(self._buf), ctypes.byref(c)),
                  "qcw_server_poll")
            for i in range(c.value):
                r = self._buf[i]
                out.append({"id": r.id, "n": r.nqubits, "status": r.status, "trace": r.trace, "purity": r.purity,
                            "p1": np.array(r.p1[:r.nqubits]), "t_submit": r.t_submit, "t_done": r.t_done})
            if c.value < len(self._buf):
                return out

    def stats(self) -> dict:
        w, l, c, b = LL(), LL(), LL(), LL()
        check(lib().qcw_server_stats(self.h, ctypes.byref(w), ctypes.byref(l), ctypes.byref(c), ctypes.byref(b)),
              "qcw_server_stats")
        return {"waiting": w.value, "live": l.value, "completed": c.value, "bytes_in_use": b.value}

    def set_limits(self, wait_limit_s: float, polls: int, stall_next_step: bool = False):
        check(lib().qcw_server_set_limits(self.h, float(wait_limit_s), int(polls), int(bool(stall_next_step))),
              "qcw_server_set_limits")

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().qcw_server_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
