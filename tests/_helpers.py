"""Shared test helpers: golden-file parsing and brute-force full-space operators.

Nothing here calls the CUDA library; the brute-force embedding is an independent
definition used to pin the oracle (a dense 2^n x 2^n operator built entry by entry).
"""

from __future__ import annotations

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name: str):
    """Parse a golden file: '#' comments, then 'key v1 v2 ...' lines (numbers where possible)."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            vals = []
            for p in parts[1:]:
                try:
                    vals.append(int(p))
                except ValueError:
                    try:
                        vals.append(float(p))
                    except ValueError:
                        vals.append(p)
            rows.append((parts[0], vals))
    return rows


def embed(u: np.ndarray, qubits, n: int, controls=()) -> np.ndarray:
    """Full 2^n x 2^n operator, entry by entry from its definition.

    <r'|U_full|r> = U[idx(r'), idx(r)] when r' and r agree on every qubit outside ``qubits``
    (and all ``controls`` are 1 in r); identity on labels whose controls are not all 1.
    Qubit q carries weight 2^(n-1-q); idx() reads the struck qubits in the given order.
    """
    d = 1 << n
    k = len(qubits)
    w = [1 << (n - 1 - q) for q in qubits]
    cw = [1 << (n - 1 - q) for q in controls]
    tmask = sum(w)
    full = np.zeros((d, d), dtype=np.complex128)

    def idx(x):
        return sum(((x >> (n - 1 - q)) & 1) << (k - 1 - j) for j, q in enumerate(qubits))

    for r in range(d):
        if not all(r & c for c in cw):
            full[r, r] = 1.0
            continue
        for r2 in range(d):
            if (r & ~tmask) != (r2 & ~tmask):
                continue
            full[r2, r] = u[idx(r2), idx(r)]
    return full


def kron_single(u: np.ndarray, q: int, n: int) -> np.ndarray:
    """I_{2^q} (x) u (x) I_{2^(n-1-q)}: qubit 0 is the leftmost (most significant) factor."""
    return np.kron(np.kron(np.eye(1 << q), u), np.eye(1 << (n - 1 - q)))


def haar_unitary(rng, dim):
    z = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))[None, :]


def random_rho(rng, n, rank=None):
    d = 1 << n
    r = d if rank is None else rank
    a = rng.standard_normal((d, r)) + 1j * rng.standard_normal((d, r))
    m = a @ a.conj().T
    return m / np.trace(m).real


def bloch(rho1: np.ndarray) -> np.ndarray:
    """Polarisation P = Tr[sigma rho] of a one-qubit density matrix (Sec. 5.2)."""
    sx = np.array([[0, 1], [1, 0]])
    sy = np.array([[0, -1j], [1j, 0]])
    sz = np.array([[1, 0], [0, -1]])
    return np.array([np.trace(s @ rho1).real for s in (sx, sy, sz)])


def numpy_partial_trace(rho: np.ndarray, keep, n: int) -> np.ndarray:
    """Partial trace by reshaping to a rank-2n tensor and contracting with numpy.einsum."""
    keep = sorted(keep)
    t = rho.reshape([2] * (2 * n))
    letters = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"
    rin = list(letters[:n])
    cin = list(letters[n:2 * n])
    for q in range(n):
        if q not in keep:
            cin[q] = rin[q]
    out = "".join(rin[q] for q in keep) + "".join(cin[q] for q in keep)
    res = np.einsum("".join(rin) + "".join(cin) + "->" + out, t)
    da = 1 << len(keep)
    return res.reshape(da, da)


def gather_elements(d, rows, cols) -> np.ndarray:
    """Elements (rows[i], cols[i]) of a qcw Density's rho, gathered on the device and returned as
    complex128 (the library completes the state and orders it on the context's stream before it
    hands out the pointer).  Reads a few elements of a state too large to copy to the host."""
    import torch

    ptr, sp = d.device_state()
    torch.cuda.ExternalStream(sp).synchronize()
    dim = 1 << d.n

    class _Buf:
        pass

    buf = _Buf()
    buf.__cuda_array_interface__ = {"shape": (dim, 2 * dim), "typestr": "<f4", "data": (ptr, False), "version": 2}
    view = torch.as_tensor(buf, device="cuda")
    r = torch.as_tensor(np.asarray(rows, dtype=np.int64), device="cuda")
    c2 = torch.as_tensor(2 * np.asarray(cols, dtype=np.int64), device="cuda")
    return view[r, c2].double().cpu().numpy() + 1j * view[r, c2 + 1].double().cpu().numpy()
