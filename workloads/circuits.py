"""Seeded circuit and state generators (inputs only; no simulation arithmetic).

Every random draw goes through numpy's PCG64 with a seed derived from the workload:
configuration c uses base seed 20261100 + c and circuit j inside it uses
base * 1000003 + j.

Gate set.  The paper defines NOT (sigma_x), the Hadamard and the Pauli operators
(Sec. 3, Sec. 3.1) and names CNOT and the controlled phase as its typical two-qubit gates
(Sec. 4.2).  The remaining members are the standard ones: S = diag(1, i),
T = diag(1, e^{i pi/4}), CZ = diag(1, 1, 1, -1) and a Haar-random SU(2) built from four
N(0,1) draws (a, b, c, d) normalised to unit length, U = [[a+ib, c+id], [-c+id, a-ib]].

Noise.  The paper's ensemble form (Eq. rhoE1 / rhoE2) is a Kraus sum; the channels used
by the workloads are amplitude damping, phase damping and depolarising (Pauli multiverse
with n_p = 3 and epsilon = p), with the textbook Kraus operators.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

BASE_SEED = 20261100
GATE_KINDS_MIXED = ("H", "X", "Z", "S", "T", "CNOT", "HAAR")

_SQ2 = 1.0 / np.sqrt(2.0)
_FIXED = {
    "I": np.eye(2, dtype=np.complex128),
    "H": np.array([[_SQ2, _SQ2], [_SQ2, -_SQ2]], dtype=np.complex128),
    "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    "Z": np.array([[1, 0], [0, -1]], dtype=np.complex128),
    "S": np.array([[1, 0], [0, 1j]], dtype=np.complex128),
    "T": np.array([[1, 0], [0, np.exp(1j * np.pi / 4)]], dtype=np.complex128),
    "CNOT": np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=np.complex128),
    "CZ": np.diag([1, 1, 1, -1]).astype(np.complex128),
    "SWAP": np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128),
}


def seed_for(config: int, index: int = 0) -> int:
    """Seed of circuit ``index`` inside workload configuration ``config``."""
    return (BASE_SEED + config) * 1000003 + index


def gate_matrix(name: str) -> np.ndarray:
    """Fixed gate matrix by name (copy)."""
    return _FIXED[name].copy()


def haar_su2(rng: np.random.Generator) -> np.ndarray:
    a, b, c, d = rng.standard_normal(4)
    nrm = np.sqrt(a * a + b * b + c * c + d * d)
    a, b, c, d = a / nrm, b / nrm, c / nrm, d / nrm
    return np.array([[a + 1j * b, c + 1j * d], [-c + 1j * d, a - 1j * b]], dtype=np.complex128)


def haar_unitary(rng: np.random.Generator, dim: int) -> np.ndarray:
    """Haar unitary of size dim (QR of a complex Ginibre matrix with phase fix)."""
    z = (rng.standard_normal((dim, dim)) + 1j * rng.standard_normal((dim, dim))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return q * ph[None, :]


def haar_state(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return v / np.linalg.norm(v)


def kraus_ad(gamma: float) -> np.ndarray:
    """Amplitude damping: K0 = diag(1, sqrt(1-g)), K1 = [[0, sqrt(g)], [0, 0]]."""
    k0 = np.array([[1, 0], [0, np.sqrt(1 - gamma)]], dtype=np.complex128)
    k1 = np.array([[0, np.sqrt(gamma)], [0, 0]], dtype=np.complex128)
    return np.stack([k0, k1])


def kraus_pd(lam: float) -> np.ndarray:
    """Phase damping: K0 = diag(1, sqrt(1-l)), K1 = diag(0, sqrt(l))."""
    k0 = np.array([[1, 0], [0, np.sqrt(1 - lam)]], dtype=np.complex128)
    k1 = np.array([[0, 0], [0, np.sqrt(lam)]], dtype=np.complex128)
    return np.stack([k0, k1])


def kraus_pauli_multiverse(p: float, eps: float, omegas: Sequence[np.ndarray]) -> np.ndarray:
    """Kraus set of the paper's ensemble (Eq. rhoE2): sqrt(p) 1 and sqrt(eps/n_p) Omega_n."""
    d = omegas[0].shape[0]
    npth = len(omegas)
    ks = [np.sqrt(p) * np.eye(d, dtype=np.complex128)]
    ks += [np.sqrt(eps / npth) * np.asarray(o, dtype=np.complex128) for o in omegas]
    return np.stack(ks)


def kraus_depolarising(p: float) -> np.ndarray:
    """(1-p) rho + p/3 (X rho X + Y rho Y + Z rho Z): Eq. rhoE2 with n_p = 3, eps = p."""
    return kraus_pauli_multiverse(1.0 - p, p, [_FIXED["X"], _FIXED["Y"], _FIXED["Z"]])


@dataclass
class Op:
    """One circuit element.  ``mats`` has shape (m, d, d), d = 2**len(qubits); a gate has m = 1."""

    kind: str  # "gate" or "kraus"
    qubits: Tuple[int, ...]
    mats: np.ndarray
    name: str = ""

    @property
    def k(self) -> int:
        return len(self.qubits)


@dataclass
class Circuit:
    n: int
    ops: List[Op] = field(default_factory=list)
    init: str = "zero"  # "zero" or "matrix"
    rho0: np.ndarray | None = None  # complex128 (2^n, 2^n) when init == "matrix"
    seed: int = 0
    measure_qubit: int | None = None

    @property
    def n_gates(self) -> int:
        return sum(1 for o in self.ops if o.kind == "gate")

    @property
    def n_channels(self) -> int:
        return sum(1 for o in self.ops if o.kind == "kraus")

    def gate_prefix(self, ngates: int) -> "Circuit":
        """Ops up to and including the channels attached to gate number ``ngates``."""
        out, seen = [], 0
        for o in self.ops:
            if o.kind == "gate":
                if seen == ngates:
                    break
                seen += 1
            out.append(o)
        return Circuit(self.n, out, self.init, self.rho0, self.seed, self.measure_qubit)


def zero_state(n: int) -> np.ndarray:
    rho = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    rho[0, 0] = 1.0
    return rho


def mixed_plus_haar_state(rng: np.random.Generator, n: int, weight: float = 0.5) -> np.ndarray:
    """(1 - w) I / 2^n + w |psi><psi| with psi Haar-random."""
    psi = haar_state(rng, n)
    d = 1 << n
    return (1.0 - weight) * np.eye(d, dtype=np.complex128) / d + weight * np.outer(psi, psi.conj())


def random_density_matrix(rng: np.random.Generator, n: int, rank: int | None = None) -> np.ndarray:
    """A A^dagger / Tr with A complex Gaussian (d x rank): Hermitian, PSD, unit trace."""
    d = 1 << n
    r = d if rank is None else rank
    a = rng.standard_normal((d, r)) + 1j * rng.standard_normal((d, r))
    m = a @ a.conj().T
    return m / np.trace(m).real


def _pick_qubits(rng: np.random.Generator, n: int, k: int) -> Tuple[int, ...]:
    return tuple(int(q) for q in rng.choice(n, size=k, replace=False))


def _noise_ops(noise: str, qubits: Sequence[int], params: dict) -> List[Op]:
    out: List[Op] = []
    for q in qubits:
        if noise == "adpd":
            out.append(Op("kraus", (q,), kraus_ad(params.get("gamma", 0.01)), "AD"))
            out.append(Op("kraus", (q,), kraus_pd(params.get("lam", 0.02)), "PD"))
        elif noise == "dep":
            out.append(Op("kraus", (q,), kraus_depolarising(params.get("p", 1e-3)), "DEP"))
        elif noise == "none":
            pass
        else:
            raise ValueError(noise)
    return out


def random_circuit(
    n: int,
    ngates: int,
    seed: int,
    mix: str = "mixed",
    noise: str = "adpd",
    noise_params: dict | None = None,
) -> Circuit:
    """Seeded random circuit.

    mix="mixed": kinds uniform over {H, X, Z, S, T, CNOT, HAAR}; CNOT on an ordered distinct
    pair (first = control).  mix="haar70": 70 % Haar SU(2), 30 % CNOT/CZ (1:1).
    After each gate the noise channel acts on every touched qubit (AD then PD for "adpd").
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    params = dict(noise_params or {})
    ops: List[Op] = []
    for _ in range(ngates):
        if mix == "mixed":
            kind = GATE_KINDS_MIXED[int(rng.integers(len(GATE_KINDS_MIXED)))]
        elif mix == "haar70":
            if rng.random() < 0.7:
                kind = "HAAR"
            else:
                kind = "CNOT" if rng.random() < 0.5 else "CZ"
        else:
            raise ValueError(mix)
        if kind in ("CNOT", "CZ"):
            if n < 2:
                kind = "HAAR"
            else:
                qs = _pick_qubits(rng, n, 2)
                ops.append(Op("gate", qs, gate_matrix(kind)[None], kind))
                ops.extend(_noise_ops(noise, qs, params))
                continue
        q = int(rng.integers(n))
        mat = haar_su2(rng) if kind == "HAAR" else gate_matrix(kind)
        ops.append(Op("gate", (q,), mat[None], kind))
        ops.extend(_noise_ops(noise, (q,), params))
    return Circuit(n, ops, seed=seed)


def config1_circuit(index: int = 0) -> Circuit:
    """4 qubits from |0000><0000|, 40 mixed gates, AD(0.01)+PD(0.02), measure qubit 0."""
    c = random_circuit(4, 40, seed_for(1, index), "mixed", "adpd", {"gamma": 0.01, "lam": 0.02})
    c.measure_qubit = 0
    return c


def config2_circuit(index: int = 0, n: int = 12, ngates: int = 500) -> Circuit:
    """12 qubits from I/2^n/2 + |psi><psi|/2, 500 gates (70 % Haar, 30 % CNOT/CZ), dep 1e-3."""
    seed = seed_for(2, index)
    c = random_circuit(n, ngates, seed, "haar70", "dep", {"p": 1e-3})
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    c.init = "matrix"
    c.rho0 = mixed_plus_haar_state(rng, n, 0.5)
    return c


def config3_circuit(index: int = 0, n: int = 14, ngates: int = 1000) -> Circuit:
    """14 qubits from |0><0|, 1000 mixed gates with AD(0.01)+PD(0.02) on touched qubits."""
    c = random_circuit(n, ngates, seed_for(3, index), "mixed", "adpd", {"gamma": 0.01, "lam": 0.02})
    c.measure_qubit = 0
    return c


def config4_batch(ncirc: int = 512, nmin: int = 4, nmax: int = 10, dmin: int = 50, dmax: int = 400,
                  index: int = 0) -> List[Circuit]:
    """Independent circuits: n ~ U{nmin..nmax}, depth ~ U{dmin..dmax}, gamma ~ U[.001,.05]."""
    rng = np.random.Generator(np.random.PCG64(seed_for(4, index)))
    out = []
    for j in range(ncirc):
        n = int(rng.integers(nmin, nmax + 1))
        depth = int(rng.integers(dmin, dmax + 1))
        gamma = float(rng.uniform(0.001, 0.05))
        c = random_circuit(n, depth, seed_for(4, index) + 1 + j, "mixed", "adpd",
                           {"gamma": gamma, "lam": 0.02})
        out.append(c)
    return out


def config5_requests(rate: float = 2000.0, duration: float = 60.0, nmin: int = 3, nmax: int = 13,
                     dmin: int = 20, dmax: int = 500, index: int = 0, limit: int | None = None):
    """Poisson request stream: list of (arrival_time_s, Circuit).

    n in nmin..nmax with P(n) proportional to 2^-(n - nmin); depth ~ U{dmin..dmax};
    noise uniform over {AD+PD, depolarising, none}.
    """
    rng = np.random.Generator(np.random.PCG64(seed_for(5, index)))
    ns = np.arange(nmin, nmax + 1)
    w = 2.0 ** (-(ns - nmin).astype(np.float64))
    w /= w.sum()
    t = 0.0
    out = []
    j = 0
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration or (limit is not None and j >= limit):
            break
        n = int(rng.choice(ns, p=w))
        depth = int(rng.integers(dmin, dmax + 1))
        noise = ("adpd", "dep", "none")[int(rng.integers(3))]
        c = random_circuit(n, depth, seed_for(5, index) + 1 + j, "mixed", noise,
                           {"gamma": 0.01, "lam": 0.02, "p": 1e-3})
        out.append((t, c))
        j += 1
    return out


# ----------------------------------------------------------------------------- multiverse noise experiments
# The paper's noise studies (Sec. 5.2-5.4; notebooks MV1-Noise, MV2-Noise, MVn-Noise): a short
# algorithm on 1, 2 or 5 qubits, and at every step the ensemble average of Eq. rhoE4 over n_p
# noise paths.  The ideal path keeps rho with probability p (the storage case: p = 0.8,
# eps = 0.2); path k applies, with probability eps p_1 / n_p, a Pauli to one random qubit and,
# with probability eps p_2 / n_p, Paulis to two distinct random qubits (p_1 = 0.95, p_2 = 0.05;
# a one-qubit register has only the one-hit case, weight eps / n_p).  The noise operators are
# drawn once and held fixed.  Switching a Pauli off (the notebooks' ss[i] -> s[0]) replaces it
# by the identity after the draw, so every noise setting shares the same random structure.
# This module only draws these inputs; both sides apply them.

PAULI_NAMES = ("I", "X", "Y", "Z")
NOISE_SWITCHES = {"xyz": (1, 2, 3), "yz": (2, 3), "z": (3,), "none": ()}

MV_ALGORITHMS = {
    # |0>, Hadamard at step 1, another at step 3, then noise only (caption of the MV1 figure)
    "MV1": (1, {1: [("H", (0,))], 3: [("H", (0,))]}),
    # |00>, H on qubit 1 then CNOT_12 (the Bell preparation), later CNOT_12 then H_1 (its
    # inverse), then noise only (Sec. 5.3, MV2-Noise)
    "MV2": (2, {1: [("H", (0,))], 2: [("CNOT", (0, 1))], 3: [("CNOT", (0, 1))], 4: [("H", (0,))]}),
    # |00000>, H_1 then CNOT_12, CNOT_13, CNOT_14, CNOT_15: the GHZ chain (Sec. 5.4, MVn-Noise)
    "MVn": (5, {1: [("H", (0,))], 2: [("CNOT", (0, 1))], 3: [("CNOT", (0, 2))], 4: [("CNOT", (0, 3))],
                5: [("CNOT", (0, 4))]}),
}


@dataclass
class MVExperiment:
    name: str
    n: int
    nsteps: int
    n_p: int
    noise: str
    p: float = 0.8
    eps: float = 0.2
    ps: Tuple[float, float] = (0.95, 0.05)
    algorithm: dict = field(default_factory=dict)
    hits: list = field(default_factory=list)  # hits[step - 1][k] = (one-hit [(q, a)], two-hit [(q, a), (q, a)])

    def _on(self, a: int) -> int:
        return a if a in NOISE_SWITCHES[self.noise] else 0

    def noise_terms(self, step: int):
        """Terms (weight, [(qubit, Pauli index 0..3), ...]) of the noise average at `step` (1-based);
        the first term is the ideal path.  Weights sum to 1."""
        terms = [(self.p, [])]
        for one, two in self.hits[step - 1]:
            if self.n == 1:
                terms.append((self.eps / self.n_p, [(q, self._on(a)) for q, a in one]))
            else:
                terms.append((self.eps * self.ps[0] / self.n_p, [(q, self._on(a)) for q, a in one]))
                terms.append((self.eps * self.ps[1] / self.n_p, [(q, self._on(a)) for q, a in two]))
        return terms

    def pauli_string(self, hits) -> np.ndarray:
        """The full-register operator of a term's hits (qubit 0 the leftmost Kronecker factor)."""
        ops = [_FIXED["I"]] * self.n
        ops = list(ops)
        for q, a in hits:
            ops[q] = _FIXED[PAULI_NAMES[a]]
        m = np.ones((1, 1), dtype=np.complex128)
        for o in ops:
            m = np.kron(m, o)
        return m

    def kraus(self, step: int) -> np.ndarray:
        """Kraus form of the step's noise average (Eq. rhoE2): sqrt(w) times each term's operator,
        acting on all qubits 0..n-1 in order."""
        return np.stack([np.sqrt(w) * self.pauli_string(h) for w, h in self.noise_terms(step)])

    def gates(self, step: int):
        """Algorithm operators of `step` as (matrix, qubits), applied after the step's noise."""
        return [(gate_matrix(name), qs) for name, qs in self.algorithm.get(step, [])]

    def psi0(self) -> np.ndarray:
        v = np.zeros(1 << self.n, dtype=np.complex128)
        v[0] = 1.0
        return v

    def rho0(self) -> np.ndarray:
        return zero_state(self.n)


def mv_experiment(name: str, noise: str = "xyz", nsteps: int | None = None, n_p: int = 8,
                  index: int = 0) -> MVExperiment:
    """One of the paper's noise experiments with its noise operators drawn (seeded, held fixed)."""
    n, algo = MV_ALGORITHMS[name]
    nsteps = nsteps if nsteps is not None else {"MV1": 30, "MV2": 40, "MVn": 24}[name]
    rng = np.random.Generator(np.random.PCG64(seed_for(6, 10 * index + ("MV1", "MV2", "MVn").index(name))))
    hits = []
    for _ in range(nsteps):
        step = []
        for _ in range(n_p):
            q = int(rng.integers(n))
            one = [(q, int(rng.integers(1, 4)))]
            two = []
            if n > 1:
                q1, q2 = (int(x) for x in rng.choice(n, size=2, replace=False))
                two = [(q1, int(rng.integers(1, 4))), (q2, int(rng.integers(1, 4)))]
            step.append((one, two))
        hits.append(step)
    return MVExperiment(name, n, nsteps, n_p, noise, algorithm=algo, hits=hits)


def mv_trajectories(exp: MVExperiment, nvec: int, index: int = 0) -> np.ndarray:
    """Sampled paths of the statevector form of the same experiment: choice[step - 1, v] is the
    index of the noise term (into exp.noise_terms(step)) that vector v takes at that step, drawn
    with the terms' weights.  The average of the nvec pure states estimates rho."""
    rng = np.random.Generator(np.random.PCG64(seed_for(7, index)))
    out = np.zeros((exp.nsteps, nvec), dtype=np.int32)
    for s in range(1, exp.nsteps + 1):
        w = np.array([t[0] for t in exp.noise_terms(s)])
        out[s - 1] = rng.choice(len(w), size=nvec, p=w / w.sum())
    return out
