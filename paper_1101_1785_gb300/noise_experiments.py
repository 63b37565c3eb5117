"""The paper's noise experiments on the qcw library (Sec. 5.2-5.4; notebooks MV1-Noise,
MV2-Noise and MVn-Noise).

Each experiment is a short algorithm on 1, 2 or 5 qubits (two Hadamards; the Bell preparation
and its inverse; the 5-qubit GHZ chain) in which every step first forms the ensemble average
of Eq. rhoE4 over the ideal path and n_p noise paths, then applies the step's algorithm
operators.  The noise operators (random Paulis on one qubit, or on two distinct qubits, held
fixed once drawn) and the on/off switches of the X, Y and Z noise come with the experiment
object (``workloads.mv_experiment``).  At every step the entropy, purity, fidelity with the
initial state, eigenvalues, polarisation vectors and (two or more qubits) the spin correlation
tensor of qubits 0 and 1 are read out, as the notebooks track them.

Two forms, both on the GPU through the C ABI:
  * ``run_density``: the density matrix itself; the noise average is one Kraus channel
    (Eq. rhoE2: sqrt(p) 1 and sqrt(eps p_s / n_p) Omega_ks) on the whole register.
  * ``run_trajectories``: the multiverse of state vectors (Sec. 5.2.1): each vector follows one
    sampled path per step (Op1 on every hit qubit), the algorithm acts on all vectors, and rho is
    the equal-weight average of the vectors' projectors, formed on the GPU.

``python -m paper_1101_1785_gb300.noise_experiments`` prints the fidelity, purity and entropy
curves of the three experiments under XYZ, YZ, Z-only and no noise.
"""

from __future__ import annotations

import numpy as np

from ._binding import QCW_MODE_FUSED, Density, Ensemble

_SQ = np.array


def _pauli_set() -> np.ndarray:
    return np.stack([
        _SQ([[1, 0], [0, 1]], dtype=np.complex128),
        _SQ([[0, 1], [1, 0]], dtype=np.complex128),
        _SQ([[0, -1j], [1j, 0]], dtype=np.complex128),
        _SQ([[1, 0], [0, -1]], dtype=np.complex128),
    ])


def readouts(d: Density, rho0: np.ndarray) -> dict:
    """The quantities the notebooks track, from the library's readouts of the whole register."""
    allq = list(range(d.n))
    r = {
        "trace": d.trace().real,
        "purity": d.purity(),
        "entropy": d.entropy(allq),
        "fidelity": d.fidelity(allq, rho0),
        "eigenvalues": d.eigenvalues(allq),
        "polarization": d.polarization(),
    }
    if d.n >= 2:
        r["correlation"] = d.correlation(0, 1)
    return r


def _apply_gates(target, exp, step):
    for u, qs in exp.gates(step):
        if len(qs) == 1:
            target.apply_gate1(u, qs[0])
        else:
            target.apply_gate2(u, qs[0], qs[1])


def run_density(exp, mode: str = "plain", fuse_k: int = 0, states: bool = False) -> list:
    """Readouts after step 0 .. exp.nsteps of the density-matrix form (plain or fused path)."""
    d = Density(exp.n)
    if mode == "fused":
        d.set_mode(QCW_MODE_FUSED, fuse_k)
    rho0 = exp.rho0()
    allq = list(range(exp.n))
    out = [readouts(d, rho0)]
    if states:
        out[-1]["rho"] = d.get_state()
    for s in range(1, exp.nsteps + 1):
        d.apply_kraus(exp.kraus(s), allq)
        _apply_gates(d, exp, s)
        out.append(readouts(d, rho0))
        if states:
            out[-1]["rho"] = d.get_state()
    d.close()
    return out


def run_trajectories(exp, choices: np.ndarray, states: bool = False) -> list:
    """Readouts after step 0 .. exp.nsteps of the statevector multiverse: choices[s - 1, v] is
    the noise term (index into exp.noise_terms(s)) vector v takes at step s."""
    nvec = choices.shape[1]
    ens = Ensemble(exp.n, nvec)
    ens.set(np.tile(exp.psi0(), (nvec, 1)))
    d = Density(exp.n)
    w = np.full(nvec, 1.0 / nvec)
    omegas = _pauli_set()
    rho0 = exp.rho0()
    ens.density(w, d)
    out = [readouts(d, rho0)]
    if states:
        out[-1]["rho"] = d.get_state()
    for s in range(1, exp.nsteps + 1):
        terms = exp.noise_terms(s)
        for q in range(exp.n):
            pick = np.zeros(nvec, dtype=np.int32)
            for t, (_, hits) in enumerate(terms):
                a = dict(hits).get(q, 0)
                if a:
                    pick[choices[s - 1] == t] = a
            if pick.any():
                ens.apply_noise1(omegas, q, pick)
        _apply_gates(ens, exp, s)
        ens.density(w, d)
        out.append(readouts(d, rho0))
        if states:
            out[-1]["rho"] = d.get_state()
    d.close()
    ens.close()
    return out


def main():
    import os
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import workloads as wl

    for name in ("MV1", "MV2", "MVn"):
        for noise in ("xyz", "yz", "z", "none"):
            exp = wl.mv_experiment(name, noise)
            res = run_density(exp)
            print(f"{name} noise={noise}: n={exp.n}, n_p={exp.n_p}, p={exp.p}, eps={exp.eps}")
            print("  step  fidelity  purity   entropy  eigenvalues")
            for s, r in enumerate(res):
                ev = " ".join(f"{x:.4f}" for x in r["eigenvalues"][-min(4, len(r['eigenvalues'])):])
                print(f"  {s:4d}  {r['fidelity']:.5f}  {r['purity']:.5f}  {r['entropy']:.5f}  {ev}")


if __name__ == "__main__":
    main()
