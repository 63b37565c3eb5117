#!/usr/bin/env python
"""Write the full-depth oracle readouts of the two large seeded circuits.

    python tests/golden/make_deep_goldens.py config2   # -> tests/golden/config2_n12.txt
    python tests/golden/make_deep_goldens.py config3   # -> tests/golden/config3_n14.txt

This script calls only the complex128 CPU oracle (``oracle/``) and the seeded input
generators (``workloads/``).  The circuits are too large for the oracle to replay inside a
GPU test (the 14-qubit one takes hours of host time), so their readouts are computed once
here and the GPU tests compare against the stored values.

What is recorded, in the order the benchmark reads it:
  * config2 (12 qubits, rho0 = I/2^n/2 + |psi><psi|/2, 500 gates, depolarising 1e-3, the
    Kraus sum of Eq. rhoE2 per touched qubit): the final trace, purity, per-qubit
    probabilities, two partial traces and 1024 seeded elements of the lower triangle
    (256 on the diagonal).
  * config3 (14 qubits from |0..0><0..0|, 1000 gates, AD(0.01) + PD(0.02) per touched qubit):
    trace, purity and per-qubit probabilities after every 100 gates; then 1024 seeded
    elements and the partial traces over qubits (0, 1) and (6, 13) of the final state; then
    the u-driven measurement of qubit 0 (u = 0.37, outcome 0 iff u < p_0, the reading of the
    measurement rule used throughout) with its outcome and probability, and the partial trace
    over (0, 1) and the purity of the renormalised post-measurement state.

``--state-dir`` keeps the oracle state every 100 gates so that an interrupted run resumes.
The 14-qubit state is 4 GiB of complex128: run with ``GLIBC_TUNABLES=glibc.malloc.hugetlb=1``
(transparent huge pages for large allocations), else page faults take most of the host time
(about three hours on 8 cores with them).
"""

from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as wl  # noqa: E402

NSAMPLE_OFF = 768
NSAMPLE_DIAG = 256
SAMPLE_SEED = 1101178500


def sample_positions(n: int):
    """Seeded (row, column) positions: NSAMPLE_DIAG on the diagonal, the rest strictly below it."""
    rng = np.random.Generator(np.random.PCG64(SAMPLE_SEED + n))
    d = 1 << n
    diag = rng.choice(d, size=NSAMPLE_DIAG, replace=False)
    pos = [(int(r), int(r)) for r in np.sort(diag)]
    seen = set()
    while len(seen) < NSAMPLE_OFF:
        r, c = (int(x) for x in rng.integers(0, d, size=2))
        if r == c:
            continue
        r, c = max(r, c), min(r, c)
        seen.add((r, c))
    return pos + sorted(seen)


def fmt(x: float) -> str:
    return repr(float(x))


def cplx_list(a) -> str:
    return " ".join(f"{fmt(z.real)} {fmt(z.imag)}" for z in np.asarray(a).ravel())


def readout_lines(rho, tag: str):
    tr = oracle.trace(rho)
    return [f"{tag} {fmt(tr.real)} {fmt(tr.imag)} {fmt(oracle.purity(rho))} "
            + " ".join(fmt(p) for p in oracle.probabilities(rho))]


def element_lines(rho, n):
    return [f"elem {r} {c} {fmt(rho[r, c].real)} {fmt(rho[r, c].imag)}" for r, c in sample_positions(n)]


def log(msg):
    print(f"[{time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def run_chunked(circuit, chunk: int, state_dir: str | None, tag: str, on_chunk=None):
    """Replay ``circuit`` chunk by chunk of gates (with their channels); on_chunk(g, rho) after each."""
    ng = circuit.n_gates
    bounds = list(range(0, ng + 1, chunk))
    if bounds[-1] != ng:
        bounds.append(ng)
    rho = oracle.initial_state(circuit)
    done = 0
    if state_dir:
        os.makedirs(state_dir, exist_ok=True)
        for g in reversed(bounds[1:]):
            path = os.path.join(state_dir, f"{tag}_g{g}.npy")
            if os.path.exists(path):
                rho = np.load(path)
                done = g
                log(f"resumed {tag} at gate {g}")
                break
    lines_by_g = {}
    if state_dir:
        for g in bounds[1:]:
            lp = os.path.join(state_dir, f"{tag}_g{g}.lines")
            if g <= done and os.path.exists(lp):
                with open(lp) as f:
                    lines_by_g[g] = f.read().splitlines()
    t0 = time.time()
    for i in range(len(bounds) - 1):
        g0, g1 = bounds[i], bounds[i + 1]
        if g1 <= done:
            continue
        ops = circuit.gate_prefix(g1).ops[len(circuit.gate_prefix(g0).ops):]
        for op in ops:
            oracle.apply_op(rho, op)
        lines = on_chunk(g1, rho) if on_chunk else []
        lines_by_g[g1] = lines
        log(f"{tag}: {g1}/{ng} gates, {time.time() - t0:.0f} s")
        if state_dir:
            np.save(os.path.join(state_dir, f"{tag}_g{g1}.npy.tmp.npy"), rho)
            os.replace(os.path.join(state_dir, f"{tag}_g{g1}.npy.tmp.npy"), os.path.join(state_dir, f"{tag}_g{g1}.npy"))
            with open(os.path.join(state_dir, f"{tag}_g{g1}.lines"), "w") as f:
                f.write("\n".join(lines))
            prev = os.path.join(state_dir, f"{tag}_g{g0}.npy")
            if g0 and os.path.exists(prev):
                os.remove(prev)
    out = []
    for g in bounds[1:]:
        out += lines_by_g.get(g, [])
    return rho, out


def make_config2(state_dir):
    c = wl.config2_circuit()
    n = c.n
    rho, _ = run_chunked(c, 100, state_dir, "config2")
    lines = [
        "# Full-depth oracle readouts of the 12-qubit circuit: rho0 = I/2^n/2 + |psi><psi|/2 (psi Haar),",
        "# 500 seeded gates (70 % Haar SU(2), 30 % CNOT / CZ), the depolarising channel p = 1e-3 of",
        "# Eq. rhoE1 / rhoE2 (n_p = 3, Omega in {X, Y, Z}, eps = p) on every touched qubit; the gate",
        "# sweeps of Sec. 3.1-3.2 (Eqs. resmat1, resmat2) on rows with U and columns with conj(U).",
        "# Written by tests/golden/make_deep_goldens.py from the complex128 oracle.",
        f"n {n}",
        f"gates {c.n_gates}",
        f"channels {c.n_channels}",
    ]
    lines += readout_lines(rho, "final")
    lines.append("ptrace 0 1 " + cplx_list(oracle.partial_trace(rho, [0, 1])))
    q2 = [n // 2 - 1, n - 1]
    lines.append(f"ptrace {q2[0]} {q2[1]} " + cplx_list(oracle.partial_trace(rho, q2)))
    lines += element_lines(rho, n)
    return "\n".join(lines) + "\n"


def make_config3(state_dir, u=0.37):
    c = wl.config3_circuit()
    n = c.n

    def ckpt(g, rho):
        return readout_lines(rho, f"ckpt {g}")

    rho, ck = run_chunked(c, 100, state_dir, "config3", ckpt)
    lines = [
        "# Full-depth oracle readouts of the 14-qubit benchmark circuit: |0..0><0..0|, 1000 seeded",
        "# gates uniform over {H, X, Z, S, T, CNOT, Haar SU(2)}, amplitude damping (gamma = 0.01) then",
        "# phase damping (lambda = 0.02) on every touched qubit (Kraus sums, Eq. rhoE2); gate sweeps",
        "# of Sec. 3.1-3.2 (Eqs. resmat1, resmat2) on rows with U and columns with conj(U).",
        "# ckpt lines: gate count, Re tr, Im tr, purity, P(q = 1) for q = 0..13.  elem lines: row,",
        "# column, Re, Im of the final state before the measurement.  measure: qubit, u, outcome,",
        "# p_outcome (outcome 0 iff u < p_0).  Written by tests/golden/make_deep_goldens.py from the",
        "# complex128 oracle.",
        f"n {n}",
        f"gates {c.n_gates}",
        f"channels {c.n_channels}",
    ]
    lines += ck
    lines.append("ptrace 0 1 " + cplx_list(oracle.partial_trace(rho, [0, 1])))
    q2 = [n // 2 - 1, n - 1]
    lines.append(f"ptrace {q2[0]} {q2[1]} " + cplx_list(oracle.partial_trace(rho, q2)))
    lines += element_lines(rho, n)
    m, pm = oracle.measure(rho, 0, -1, u)
    lines.append(f"measure 0 {fmt(u)} {m} {fmt(pm)}")
    lines.append("post_ptrace 0 1 " + cplx_list(oracle.partial_trace(rho, [0, 1])))
    lines.append(f"post_purity {fmt(oracle.purity(rho))}")
    return "\n".join(lines) + "\n"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("which", choices=["config2", "config3"])
    ap.add_argument("--state-dir", default=None)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    oracle.set_threads(0)
    text = make_config2(a.state_dir) if a.which == "config2" else make_config3(a.state_dir)
    out = a.out or os.path.join(HERE, "config2_n12.txt" if a.which == "config2" else "config3_n14.txt")
    with open(out + ".tmp", "w") as f:
        f.write(text)
    os.replace(out + ".tmp", out)
    log(f"wrote {out}")


if __name__ == "__main__":
    main()
