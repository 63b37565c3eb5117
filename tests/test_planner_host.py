"""CPU tests of the fusion planner and tile-plan packing (host code).

The planner's passes and composed phase superoperators, replayed in order with numpy, must
reproduce the oracle applying the original operations in order (up to complex128 rounding):
this checks the commutation-based reordering, the phase composition and the product-phase
split.  The packed tile plan (what the kernels receive) is replayed with the kernels'
arithmetic -- Pauli butterflies and real transfer matrices (16 x 16 for two-qubit phases, 4 x 4
per qubit for product and one-qubit phases) -- against the oracle to FP32 accuracy: this checks
the transfer-matrix conventions and every coefficient layout without a GPU."""

import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import workloads as wl
from tests._helpers import haar_unitary, random_rho

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1101_1785_gb300", "csrc")
SHIM = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cpp", "planner_shim.cpp")


def _cuda_include():
    for d in ("/usr/local/cuda/include",):
        if os.path.exists(os.path.join(d, "cuda_runtime.h")):
            return d
    pytest.skip("CUDA headers not found")


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("planner") / "libplanner_shim.so")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-I", os.path.join(ROOT, "include"),
                           "-I", CSRC, "-I", _cuda_include(), "-o", out, SHIM, os.path.join(CSRC, "planner.cpp"),
                           os.path.join(CSRC, "tile.cpp")])
    lib = ctypes.CDLL(out)
    lib.planner_phases.restype = ctypes.c_int
    lib.planner_count_only_mismatch.restype = ctypes.c_int
    lib.tile_plan.restype = ctypes.c_int
    return lib


def _superop_kraus(ks):
    return sum(np.kron(K, K.conj()) for K in ks)


def _random_ops(rng, n, count):
    ops = []
    for _ in range(count):
        r = rng.random()
        if r < 0.4:
            ops.append(("u", (int(rng.integers(n)),), haar_unitary(rng, 2)))
        elif r < 0.6:
            a, b = [int(x) for x in rng.permutation(n)[:2]]
            ops.append(("u", (a, b), haar_unitary(rng, 4)))
        elif r < 0.9:
            q = int(rng.integers(n))
            ks = [np.sqrt(w) * haar_unitary(rng, 2) for w in (0.7, 0.3)]
            ops.append(("k", (q,), ks))
        else:
            a, b = [int(x) for x in rng.permutation(n)[:2]]
            ks = [np.sqrt(w) * haar_unitary(rng, 4) for w in (0.5, 0.5)]
            ops.append(("k", (a, b), ks))
    return ops


def _marshal(ops):
    """Op arrays in the shim's layout: kind, k, qubits (two per op), matrices, offsets."""
    kinds = np.array([0 if o[0] == "u" else 1 for o in ops], dtype=np.int32)
    ks = np.array([len(o[1]) for o in ops], dtype=np.int32)
    qs = np.zeros(2 * len(ops), dtype=np.int32)
    mats, offs, off = [], [], 0
    for i, o in enumerate(ops):
        qs[2 * i:2 * i + len(o[1])] = o[1]
        m = o[2] if o[0] == "u" else _superop_kraus(o[2])
        mats.append(np.ascontiguousarray(m, dtype=np.complex128).ravel())
        offs.append(off)
        off += m.size
    return kinds, ks, qs, np.concatenate(mats), np.array(offs, dtype=np.int64)


def _plan(shim, n, kmax, ops, search=0):
    kinds, ks, qs, mats, offs = _marshal(ops)
    maxp = 4 * len(ops) + 8
    pp = np.zeros(maxp, np.int32)
    pnq = np.zeros(maxp, np.int32)
    pq = np.zeros(2 * maxp, np.int32)
    pprod = np.zeros(maxp, np.int32)
    pS = np.zeros(512 * maxp, np.float64)
    passq = np.zeros(maxp, np.int32)
    P = ctypes.c_void_p
    r = shim.planner_phases(n, kmax, search, len(ops), kinds.ctypes.data_as(P), ks.ctypes.data_as(P), qs.ctypes.data_as(P),
                            mats.ctypes.data_as(P), offs.ctypes.data_as(P), maxp, pp.ctypes.data_as(P),
                            pnq.ctypes.data_as(P), pq.ctypes.data_as(P), pprod.ctypes.data_as(P),
                            pS.ctypes.data_as(P), passq.ctypes.data_as(P))
    assert r >= 0
    nph, npass = r // 1000, r % 1000
    phases = []
    for i in range(nph):
        S = pS[512 * i:512 * i + 512].view(np.complex128)
        phases.append((int(pp[i]), int(pnq[i]), (int(pq[2 * i]), int(pq[2 * i + 1])), bool(pprod[i]), S.copy()))
    return phases, passq[:npass]


def _apply_superop(rho, n, S, qubits):
    """rho <- S acting on (row bits, column bits) of `qubits`; index (R, C) with R, C the
    binary numbers of the qubits' row / column bits (first qubit most significant)."""
    k = len(qubits)
    t = rho.reshape([2] * (2 * n))
    S = S.reshape([2] * (4 * k))
    letters = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ"
    src = list(letters[:2 * n])
    out = list(src)
    new = letters[2 * n:2 * n + 2 * k]
    s_out = []
    s_in = []
    for j, q in enumerate(qubits):  # row bits
        s_in.append(src[q])
        s_out.append(new[j])
        out[q] = new[j]
    for j, q in enumerate(qubits):  # column bits
        s_in.append(src[n + q])
        s_out.append(new[k + j])
        out[n + q] = new[k + j]
    expr = "".join(s_out) + "".join(s_in) + "," + "".join(src) + "->" + "".join(out)
    return np.einsum(expr, S, t).reshape(rho.shape)


@pytest.mark.parametrize("search", [0, 1, 2])
@pytest.mark.parametrize("n,kmax,seed", [(3, 2, 1), (4, 3, 2), (5, 4, 3), (6, 5, 4), (6, 2, 5), (9, 4, 6)])
def test_planner_replay_matches_oracle(shim, n, kmax, seed, search):
    rng = np.random.default_rng(seed)
    ops = _random_ops(rng, n, 60)
    rho0 = random_rho(rng, n)
    want = rho0.copy()
    for kind, qs, m in ops:
        if kind == "u":
            oracle.apply_unitary(want, m, qs)
        else:
            oracle.apply_kraus(want, np.stack(m), qs)
    phases, pass_nq = _plan(shim, n, kmax, ops, search)
    assert (pass_nq <= kmax).all() and len(pass_nq) >= 1
    assert np.abs(_replay(phases, n, rho0) - want).max() < 1e-12


def _replay(phases, n, rho0):
    """The planned phases applied in order with numpy."""
    got = rho0.copy()
    for _, nq, (qa, qb), product, S in phases:
        if nq == 1:
            got = _apply_superop(got, n, S[:16], (qa,))
        elif product:
            got = _apply_superop(got, n, S[:16], (qa,))
            got = _apply_superop(got, n, S[16:32], (qb,))
        else:
            got = _apply_superop(got, n, S, (qa, qb))
    return got


def _oracle_run(ops, rho0):
    want = rho0.copy()
    for kind, qs, m in ops:
        if kind == "u":
            oracle.apply_unitary(want, m, qs)
        else:
            oracle.apply_kraus(want, np.stack(m), qs)
    return want


def _structure(phases):
    return [(nq, q if nq == 2 else (q[0],), prod) for _, nq, q, prod, _ in phases]


def test_phases_anchor_on_two_qubit_operations(shim):
    """A two-qubit operation opens a phase that takes the single-qubit operations on its qubits
    placed so far; later single-qubit operations and a second operation on the same pair join
    it; a qubit with no two-qubit operation in the pass gets its own phase, placed first."""
    rng = np.random.default_rng(5)
    ops = [("u", (0,), haar_unitary(rng, 2)), ("u", (2,), haar_unitary(rng, 2)),
           ("u", (0, 1), haar_unitary(rng, 4)), ("u", (0,), haar_unitary(rng, 2)),
           ("k", (1,), [np.sqrt(w) * haar_unitary(rng, 2) for w in (0.6, 0.4)]),
           ("u", (1, 0), haar_unitary(rng, 4)), ("u", (1,), haar_unitary(rng, 2))]
    phases, pass_nq = _plan(shim, 3, 3, ops)
    assert len(pass_nq) == 1
    assert _structure(phases) == [(1, (2,), False), (2, (0, 1), False)]
    rho0 = random_rho(rng, 3)
    assert np.abs(_replay(phases, 3, rho0) - _oracle_run(ops, rho0)).max() < 1e-12


def test_single_qubit_operation_joins_the_last_phase_on_its_qubit(shim):
    """After phases on (0, 1) and (1, 2), an operation on qubit 0 commutes past the (1, 2) phase
    into the (0, 1) one and an operation on qubit 1 joins (1, 2); a two-qubit operation on (0, 2)
    whose qubits' last phases differ opens a new phase."""
    rng = np.random.default_rng(6)
    ops = [("u", (0, 1), haar_unitary(rng, 4)), ("u", (1, 2), haar_unitary(rng, 4)),
           ("u", (0,), haar_unitary(rng, 2)), ("u", (1,), haar_unitary(rng, 2)),
           ("u", (0, 2), haar_unitary(rng, 4)), ("u", (2,), haar_unitary(rng, 2))]
    phases, pass_nq = _plan(shim, 3, 3, ops)
    assert len(pass_nq) == 1
    assert _structure(phases) == [(2, (0, 1), False), (2, (1, 2), False), (2, (0, 2), False)]
    rho0 = random_rho(rng, 3)
    assert np.abs(_replay(phases, 3, rho0) - _oracle_run(ops, rho0)).max() < 1e-12


def test_qubits_without_two_qubit_operations_pair_into_product_phases(shim):
    """Five qubits with single-qubit operations only: product phases on (0, 1) and (2, 3) and a
    one-qubit phase on 4, whatever the order of the operations."""
    rng = np.random.default_rng(7)
    ops = [("u", (q,), haar_unitary(rng, 2)) for q in (4, 2, 0, 3, 1, 0, 4, 2)]
    ops.append(("k", (3,), [np.sqrt(w) * haar_unitary(rng, 2) for w in (0.5, 0.5)]))
    phases, pass_nq = _plan(shim, 5, 5, ops)
    assert len(pass_nq) == 1
    assert _structure(phases) == [(2, (0, 1), True), (2, (2, 3), True), (1, (4,), False)]
    rho0 = random_rho(rng, 5)
    assert np.abs(_replay(phases, 5, rho0) - _oracle_run(ops, rho0)).max() < 1e-12


def test_planner_packs_disjoint_work(shim):
    """Ops on disjoint qubits commute: a run alternating between two qubit pairs fits one pass."""
    rng = np.random.default_rng(9)
    ops = []
    for i in range(20):
        pair = (0, 1) if i % 2 == 0 else (2, 3)
        ops.append(("u", pair, haar_unitary(rng, 4)))
    phases, pass_nq = _plan(shim, 4, 4, ops)
    assert len(pass_nq) == 1 and len(phases) == 2


@pytest.mark.parametrize("search", [0, 1, 2])
@pytest.mark.parametrize("n,kmax", [(5, 3), (8, 4), (10, 5)])
def test_count_only_plan_has_the_same_structure(shim, n, kmax, search):
    """The width search plans without composing superoperators; its passes and phases must be
    the ones the full plan produces."""
    rng = np.random.default_rng(n * 31 + kmax)
    ops = _random_ops(rng, n, 120)
    kinds, ks, qs, mats, offs = _marshal(ops)
    P = ctypes.c_void_p
    bad = shim.planner_count_only_mismatch(n, kmax, search, len(ops), kinds.ctypes.data_as(P), ks.ctypes.data_as(P),
                                           qs.ctypes.data_as(P), mats.ctypes.data_as(P), offs.ctypes.data_as(P))
    assert bad == 0


def _tile_plan(shim, n, kmax, herm, tbmax, ops, search=0):
    kinds, ks, qs, mats, offs = _marshal(ops)
    maxp, maxc = 4 * len(ops) + 8, 256 * (4 * len(ops) + 8)
    kind = np.zeros(maxp, np.int32)
    pos = np.zeros(4 * maxp, np.int32)
    coef = np.zeros(maxp, np.int32)
    ppass = np.zeros(maxp, np.int32)
    tb = np.zeros(maxp, np.int32)
    tbits = np.zeros(16 * maxp, np.int32)
    coefs = np.zeros(2 * maxc, np.float32)
    ncoefs = ctypes.c_int(0)
    P = ctypes.c_void_p
    nph = shim.tile_plan(n, kmax, search, int(herm), tbmax, len(ops), kinds.ctypes.data_as(P), ks.ctypes.data_as(P),
                         qs.ctypes.data_as(P), mats.ctypes.data_as(P), offs.ctypes.data_as(P), maxp,
                         kind.ctypes.data_as(P), pos.ctypes.data_as(P), coef.ctypes.data_as(P),
                         ppass.ctypes.data_as(P), maxp, tb.ctypes.data_as(P), tbits.ctypes.data_as(P), maxc,
                         coefs.ctypes.data_as(P), ctypes.byref(ncoefs))
    assert nph >= 0
    cf = coefs[:2 * ncoefs.value].astype(np.float64).view(np.complex128)
    return [(int(kind[i]), [int(x) for x in pos[4 * i:4 * i + 4]], int(coef[i]), int(tb[ppass[i]]),
             [int(x) for x in tbits[16 * ppass[i]:16 * ppass[i] + 16]]) for i in range(nph)], cf


def _pauli_odd(e):
    return (((e >> 3) & 1) and not ((e >> 1) & 1)) != (((e >> 2) & 1) and not (e & 1))


def _butterflies(x):
    """The kernels' per-qubit butterflies on axis 0 of x (16 members, bits r_a c_a r_b c_b as
    8, 2, 4, 1): (b00, b01, b10, b11) -> (b00 + b11, b01 + b10, b01 - b10, b00 - b11)."""
    x = x.copy()
    for s1, s2, offs in ((8, 2, (0, 1, 4, 5)), (4, 1, (0, 2, 8, 10))):
        for o in offs:
            a, b, c, d = x[o].copy(), x[o + s2].copy(), x[o + s1].copy(), x[o + s1 + s2].copy()
            x[o], x[o + s2], x[o + s1], x[o + s1 + s2] = a + d, b + c, b - c, a - d
    return x


def _pauli_quartet(q, R):
    """One qubit's quartet (b00, b01, b10, b11) as the kernels treat it: butterflies to
    (I, X, D, Z), v = (I, X, i D, Z), c = R v, back with (c_I, c_X, -i c_D, c_Z) and the same
    butterflies."""
    def bfly(t):
        return np.stack([t[0] + t[3], t[1] + t[2], t[1] - t[2], t[0] - t[3]])
    u = bfly(q)
    u[2] = 1j * u[2]
    c = R @ u
    c[2] = -1j * c[2]
    return bfly(c)


def _replay_tile_plan(rho, n, phases, cf):
    """Apply the packed phases to rho (2^n x 2^n) the way the kernels do, in float64."""
    flat = rho.reshape(-1).copy()
    vbits = 2 * n
    for kind, pos, coff, tb, tbits in phases:
        # virtual bit of each phase position; members are flat indices differing in those bits
        vb = [tbits[p] for p in pos[:4 if kind != 1 else 2]]
        others = [v for v in range(vbits) if v not in vb]
        base = np.zeros(1, dtype=np.int64)
        for v in others:
            base = np.concatenate([base, base | (1 << v)])
        if kind == 1:
            R = cf[coff:coff + 16].real.reshape(4, 4)
            mem = [base | (r << vb[0]) | (c << vb[1]) for r in (0, 1) for c in (0, 1)]
            x = np.stack([flat[m] for m in mem])
            y = _pauli_quartet(x, R)
            for i, m in enumerate(mem):
                flat[m] = y[i]
            continue
        mem = []
        for e in range(16):
            idx = base.copy()
            for j in range(4):
                if (e >> (3 - j)) & 1:
                    idx = idx | (1 << vb[j])
            mem.append(idx)
        x = np.stack([flat[m] for m in mem])
        if kind == 3:  # product: R_a on (r_a, c_a) = bits (8, 2), R_b on (r_b, c_b) = (4, 1)
            for R, (s1, s2, offs) in ((cf[coff:coff + 16].real.reshape(4, 4), (8, 2, (0, 1, 4, 5))),
                                      (cf[coff + 16:coff + 32].real.reshape(4, 4), (4, 1, (0, 2, 8, 10)))):
                for o in offs:
                    q = np.stack([x[o], x[o + s2], x[o + s1], x[o + s1 + s2]])
                    x[o], x[o + s2], x[o + s1], x[o + s1 + s2] = _pauli_quartet(q, R)
        else:  # two-qubit phase in the Pauli basis
            pairs = cf[coff:coff + 128]  # (R[2p][f], R[2p+1][f]) at f * 8 + p
            R = np.zeros((16, 16))
            for f in range(16):
                for p in range(8):
                    R[2 * p, f] = pairs[f * 8 + p].real
                    R[2 * p + 1, f] = pairs[f * 8 + p].imag
            u = _butterflies(x)
            v = np.stack([1j * u[f] if _pauli_odd(f) else u[f] for f in range(16)])
            c = R @ v
            w = np.stack([-1j * c[e] if _pauli_odd(e) else c[e] for e in range(16)])
            x = _butterflies(w)
        for e in range(16):
            flat[mem[e]] = x[e]
    return flat.reshape(rho.shape)


@pytest.mark.parametrize("search", [0, 1, 2])
@pytest.mark.parametrize("n,kmax,herm,seed", [(6, 2, True, 11), (6, 4, True, 12), (5, 3, False, 13), (7, 5, True, 14)])
def test_tile_plan_coefficients_replay_matches_oracle(shim, n, kmax, herm, seed, search):
    """The packed coefficients of every phase kind, applied with the kernels' arithmetic."""
    rng = np.random.default_rng(seed)
    ops = _random_ops(rng, n, 50)
    rho0 = random_rho(rng, n)
    want = rho0.copy()
    for kind, qs, m in ops:
        if kind == "u":
            oracle.apply_unitary(want, m, qs)
        else:
            oracle.apply_kraus(want, np.stack(m), qs)
    phases, cf = _tile_plan(shim, n, kmax, herm, 12 if herm else 13, ops, search)
    assert {p[0] for p in phases} >= {2}
    got = _replay_tile_plan(rho0, n, phases, cf)
    assert np.abs(got - want).max() < 2e-5  # FP32 coefficients



def test_best_search_packs_no_more_passes_than_order(shim):
    """The best-absorption pass search never needs more passes than the in-order greedy one on
    random circuits (and usually far fewer)."""
    rng = np.random.default_rng(77)
    n = 10
    ops = _random_ops(rng, n, 300)
    _, order = _plan(shim, n, 4, ops, 0)
    _, best = _plan(shim, n, 4, ops, 1)
    assert len(best) <= len(order)
    assert len(best) < 0.9 * len(order)


def test_beam_search_packs_no_more_passes_than_best(shim):
    """The beam search over pass sequences never needs more passes than the greedy
    best-absorption choice (its first partial sequence is the greedy one), on random circuits and
    on the 100-gate segments of the 14-qubit benchmark circuit at width 5."""
    rng = np.random.default_rng(78)
    for n, kmax in ((10, 4), (9, 5)):
        ops = _random_ops(rng, n, 300)
        _, best = _plan(shim, n, kmax, ops, 1)
        _, beam = _plan(shim, n, kmax, ops, 2)
        assert len(beam) <= len(best)
    c = wl.config3_circuit()
    bounds = [len(c.gate_prefix(g).ops) for g in range(0, 1001, 100)]
    tot_best = tot_beam = 0
    for i in range(10):
        seg = [(("u" if o.kind == "gate" else "k"), o.qubits, o.mats[0] if o.kind == "gate" else list(o.mats))
               for o in c.ops[bounds[i]:bounds[i + 1]]]
        _, best = _plan(shim, 14, 5, seg, 1)
        _, beam = _plan(shim, 14, 5, seg, 2)
        assert len(beam) <= len(best)
        tot_best += len(best)
        tot_beam += len(beam)
    print(f"benchmark circuit at width 5: {tot_best} passes (greedy best), {tot_beam} (beam)")


def test_trace_row_of_two_qubit_transfer_matrices(shim):
    """Trace-preserving operations (unitaries, channels cut from isometries) give two-qubit
    transfer matrices whose row 0 -- the trace component in the Pauli basis -- is (1/4, 0, ..., 0)
    up to rounding residue, so the tensor-core phases, which round R to TF32 pieces, leave the
    trace exact (0.25 and 0 are TF32 numbers)."""
    rng = np.random.default_rng(71)
    n = 5
    ops = []
    for _ in range(80):
        r = rng.random()
        if r < 0.3:
            ops.append(("u", (int(rng.integers(n)),), haar_unitary(rng, 2)))
        elif r < 0.6:
            a, b = [int(x) for x in rng.permutation(n)[:2]]
            ops.append(("u", (a, b), haar_unitary(rng, 4)))
        elif r < 0.85:
            iso = haar_unitary(rng, 6)[:, :2]
            ops.append(("k", (int(rng.integers(n)),), [iso[2 * j:2 * j + 2] for j in range(3)]))
        else:
            a, b = [int(x) for x in rng.permutation(n)[:2]]
            iso = haar_unitary(rng, 8)[:, :4]
            ops.append(("k", (a, b), [iso[4 * j:4 * j + 4] for j in range(2)]))
    phases, cf = _tile_plan(shim, n, 4, True, 12, ops)
    two = [off for kind, _, off, _, _ in phases if kind == 2]
    assert len(two) >= 10
    for off in two:
        row0 = np.array([cf[off + 8 * f].real for f in range(16)])
        assert abs(row0[0] - 0.25) < 1e-12
        assert np.abs(row0[1:]).max() < 1e-12


# ----------------------------------------------------------------------------- plain-path transfer form
def _pauli_apply_plain(R, x, k):
    """The plain kernels' arithmetic on one group (k_super1 / k_super2): butterflies per qubit,
    i on the odd members, c = R v, -i back, the same butterflies.  x: 4^k members, index
    (row bits, column bits) as 2 r + c (k = 1) or 8 r1 + 4 r2 + 2 c1 + c2 (k = 2)."""
    x = np.array(x, dtype=np.complex128)

    def fly(v):
        v = v.copy()
        quads = [(2, 1, 0)] if k == 1 else [(8, 2, o) for o in (0, 1, 4, 5)] + [(4, 1, o) for o in (0, 2, 8, 10)]
        for s1, s2, o in quads:
            a, b, c, d = v[o], v[o + s2], v[o + s1], v[o + s1 + s2]
            v[o], v[o + s2], v[o + s1], v[o + s1 + s2] = a + d, b + c, b - c, a - d
        return v

    def odd(e):
        if k == 1:
            return e == 2
        return bool(((e >> 3) & 1) and not ((e >> 1) & 1)) != bool(((e >> 2) & 1) and not (e & 1))

    v = fly(x)
    v = np.array([1j * v[f] if odd(f) else v[f] for f in range(4 ** k)])
    c = R @ v
    c = np.array([-1j * c[e] if odd(e) else c[e] for e in range(4 ** k)])
    return fly(c)


@pytest.mark.parametrize("k", [1, 2])
def test_plain_transfer_form_reproduces_the_superoperator(shim, k):
    """For gates (S = U (x) conj U) and Kraus sets, the transfer matrix the library computes for
    the plain kernels, applied with their butterfly arithmetic, gives S x; for trace-preserving
    maps its first row is exactly (2^-k, 0, ...) in FP32, so the kernels keep the trace."""
    rng = np.random.default_rng(1700 + k)
    d = 1 << k
    P = ctypes.c_void_p
    for trial in range(6):
        if trial % 2 == 0:
            u = haar_unitary(rng, d)
            S = np.kron(u, u.conj())
        else:
            ks = [np.sqrt(w) * haar_unitary(rng, d) for w in rng.dirichlet(np.ones(3))]
            S = _superop_kraus(ks)
        # S's index (row, column) of the member: reorder kron's (r1 c1 | ...) -- np.kron(K, conj K)
        # indexes (r, c) as r * d + c with r, c the whole row / column labels, i.e. the members'
        # row bits above their column bits, as the kernels use
        Sd = np.ascontiguousarray(S, dtype=np.complex128)
        R = np.zeros((4 ** k) ** 2)
        shim.pauli_transfer_k(k, Sd.ctypes.data_as(P), R.ctypes.data_as(P))
        R = R.reshape(4 ** k, 4 ** k)
        x = rng.standard_normal(4 ** k) + 1j * rng.standard_normal(4 ** k)
        np.testing.assert_allclose(_pauli_apply_plain(R, x, k), Sd @ x, atol=1e-12)
        R32 = R.astype(np.float32)
        assert R32[0, 0] == np.float32(2.0 ** -k) and not R32[0, 1:].any()
