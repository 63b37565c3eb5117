"""GPU parity of the fused path (planner + fused-pass kernel) against the CPU oracle.

Tolerance as everywhere: max |delta rho| <= 1e-5, |tr rho - 1| <= 1e-6 (FP32 state vs the
FP64 oracle).  The 14-qubit cases run in the launch configuration the benchmark times
(fusion width 5, 2^12-element Hermitian tiles); the 17-qubit cases run at the largest
register the library takes (QCW_MAX_QUBITS, rho = 128 GiB).
"""

import numpy as np
import pytest

import oracle
import workloads as wl
from tests._helpers import gather_elements, haar_unitary, random_rho

pytestmark = pytest.mark.gpu

ATOL = 1e-5
TRACE_TOL = 1e-6


@pytest.fixture(scope="module")
def q():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1101_1785_gb300 as q

    return q


def _run(q, c, mode, k=0, rho0=None):
    d = q.Density(c.n)
    d.set_mode(mode, k)
    if rho0 is not None:
        d.set_state(rho0)
    elif c.init == "matrix":
        d.set_state(c.rho0)
    for op in c.ops:
        d.apply_op(op)
    return d


@pytest.mark.parametrize("n,k", [(2, 2), (3, 2), (3, 3), (4, 4), (5, 3), (6, 5), (7, 4), (8, 5)])
def test_fused_random_noisy_circuits(q, n, k):
    for noise, seed in (("adpd", 1), ("dep", 2), ("none", 3)):
        c = wl.random_circuit(n, 50, 1000 * n + seed, "mixed", noise)
        rho0 = random_rho(np.random.default_rng(seed + n), n)
        want = oracle.run_circuit(c, rho0.copy())
        d = _run(q, c, q.QCW_MODE_FUSED, k, rho0)
        got = d.get_state()
        err = np.abs(got - want).max()
        assert err <= ATOL, (noise, err)
        assert abs(d.trace() - oracle.trace(want)) <= TRACE_TOL
        d.close()


def test_fused_two_qubit_channels_and_dense_gates(q):
    rng = np.random.default_rng(77)
    n = 6
    rho = random_rho(rng, n)
    want = rho.copy()
    d = q.Density(n)
    d.set_state(rho)
    d.set_mode(q.QCW_MODE_FUSED, 4)
    for step in range(12):
        a, b = [int(x) for x in rng.permutation(n)[:2]]
        ks = np.stack([np.sqrt(w) * haar_unitary(rng, 4) for w in (0.6, 0.4)])
        d.apply_kraus(ks, [a, b])
        oracle.apply_kraus(want, ks, [a, b])
        u = haar_unitary(rng, 2)
        d.apply_gate1(u, (a + step) % n)
        oracle.apply_unitary(want, u, [(a + step) % n])
        if step % 4 == 0:  # dense 3-qubit gate: a barrier for the planner
            qs = [int(x) for x in rng.permutation(n)[:3]]
            u3 = haar_unitary(rng, 8)
            d.apply_gate(u3, qs)
            oracle.apply_unitary(want, u3, qs)
        if step % 3 == 0:  # controlled gates: 1 + 1 is lowered, 1 + 2 runs on its own
            u = haar_unitary(rng, 2)
            d.apply_gate1(u, b, [a])
            oracle.apply_unitary(want, u, [b], [a])
            c2 = [x for x in range(n) if x not in (a, b)][:2]
            d.apply_gate1(u, b, c2)
            oracle.apply_unitary(want, u, [b], c2)
    assert np.abs(d.get_state() - want).max() <= ATOL
    d.close()


def test_fused_matches_plain_and_is_deterministic(q):
    c = wl.random_circuit(9, 200, 4242, "mixed", "adpd")
    a = _run(q, c, q.QCW_MODE_PLAIN).get_state()
    f1 = _run(q, c, q.QCW_MODE_FUSED, 5).get_state()
    f2 = _run(q, c, q.QCW_MODE_FUSED, 5).get_state()
    assert np.abs(a - f1).max() <= 1e-6
    np.testing.assert_array_equal(f1, f2)


def test_config1_fused_with_measurement(q):
    c = wl.config1_circuit()
    want = oracle.run_circuit(c)
    for forced in (0, 1):
        d = _run(q, c, q.QCW_MODE_FUSED, 4)
        assert np.abs(d.get_state() - want).max() <= ATOL
        assert abs(d.trace() - 1) <= TRACE_TOL
        ref = want.copy()
        m_ref, p_ref = oracle.measure(ref, 0, forced)
        m, p = d.measure(0, forced)
        assert m == m_ref and abs(p - p_ref) <= 1e-6
        assert np.abs(d.get_state() - ref).max() <= ATOL
        d.close()


def test_plan_cache_reuse_and_miss(q):
    c1 = wl.random_circuit(7, 80, 11, "mixed", "adpd")
    c2 = wl.random_circuit(7, 80, 12, "mixed", "adpd")
    d = q.Density(7)
    d.set_mode(q.QCW_MODE_FUSED, 5)
    for c in (c1, c2, c1, c2):
        d.reset()
        for op in c.ops:
            d.apply_op(op)
        np.testing.assert_allclose(d.get_state(), oracle.run_circuit(c), atol=ATOL, rtol=0)
    d.close()


def test_config2_prefix_n12_fused_and_plain(q):
    c = wl.config2_circuit()
    pre = c.gate_prefix(30)
    want = oracle.run_circuit(pre)
    for mode in (q.QCW_MODE_PLAIN, q.QCW_MODE_FUSED):
        d = _run(q, pre, mode, 5)
        err = np.abs(d.get_state() - want).max()
        assert err <= ATOL, err
        assert abs(d.trace() - 1) <= TRACE_TOL
        d.close()


def test_full_size_n14_embedded_subsystem(q):
    """n = 14 in the benchmark's launch configuration, on a circuit confined to five qubits
    spread over the register: rho = rho_S (x) |0><0| on the rest, with rho_S from the oracle."""
    n, S = 14, [0, 3, 7, 12, 13]
    small = wl.random_circuit(5, 120, 314, "mixed", "adpd")
    want_s = oracle.run_circuit(small)
    d = q.Density(n)
    d.set_mode(q.QCW_MODE_FUSED, 5)
    for op in small.ops:
        mapped = [S[x] for x in op.qubits]
        if op.kind == "gate":
            if op.k == 1:
                d.apply_gate1(op.mats[0], mapped[0])
            else:
                d.apply_gate2(op.mats[0], mapped[0], mapped[1])
        else:
            d.apply_kraus(op.mats, mapped)
    got = d.get_state()
    assert abs(d.trace() - 1) <= TRACE_TOL
    d.close()
    t = got.reshape([2] * (2 * n))
    idx = tuple(slice(None) if (ax % n) in S else 0 for ax in range(2 * n))
    block = t[idx].reshape(32, 32)
    assert np.abs(block - want_s).max() <= ATOL
    t[idx] = 0
    assert np.abs(got).max() == 0.0


def _embedded_index(n, S):
    """Row (or column) indices of rho whose bits outside the qubits S are 0, in the order of the
    subsystem's own index (qubit 0 the most significant bit, as everywhere)."""
    out = np.zeros(1 << len(S), dtype=np.int64)
    for s in range(1 << len(S)):
        for j, qb in enumerate(S):
            if (s >> (len(S) - 1 - j)) & 1:
                out[s] |= 1 << (n - 1 - qb)
    return out


@pytest.mark.parametrize("mode", ["fused", "plain"])
def test_max_size_n17_embedded_subsystem(q, mode):
    """The largest register, 17 qubits (rho = 2^34 complex64 = 128 GiB: element offsets beyond
    32 bits in every kernel on the path), on a noisy circuit confined to five qubits spread over
    the register: the 32 x 32 block rho_S against the oracle, seeded elements outside it exactly
    0, and the trace, purity and per-qubit probabilities."""
    import torch

    from paper_1101_1785_gb300._binding import QCW_MAX_QUBITS

    n = QCW_MAX_QUBITS
    free, _ = torch.cuda.mem_get_info()
    if free < (8 << (2 * n)) + (16 << 30):
        pytest.skip(f"needs {(8 << (2 * n)) >> 30} GiB of free device memory and some headroom")
    S = [0, 5, 9, 14, 16]
    small = wl.random_circuit(5, 120 if mode == "fused" else 30, 1717, "mixed", "adpd")
    want_s = oracle.run_circuit(small)
    d = q.Density(n)
    if mode == "fused":
        d.set_mode(q.QCW_MODE_FUSED, 5)
    for op in small.ops:
        mapped = [S[x] for x in op.qubits]
        if op.kind == "gate":
            if op.k == 1:
                d.apply_gate1(op.mats[0], mapped[0])
            else:
                d.apply_gate2(op.mats[0], mapped[0], mapped[1])
        else:
            d.apply_kraus(op.mats, mapped)
    idx = _embedded_index(n, S)
    rr, cc = np.meshgrid(idx, idx, indexing="ij")
    block = gather_elements(d, rr.ravel(), cc.ravel()).reshape(32, 32)
    assert np.abs(block - want_s).max() <= ATOL
    rng = np.random.default_rng(17)
    rows = rng.integers(0, 1 << n, 8192)
    cols = rng.integers(0, 1 << n, 8192)
    outside = ~(np.isin(rows, idx) & np.isin(cols, idx))
    assert np.all(gather_elements(d, rows[outside], cols[outside]) == 0)
    assert abs(d.trace() - 1) <= TRACE_TOL
    assert abs(d.purity() - oracle.purity(want_s)) <= 2 * TRACE_TOL
    p = d.probabilities()
    np.testing.assert_allclose(p[S], oracle.probabilities(want_s), atol=1e-6)
    assert np.all(np.delete(p, S) == 0)
    d.close()


def test_full_size_n14_config3_prefix(q):
    """First three gates of the 14-qubit benchmark circuit, fused k = 5, against the oracle."""
    c = wl.config3_circuit().gate_prefix(3)
    want = oracle.run_circuit(c)
    d = _run(q, c, q.QCW_MODE_FUSED, 5)
    got = d.get_state()
    assert np.abs(got - want).max() <= ATOL
    assert abs(d.trace() - 1) <= TRACE_TOL
    d.close()


def test_contexts_of_different_sizes_interleave(q):
    """Kernel attributes are per process: a small context must not break a big one."""
    big = wl.random_circuit(10, 30, 21, "mixed", "adpd")
    small = wl.random_circuit(3, 30, 22, "mixed", "adpd")
    db, ds = q.Density(10), q.Density(3)
    db.set_mode(q.QCW_MODE_FUSED, 5)
    ds.set_mode(q.QCW_MODE_FUSED, 0)
    for c, d in ((big, db), (small, ds), (big, db), (small, ds)):
        d.reset()
        for op in c.ops:
            d.apply_op(op)
        assert np.abs(d.get_state() - oracle.run_circuit(c)).max() <= ATOL
    db.close()
    ds.close()


def test_persistent_pipeline_matches_plain_n12(q):
    """n = 12 has 2^11 tiles per pass, enough for the persistent double-buffered kernel."""
    c = wl.random_circuit(12, 150, 1212, "mixed", "adpd")
    a = _run(q, c, q.QCW_MODE_PLAIN).get_state()
    f = _run(q, c, q.QCW_MODE_FUSED, 5).get_state()
    assert np.abs(a - f).max() <= 1e-6


@pytest.mark.parametrize("n", [6, 8, 11])
def test_hermitian_kernel_matches_general_kernels(q, n):
    """The Hermitian pass kernels (tiles on or above the diagonal, mirrors written as conjugate
    transposes; one CTA per tile pair, the warp-specialised persistent one and its tensor-core
    variant) against the general per-tile kernel and, at n = 6 and 8, the oracle."""
    c = wl.random_circuit(n, 80, 808 + n, "mixed", "adpd")
    got = {}
    for which in (1, 2, 3, 4):
        d = q.Density(n)
        d.set_mode(q.QCW_MODE_FUSED, 5)
        d.set_fused_kernel(which)
        for op in c.ops:
            d.apply_op(op)
        got[which] = d.get_state()
        d.close()
    assert np.abs(got[2] - got[1]).max() <= 1e-6
    assert np.abs(got[2] - got[2].conj().T).max() <= 1e-7
    # same tile layout and phase arithmetic: the two Hermitian kernels agree bit for bit
    np.testing.assert_array_equal(got[3], got[2])
    # 3xTF32 tensor-core phases: FP32-level agreement, not bitwise
    assert np.abs(got[4] - got[3]).max() <= 1e-6
    if n <= 8:
        want = oracle.run_circuit(c)
        assert np.abs(got[3] - want).max() <= ATOL
        assert np.abs(got[4] - want).max() <= ATOL


@pytest.mark.parametrize("k", [4, 5])
def test_hermitian_kernel_at_n12(q, k):
    """The Hermitian pass kernel at a size with thousands of tile pairs per pass, against the
    general per-tile kernel."""
    c = wl.random_circuit(12, 60, 1200 + k, "mixed", "adpd")
    got = {}
    for w in (1, 2, 3, 4):
        d = q.Density(12)
        d.set_mode(q.QCW_MODE_FUSED, k)
        d.set_fused_kernel(w)
        for op in c.ops:
            d.apply_op(op)
        got[w] = d.get_state()
        d.close()
    assert np.abs(got[2] - got[1]).max() <= 1e-6
    np.testing.assert_array_equal(got[3], got[2])
    assert np.abs(got[4] - got[3]).max() <= 1e-6


@pytest.mark.parametrize("kernel", [3, 4])
def test_warp_specialised_wait_runs_out_and_context_recovers(q, kernel):
    """The first CTA skips the load of its first tile: its consumers' bounded wait runs out,
    the producer's wait for them runs out next, the kernel ends and the following readout
    reports QCW_ETIMEOUT (sticky until reset).  After a reset the context works again."""
    n = 9
    c = wl.random_circuit(n, 40, 4040, "mixed", "adpd")
    d = q.Density(n)
    d.set_mode(q.QCW_MODE_FUSED, 4)
    d.set_fused_kernel(kernel)
    d.set_fused_wait_limit(2000, 0)
    for op in c.ops:
        d.apply_op(op)
    for _ in range(2):
        with pytest.raises(q.QcwError) as e:
            d.trace()
        assert e.value.status == q.QCW_ETIMEOUT
    d.set_fused_wait_limit(0, -1)
    d.reset()
    for op in c.ops:
        d.apply_op(op)
    d.sync()
    assert np.abs(d.get_state() - oracle.run_circuit(c)).max() <= ATOL
    d.close()


@pytest.mark.parametrize("kernel", [3, 4])
@pytest.mark.parametrize("n", [6, 9, 11])
def test_half_storage_readouts(q, n, kernel):
    """The warp-specialised pass leaves only the lower triangle current.  Readouts taken in that
    state (trace and probabilities from the diagonal, purity from the lower triangle, the
    measurement's projection of the lower triangle, partial traces that read each upper element
    as the conjugate of its mirror) and the completed state all match the oracle; a later pass
    on another kernel sees the full matrix."""
    c = wl.random_circuit(n, 60, 9100 + n, "mixed", "adpd")
    want = oracle.run_circuit(c)
    d = q.Density(n)
    d.set_mode(q.QCW_MODE_FUSED, 4)
    d.set_fused_kernel(kernel)
    for op in c.ops:
        d.apply_op(op)
    assert abs(d.trace() - oracle.trace(want)) <= TRACE_TOL
    assert abs(d.purity() - oracle.purity(want)) <= 1e-6
    np.testing.assert_allclose(d.probabilities(), oracle.probabilities(want), atol=1e-6, rtol=0)
    m_ref, p_ref = oracle.measure(want, 1, 0)
    m, p = d.measure(1, 0)
    assert m == m_ref and abs(p - p_ref) <= 1e-6
    assert abs(d.purity() - oracle.purity(want)) <= 1e-5
    for keep in ([0, n - 1], [1, n // 2, n - 2]):
        np.testing.assert_allclose(d.partial_trace(keep), oracle.partial_trace(want, keep), atol=1e-6, rtol=0)
    # more work on the warp-specialised kernel, then on the per-tile Hermitian kernel
    tail = wl.random_circuit(n, 20, 9200 + n, "mixed", "adpd")
    for op in tail.ops:
        d.apply_op(op)
        oracle.apply_op(want, op)
    d.set_fused_kernel(2)
    for op in tail.ops:
        d.apply_op(op)
        oracle.apply_op(want, op)
    got = d.get_state()
    assert np.abs(got - want).max() <= ATOL
    assert np.abs(got - got.conj().T).max() == 0.0
    d.close()


@pytest.mark.parametrize("kernel", [3, 4])
def test_pass_with_more_phases_than_the_parameter_block_holds(q, kernel):
    """Alternating two-qubit channels on five qubits at width 5 make one pass with dozens of
    phases: the warp-specialised kernel then stages each phase's coefficients itself."""
    n = 8
    rng = np.random.default_rng(4242)
    rho = random_rho(rng, n)
    want = rho.copy()
    d = q.Density(n)
    d.set_state(rho)
    d.set_mode(q.QCW_MODE_FUSED, 5)
    d.set_fused_kernel(kernel)
    pairs = [(0, 1), (1, 2), (2, 3), (3, 4), (0, 4), (1, 3)]
    for step in range(40):
        a, b = pairs[step % len(pairs)]
        ks = np.stack([np.sqrt(w) * haar_unitary(rng, 4) for w in (0.7, 0.3)])
        d.apply_kraus(ks, [a, b])
        oracle.apply_kraus(want, ks, [a, b])
    assert abs(d.purity() - oracle.purity(want)) <= 1e-6
    assert np.abs(d.get_state() - want).max() <= ATOL
    d.close()


@pytest.mark.parametrize("kernel", [3, 4])
def test_purity_from_the_pass_epilogue(q, kernel):
    """The last fused pass of a flush also sums w |rho_rc|^2 over the elements it writes (w = 2
    below the diagonal, 1 on it).  That purity matches the oracle and the standalone reduction
    (taken after direct device access invalidates the pass's sums), is bitwise reproducible,
    and is not reused once the state changes (gate, measurement)."""
    n = 10
    c = wl.random_circuit(n, 60, 6100 + kernel, "mixed", "adpd")
    want = oracle.run_circuit(c)
    vals = []
    for _ in range(2):
        d = q.Density(n)
        d.set_mode(q.QCW_MODE_FUSED, 5)
        d.set_fused_kernel(kernel)
        for op in c.ops:
            d.apply_op(op)
        vals.append(d.purity())
        d.device_state()  # the caller may write rho: the pass's sums no longer count
        standalone = d.purity()
        assert abs(standalone - vals[-1]) <= 1e-6
        d.close()
    assert vals[0] == vals[1]
    assert abs(vals[0] - oracle.purity(want)) <= 1e-6
    # a state change after the pass: the next purity comes from the new state
    d = q.Density(n)
    d.set_mode(q.QCW_MODE_FUSED, 5)
    d.set_fused_kernel(kernel)
    for op in c.ops:
        d.apply_op(op)
    d.trace()  # flushes; the pass's sums describe rho
    m_ref, _ = oracle.measure(want, 2, 1)
    m, _ = d.measure(2, 1)
    assert m == m_ref
    assert abs(d.purity() - oracle.purity(want)) <= 1e-6
    d.close()


@pytest.mark.parametrize("mode,kernel", [("fused", 3), ("fused", 4), ("plain", 0)])
def test_checkpoints_match_synchronous_readouts(q, mode, kernel):
    """Asynchronous checkpoints after each third of a circuit hold exactly the values the
    synchronous readouts give on an identical context at the same points (same kernels, same
    summation order), and the last one matches the oracle."""
    n = 9
    c = wl.random_circuit(n, 90, 7300 + kernel, "mixed", "adpd")
    ctxs = []
    for _ in range(2):
        d = q.Density(n)
        if mode == "fused":
            d.set_mode(q.QCW_MODE_FUSED, 5)
            d.set_fused_kernel(kernel)
        ctxs.append(d)
    d, ref = ctxs
    thirds = np.array_split(np.arange(len(c.ops)), 3)
    tickets, want = [], []
    for part in thirds:
        for i in part:
            d.apply_op(c.ops[i])
            ref.apply_op(c.ops[i])
        tickets.append(d.checkpoint())
        want.append((ref.trace(), ref.purity(), ref.probabilities()))
    for t, (tr, pu, pr) in zip(tickets, want):
        gtr, gpu, gpr = d.checkpoint_read(t)
        assert gtr == tr and gpu == pu
        np.testing.assert_array_equal(gpr, pr)
    rho = oracle.run_circuit(c)
    gtr, gpu, gpr = d.checkpoint_read(tickets[-1])
    assert abs(gtr - oracle.trace(rho)) <= TRACE_TOL
    assert abs(gpu - oracle.purity(rho)) <= 1e-6
    np.testing.assert_allclose(gpr, oracle.probabilities(rho), atol=1e-6, rtol=0)
    d.close()
    ref.close()


def test_checkpoint_tickets(q):
    """Unknown and future tickets are rejected; the ring keeps the last QCW_CHECKPOINT_SLOTS."""
    d = q.Density(3)
    with pytest.raises(q.QcwError) as e:
        d.checkpoint_read(0)
    assert e.value.status == q.QCW_EINVAL
    tickets = [d.checkpoint() for _ in range(65)]
    assert tickets == list(range(65))
    with pytest.raises(q.QcwError) as e:
        d.checkpoint_read(0)
    assert e.value.status == q.QCW_EINVAL
    with pytest.raises(q.QcwError) as e:
        d.checkpoint_read(65)
    assert e.value.status == q.QCW_EINVAL
    tr, pu, pr = d.checkpoint_read(64)
    assert tr == 1.0 and pu == 1.0 and (pr == 0.0).all()
    d.close()


def test_checkpoint_reports_a_wait_that_ran_out(q):
    """A fused pass whose bounded wait ran out before the checkpoint: the read returns
    QCW_ETIMEOUT (the error word travels with the checkpoint's values)."""
    n = 9
    c = wl.random_circuit(n, 40, 4041, "mixed", "adpd")
    d = q.Density(n)
    d.set_mode(q.QCW_MODE_FUSED, 4)
    d.set_fused_kernel(3)
    d.set_fused_wait_limit(2000, 0)
    for op in c.ops:
        d.apply_op(op)
    t = d.checkpoint()
    with pytest.raises(q.QcwError) as e:
        d.checkpoint_read(t)
    assert e.value.status == q.QCW_ETIMEOUT
    d.set_fused_wait_limit(0, -1)
    d.reset()
    d.close()
