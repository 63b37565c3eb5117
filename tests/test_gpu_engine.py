"""GPU tests of the batched runner (one graph launch over many circuits) and the serving
loop (continuous batching), against the CPU oracle, plus their bounded-wait error paths.

Tolerance: max |delta rho| <= 1e-5, readouts (trace, purity, P(q=1)) within 1e-6 of the
oracle; a circuit's results must be bitwise identical alone and in a mix.
"""

import numpy as np
import pytest

import oracle
import workloads as wl

pytestmark = pytest.mark.gpu

ATOL = 1e-5
RTOL_READ = 1e-6


@pytest.fixture(scope="module")
def q():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1101_1785_gb300 as q

    return q


def _mixed_circuits(seed, ns, depth=40):
    rng = np.random.default_rng(seed)
    out = []
    for j, n in enumerate(ns):
        noise = ("adpd", "dep", "none")[j % 3]
        out.append(wl.random_circuit(n, int(rng.integers(depth // 2, depth + 1)), seed * 1000 + j, "mixed", noise,
                                     {"gamma": float(rng.uniform(0.001, 0.05)), "lam": 0.02, "p": 1e-3}))
    return out


def _readouts(rho):
    return oracle.probabilities(rho), oracle.purity(rho), oracle.trace(rho).real


def test_batch_against_oracle(q):
    circs = _mixed_circuits(1, [1, 2, 3, 4, 5, 6, 7, 8, 9, 4, 7, 2])
    b = q.Batch(circs)
    b.run()
    p1, pur, tr = b.results()
    for j, c in enumerate(circs):
        want = oracle.run_circuit(c)
        got = b.get_state(j)
        assert np.abs(got - want).max() <= ATOL, (j, c.n)
        wp1, wpur, wtr = _readouts(want)
        np.testing.assert_allclose(p1[j], wp1, atol=RTOL_READ, rtol=0)
        assert abs(pur[j] - wpur) <= RTOL_READ and abs(tr[j] - wtr) <= RTOL_READ
    info = b.info()
    assert info["items"] > len(circs) and info["passes"] >= len(circs)
    # a second launch of the captured graph starts over and gives the same results
    b.run()
    p1b, purb, trb = b.results()
    np.testing.assert_array_equal(purb, pur)
    b.close()


def test_batch_alone_equals_mixed(q):
    target = wl.random_circuit(8, 60, 77, "mixed", "adpd")
    others = _mixed_circuits(2, [9, 5, 8, 3, 7, 6, 10])
    alone = q.Batch([target])
    alone.run()
    a_p1, a_pur, a_tr = alone.results()
    a_state = alone.get_state(0)
    mixed = q.Batch(others[:3] + [target] + others[3:])
    mixed.run()
    m_p1, m_pur, m_tr = mixed.results()
    np.testing.assert_array_equal(mixed.get_state(3), a_state)
    np.testing.assert_array_equal(m_p1[3], a_p1[0])
    assert m_pur[3] == a_pur[0] and m_tr[3] == a_tr[0]
    alone.close()
    mixed.close()


def test_batch_wait_runs_out_without_hanging(q):
    circs = _mixed_circuits(3, [8, 8, 4])
    b = q.Batch(circs)
    b.run()
    good = b.results()[1].copy()
    n_items = b.info()["items"]
    b.set_wait_limit(2000, n_items - 1)  # the last item waits on a counter nothing sets
    b.run()
    with pytest.raises(q.QcwError) as e:
        b.wait(30.0)
    assert e.value.status == q.QCW_ETIMEOUT
    b.set_wait_limit(20_000_000, -1)  # normal list again: the context is still usable
    b.run()
    np.testing.assert_array_equal(b.results()[1], good)
    b.close()


def _server_results(q, srv, circs):
    ids = [srv.submit(c) for c in circs]
    srv.drain(60.0)
    res = {r["id"]: r for r in srv.poll()}
    return [res[i] for i in ids]


def test_server_against_oracle(q):
    circs = _mixed_circuits(4, [3, 5, 7, 9, 4, 8, 6, 10, 3], depth=50)
    srv = q.Server(1 << 30, passes_per_step=3)
    out = _server_results(q, srv, circs)
    for c, r in zip(circs, out):
        want = oracle.run_circuit(c)
        wp1, wpur, wtr = _readouts(want)
        assert r["status"] == q.QCW_OK
        np.testing.assert_allclose(r["p1"], wp1, atol=RTOL_READ, rtol=0)
        assert abs(r["purity"] - wpur) <= RTOL_READ and abs(r["trace"] - wtr) <= RTOL_READ
    assert srv.stats()["bytes_in_use"] == 0
    srv.close()


def test_server_alone_equals_mixed(q):
    target = wl.random_circuit(9, 80, 99, "mixed", "dep")
    srv = q.Server(1 << 30, passes_per_step=2)
    alone = _server_results(q, srv, [target])[0]
    mix = _mixed_circuits(5, [10, 3, 9, 6, 8, 4, 7], depth=60)
    got = _server_results(q, srv, mix[:4] + [target] + mix[4:])[4]
    np.testing.assert_array_equal(got["p1"], alone["p1"])
    assert got["purity"] == alone["purity"] and got["trace"] == alone["trace"]
    srv.close()


def test_server_admission_respects_budget(q):
    n = 8
    budget = 2 * 16 * 4 ** n  # room for two 8-qubit requests
    srv = q.Server(budget, passes_per_step=1)
    circs = [wl.random_circuit(n, 40, 500 + j, "mixed", "adpd") for j in range(5)]
    for c in circs:
        srv.submit(c)
    seen_live, done = 0, []
    for _ in range(10000):
        srv.step()
        st = srv.stats()
        assert st["bytes_in_use"] <= budget
        seen_live = max(seen_live, st["live"])
        done += srv.poll()
        if len(done) == len(circs):
            break
    assert len(done) == len(circs) and seen_live == 2
    with pytest.raises(q.QcwError):  # a request that can never fit is refused at submission
        srv.submit(wl.random_circuit(n + 1, 5, 1, "mixed", "none"))
    srv.close()


def test_server_bounded_waits(q):
    srv = q.Server(1 << 31, passes_per_step=4)
    big = wl.random_circuit(12, 300, 7, "mixed", "adpd")
    small = wl.random_circuit(5, 30, 8, "mixed", "adpd")
    # in-kernel wait that runs out: the step reports QCW_ETIMEOUT and the server carries on
    srv.set_limits(30.0, 2000, stall_next_step=True)
    srv.submit(small)
    srv.step()
    with pytest.raises(q.QcwError) as e:
        srv.step()
    assert e.value.status == q.QCW_ETIMEOUT
    assert [r["status"] for r in srv.poll()] == [q.QCW_ETIMEOUT]
    srv.set_limits(30.0, 20_000_000)
    # host wait limit: a zero limit cannot see the big step finish
    srv.submit(big)
    srv.step()
    srv.set_limits(0.0, 20_000_000)
    with pytest.raises(q.QcwError) as e:
        srv.step()
    assert e.value.status == q.QCW_ETIMEOUT
    srv.set_limits(60.0, 20_000_000)
    srv.submit(small)
    srv.drain(120.0)
    res = srv.poll()
    assert sorted(r["status"] for r in res) == [q.QCW_OK, q.QCW_OK]
    want = oracle.run_circuit(small)
    r = [x for x in res if x["n"] == 5][0]
    assert abs(r["purity"] - oracle.purity(want)) <= RTOL_READ
    srv.close()
