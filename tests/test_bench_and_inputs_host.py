"""CPU tests of host-side pieces without a GPU: the benchmark's stored-readout parser and its
byte accounting, and the seeded inputs of the paper's noise experiments."""

import os

import numpy as np
import pytest

import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_stored_readouts_parse(bench):
    g = bench.read_golden(bench.GOLDEN_N12)
    assert g["n"] == [12.0] and g["gates"] == [500.0]
    assert len(g["final"]) == 3 + 12
    assert abs(g["final"][0] - 1) < 1e-12 and 0 < g["final"][2] <= 1
    assert len(g["elem"]) == 1024 and all(r >= c for r, c, _, _ in g["elem"])
    assert sum(1 for r, c, _, _ in g["elem"] if r == c) == 256
    assert set(g["ptrace"]) == {(0, 1), (5, 11)}
    for pt in g["ptrace"].values():
        assert pt.shape == (4, 4)
        assert abs(np.trace(pt) - 1) < 1e-12
        assert np.abs(pt - pt.conj().T).max() < 1e-15
    if os.path.exists(bench.GOLDEN_N14):
        g = bench.read_golden(bench.GOLDEN_N14)
        assert len(g["ckpt"]) == 10 and [int(r[0]) for r in g["ckpt"]] == list(range(100, 1001, 100))
        assert all(len(r) == 4 + 14 for r in g["ckpt"])
        assert len(g["measure"]) == 4 and g["measure"][2] in (0.0, 1.0)
        assert (0, 1) in g["post_ptrace"]


def test_byte_accounting(bench):
    n = 14
    assert bench.pass_unit_bytes(n) == 16 * 4 ** n
    m = 1 << (n - 6)
    assert bench.design_pass_bytes(n, "k_fused_herm_ws") == 2 * 8 * 4 ** 6 * m * (m + 1) // 2
    assert bench.design_pass_bytes(n, "k_fused_pass") == 16 * 4 ** n
    assert bench.d2h_bytes_per_step(n) == 10 * (n + 4) * 8 + 2 * 64 * 8 + 16 * 16


def test_recorded_traffic_follows_the_source(bench, tmp_path, monkeypatch):
    """A stored DRAM figure is used only while the pass kernel's sources hash to the value it was
    recorded with."""
    h = bench.kernel_hash()
    assert h == bench.kernel_hash() and len(h) == 16
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k_fused_herm_ws_n14_traffic.txt").write_text(f"kernel_hash = {h}\ndram_bytes_per_launch = 123\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_hash", lambda: h)
    assert bench.recorded_traffic("k_fused_herm_ws") == 123.0
    monkeypatch.setattr(bench, "kernel_hash", lambda: "0" * 16)
    assert bench.recorded_traffic("k_fused_herm_ws") is None


@pytest.mark.parametrize("name", ["MV1", "MV2", "MVn"])
def test_noise_experiment_inputs(name):
    """Weights of every step's noise average sum to 1 (p = 0.8 ideal path, eps = 0.2 split
    p_1 / p_2 = .95 / .05 over the paths, one-hit only for one qubit), the Kraus form keeps the
    trace, switching noise off only replaces Paulis by the identity (same structure, same
    weights), and the draws are reproducible."""
    full = wl.mv_experiment(name, "xyz")
    n_paths = full.n_p * (1 if full.n == 1 else 2)
    for s in (1, full.nsteps):
        terms = full.noise_terms(s)
        assert len(terms) == 1 + n_paths
        assert abs(sum(w for w, _ in terms) - 1) < 1e-15
        assert terms[0] == (0.8, [])
        ks = full.kraus(s)
        assert np.abs(sum(k.conj().T @ k for k in ks) - np.eye(1 << full.n)).max() < 1e-12
        for noise in ("yz", "z", "none"):
            other = wl.mv_experiment(name, noise).noise_terms(s)
            assert [w for w, _ in other] == [w for w, _ in terms]
            for (_, h1), (_, h2) in zip(terms, other):
                assert [q for q, _ in h1] == [q for q, _ in h2]
                for (_, a1), (_, a2) in zip(h1, h2):
                    assert a2 == (a1 if a1 in wl.NOISE_SWITCHES[noise] else 0)
    again = wl.mv_experiment(name, "xyz")
    assert again.hits == full.hits
    tr = wl.mv_trajectories(full, 200)
    assert tr.shape == (full.nsteps, 200) and tr.min() >= 0 and tr.max() <= n_paths
