#!/usr/bin/env python
"""Throughput benchmark of the qcw density-matrix path on the 14-qubit noisy circuit.

Workload (one "step"): a 14-qubit density matrix (16384 x 16384 complex64 on the device)
starts in |0..0><0..0|; a seeded 1000-gate circuit (kinds uniform over H, X, Z, S, T,
CNOT, Haar SU(2)) runs with amplitude damping (gamma = 0.01) and phase damping
(lambda = 0.02) on every touched qubit after each gate, in the fused path (planner +
Hermitian fused-pass kernel, fusion width chosen per segment by the library's cost model).  After every 100 gates the step reads trace and purity
in FP64; at the end it reads the per-qubit probabilities, measures qubit 0 (u-driven
projective measurement with renormalisation) and takes the partial trace over qubits 0, 1.

Metric: gate-applications/s = gates per step x steps (x GPUs) / time.  One JSON line.

Beside the timed steps (untimed for the headline, each with its own numbers in the line): an
accuracy replay of one step against the complex128 oracle's stored readouts of the full
circuit; the oracle itself timed on a warm sample on every host core and on one; and, at one
GPU, three sub-measurements -- the 12-qubit depolarising circuit on the plain path (one launch
per gate and per channel, GB/s per launch), the 512-circuit batch in one persistent launch
against the one-circuit-at-a-time loop, 5 s of the Poisson request stream through the
continuous-batching server (p50 / p99 latency, req/s) against the same loop, and the multiverse
ensemble's density kernel at 12-14 qubits.
``--impl reference`` times the CPU oracle on a bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gate-applications/s on 14-qubit noisy rho (HBM GB/s vs peak); req/s + p99 at 1e-5"
UNIT = "gate-applications/s"
N_QUBITS = 14
N_GATES = 1000
CHUNK = 100
FUSE_K = 0  # 0: the library's cost model picks the width per segment
U_MEASURE = 0.37
PT_KEEP = [0, 1]
GOLDEN_N14 = os.path.join(ROOT, "tests", "golden", "config3_n14.txt")
GOLDEN_N12 = os.path.join(ROOT, "tests", "golden", "config2_n12.txt")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="qcw", choices=["qcw", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-gates", type=int, default=3, help="gates of the timed oracle sample (all cores)")
    ap.add_argument("--cpu-baseline-leg", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the untimed accuracy leg and the plain / batch / serve sub-measurements")
    ap.add_argument("--workload", default="circuit14", choices=["circuit14", "plain12", "batch", "serve", "ensemble"],
                    help="circuit14: the 14-qubit benchmark (default); plain12: the 12-qubit depolarising circuit "
                         "on the plain path, one launch per gate and per channel; batch: 512 circuits of 4..10 "
                         "qubits in one launch; serve: Poisson request stream through the continuous-batching server; "
                         "ensemble: the multiverse ensemble's density kernel")
    ap.add_argument("--duration", type=float, default=10.0, help="serve: seconds of arrivals")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: arrivals per second")
    ap.add_argument("--fused-kernel", default="auto", choices=["auto", "tile", "herm", "herm_ws", "herm_tc"],
                    help="kernel for large fused passes (results are identical)")
    ap.add_argument("--fuse-k", type=int, default=FUSE_K, help="qubits per fused pass")
    ap.add_argument("--qubits", type=int, default=N_QUBITS,
                    help="register size (14 is the benchmark; smaller sizes are for profiling)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, dist, device) -> float:
    """The largest of every rank's x: a job of independent replicas takes as long as its slowest
    rank.  dist is torch.distributed (None: one process); device holds the reduction's tensor
    (the GPU under NCCL, the CPU under gloo)."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(gates_per_step: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job gate applications per second of `world` replicas, each running `steps` steps of
    `gates_per_step` gates, over the slowest rank's time."""
    return gates_per_step * steps * world / seconds


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in rows for j in range(4) if r[5 + j].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- workload
def make_workload(n):
    import workloads as wl

    c = wl.config3_circuit(n=n, ngates=N_GATES)
    chunks = [c.gate_prefix(g).ops for g in range(0, N_GATES + 1, CHUNK)]
    parts = [chunks[i + 1][len(chunks[i]):] for i in range(len(chunks) - 1)]
    return c, parts


def gpu_step(d, packed, host_rho_ptr=None, loaded=False):
    """One pass of the whole path; returns the readouts (host FP64).  rho_0: |0..0><0..0| on the
    device, uploaded from host_rho_ptr, or (loaded) already uploaded by the caller."""
    if loaded:
        pass
    elif host_rho_ptr is None:
        d.reset()
    else:
        d.set_state_c64(host_rho_ptr)
    # trace and purity every CHUNK gates as asynchronous checkpoints: the host queues and plans
    # the next chunk while the GPU evolves this one
    tickets = []
    for p in packed:
        d.apply_packed(p)
        tickets.append(d.checkpoint())
    tp = [(tr, pu) for tr, pu, _ in (d.checkpoint_read(t) for t in tickets)]
    probs = d.probabilities()
    m, pm = d.measure(0, -1, U_MEASURE)
    pt = d.partial_trace(PT_KEEP)
    return tp, probs, (m, pm), pt


def d2h_bytes_per_step(n):
    """Checkpoint slots ((n + 3) values and the error word per checkpoint), the 64-double result
    block of the probabilities and the measurement readouts, and the partial trace."""
    return (N_GATES // CHUNK) * (n + 4) * 8 + 2 * 64 * 8 + 16 * (4 ** len(PT_KEEP))


def pass_unit_bytes(n):
    """Algorithmic bytes of one fused pass: one read and one write of rho in complex64."""
    return 16 * 4 ** n


def design_pass_bytes(n, kernel, tile_qubits=6):
    """HBM bytes the timed pass kernel is designed to move.  The warp-specialised kernel reads
    and writes the canonical copy of each tile pair (one tile's worth each way, M (M + 1) / 2
    pairs, M = 2^(n - 6)); the per-tile-pair Hermitian kernel reads a tile and writes it and
    its mirror; the general kernel reads and writes every element."""
    if kernel == "k_fused_pass" or n <= tile_qubits:
        return 16 * 4 ** n
    m = 1 << (n - tile_qubits)
    tile = 8 * 4 ** tile_qubits
    pairs = m * (m + 1) // 2
    return tile * 2 * pairs if kernel in ("k_fused_herm_ws", "k_fused_herm_tc") else tile * (pairs + m * m)


TIMED_KERNEL = {"auto": "k_fused_herm_ws", "herm_tc": "k_fused_herm_tc", "herm_ws": "k_fused_herm_ws",
                "herm": "k_fused_herm", "tile": "k_fused_pass"}


def kernel_hash():
    """Hash of the pass kernel's sources with comments and whitespace removed, so that a
    recorded measurement stays attached to the code it measured."""
    import re

    h = hashlib.sha256()
    for f in ("fused.cu", "planner.cpp", "qcw_device.cuh", "tile.cuh", "tile.cpp", "tc.cuh"):
        with open(os.path.join(ROOT, "paper_1101_1785_gb300", "csrc", f)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
        src = re.sub(r"//[^\n]*", " ", src)
        h.update(" ".join(src.split()).encode())
    return h.hexdigest()[:16]


def recorded_traffic(kernel):
    """dram bytes per fused-pass launch from the committed ncu summary, if it matches this source."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_n14_traffic.txt")
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if "=" in line and not line.startswith("#"):
                    k, v = line.split("=", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_hash") == kernel_hash():
            return float(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        pass
    return None


# ----------------------------------------------------------------------------- oracle timing
def oracle_timed(ngates: int, steps: int = 1, warmup: int = 0, one_core: bool = False):
    """The oracle as it stands on a bounded, warm sample of the benchmark circuit: the ops of gates
    2 .. ngates + 1 (each gate with its AD + PD channels).  The first gate runs once, untimed, on
    every core to touch the 4 GiB state's pages; then the sample runs warmup + steps times on every
    core (the first `warmup` untimed) -- the same operations each time, so every timing covers the
    same work -- and with one_core the sample's first gate once more on one thread.  Returns
    (seconds per timed sample, threads used, one-thread seconds or None)."""
    import oracle
    import workloads as wl

    c = wl.config3_circuit(n=N_QUBITS, ngates=N_GATES)
    nthreads = os.cpu_count() or 1
    used = oracle.set_threads(nthreads)
    b1, b2, bn = (len(c.gate_prefix(g).ops) for g in (1, 2, 1 + ngates))
    rho = oracle.initial_state(c)
    oracle.run_circuit(c, rho, c.ops[:b1])
    times = []
    for i in range(warmup + steps):
        t0 = time.perf_counter()
        oracle.run_circuit(c, rho, c.ops[b1:bn])
        dt = time.perf_counter() - t0
        if i >= warmup:
            times.append(dt)
    one = None
    if one_core:
        oracle.set_threads(1)
        t0 = time.perf_counter()
        oracle.run_circuit(c, rho, c.ops[b1:b2])
        one = time.perf_counter() - t0
        oracle.set_threads(nthreads)
    del rho
    return times, used, one


def cpu_baseline_subprocess(ngates: int):
    """cpu_baseline_legs in a fresh interpreter that never touches the GPU -- the environment the
    reference arm times the oracle in (inside the process that holds the CUDA context the same
    sample ran about a quarter slower)."""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-leg", "--cpu-gates", str(ngates)],
                       capture_output=True, text=True, cwd=ROOT)
    if r.returncode != 0:
        raise RuntimeError(f"CPU-baseline leg failed:\n{r.stdout[-2000:]}\n{r.stderr[-2000:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline_legs(ngates: int):
    """Every core on `ngates` warm gates (timed after one untimed pass of the same gates, as the
    reference arm's warm-up step does), then one core on the first of them."""
    times, used, one = oracle_timed(ngates, 1, 1, one_core=True)
    dt = times[0]
    sample = (f"gates 2..{ngates + 1} of the 1000-gate 14-qubit circuit with their AD+PD channels on the complex128 "
              f"oracle, {used} host threads, after one untimed warm-up gate and one untimed pass of the same gates "
              f"({dt:.1f} s); then gate 2 again on one thread ({one:.1f} s)")
    return {"value": ngates / dt, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample,
            "one_core": {"value": 1.0 / one, "unit": UNIT, "cores": 1, "seconds": one}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import workloads  # noqa: F401

    ngates = max(1, args.cpu_gates)
    t0 = time.perf_counter()
    times, threads, _ = oracle_timed(ngates, args.steps, args.warmup)
    elapsed = time.perf_counter() - t0
    total = sum(times)
    value = ngates * args.steps / total
    sample = (f"gates 2..{ngates + 1} of the 1000-gate 14-qubit circuit with their AD+PD channels per step (the same "
              f"operations each step, after one untimed warm-up gate), complex128 oracle on {threads} host threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic",
        "config": {"workload": "14-qubit noisy density matrix, 1000-gate seeded circuit, AD(0.01)+PD(0.02)",
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": elapsed,
    }), flush=True)


# ----------------------------------------------------------------------------- accuracy
def read_golden(path):
    """Stored oracle readouts (tests/golden/make_deep_goldens.py): 'key values...' lines."""
    import numpy as np

    g = {"elem": [], "ckpt": [], "ptrace": {}, "post_ptrace": {}}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            if key == "elem":
                g["elem"].append([float(x) for x in vals])
            elif key == "ckpt":
                g["ckpt"].append([float(x) for x in vals])
            elif key in ("ptrace", "post_ptrace"):
                z = np.array([float(x) for x in vals[2:]])
                g[key][(int(vals[0]), int(vals[1]))] = (z[0::2] + 1j * z[1::2]).reshape(4, 4)
            else:
                g[key] = [float(x) for x in vals]
    return g


def sampled_element_error(d, elem):
    """max |delta rho| over stored (row, column, Re, Im) elements, gathered on the device from the
    context's buffer (completed and ordered on its stream)."""
    import numpy as np
    import torch

    ptr, sp = d.device_state()
    torch.cuda.ExternalStream(sp).synchronize()
    dim = 1 << d.n

    class _Buf:
        pass

    buf = _Buf()
    buf.__cuda_array_interface__ = {"shape": (dim, 2 * dim), "typestr": "<f4", "data": (ptr, False), "version": 2}
    view = torch.as_tensor(buf, device="cuda")
    e = np.asarray(elem, dtype=np.float64)
    r = torch.as_tensor(e[:, 0].astype(np.int64), device="cuda")
    c2 = torch.as_tensor(2 * e[:, 1].astype(np.int64), device="cuda")
    got = view[r, c2].double().cpu().numpy() + 1j * view[r, c2 + 1].double().cpu().numpy()
    return float(np.abs(got - (e[:, 2] + 1j * e[:, 3])).max())


def accuracy_n14(d, packed):
    """Untimed replay of one step on the timed context, every readout against the complex128
    oracle's values for the full 1000-gate circuit."""
    import numpy as np

    if not os.path.exists(GOLDEN_N14):
        return {"vs": None, "why": "no stored oracle readouts for the 14-qubit circuit"}
    g = read_golden(GOLDEN_N14)
    d.reset()
    tickets = []
    for p in packed:
        d.apply_packed(p)
        tickets.append(d.checkpoint())
    ck = [d.checkpoint_read(t) for t in tickets]
    out = {
        "vs": "complex128 oracle, full circuit (tests/golden/config3_n14.txt)",
        "checkpoints": len(ck),
        "max_abs_trace_err": max(abs(c[0] - 1) for c in ck),
        "max_abs_dtrace": max(abs(c[0].real - w[1]) for c, w in zip(ck, g["ckpt"])),
        "max_abs_dpurity": max(abs(c[1] - w[3]) for c, w in zip(ck, g["ckpt"])),
        "max_abs_dp": max(float(np.abs(c[2] - np.asarray(w[4:])).max()) for c, w in zip(ck, g["ckpt"])),
    }
    out["max_abs_drho_sampled"] = sampled_element_error(d, g["elem"])
    out["sampled_elements"] = len(g["elem"])
    out["max_abs_drho_A"] = max(float(np.abs(d.partial_trace(list(k)) - v).max()) for k, v in g["ptrace"].items())
    m, pm = d.measure(0, -1, U_MEASURE)
    out["outcome_match"] = int(m) == int(g["measure"][2])
    out["abs_dp_outcome"] = abs(pm - g["measure"][3])
    out["post_max_abs_drho_A"] = float(np.abs(d.partial_trace([0, 1]) - g["post_ptrace"][(0, 1)]).max())
    out["post_abs_dpurity"] = abs(d.purity() - g["post_purity"][0])
    return out


# ----------------------------------------------------------------------------- GPU arm
def run_ours(args):
    rank, world, local = dist_env()
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__

    if rank == 0 or world == 1:
        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
        __graft_entry__.build()  # no-op once rank 0 compiled; also loads the module
    import paper_1101_1785_gb300 as q

    nq = args.qubits
    circuit, parts = make_workload(nq)
    packed = [q.PackedOps(p) for p in parts]
    d = q.Density(nq)
    d.set_mode(q.QCW_MODE_FUSED, args.fuse_k)
    d.set_fused_kernel({"auto": 0, "tile": 1, "herm": 2, "herm_ws": 3, "herm_tc": 4}[args.fused_kernel])
    rho_ptr, stream_ptr = d.device_state()
    ext = torch.cuda.ExternalStream(stream_ptr)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timing
    for _ in range(max(3, args.warmup)):
        gpu_step(d, packed)
    barrier()
    d.stats_reset()
    d.enable_pass_timing(True)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    phys = int(vis.split(",")[local]) if vis and vis.split(",")[local].strip().isdigit() else local
    sampler = ClockSampler(phys)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    ev0.record(ext)
    for _ in range(args.steps):
        out = gpu_step(d, packed)
    ev1.record(ext)
    barrier()
    clocks = sampler.stop()
    d.enable_pass_timing(False)
    st = d.stats()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    tp, probs, meas, pt = out
    max_tr_err = max(abs(x[0] - 1) for x in tp)

    # ---- end to end: rho_0 uploaded from pinned host memory every step, readouts to host.
    # Two contexts alternate: step k + 1's upload (an asynchronous copy on the other context's
    # stream) runs while step k evolves; every upload and readout is inside the timed region.
    host = torch.zeros(2 * (4 ** nq), dtype=torch.float32).pin_memory()
    host[0] = 1.0
    d2 = q.Density(nq)
    d2.set_mode(q.QCW_MODE_FUSED, args.fuse_k)
    d2.set_fused_kernel({"auto": 0, "tile": 1, "herm": 2, "herm_ws": 3, "herm_tc": 4}[args.fused_kernel])
    ctxs = (d, d2)
    for k in range(6):  # both contexts planned, tuned and re-planned for replay (three steps each)
        gpu_step(ctxs[k % 2], packed, host.data_ptr())
    barrier()
    t0 = time.perf_counter()
    ctxs[0].set_state_c64(host.data_ptr())
    for k in range(args.steps):
        if k + 1 < args.steps:
            ctxs[(k + 1) % 2].set_state_c64(host.data_ptr())
        gpu_step(ctxs[k % 2], packed, loaded=True)
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    d2.close()
    accuracy = None
    if rank == 0 and not args.no_extras and nq == N_QUBITS:
        accuracy = accuracy_n14(d, packed)
    d.close()

    value = replica_rate(N_GATES, args.steps, world, ms / 1e3)
    e2e_value = replica_rate(N_GATES, args.steps, world, e2e_s)

    peaks, peak_kind = load_peaks()
    per_launch_bytes = pass_unit_bytes(nq)
    avg_ms = st["fused_pass_ms"] / max(1, st["timed_passes"])
    achieved = per_launch_bytes / (avg_ms / 1e3) / 1e9
    hbm = float(peaks["hbm_gbs"])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and nq == N_QUBITS:
        cpu = cpu_baseline_subprocess(args.cpu_gates)
    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        import paper_1101_1785_gb300 as q2

        extras["plain12"] = measure_plain12(q2, steps=2, warmup=1)
        extras["batch"] = measure_batch(q2, steps=3, warmup=3)
        extras["serve"] = measure_serve(q2, rate=2000.0, duration=5.0)
        extras["ensemble_density"] = measure_ensemble(q2)

    traffic = recorded_traffic(TIMED_KERNEL[args.fused_kernel])
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": "14-qubit noisy density matrix (16384 x 16384 complex64), seeded "
                                   "1000-gate circuit {H,X,Z,S,T,CNOT,Haar}, AD(0.01)+PD(0.02) per "
                                   "touched qubit, fused (width by cost model), FP64 trace+purity every 100 gates, "
                                   "probabilities, measurement, partial trace",
                       "qubits": nq, "parallelism": f"replicas x{world}",
                       "l2": f"inputs larger than L2 ({8 * 4 ** nq / 2**20:.0f} MiB rho vs 129 MB L2)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "achieved_is": "algorithmic bytes (one read and one write of rho, 16 * 4^n) per pass "
                                        "launch / the launch's event-timed duration",
                         "dram_gbs": None if traffic is None else traffic / (avg_ms / 1e3) / 1e9,
                         "peak_kind": peak_kind, "kernel": TIMED_KERNEL[args.fused_kernel],
                         "bytes_per_launch": per_launch_bytes,
                         "design_bytes_per_launch": design_pass_bytes(nq, TIMED_KERNEL[args.fused_kernel]),
                         "avg_launch_ms": avg_ms},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * (4 ** nq),
                    "pipelining": "two contexts; step k+1's rho_0 upload overlaps step k",
                    "d2h_bytes_per_step": d2h_bytes_per_step(nq)},
            "gpu_launches": st["launches"],
            "fused_passes_per_step": st["fused_passes"] / args.steps,
            "clocks": clocks,
            "checks": {"max_abs_trace_err": max_tr_err, "final_purity": tp[-1][1],
                       "outcome_q0": meas[0], "p_outcome": meas[1], "accuracy_vs_oracle": accuracy},
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- batch / serve
def _loop_one_at_a_time(q, circuits, packed, reps=1):
    """The plain GPU path: one context per size, each circuit run and read out on its own."""
    import numpy as np

    dens = {}
    for c in circuits:
        if c.n not in dens:
            dens[c.n] = q.Density(c.n)
            dens[c.n].set_mode(q.QCW_MODE_FUSED, 0)
    out = np.zeros(len(circuits))
    t0 = time.perf_counter()
    for _ in range(reps):
        for j, (c, p) in enumerate(zip(circuits, packed)):
            d = dens[c.n]
            d.reset()
            d.apply_packed(p)
            d.probabilities()
            out[j] = d.purity()
    dt = (time.perf_counter() - t0) / reps
    for d in dens.values():
        d.close()
    return dt, out


def measure_plain12(q, steps=2, warmup=1):
    """The 12-qubit depolarising circuit on the plain path: one kernel launch per gate and per
    channel (500 gates, one Kraus channel per touched qubit).  rho_0 is uploaded before each step,
    outside the timed region; the step ends with the trace, purity and probabilities.  Each launch
    reads and writes rho once: 16 * 4^12 algorithmic bytes."""
    import numpy as np
    import torch

    import workloads as wl

    c = wl.config2_circuit()
    n = c.n
    bounds = [len(c.gate_prefix(g).ops) for g in range(0, c.n_gates + 1, CHUNK)]
    packed = [q.PackedOps(c.ops[bounds[i]:bounds[i + 1]]) for i in range(len(bounds) - 1)]
    rho0 = np.ascontiguousarray(c.rho0.astype(np.complex64))
    host = torch.from_numpy(rho0.view(np.float32).reshape(-1)).pin_memory()
    d = q.Density(n)
    _, sp = d.device_state()
    stream = torch.cuda.ExternalStream(sp)
    ms_total, readouts = 0.0, None
    d.stats_reset()
    for i in range(warmup + steps):
        d.set_state_c64(host.data_ptr())
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if i == warmup:
            d.stats_reset()
        e0.record(stream)
        for p in packed:
            d.apply_packed(p)
        tr, pu, pr = d.trace(), d.purity(), d.probabilities()
        e1.record(stream)
        e1.synchronize()
        if i >= warmup:
            ms_total += e0.elapsed_time(e1)
        readouts = (tr, pu, pr)
    st = d.stats()
    peaks, peak_kind = load_peaks()
    launches = len(c.ops)
    ms = ms_total / steps
    gbs = launches * 16 * 4 ** n / (ms / 1e3) / 1e9
    out = {
        "workload": "12-qubit density matrix, rho0 = I/2^n/2 + |psi><psi|/2, 500 gates (70 % Haar SU(2), 30 % "
                    "CNOT/CZ), depolarising 1e-3 per touched qubit; plain path, one launch per gate and per channel",
        "gate_apps_per_s": c.n_gates / (ms / 1e3), "ms_per_step": ms, "steps": steps,
        "evolution_launches_per_step": launches, "gpu_launches_per_step": st["launches"] / steps,
        "bytes_per_launch": 16 * 4 ** n, "achieved_gbs": gbs, "frac_of_hbm": gbs / float(peaks["hbm_gbs"]),
        "peak_kind": peak_kind, "l2_bytes": torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size,
        "rho_bytes": 8 * 4 ** n,
    }
    if os.path.exists(GOLDEN_N12):
        g = read_golden(GOLDEN_N12)
        tr, pu, pr = readouts
        out["accuracy_vs_oracle"] = {
            "vs": "complex128 oracle, full circuit (tests/golden/config2_n12.txt)",
            "abs_trace_err": abs(tr - 1), "abs_dpurity": abs(pu - g["final"][2]),
            "max_abs_dp": float(np.abs(pr - np.asarray(g["final"][3:])).max()),
            "max_abs_drho_sampled": sampled_element_error(d, g["elem"]), "sampled_elements": len(g["elem"]),
            "max_abs_drho_A": max(float(np.abs(d.partial_trace(list(k)) - v).max()) for k, v in g["ptrace"].items()),
        }
    d.close()
    return out


def measure_ensemble(q, sizes=((12, 64), (12, 256), (13, 64), (14, 16), (14, 64)), reps=5):
    """The multiverse ensemble's density rho = sum_v w_v |psi_v><psi_v| (the paper's ensemble
    average, formed on the GPU from nvec seeded random unit vectors with equal weights): event
    time on the density context's stream, best of `reps` after one warm-up.  Algorithmic unit:
    one write of rho (8 * 4^n bytes) and 8 nvec FP32 flops on half of its elements."""
    import numpy as np
    import torch

    peaks, _ = load_peaks()
    out = []
    for n, nvec in sizes:
        rng = np.random.default_rng(n * 1000 + nvec)
        psi = rng.standard_normal((nvec, 1 << n)) + 1j * rng.standard_normal((nvec, 1 << n))
        psi /= np.linalg.norm(psi, axis=1, keepdims=True)
        e = q.Ensemble(n, nvec)
        e.set(psi)
        d = q.Density(n)
        _, sp = d.device_state()
        st = torch.cuda.ExternalStream(sp)
        w = np.full(nvec, 1.0 / nvec)
        e.density(w, d)
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            e.density(w, d)
            e1.record(st)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = min(ts)
        flops = 8.0 * nvec * 4 ** n / 2
        out.append({"qubits": n, "vectors": nvec, "ms": ms, "write_floor_ms": 8 * 4 ** n / (float(peaks["hbm_gbs"]) * 1e9) * 1e3,
                    "tflops_fp32": flops / (ms / 1e3) / 1e12, "trace_err": abs(d.trace().real - 1)})
        d.close()
        e.close()
    return out


def measure_batch(q, steps=3, warmup=3):
    import numpy as np
    import torch

    import workloads as wl

    torch.cuda.init()
    circuits = wl.config4_batch()
    gates = sum(c.n_gates for c in circuits)
    t0 = time.perf_counter()
    b = q.Batch(circuits)
    t_create = time.perf_counter() - t0
    for _ in range(max(3, warmup)):
        b.run()
        b.wait()
    sampler = ClockSampler(0)
    t0 = time.perf_counter()
    for _ in range(steps):
        b.run()
        b.wait()
    dt = (time.perf_counter() - t0) / steps
    clocks = sampler.stop()
    _, pur, tr = b.results()
    info = b.info()
    b.close()
    packed = [q.PackedOps(c.ops) for c in circuits]
    _loop_one_at_a_time(q, circuits[:16], packed[:16])  # warm-up
    dt_loop, pur_loop = _loop_one_at_a_time(q, circuits, packed)
    return {
        "metric": "gate-applications/s, 512-circuit batch (n ~ U{4..10}, depth ~ U{50..400}, AD+PD)",
        "value": gates / dt, "unit": UNIT, "steps": steps, "warmup": max(3, warmup),
        "ms_per_step": dt * 1e3, "circuits": len(circuits), "gates": gates,
        "circuits_per_s": len(circuits) / dt,
        "plain_loop": {"value": gates / dt_loop, "ms_per_batch": dt_loop * 1e3,
                       "circuits_per_s": len(circuits) / dt_loop},
        "speedup_vs_plain_loop": dt_loop / dt,
        "max_abs_purity_diff_vs_plain": float(np.abs(pur - pur_loop).max()),
        "failed_1e-5_check": int(np.sum((np.abs(pur - pur_loop) > 1e-5) | (np.abs(tr - 1) > 1e-5))),
        "plan": info, "create_s": t_create, "clocks": clocks,
    }


def measure_serve(q, rate=2000.0, duration=10.0):
    import threading

    import numpy as np
    import torch

    import workloads as wl

    torch.cuda.init()
    reqs = wl.config5_requests(rate=rate, duration=duration)
    warm = wl.config5_requests(rate=rate, duration=0.2, index=1)
    packed = [q.PackedOps(c.ops) for _, c in reqs]
    wpacked = [q.PackedOps(c.ops) for _, c in warm]
    srv = q.Server(48 << 30, max_live=8192, passes_per_step=4)
    for (_, c), p in zip(warm, wpacked):
        srv.submit(c, p)
    srv.drain(120.0)
    srv.poll()

    start = time.monotonic() + 0.05
    arrivals = [start + t for t, _ in reqs]
    ids = {}
    done_sub = threading.Event()

    def dispatcher():
        for i, ((_, c), p) in enumerate(zip(reqs, packed)):
            wait = arrivals[i] - time.monotonic()
            if wait > 0:
                time.sleep(wait)
            ids[srv.submit(c, p)] = i
        done_sub.set()

    th = threading.Thread(target=dispatcher, daemon=True)
    sampler = ClockSampler(0)
    th.start()
    results = []
    while not (done_sub.is_set() and len(results) == len(reqs)):
        srv.step()
        results += srv.poll()
        if not results and time.monotonic() - start > duration + 600:
            break
    th.join()
    clocks = sampler.stop()
    srv.close()
    lat = np.array([r["t_done"] - arrivals[ids[r["id"]]] for r in results])
    t_end = max(r["t_done"] for r in results)
    bad = sum(1 for r in results if r["status"] != 0 or abs(r["trace"] - 1) > 1e-5)
    gates = sum(c.n_gates for _, c in reqs)
    sample = min(len(reqs), 2000)
    dt_loop, _ = _loop_one_at_a_time(q, [c for _, c in reqs[:sample]], packed[:sample])
    return {
        "metric": "req/s and p99 latency, Poisson request stream (n 3..13, depth 20..500, mixed noise)",
        "value": len(results) / (t_end - start), "unit": "req/s",
        "config": {"workload": f"Poisson {rate:g} req/s for {duration:g} s, budget 48 GiB (16*4^n per "
                               f"request), 4 passes per engine step", "requests": len(reqs)},
        "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3),
                       "max": float(lat.max() * 1e3)},
        "gate_apps_per_s": gates / (t_end - start), "offered_req_per_s": rate,
        "failed_1e-5_check": bad,
        "plain_loop": {"req_per_s": sample / dt_loop, "sample": sample},
        "clocks": clocks,
    }


def _standalone(args, what):
    import __graft_entry__

    __graft_entry__.build()
    import torch

    import paper_1101_1785_gb300 as q

    torch.cuda.set_device(0)
    if what == "plain12":
        r = measure_plain12(q, steps=args.steps, warmup=max(1, args.warmup))
        r.update({"metric": "gate-applications/s, 12-qubit plain path (GB/s per launch vs peak)", "value":
                  r["gate_apps_per_s"], "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "c64",
                  "data": "synthetic"})
    elif what == "batch":
        r = measure_batch(q, steps=args.steps, warmup=args.warmup)
        r.update({"n_gpus": 1, "higher_is_better": True, "dtype": "c64", "data": "synthetic"})
    elif what == "ensemble":
        r = {"metric": "ensemble density: ms per rho = sum_v w_v |psi_v><psi_v|", "unit": "ms", "n_gpus": 1,
             "higher_is_better": False, "dtype": "c64", "data": "synthetic", "sizes": measure_ensemble(q)}
    else:
        r = measure_serve(q, rate=args.rate, duration=args.duration)
        r.update({"n_gpus": 1, "higher_is_better": True, "dtype": "c64", "data": "synthetic"})
    print(json.dumps(r), flush=True)


def main():
    args = parse_args()
    if args.cpu_baseline_leg:
        print(json.dumps(cpu_baseline_legs(args.cpu_gates)), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload in ("plain12", "batch", "serve", "ensemble"):
        _standalone(args, args.workload)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
