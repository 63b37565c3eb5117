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


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="qcw", choices=["qcw", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-gates", type=int, default=1, help="gates of the oracle sample")
    ap.add_argument("--workload", default="circuit14", choices=["circuit14", "batch", "serve"],
                    help="circuit14: the 14-qubit benchmark (default); batch: 512 circuits of 4..10 qubits in "
                         "one launch; serve: Poisson request stream through the continuous-batching server")
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
def oracle_sample(ngates: int):
    """Oracle on the first `ngates` gates (+ channels) of the same circuit; returns (gates/s, s, threads)."""
    import oracle
    import workloads as wl

    c = wl.config3_circuit(n=N_QUBITS, ngates=N_GATES).gate_prefix(ngates)
    threads = oracle.set_threads(0)
    rho = oracle.initial_state(c)
    t0 = time.perf_counter()
    oracle.run_circuit(c, rho)
    dt = time.perf_counter() - t0
    del rho
    return ngates / dt, dt, threads


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import workloads  # noqa: F401

    for _ in range(args.warmup):
        oracle_sample(args.cpu_gates)
    t0 = time.perf_counter()
    total = 0.0
    threads = 0
    for _ in range(args.steps):
        _, dt, threads = oracle_sample(args.cpu_gates)
        total += dt
    elapsed = time.perf_counter() - t0
    value = args.cpu_gates * args.steps / total
    sample = (f"first {args.cpu_gates} gate(s) of the 1000-gate 14-qubit circuit with their AD+PD "
              f"channels, complex128 oracle, per step")
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
    ms = ev0.elapsed_time(ev1)
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
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
    for k in range(4):  # both contexts planned and tuned
        gpu_step(ctxs[k % 2], packed, host.data_ptr())
    barrier()
    t0 = time.perf_counter()
    ctxs[0].set_state_c64(host.data_ptr())
    for k in range(args.steps):
        if k + 1 < args.steps:
            ctxs[(k + 1) % 2].set_state_c64(host.data_ptr())
        gpu_step(ctxs[k % 2], packed, loaded=True)
    barrier()
    e2e_s = time.perf_counter() - t0
    d2.close()
    if dist is not None:
        t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    d.close()

    total_gates = N_GATES * args.steps * world
    value = total_gates / (ms / 1e3)
    e2e_value = total_gates / e2e_s

    peaks, peak_kind = load_peaks()
    per_launch_bytes = pass_unit_bytes(nq)
    avg_ms = st["fused_pass_ms"] / max(1, st["timed_passes"])
    achieved = per_launch_bytes / (avg_ms / 1e3) / 1e9
    hbm = float(peaks["hbm_gbs"])

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and nq == N_QUBITS:
        v, dt, threads = oracle_sample(args.cpu_gates)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"first {args.cpu_gates} gate(s) of the same circuit with their AD+PD channels "
                         f"on the complex128 oracle ({dt:.1f} s)"}

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
                         "frac": achieved / hbm, "traffic": recorded_traffic(TIMED_KERNEL[args.fused_kernel]),
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
                       "outcome_q0": meas[0], "p_outcome": meas[1]},
        }
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


def run_batch(args):
    import numpy as np
    import torch

    import __graft_entry__
    import workloads as wl

    __graft_entry__.build()
    import paper_1101_1785_gb300 as q

    torch.cuda.init()
    circuits = wl.config4_batch()
    gates = sum(c.n_gates for c in circuits)
    t0 = time.perf_counter()
    b = q.Batch(circuits)
    t_create = time.perf_counter() - t0
    for _ in range(max(3, args.warmup)):
        b.run()
        b.wait()
    sampler = ClockSampler(0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        b.run()
        b.wait()
    dt = (time.perf_counter() - t0) / args.steps
    clocks = sampler.stop()
    _, pur, _ = b.results()
    info = b.info()
    b.close()
    packed = [q.PackedOps(c.ops) for c in circuits]
    _loop_one_at_a_time(q, circuits[:16], packed[:16])  # warm-up
    dt_loop, pur_loop = _loop_one_at_a_time(q, circuits, packed)
    print(json.dumps({
        "metric": "gate-applications/s, 512-circuit batch (n ~ U{4..10}, depth ~ U{50..400}, AD+PD)",
        "value": gates / dt, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
        "ms_per_step": dt * 1e3, "higher_is_better": True, "dtype": "c64", "data": "synthetic",
        "config": {"workload": "512 seeded circuits, one persistent graph-captured launch", "circuits": len(circuits),
                   "gates": gates},
        "circuits_per_s": len(circuits) / dt,
        "plain_loop": {"value": gates / dt_loop, "ms_per_batch": dt_loop * 1e3,
                       "circuits_per_s": len(circuits) / dt_loop},
        "speedup_vs_plain_loop": dt_loop / dt,
        "max_abs_purity_diff_vs_plain": float(np.abs(pur - pur_loop).max()),
        "plan": info, "create_s": t_create, "clocks": clocks,
    }), flush=True)


def run_serve(args):
    import threading

    import numpy as np
    import torch

    import __graft_entry__
    import workloads as wl

    __graft_entry__.build()
    import paper_1101_1785_gb300 as q

    torch.cuda.init()
    reqs = wl.config5_requests(rate=args.rate, duration=args.duration)
    warm = wl.config5_requests(rate=args.rate, duration=0.2, index=1)
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
        if not results and time.monotonic() - start > args.duration + 600:
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
    print(json.dumps({
        "metric": "req/s and p99 latency, Poisson request stream (n 3..13, depth 20..500, mixed noise)",
        "value": len(results) / (t_end - start), "unit": "req/s", "n_gpus": 1, "higher_is_better": True,
        "dtype": "c64", "data": "synthetic",
        "config": {"workload": f"Poisson {args.rate:g} req/s for {args.duration:g} s, budget 48 GiB (16*4^n per "
                               f"request), 4 passes per engine step", "requests": len(reqs)},
        "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3),
                       "max": float(lat.max() * 1e3)},
        "gate_apps_per_s": gates / (t_end - start), "offered_req_per_s": args.rate,
        "bad_results": bad,
        "plain_loop": {"req_per_s": sample / dt_loop, "sample": sample},
        "clocks": clocks,
    }), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
