#!/usr/bin/env python3
"""Benchmark of the GB300 state-vector simulator on the paper's random-circuit workload.

Workload (one step): a 30-qubit complex128 state set to |0...0>, the seeded depth-20 random
circuit (each layer U3 on every qubit, then CZ on (i, i+1) of the layer's parity; 890 gates),
applied through a fusion plan whose width the library's autotuner picks, then <Z0 Z1>.
The 16 GiB state is larger than L2, so every pass streams from HBM.

value = gates/s (original gate count / device time per step; fusion shows up as a gain).
roofline: the kernel with the largest share of device time, its algorithmic bytes per launch
(2 x 16 B x the amplitudes it must update) over its event-timed duration, against the measured
HBM copy bandwidth. e2e: the same metric through the public API call a user makes, wall clock,
including planning, matrix uploads and the host read of the result.

--impl reference times the FP64 CPU oracle on the same workload (bounded sample of gates per
step). Multi-GPU (torchrun): independent replicas, one per rank, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "state-vector GB/s & gates/s at n=30 c128 vs HBM peak; adjoint-grad ms; circuits/s"
HBM_PEAK_FALLBACK = 6800.0
# DRAM bytes (read + write) per launch of a kernel, from one ncu capture of the kernel as it is
# built now, at a smaller state than the bench's and scaled to n = 30 by the amplitudes a launch
# updates (the traffic of these kernels grows in proportion to the state): (kernel, n) -> bytes.
# k_dense_oz5 at n = 27: the mean of two launches, (2163699712 + 2085241088) and
# (2203977728 + 2082443776) bytes read + written.
NCU_TRAFFIC = {("dense_df", 27): 4232672512, ("dense_df", 30): 4232672512 * 8,
               ("dense_oz5", 27): 4267681152, ("dense_oz5", 30): 4267681152 * 8}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=30)
    p.add_argument("--depth", type=int, default=20)
    p.add_argument("--seed", type=int, default=20201127)
    p.add_argument("--fusion", type=int, default=-1, help="-1 autotune, 0 gate by gate, 1..6 width")
    p.add_argument("--math", default="auto", choices=["auto", "fp64", "df"])
    p.add_argument("--tensor", type=int, default=-1,
                   help="tensor-core path mask (2 complex128 double-float, 4 complex64 bf16 slices); -1 = library default")
    p.add_argument("--extras", type=int, default=1, help="also measure unfused, c64, adjoint (rank 0)")
    p.add_argument("--cpu-sample-gates", type=int, default=27, help="gates of the oracle sample timed (<= 90)")
    p.add_argument("--only", default="", choices=["", "batch"],
                   help="profiling aid: time only the batched workload and print its numbers")
    p.add_argument("--batch-count", type=int, default=4096)
    return p.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_PEAK_FALLBACK, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_circuit(args, rank):
    """Each rank simulates its own replica of the workload (its own seed): no data is shared."""
    return W.u3cz_circuit(args.n, args.depth, args.seed + rank)


def max_over_ranks(ms, pg, device):
    """The slowest rank's time (timing only; the one collective of the multi-GPU run)."""
    if pg is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, gates, steps, max_ms):
    """Gates of all replicas per second of the slowest rank."""
    return world * gates * steps / (max_ms / 1e3)


def zz_obs(n):
    return W.PauliObservable(n, np.array([1.0]), np.array([0], dtype=np.uint64), np.array([3], dtype=np.uint64))


# ---------------------------------------------------------------- CPU oracle timing
# One gate mix for both CPU numbers (the cpu_baseline leg and the --impl reference arm): triples
# of two U3 gates and one CZ taken in circuit order (the circuit has 600 U3 and 290 CZ, about 2:1),
# 30 triples (90 gates), applied to a 2^n complex128 state. The cpu_baseline leg times the first
# 9 triples; each step of the reference arm applies the next triple. The per-gate cost does not
# depend on the amplitudes.
ORACLE_SAMPLE = 90


def oracle_sample(circuit, m=ORACLE_SAMPLE):
    u3 = [g for g in circuit.gates if g.name == "U3"]
    cz = [g for g in circuit.gates if g.name == "CZ"]
    out = []
    for t in range(m // 3):
        out += [u3[(2 * t) % len(u3)], u3[(2 * t + 1) % len(u3)], cz[t % len(cz)]]
    return out


def oracle_gates_per_s(n, circuit, n_gates):
    """The oracle (FP64, OpenMP over B(0)) on the first n_gates gates of the sample."""
    import oracle
    psi = oracle.zero_state(n)
    sample = oracle_sample(circuit)[:n_gates]
    t0 = time.perf_counter()
    for g in sample:
        oracle.apply_gate(psi, n, g)
    dt = time.perf_counter() - t0
    names = sorted({g.name for g in sample})
    return len(sample) / dt, oracle.threads(), dt, names


def run_reference(args):
    """The FP64 oracle on the benchmark's workload: each step applies the next triple (two U3,
    one CZ) of the sample, on the host cores."""
    ws, rank, _ = dist()
    if rank != 0:
        return
    import oracle
    circuit = W.u3cz_circuit(args.n, args.depth, args.seed)
    sample = oracle_sample(circuit)
    n = args.n
    psi = oracle.zero_state(n)
    per_step = 3
    rates = []
    gi = 0
    total_t = 0.0
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for _ in range(per_step):
            oracle.apply_gate(psi, n, sample[gi % len(sample)])
            gi += 1
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            rates.append(per_step / dt)
            total_t += dt
    v = len(rates) * per_step / total_t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "gates/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"random U3+CZ brickwork, n={n}, depth={args.depth}, complex128, |0..0>, "
                                   f"fused (autotuned width), then <Z0Z1>",
                       "n": n, "depth": args.depth, "gates": len(circuit.gates), "seed": args.seed},
            "cpu_baseline": {"value": v, "unit": "gates/s", "cores": oracle.threads(), "kind": "oracle",
                             "sample": f"{per_step} gates per step (two U3, one CZ: the circuit's 2:1 mix) from the "
                                       f"{len(sample)}-gate sample of the circuit, on a 2^{n} complex128 state"},
            "e2e": {"value": v, "unit": "gates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def run_ours(args):
    import torch
    import paper_2011_13524_gb300 as qs

    ws, rank, local = dist()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        pg = tdist
    qs.lib()
    # complex128 gate arithmetic: double-float on the FP32 pipes unless FP64 is asked for
    math_mode = {"fp64": qs.QS_MATH_FP64, "df": qs.QS_MATH_DF, "auto": qs.QS_MATH_DF}[args.math]
    qs.set_c128_math(math_mode)
    if args.tensor >= 0:
        qs.set_tensor_cores(args.tensor)
    n, dtype = args.n, qs.QS_C128
    circuit = replica_circuit(args, rank)
    G = len(circuit.gates)
    zz = zz_obs(n)
    stream = torch.cuda.current_stream()

    t_plan0 = time.perf_counter()
    if args.fusion < 0:
        k, pred = qs.autotune_fusion(circuit, dtype)
    else:
        k, pred = args.fusion, None
    plan = qs.FusedCircuit(circuit, k) if k > 0 else qs.FusedCircuit(circuit, 1)
    plan_s = time.perf_counter() - t_plan0
    if k == 0:
        plan = None
    st = qs.State(n, dtype)

    costs = None
    if plan is not None:
        costs = [plan.block_cost(b, dtype) for b in range(plan.n_blocks)]

    def step(timed_blocks=None):
        st.set_basis(0)
        if plan is None:
            for g in circuit.gates:
                st.apply_gate(g)
        elif timed_blocks is not None:
            timed_blocks.append(st.apply_plan_timed(plan))
        else:
            st.apply_plan(plan)
        return st.expectation(zz)[0]

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clocks = Clocks(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    block_times = []
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        result = step(block_times if plan is not None else None)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms, pg, "cuda")
    if pg:
        pg.barrier()
    ms_per_step = ms / args.steps
    value = whole_job_rate(ws, G, args.steps, ms)

    # roofline of the dominant kernel, from the per-block events of the timed steps
    peak, peak_kind = measured_peaks()
    roof = None
    bytes_per_step = None
    kernels_per_step = None
    if plan is not None and block_times:
        bt = np.mean(np.array(block_times), axis=0)
        per_kernel = {}
        for (kname, launches, by), t in zip(costs, bt):
            if launches == 0:
                continue
            d = per_kernel.setdefault(kname, {"ms": 0.0, "bytes": 0.0, "launches": 0})
            d["ms"] += float(t)
            d["bytes"] += by
            d["launches"] += launches
        dom = max(per_kernel, key=lambda k_: per_kernel[k_]["ms"])
        d = per_kernel[dom]
        achieved = d["bytes"] / (d["ms"] / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": NCU_TRAFFIC.get((dom, n)),
                "bytes_per_launch": d["bytes"] / d["launches"], "ms_per_launch": d["ms"] / d["launches"],
                "share_of_step": d["ms"] / ms_per_step,
                "per_kernel_ms": {k_: round(v["ms"], 3) for k_, v in per_kernel.items()}}
        bytes_per_step = sum(c[2] for c in costs)
        kernels_per_step = sum(c[1] for c in costs)
    # separate in-place layout changes of a double-float run (entry and exit, unless folded into
    # the plan's first and last passes; per gate when gates are applied one by one)
    if plan is not None:
        conversions = plan.layout_passes(dtype)
    else:
        conversions = 2 * G if math_mode == qs.QS_MATH_DF else 0
    launches_per_step = (kernels_per_step if kernels_per_step is not None else G) + 1 + 2 + conversions

    # e2e through the public API: host circuit in, host result out, planning included
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 2))
    for _ in range(e2e_steps):
        st.set_basis(0)
        st.run(circuit, args.fusion)
        st.expectation(zz)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    gate_desc = 120 * G  # sizeof(qs_gate) per gate descriptor read by the planner
    wide = 0 if plan is None else sum(16 * (1 << len(plan.block(b)[0])) ** 2 for b in range(plan.n_blocks)
                                       if len(plan.block(b)[0]) >= 4)
    # the same with nothing cached from earlier runs of the circuit: the fusion planner partitions
    # it again for every width the autotuner compares (the autotuner's per-kernel timings of this
    # GPU stay)
    qs.clear_plan_cache()
    t0 = time.perf_counter()
    st.set_basis(0)
    st.run(circuit, args.fusion)
    st.expectation(zz)
    e2e_cold_s = time.perf_counter() - t0
    e2e = {"value": ws * G / e2e_s, "unit": "gates/s", "h2d_bytes_per_step": gate_desc + wide,
           "d2h_bytes_per_step": 16, "wall_ms_per_step": 1e3 * e2e_s,
           "cold": {"value": ws * G / e2e_cold_s, "unit": "gates/s", "wall_ms_per_step": 1e3 * e2e_cold_s,
                    "what": "one step after qs_clear_plan_cache: planning of every width included"}}

    line = {"metric": METRIC, "value": value, "unit": "gates/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if qs.get_c128_math() == qs.QS_MATH_FP64 else "f32x2",
            "data": "synthetic",
            "config": {"workload": f"random U3+CZ brickwork, n={n}, depth={args.depth}, complex128, |0..0>, "
                                   f"fused (autotuned width), then <Z0Z1>",
                       "n": n, "depth": args.depth, "gates": G, "seed": args.seed, "fusion_k": k,
                       "autotune_pred_ms": pred, "plan_blocks": None if plan is None else plan.n_blocks,
                       "l2": "state 16 GiB > 129 MB L2 (no flush needed)", "replicas": ws},
            "roofline": roof, "e2e": e2e, "clocks": clk, "gpu_launches": launches_per_step * args.steps,
            "result_z0z1": result, "plan_ms": 1e3 * plan_s}
    if bytes_per_step is not None:
        line["state_gbps"] = bytes_per_step / (ms_per_step / 1e3) / 1e9
        line["state_frac_hbm"] = line["state_gbps"] / peak

    if rank == 0 and ws == 1:
        extras = {}
        if args.extras:
            del st
            torch.cuda.empty_cache()
            extras = measure_extras(args, qs, torch, circuit)
        line["extras"] = extras
        rate, cores, dt, names = oracle_gates_per_s(n, circuit, args.cpu_sample_gates)
        line["cpu_baseline"] = {"value": rate, "unit": "gates/s", "cores": cores, "kind": "oracle",
                                "sample": f"the first {args.cpu_sample_gates} gates ({'/'.join(names)}; two U3 and one "
                                          f"CZ per triple, the circuit's 2:1 mix) of the {ORACLE_SAMPLE}-gate sample "
                                          f"of the circuit, applied to a 2^{n} complex128 state, {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()


def measure_extras(args, qs, torch, circuit):
    """Secondary numbers of the same run: unfused per-gate rate, complex64, adjoint gradient."""
    out = {}
    n = args.n
    G = len(circuit.gates)
    stream = torch.cuda.current_stream()

    def timed(fn, reps=1):
        fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    st = qs.State(n, qs.QS_C128)
    ms = timed(lambda: (st.set_basis(0), st.run(circuit, 0)))
    out["c128_unfused_gates_per_s"] = G / (ms / 1e3)
    # the same circuit fused on the CUDA cores (double-float, tensor cores off) and with plain
    # FP64 arithmetic, each at its own autotuned width
    old_tc, old_math = qs.get_tensor_cores(), qs.get_c128_math()
    for label, tc, math_mode in (("c128_df_cuda_cores", 0, qs.QS_MATH_DF), ("c128_fp64", 0, qs.QS_MATH_FP64)):
        qs.set_tensor_cores(tc)
        qs.set_c128_math(math_mode)
        kk, _ = qs.autotune_fusion(circuit, qs.QS_C128)
        pl = qs.FusedCircuit(circuit, max(kk, 1))
        ms = timed(lambda: (st.set_basis(0), st.apply_plan(pl)))
        out[label + "_gates_per_s"] = G / (ms / 1e3)
        out[label + "_fusion_k"] = kk
        # rows per thread of the shared-memory dense kernel the autotuner timed and kept, per width
        out[label + "_tile_rows"] = {m: qs.dense_tile_rows(qs.QS_C128, m)[0] for m in (4, 5, 6)}
    qs.set_tensor_cores(old_tc)
    qs.set_c128_math(old_math)
    del st
    torch.cuda.empty_cache()
    st = qs.State(n, qs.QS_C64)
    k64, _ = qs.autotune_fusion(circuit, qs.QS_C64)
    plan64 = qs.FusedCircuit(circuit, max(k64, 1))
    ms = timed(lambda: (st.set_basis(0), st.apply_plan(plan64) if k64 else st.run(circuit, 0)), reps=2)
    out["c64_fused_gates_per_s"] = G / (ms / 1e3)
    out["c64_fusion_k"] = k64
    # fused width 6 on the tensor cores (bf16 slices, exact FP32 sums) and on the FP32 CUDA cores
    old_tc = qs.get_tensor_cores()
    plan6 = qs.FusedCircuit(circuit, 6)
    for tc in (qs.QS_TENSOR_C64X, 0):
        qs.set_tensor_cores(tc)
        if not tc:  # the CUDA-core tile shapes timed by the autotuner
            qs.autotune_fusion(circuit, qs.QS_C64)
            out["c64_cuda_cores_tile_rows"] = {m: qs.dense_tile_rows(qs.QS_C64, m)[0] for m in (5, 6)}
        ms6 = timed(lambda: (st.set_basis(0), st.apply_plan(plan6)), reps=2)
        out["c64_k6_%s_gates_per_s" % ("tensor" if tc else "cuda_cores")] = G / (ms6 / 1e3)
    qs.set_tensor_cores(old_tc)
    ms = timed(lambda: (st.set_basis(0), st.run(circuit, 0)))
    out["c64_unfused_gates_per_s"] = G / (ms / 1e3)
    del st
    torch.cuda.empty_cache()
    # adjoint: n = 20 hardware-efficient ansatz, 20 layers, H = sum ZZ + sum X, complex128
    hea = W.hea_circuit(20, 20, args.seed)
    H = W.tfim_observable(20, 1.0)
    qs.adjoint_grad(hea, H)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e, g = qs.adjoint_grad(hea, H)
    out["adjoint_ms_n20_l20_c128"] = 1e3 * (time.perf_counter() - t0)
    out["adjoint_params"] = int(hea.n_params)
    # batch: 4096 HEA circuits, n ~ U{8..20}, 2..12 layers, 4-term Pauli observables, complex64,
    # energies + adjoint gradients, one persistent launch replayed from a CUDA graph
    items = W.batch_workload(args.batch_count, args.seed)
    b = qs.Batch([i.circuit for i in items], [i.observable for i in items])
    theta = np.concatenate([i.circuit.parameters() for i in items])
    b.run(theta, use_graph=True)
    reps = 3
    t0 = time.perf_counter()
    for _ in range(reps):
        b.run(theta, use_graph=True)
    dt = (time.perf_counter() - t0) / reps
    out["batch_circuits_per_s"] = args.batch_count / dt
    out["batch_ms"] = 1e3 * dt
    out["batch_params"] = b.total_params
    out["batch_workspace_gib"] = b.workspace_bytes / 2**30
    peak, _ = measured_peaks()
    out["batch_roofline"] = {"bound": "hbm", "achieved": b.traffic_bytes / dt / 1e9, "peak": peak, "unit": "GB/s",
                             "frac": b.traffic_bytes / dt / 1e9 / peak, "bytes_per_run": b.traffic_bytes,
                             "note": "psi/lambda passes of the circuits wider than 13 qubits; the narrower "
                                     "ones run in shared memory (latency-bound, no HBM traffic)"}
    del b
    # precision: the same circuit as complex64 and complex128 (double-float) on the GPU, n = 30;
    # max-abs amplitude difference, 1 - fidelity and the transverse-field Ising energy (h = 1)
    a = qs.State(n, qs.QS_C128)
    a.run(circuit, 2)
    c = qs.State(n, qs.QS_C64)
    c.run(circuit, 4)
    tf = W.tfim_observable(n, 1.0)
    e128 = a.expectation(tf)[0]
    e64 = c.expectation(tf)[0]
    d = (a.tensor - c.tensor.to(torch.complex128)).abs().max().item()
    ov = torch.vdot(a.tensor, c.tensor.to(torch.complex128)).abs().item() ** 2
    out["precision_n30"] = {"max_abs_c64_vs_c128": d, "one_minus_fidelity": 1.0 - ov / (a.norm2() * c.norm2()),
                            "tfim_energy_c128": e128, "tfim_energy_err_c64": abs(e64 - e128),
                            "norm2_c64": c.norm2(), "norm2_c128": a.norm2()}
    # Pauli expectation of that Ising chain (2n - 1 terms, n + 1 flip-mask groups): tiled reads,
    # each evaluating every group whose flip mask lies in its tile, double-float arithmetic
    masks, single = qs.expectation_plan(n, tf)
    reads = len(masks) + single
    groups = len(set(int(x) for x in tf.x_mask))
    for label, stt, S in (("c128", a, 16), ("c64", c, 8)):
        ms = timed(lambda: stt.expectation(tf), reps=3)
        out["tfim_expectation_n30_%s_ms" % label] = ms
        out["tfim_expectation_n30_%s_read_gbps" % label] = reads * S * 2.0 ** n / (ms / 1e3) / 1e9
    out["tfim_expectation_n30_reads"] = reads
    out["tfim_expectation_n30_groups"] = groups
    del a, c
    torch.cuda.empty_cache()
    # the comparison circuit of Sec. 7 (RZ RX RZ layers, CNOT ring, 10 repetitions), n = 30,
    # complex128 at the autotuned width
    cc = W.rzrxrz_cnot_circuit(n, 10, args.seed)
    kc, _ = qs.autotune_fusion(cc, qs.QS_C128)
    plc = qs.FusedCircuit(cc, max(kc, 1))
    stc = qs.State(n, qs.QS_C128)
    ms = timed(lambda: (stc.set_basis(0), stc.apply_plan(plc)))
    out["comparison_circuit_gates"] = len(cc.gates)
    out["comparison_circuit_fusion_k"] = kc
    out["comparison_circuit_blocks"] = plc.n_blocks
    out["comparison_circuit_gates_per_s"] = len(cc.gates) / (ms / 1e3)
    del stc
    torch.cuda.empty_cache()
    # Pauli rotation of an n-qubit X/Y/Z string (one pass over amplitude pairs), and one Trotter
    # slice of the transverse-field Ising chain (2n - 1 Pauli rotations), complex128 double-float
    stp = qs.State(n, qs.QS_C128)
    xm = sum(1 << q for q in range(n) if q % 3 != 2)
    zm = sum(1 << q for q in range(n) if q % 3 != 0)
    ms = timed(lambda: stp.apply_pauli_rotation(xm, zm, 0.3), reps=3)
    out["pauli_rotation_call_n30_ms"] = ms  # one public call: includes the double-float layout passes
    tf = W.tfim_observable(n, 1.0)
    ms = timed(lambda: stp.apply_observable_rotation(tf, 0.1, 1))
    out["tfim_trotter_slice_n30_ms"] = ms
    out["pauli_rotation_in_trotter_n30_gbps"] = tf.n_terms * 2 * 16 * 2.0 ** n / (ms / 1e3) / 1e9
    del stp
    torch.cuda.empty_cache()
    # analysis calls at n = 30 complex128: transition amplitude of the TFIM observable between two
    # states, and 100000 Z-basis samples (uniforms from the seeded generator)
    sa, sb = qs.State(n, qs.QS_C128), qs.State(n, qs.QS_C128)
    sa.run(W.u3cz_circuit(n, 4, args.seed + 1), 4)
    sb.run(W.u3cz_circuit(n, 4, args.seed + 2), 4)
    ms = timed(lambda: sa.transition_amplitude(tf, sb))
    out["transition_amplitude_tfim_n30_ms"] = ms
    rng = W.SplitMix64(args.seed)
    uni = np.array([rng.uniform() for _ in range(100000)])
    t0 = time.perf_counter()
    sb.sample(uni)
    out["sample_1e5_n30_ms"] = 1e3 * (time.perf_counter() - t0)
    del sa, sb
    torch.cuda.empty_cache()
    # a commuting (IQP-like) circuit: H layers around 20 diagonal layers, n = 30 complex128
    ci = W.iqp_circuit(n, 20, args.seed)
    ki, _ = qs.autotune_fusion(ci, qs.QS_C128)
    pli = qs.FusedCircuit(ci, max(ki, 1))
    sti = qs.State(n, qs.QS_C128)
    ms = timed(lambda: (sti.set_basis(0), sti.apply_plan(pli)))
    out["iqp_circuit_gates"] = len(ci.gates)
    out["iqp_circuit_fusion_k"] = ki
    out["iqp_circuit_blocks"] = pli.n_blocks
    out["iqp_circuit_gates_per_s"] = len(ci.gates) / (ms / 1e3)
    del sti
    torch.cuda.empty_cache()
    # n = 33 complex128 (128 GiB state), same circuit family at depth 20, autotuned width
    try:
        c33 = W.u3cz_circuit(33, args.depth, args.seed)
        s33 = qs.State(33, qs.QS_C128)
        k33, _ = qs.autotune_fusion(c33, qs.QS_C128)
        plan33 = qs.FusedCircuit(c33, max(k33, 1))
        out["c128_n33_fusion_k"] = k33
        ms33 = timed(lambda: (s33.set_basis(0), s33.apply_plan(plan33)))
        out["c128_n33_gates_per_s"] = len(c33.gates) / (ms33 / 1e3)
        out["c128_n33_ms"] = ms33
        del s33
    except Exception as e:  # not enough free device memory on this GPU
        out["c128_n33_error"] = str(e)[:200]
    torch.cuda.empty_cache()
    return out


def batch_shard(args, rank, ws):
    """The 4096-pair batch workload, split across ranks by cost (every rank computes the same
    split); this rank's (indices, items)."""
    from paper_2011_13524_gb300 import shard
    items = W.batch_workload(args.batch_count, args.seed)
    parts = shard.split([shard.pair_cost(i.circuit) for i in items], ws)
    idx = parts[rank]
    return idx, [items[i] for i in idx], len(items)


def run_batch_only(args):
    """The batched workload alone: each rank evaluates its share of the pairs (split by cost, no
    data exchanged), the results are gathered on rank 0, which prints one JSON line."""
    import torch
    import paper_2011_13524_gb300 as qs
    from paper_2011_13524_gb300 import shard
    ws, rank, local = dist()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        pg = tdist
    idx, items, count = batch_shard(args, rank, ws)
    b = qs.Batch([i.circuit for i in items], [i.observable for i in items])
    theta = np.concatenate([i.circuit.parameters() for i in items])
    for _ in range(args.warmup):
        b.run(theta, use_graph=True)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e, g = b.run(theta, use_graph=True)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.steps
    dt = max_over_ranks(1e3 * dt, pg, "cuda") / 1e3
    e_all, g_all = shard.gather(pg, count, idx, e, g)
    traffic = b.traffic_bytes
    if pg:
        t = torch.tensor([traffic], device="cuda", dtype=torch.float64)
        pg.all_reduce(t)
        traffic = float(t.item())
    peak, peak_kind = measured_peaks()
    if rank == 0:
        print(json.dumps({"batch_circuits": count, "ranks": ws, "batch_ms": 1e3 * dt,
                          "batch_circuits_per_s": count / dt, "passes_rank0": b.total_passes,
                          "energies_finite": bool(np.all(np.isfinite(e_all))),
                          "roofline": {"bound": "hbm", "achieved": traffic / dt / 1e9 / ws, "peak": peak,
                                       "unit": "GB/s per GPU", "frac": traffic / dt / 1e9 / ws / peak,
                                       "peak_source": peak_kind,
                                       "bytes_per_run": traffic,
                                       "note": "psi/lambda traffic of the circuits wider than 13 qubits; "
                                               "narrower ones run in shared memory"}}), flush=True)
    if pg:
        pg.destroy_process_group()


def main():
    args = parse()
    if args.only == "batch":
        run_batch_only(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
