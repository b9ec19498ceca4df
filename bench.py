"""Benchmark: elements/s of the Newton-Schur tangent assembly on GB300.

One step = one vms_assemble_newton_schur call over the whole mesh: gather, quadrature-point
geometry and fields, FP64 residual, tangent blocks, Schur condensation of the bubble unknowns,
scatter-add into the CSR system and the Dirichlet rows/columns. The CSR pattern is built once per
mesh, outside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

Multi-GPU (torchrun): every rank assembles its own copy of the workload (independent problems, no
collective on the data path); `value` sums the elements over ranks and divides by the slowest
rank's time (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "elements/s Newton-Schur tangent assembly"  # plus "newton": wall time per Newton solve
UNIT = "elements/s"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")

# FP64 peak of the GB300: 152 SMs x 2 FP64 FMA lanes per clock x 2 flops x 2.07 GHz (maximum SM
# clock) = 1.259 TFLOP/s (the nominal 1.25 TFLOP/s FP64 figure); FP32: 152 x 128 x 2 x 2.07 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12

# Executed FP64 flops per element (FMA = 2, add/mul = 1) of each kernel as implemented, 27-point
# rule, from ncu's per-opcode counts on the 32^3 cavity (sass__thread_inst_executed_true_per_opcode
# divided by the 32,768 elements): residual 5,967 DFMA + 1,759 DMUL + 1,098 DADD; FP64 tangent
# 51,034 DFMA + 15,673 DMUL + 11,956 DADD; tetrahedral kernel below.
FP64_FLOPS_PER_ELEM = {
    "residual": 14_791,
    "tangent_fp64": 129_697,
    # tetrahedral assembly kernel (one kernel: residual, tangent, condensation, scatter from the
    # reference moments, four lanes per element): 2,316 DFMA + 1,432 DMUL + 534 DADD per element
    # (ncu thread-instruction counts on the 21^3 Kuhn cavity, 55,566 elements)
    "tet": 5_866,
}

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of the
# same workload (profiles/residual_kernel_cavity32_re400.md,
# profiles/tet_assembly_kernel_tetcavity21_re400.md); None where not captured for the current
# kernel.
NCU_TRAFFIC_BYTES = {("residual", "cavity32_re400_mixed"): 4_203_776,
                     ("residual", "cavity32_re400_fp64"): 4_203_776,
                     # profiles/tet_assembly_kernel_tetcavity21_re400.md
                     ("tangent", "tetcavity21_re400_mixed"): 20_044_288}

WORKLOADS = {
    # the 32^3 jittered lid-driven cavity at Re 400, random state (mixed precision by default)
    "cavity32_re400_mixed": dict(n=32, re=400.0, jitter=0.15, state="random", seed=1002, prec=1),
    "cavity32_re400_fp64": dict(n=32, re=400.0, jitter=0.15, state="random", seed=1002, prec=0),
    # the 8^3 cavity at Re 100 (small case)
    "cavity8_re100_fp64": dict(n=8, re=100.0, jitter=0.0, state="noise", seed=1001, prec=0),
    "cavity16_re400_fp64": dict(n=16, re=400.0, jitter=0.15, state="random", seed=1002, prec=0),
    "cavity16_re400_mixed": dict(n=16, re=400.0, jitter=0.15, state="random", seed=1002, prec=1),
    # backward-facing step, h = 1/13: 518,492 elements, Re 800, rest state with parabolic inflow
    "bfs_re800_mixed": dict(kind="bfs", prec=1),
    "bfs_re800_fp64": dict(kind="bfs", prec=0),
    # channel past a cube, 300x56x56 lattice: 937,860 elements, Re 1000, backward Euler dt 0.01
    "channel_re1000_mixed": dict(kind="channel", prec=1),
    # serving-style mix: 64 jittered cavities, edges drawn from {8,12,16,24,32,48}, Re ~ U[100,1000],
    # random states, one merged mesh (1,677,504 elements) assembled per CUDA-graph launch, autotuned
    "batch64_mixed": dict(kind="batch", prec=1),
    # tetrahedral P1 + bubble cavities sized like the paper's Table 1 meshes (fine DOF = 3 x
    # elements): 39^3 Kuhn lattice, 355,914 elements (mesh E: 353,719); 21^3, 55,566 (mesh A:
    # 55,763); jittered 0.15 h, Re 400, random state
    "tetcavity39_re400_mixed": dict(kind="tet", n=39, re=400.0, jitter=0.15, state="random", seed=1002, prec=1),
    "tetcavity39_re400_fp64": dict(kind="tet", n=39, re=400.0, jitter=0.15, state="random", seed=1002, prec=0),
    "tetcavity21_re400_mixed": dict(kind="tet", n=21, re=400.0, jitter=0.15, state="random", seed=1002, prec=1),
    # transient runs with the learned warm start: a decaying vortex in a closed, jittered box
    # (--ws-n cells per edge), and the channel past a cube (--ws-nx, --ws-nyz; its systems carry
    # the nearly singular equal-order pressure modes of the hexahedral element, on which
    # GMRES + ILU(0) stalls, see the design notes)
    "vortex_warmstart_fp64": dict(kind="warmstart", flow="vortex", prec=0),
    "channel_warmstart_mixed": dict(kind="warmstart", flow="channel", prec=1),
}
DEFAULT_WORKLOAD = "cavity32_re400_mixed"
WS_SIZE = {"nx": 150, "nyz": 28, "n": 16}   # set from --ws-nx / --ws-nyz / --ws-n


def make_workload(name, with_batch=False):
    from paper_0809_4802_gb300 import inputs
    w = WORKLOADS[name]
    kind = w.get("kind", "cavity")
    batch = None
    if kind == "batch":
        batch = inputs.batched_workload(64, seed=1004)
        wl = batch.work
    elif kind == "bfs":
        wl = inputs.bfs_workload(13, re=800.0, jitter_frac=0.1, seed=1003)
    elif kind == "channel":
        wl = inputs.channel_workload(300, 56, re=1000.0, dt=0.01, seed=1005)
    elif kind == "tet":
        wl = inputs.tet_cavity_workload(w["n"], re=w["re"], jitter_frac=w["jitter"], state=w["state"],
                                        seed=w["seed"])
    elif kind == "warmstart" and w["flow"] == "channel":
        wl = inputs.channel_workload(WS_SIZE["nx"], WS_SIZE["nyz"], re=1000.0, dt=0.01, seed=1005)
    elif kind == "warmstart":
        wl = inputs.vortex_box_workload(WS_SIZE["n"], re=200.0, dt=0.02, jitter_frac=0.1)
    else:
        wl = inputs.cavity_workload(w["n"], re=w["re"], jitter_frac=w["jitter"], state=w["state"],
                                    seed=w["seed"])
    if with_batch:
        return wl, w["prec"], batch
    return wl, w["prec"]


# ----------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.p = None
        self.path = f"/tmp/vms_clocks_{os.getpid()}.csv"

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[4:]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = np.array([r[0] for r in rows])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[3][1:]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(rows[0][1]),
                "power_w_max": float(max(r[2] for r in rows)), "samples": len(rows),
                "reasons": reasons}


# ----------------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the same workload
# ----------------------------------------------------------------------------------------------
def oracle_assembly_rate(wl, target_s=10.0, max_elems=None):
    """Elements/s of the oracle's assembly (element kernel, condensation, CSR assembly, Dirichlet)
    on the first elements of the workload's mesh, sized to take about target_s seconds."""
    import oracle
    from oracle import Params
    mesh = wl.mesh
    p = Params(nu=wl.nu, dt=wl.dt, element="tet" if mesh.conn.shape[1] == 4 else "hex")
    beta = wl.beta

    def run(n):
        t0 = time.perf_counter()
        X, U, b, Up = oracle.gather(mesh.conn[:n], mesh.xyz, wl.u, beta[:n], wl.u_prev)
        k = oracle.element_kernel(X, U, b, p, Up)
        S, r, _, _ = oracle.condense(*oracle.pack_element(k))
        A, rhs = oracle.assemble(mesh.conn[:n], mesh.n_nodes, S, r)
        oracle.apply_dirichlet(A, rhs, wl.bc.dofs)
        return time.perf_counter() - t0

    n0 = min(256, mesh.n_elems)
    t0 = run(n0)
    n = int(min(mesh.n_elems if max_elems is None else max_elems,
                max(n0, n0 * target_s / max(t0, 1e-6))))
    t = run(n)
    return n / t, n, t


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float) -> float:
    """The slowest rank's value (the benchmark's time is the maximum over ranks); x itself when
    torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reference_arm(args):
    ws, rank, local = dist_setup()
    if rank != 0:
        return
    wl, prec = make_workload(args.workload)
    # bounded sample: about 150k oracle elements in total (~45 s on one core), at least 64 a step
    per_step = max(64, min(args.ref_sample, 150_000 // max(args.steps, 1)))
    for _ in range(args.warmup):
        oracle_assembly_rate(wl, target_s=0.0, max_elems=64)
    rates = []
    t_total = 0.0
    for _ in range(args.steps):
        rate, n, t = oracle_assembly_rate(wl, target_s=0.0, max_elems=per_step)
        rates.append(rate)
        t_total += t
    value = float(np.mean(rates))
    newton = None
    if args.newton != "off":
        import oracle
        small, _ = make_workload("cavity8_re100_fp64")
        t0 = time.perf_counter()
        _, _, norms = oracle.newton_solve(small.mesh.xyz, small.mesh.conn, small.u, small.beta,
                                          small.bc.dofs, oracle.Params(nu=small.nu), tol=1e-10,
                                          maxit=20)
        newton = {"metric": "wall time per Newton solve to 1e-10 rel", "value": time.perf_counter() - t0,
                  "unit": "s", "workload": "cavity8_re100_fp64", "newton_iterations": len(norms) - 1,
                  "final_rel": norms[-1] / norms[0],
                  "linear_solver": "scipy sparse direct solve (oracle)"}
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * t_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.workload, wl, prec, None),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"first {per_step} elements of the mesh per step (numpy FP64 oracle)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "newton": newton,
    }
    print(json.dumps(line), flush=True)


NEWTON_METRIC = "wall time per Newton solve to 1e-8 rel"


def newton_timing(vms, wl, prec, device, stream, rtol=1e-8, repeats=2, maxit=30):
    """Wall time of vms_newton_solve from the workload's initial state to ||R|| <= rtol ||R^0||:
    host clock around the call with the device synchronised on both sides; the state is uploaded
    again (outside the timed region) before each repeat; one untimed solve first builds the
    ILU(0) pattern and the Krylov work space. Median over the repeats."""
    import torch
    ctx = vms.Context(device, prec)
    ctx.set_stream(stream)
    ctx.mesh_upload(wl.mesh.xyz, wl.mesh.conn, wl.bc.dofs, wl.bc.vals)
    ctx.set_params(wl.nu, dt=wl.dt)
    ctx.state_upload(wl.u, wl.beta, wl.u_prev)
    try:
        ctx.newton_solve(rtol=rtol, maxit=maxit)
    except vms.VmsError as e:
        ctx.close()
        return {"metric": NEWTON_METRIC.replace("1e-8", f"{rtol:g}"), "value": None, "unit": "s",
                "precision": "mixed" if prec == 1 else "fp64", "failed": str(e)}
    times, its, hist, stats = [], 0, None, (0, 0)
    for _ in range(repeats):
        ctx.state_upload(wl.u, wl.beta, wl.u_prev)
        torch.cuda.synchronize(device)
        ctx.solver_stats(reset=True)
        t0 = time.perf_counter()
        its, hist = ctx.newton_solve(rtol=rtol, maxit=maxit)
        torch.cuda.synchronize(device)
        times.append(time.perf_counter() - t0)
        stats = ctx.solver_stats(reset=True)
    ctx.close()
    return {"metric": NEWTON_METRIC.replace("1e-8", f"{rtol:g}"), "value": float(np.median(times)),
            "unit": "s", "higher_is_better": False, "precision": "mixed" if prec == 1 else "fp64",
            "newton_iterations": int(its), "linear_solves": int(stats[0]),
            "krylov_iterations": int(stats[1]), "final_rel": float(hist[-1] / hist[0]),
            "krylov": "GMRES(150), block ILU(0) right preconditioner, inexact Newton",
            "repeats": repeats, "times": [round(t, 4) for t in times]}


def warmstart_study(vms, ctx, wl, args, dev):
    """Backward-Euler steps from rest: record args.ws_train steps (previous-step start), train the
    network, then run the next args.ws_eval steps twice from the same state: previous-step start
    and learned start; Newton to the same absolute target (1e-8 of the previous-step start's
    residual) in both."""
    import torch
    from paper_0809_4802_gb300 import transient as tr
    ctx.set_graph(False)
    ctx.state_upload(wl.u, wl.beta, wl.u_prev)
    rec = tr.Recorder()
    t0 = time.perf_counter()
    tr.run_steps(vms, ctx, args.ws_train, rtol=1e-8, record=rec)
    t_record = time.perf_counter() - t0
    u, beta = ctx.state_download()
    up = ctx.state_download_prev()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ws = tr.WarmStart(vms, dev.index or 0, seed=7)
    loss = ws.fit(rec, epochs=args.ws_epochs, batch=4096, lr=2e-3)
    torch.cuda.synchronize(dev)
    t_train = time.perf_counter() - t0
    base = tr.run_steps(vms, ctx, args.ws_eval, rtol=1e-8, first_step=args.ws_train)
    ctx.state_upload(u, beta, up)
    learned = tr.run_steps(vms, ctx, args.ws_eval, rtol=1e-8, warm=ws, first_step=args.ws_train)
    ws.mlp.close()

    def summary(st):
        return {"newton_iterations": int(sum(s.newton_iterations for s in st)),
                "krylov_iterations": int(sum(s.krylov_iterations for s in st)),
                "wall_s": float(sum(s.seconds for s in st)),
                "start_residual_ratio_mean": float(np.mean([s.start_residual / s.reference_residual for s in st]))}
    return {"steps_recorded": args.ws_train, "steps_evaluated": args.ws_eval,
            "record_wall_s": t_record, "train_wall_s": t_train, "train_epochs": args.ws_epochs,
            "final_loss": loss, "previous_step_start": summary(base), "learned_start": summary(learned),
            "newton_iterations_saved": summary(base)["newton_iterations"] - summary(learned)["newton_iterations"],
            "note": "warm start applied to the velocity; Newton to the same absolute target"}


def workload_config(name, wl, prec, scatter, batch=None):
    c = {"workload": name, "elements": wl.mesh.n_elems, "nodes": wl.mesh.n_nodes,
         "reynolds": round(1.0 / wl.nu, 3), "dt": wl.dt, "precision": "mixed" if prec == 1 else "fp64",
         "quad_points": 27, "l2": "flushed between timed steps (256 MB write)"}
    if batch is not None:
        edges = [int(round(w.mesh.n_elems ** (1 / 3))) for w in batch.members]
        c.update(instances=len(batch.members), reynolds="per instance, U[100, 1000]",
                 edge_counts={str(k): edges.count(k) for k in sorted(set(edges))})
    if scatter is not None:
        c["scatter"] = "colour" if scatter == 1 else "atomic"
    return c


def ours(args):
    import torch
    ws, rank, local = dist_setup()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    from paper_0809_4802_gb300 import build as vbuild, vms
    if rank == 0 or ws == 1:
        vbuild.build()
    if ws > 1:
        torch.distributed.barrier()
    vms.load_library()

    wl, prec, batch = make_workload(args.workload, with_batch=True)
    if args.precision is not None:
        prec = {"mixed": 1, "fp64": 0}[args.precision]
    mesh = wl.mesh
    E = mesh.n_elems
    stream = torch.cuda.current_stream(dev)
    ctx = vms.Context(local, prec)
    ctx.set_stream(stream.cuda_stream)
    ctx.mesh_upload(mesh.xyz, mesh.conn, wl.bc.dofs, wl.bc.vals)
    ctx.set_params(wl.nu, dt=wl.dt, scatter_mode=args.scatter)
    tuning = None
    if batch is not None:
        ctx.set_element_viscosity(batch.nu_e)
        ctx.set_instances(batch.node_offsets, batch.elem_offsets)
    u_host = torch.from_numpy(np.ascontiguousarray(wl.u)).pin_memory()
    beta_host = torch.from_numpy(np.ascontiguousarray(wl.beta)).pin_memory()
    u_prev_host = (torch.from_numpy(np.ascontiguousarray(wl.u_prev)).pin_memory()
                   if wl.u_prev is not None else None)
    ctx.state_upload(wl.u, wl.beta, wl.u_prev)
    if batch is not None or args.autotune:
        tuning = ctx.autotune(repeats=3)
    if batch is not None or args.graph:
        ctx.set_graph(True)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        ctx.assemble()
    barrier()

    # ---- timed region: device-resident inputs ----
    ctx.profile_read(reset=True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        barrier()
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            ctx.assemble()
            ends[k].record(stream)
        barrier()
    counts = ctx.profile_read(reset=True)
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    gpu_launches = int(sum(v[1] for v in counts.values()))
    ms = max_over_ranks(ms)
    value = ws * E * args.steps / (ms / 1000.0)

    # ---- per-kernel times (events inside the library, same stream) for the roofline ----
    ctx.profile_enable(True)
    for _ in range(args.steps):
        flush.zero_()
        ctx.assemble()
    prof = ctx.profile_read(reset=True)
    ctx.profile_enable(False)
    kern = {k: v for k, v in prof.items() if v[1] > 0}
    # the kernel on the FP64 critical path: the residual in mixed precision (the FP32 tangent runs
    # beside it on a second stream), the tangent in FP64 mode
    tet = mesh.conn.shape[1] == 4
    dom = "tangent" if (tet or prec == 0) else "residual"
    dom_ms = kern[dom][0] / kern[dom][1]
    key = "tet" if tet else ("residual" if dom == "residual" else "tangent_fp64")
    fpe = FP64_FLOPS_PER_ELEM.get(key)
    achieved = fpe * E / (dom_ms / 1000.0) / 1e12 if fpe else None
    roofline = {"bound": "alu", "kernel": "tet_assembly" if tet else dom, "achieved": achieved,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS if achieved else None,
                "traffic": NCU_TRAFFIC_BYTES.get((dom, args.workload)),
                "pipe": "fp64", "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 x 2.07 GHz",
                "flops_per_element": fpe,
                "concurrent": "residual (stream 1) and tangent (stream 2) overlap; times are in situ",
                "kernel_ms": {k: round(v[0] / v[1], 4) for k, v in kern.items()}}

    # ---- end to end through the C-ABI with host buffers ----
    rhs_host = torch.empty(4 * mesh.n_nodes, dtype=torch.float64).pin_memory()
    e_starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e_ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    barrier()
    for k in range(args.steps):
        flush.zero_()
        e_starts[k].record(stream)
        ctx.state_upload(u_host, beta_host, u_prev_host)
        view = ctx.assemble()
        rhs_dev = ctx.csr_device(view)[3]
        rhs_host.copy_(rhs_dev, non_blocking=True)
        e_ends[k].record(stream)
    barrier()
    e_ms = sum(s.elapsed_time(e) for s, e in zip(e_starts, e_ends))
    e_ms = max_over_ranks(e_ms)
    e2e = {"value": ws * E * args.steps / (e_ms / 1000.0), "unit": UNIT,
           "h2d_bytes_per_step": int(u_host.numel() * 8 + beta_host.numel() * 8
                                     + (u_prev_host.numel() * 8 if u_prev_host is not None else 0)),
           "d2h_bytes_per_step": int(rhs_host.numel() * 8)}

    # ---- wall time per Newton solve (same mesh and initial state; mixed and plain FP64) ----
    newton = None
    if args.newton == "on" or (args.newton == "auto" and (args.workload.startswith("cavity")
                                                          or args.workload.startswith("tetcavity"))):
        newton = newton_timing(vms, wl, prec, local, stream.cuda_stream)
        other = newton_timing(vms, wl, 1 - prec, local, stream.cuda_stream)
        newton["other_precision"] = {k: other.get(k) for k in ("precision", "value", "newton_iterations",
                                                               "krylov_iterations", "final_rel", "failed")}
        small, _ = make_workload("cavity8_re100_fp64")
        newton["cavity8_re100_fp64_to_1e-10"] = {
            k: v for k, v in newton_timing(vms, small, 0, local, stream.cuda_stream, rtol=1e-10,
                                           repeats=3).items()
            if k in ("value", "unit", "newton_iterations", "krylov_iterations", "final_rel")}
        if newton["value"] is not None:
            newton["value"] = max_over_ranks(newton["value"])

    # ---- transient: learned warm start against the previous-step start ----
    warm = None
    if WORKLOADS[args.workload].get("kind") == "warmstart":
        warm = warmstart_study(vms, ctx, wl, args, dev)

    # ---- batch: one linear solve per instance (the first inexact-Newton system, eta = 1e-2) ----
    per_instance = None
    if batch is not None:
        ctx.assemble()
        times, iters, fails = [], [], 0
        for i in range(len(batch.members)):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            try:
                it, _ = ctx.solve_instance(i, rtol=1e-2, maxit=3000, restart=150, update=False)
                iters.append(it)
            except vms.VmsError:
                fails += 1
            times.append(time.perf_counter() - t0)
        ms_i = np.array(times) * 1e3
        per_instance = {"metric": "per-instance linear solve time (first Newton system, rtol 1e-2)",
                        "unit": "ms", "instances": len(times), "failures": fails,
                        "median": float(np.median(ms_i)), "p90": float(np.percentile(ms_i, 90)),
                        "max": float(ms_i.max()), "total": float(ms_i.sum()),
                        "krylov_iterations_median": float(np.median(iters)) if iters else None,
                        "solver": "FP32 GMRES(150) + FP64 refinement, block ILU(0) (FP64-eliminated, FP32 sweeps)"}

    cpu = None
    if rank == 0 and not args.skip_cpu_baseline:
        src = batch.members[0] if batch is not None else wl
        rate, n, t = oracle_assembly_rate(src, target_s=args.cpu_seconds)
        what = "of the first instance" if batch is not None else f"of {E}"
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {n} elements {what}, numpy FP64 oracle assembly ({t:.1f} s)"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == 1 else "f64", "data": "synthetic",
            "config": workload_config(args.workload, wl, prec, args.scatter, batch),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "newton": newton,
            "tuning": tuning, "graph": bool(batch is not None or args.graph),
            "per_instance_solve": per_instance, "warm_start": warm,
            "gpu_launches": gpu_launches, "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default=None)
    ap.add_argument("--scatter", type=int, choices=[0, 1], default=0)
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-sample", type=int, default=2048)
    ap.add_argument("--autotune", action="store_true", help="autotune launch shapes first")
    ap.add_argument("--ws-n", type=int, default=16)
    ap.add_argument("--ws-nx", type=int, default=150)
    ap.add_argument("--ws-nyz", type=int, default=28)
    ap.add_argument("--ws-train", type=int, default=100)
    ap.add_argument("--ws-eval", type=int, default=200)
    ap.add_argument("--ws-epochs", type=int, default=60)
    ap.add_argument("--graph", action="store_true", help="replay the assembly as a CUDA graph")
    ap.add_argument("--newton", choices=["auto", "on", "off"], default="auto",
                    help="also time Newton solves to 1e-8 (auto: on for the cavity workloads)")
    args = ap.parse_args()
    WS_SIZE.update(nx=args.ws_nx, nyz=args.ws_nyz, n=args.ws_n)
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        reference_arm(args)
    else:
        ours(args)


if __name__ == "__main__":
    main()
