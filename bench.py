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

# Algorithmic flops per element of the two hexahedral element kernels, 27-point rule: the
# per-point cost of a direct evaluation of the formulas (geometry and fields ~600 flops, residual
# ~300, tangent blocks K_vv ~1.7k + K_vp ~0.4k + fine-coupled blocks ~0.5k) plus the condensation
# (~7k flops per element). The kernels execute fewer flops than these counts where their
# formulation needs fewer; `executed` gives ncu opcode counts (FMA = 2 flops) on the 32^3 cavity:
# the FP64 residual's line-factored monomial form 8,614, the FP64 tangent's factorised sums 41,472,
# the fused kernel's FP64 part (residual + the tangent's FP64 K_ff work) 9,066, the tetrahedral
# kernel 5,894 (21^3 tetrahedral cavity).
ALG_FLOPS = {"residual": (600 + 300) * 27, "tangent": (600 + 1700 + 400 + 500) * 27 + 7000}
EXECUTED_FLOPS = {"residual": 8_614, "tangent_fp64": 41_472, "fused_fp64": 9_066, "tet": 5_894}

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from ncu captures of the
# current kernels on the named workloads (profiles/); no entry where none was taken.
NCU_TRAFFIC_BYTES = {("fused", "cavity32_re400_mixed"): 68_553_472 + 34_592_256,
                     ("fused", "channel_re1000_mixed"): 2_074_687_744 + 3_088_019_200,
                     ("residual", "cavity32_re400_fp64"): 4_223_232 + 0,
                     ("tangent", "cavity32_re400_fp64"): 119_540_480 + 101_472_512,
                     ("tangent", "tetcavity21_re400_mixed"): 15_459_584 + 27_136}

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
DEFAULT_WORKLOAD = "channel_re1000_mixed"
# the library's precision modes (VMS_PREC_*)
PREC_NAMES = {0: "fp64", 1: "mixed", 2: "tc_bf16", 3: "tc_tf32"}
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
def _oracle_chunk(job):
    """One oracle work unit (runs in a worker process): element residuals and tangents,
    condensation and CSR assembly of a chunk of elements into a partial system."""
    import oracle
    from oracle import Params
    conn, xyz, u, beta, u_prev, nu, dt, tet = job
    p = Params(nu=nu, dt=dt, element="tet" if tet else "hex")
    X, U, b, Up = oracle.gather(conn, xyz, u, beta, u_prev)
    k = oracle.element_kernel(X, U, b, p, Up)
    S, r, _, _ = oracle.condense(*oracle.pack_element(k))
    return oracle.assemble(conn, xyz.shape[0], S, r)


def _oracle_sample(wl, n):
    """The first n elements of the workload as a mesh of their own (nodes renumbered in order of
    first use, Dirichlet dofs restricted to those nodes): the oracle's inputs for a bounded sample."""
    conn = wl.mesh.conn[:n]
    used, inv = np.unique(conn, return_inverse=True)
    local = np.full(wl.mesh.n_nodes, -1, np.int64)
    local[used] = np.arange(used.size)
    dofs = wl.bc.dofs[local[wl.bc.dofs // 4] >= 0]
    return {"conn": inv.reshape(conn.shape).astype(np.int32), "xyz": wl.mesh.xyz[used],
            "u": wl.u[used], "beta": wl.beta[:n],
            "u_prev": None if wl.u_prev is None else wl.u_prev[used],
            "dofs": 4 * local[dofs // 4] + dofs % 4, "nu": wl.nu, "dt": wl.dt,
            "tet": wl.mesh.conn.shape[1] == 4}


def _oracle_jobs(smp, parts):
    n = smp["conn"].shape[0]
    cuts = np.linspace(0, n, parts + 1).astype(int)
    return [(smp["conn"][cuts[i]:cuts[i + 1]], smp["xyz"], smp["u"], smp["beta"][cuts[i]:cuts[i + 1]],
             smp["u_prev"], smp["nu"], smp["dt"], smp["tet"]) for i in range(parts) if cuts[i + 1] > cuts[i]]


def _oracle_run(pool, smp, parts):
    """Seconds of one oracle assembly of a sample (_oracle_sample): the element chunks on the
    pool's workers, the partial systems summed and the Dirichlet rows applied in this process."""
    import oracle
    jobs = _oracle_jobs(smp, parts)
    t0 = time.perf_counter()
    out = pool.map(_oracle_chunk, jobs)
    A, rhs = out[0]
    for Ai, ri in out[1:]:
        A = A + Ai
        rhs = rhs + ri
    oracle.apply_dirichlet(A, rhs, smp["dofs"])
    return time.perf_counter() - t0


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_baseline(wl, target_s=8.0, cores=None):
    """The FP64 oracle (as it stands) timed on the host's cores: one worker process, then one per
    core, on the same first elements of the workload's mesh (sized so that the one-worker run
    takes about target_s). Workers are spawned processes with one math-library thread each."""
    import multiprocessing as mp
    cores = cores or os.cpu_count() or 1
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"
    ctx = mp.get_context("spawn")
    try:
        with ctx.Pool(1) as pool:
            _oracle_run(pool, _oracle_sample(wl, min(64, wl.mesh.n_elems)), 1)  # start-up
            n0 = min(512, wl.mesh.n_elems)
            t0 = _oracle_run(pool, _oracle_sample(wl, n0), 1)
            n = int(min(wl.mesh.n_elems, max(n0, n0 * target_s / max(t0, 1e-6))))
            smp = _oracle_sample(wl, n)
            t1 = _oracle_run(pool, smp, 1)
        with ctx.Pool(cores) as pool:
            _oracle_run(pool, _oracle_sample(wl, min(64 * cores, wl.mesh.n_elems)), cores)
            tc = _oracle_run(pool, smp, 4 * cores)
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return {"elements": n, "one_core_s": t1, "all_cores_s": tc, "one_core": n / t1,
            "all_cores": n / tc, "cores": cores, "cpu": cpu_model()}


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
    """The oracle as the reference arm: each step is one oracle assembly (element kernels,
    condensation, CSR assembly, Dirichlet rows) of a bounded sample of the workload's elements, in
    element chunks on one spawned worker process per host core."""
    ws, rank, local = dist_setup()
    if rank != 0:
        return
    import multiprocessing as mp
    wl, prec, batch = make_workload(args.workload, with_batch=True)
    cores = os.cpu_count() or 1
    # bounded sample: about 64 x per_step x steps oracle element evaluations in all
    per_step = max(64, min(args.ref_sample, 400_000 // max(args.steps, 1)))
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    times = []
    n = min(per_step, wl.mesh.n_elems)
    smp = _oracle_sample(wl, n)
    with mp.get_context("spawn").Pool(cores) as pool:
        _oracle_run(pool, _oracle_sample(wl, min(64 * cores, wl.mesh.n_elems)), cores)
        for _ in range(args.warmup):
            _oracle_run(pool, smp, 4 * cores)
        for _ in range(args.steps):
            times.append(_oracle_run(pool, smp, 4 * cores))
    value = n * len(times) / sum(times)
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
    sample = (f"first {n} elements of the mesh per step, numpy FP64 oracle in {4 * cores} chunks on "
              f"{cores} worker processes ({cpu_model()})")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.workload, wl, prec, batch),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "newton": newton,
    }
    print(json.dumps(line), flush=True)


NEWTON_METRIC = "wall time per Newton solve to 1e-8 rel"


def newton_timing(vms, wl, prec, device, stream, rtol=1e-8, repeats=2, maxit=30):
    """Wall time of vms_newton_solve from the workload's initial state to ||R|| <= rtol ||R^0||:
    host clock around the call with the device synchronised on both sides (`value`), and around
    the upload of the initial state from host arrays, the solve and the download of the solution
    to host arrays (`host_to_host_s`); one untimed solve first builds the ILU(0) pattern and the
    Krylov work space. Medians over the repeats."""
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
                "precision": PREC_NAMES[prec], "failed": str(e)}
    times, h2h, its, hist, stats = [], [], 0, None, (0, 0)
    u_out = np.empty((wl.mesh.n_nodes, 4))
    b_out = np.empty((wl.mesh.n_elems, 3))
    for _ in range(repeats):
        torch.cuda.synchronize(device)
        ctx.solver_stats(reset=True)
        th = time.perf_counter()
        ctx.state_upload(wl.u, wl.beta, wl.u_prev)   # host arrays
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        its, hist = ctx.newton_solve(rtol=rtol, maxit=maxit)
        torch.cuda.synchronize(device)
        t1 = time.perf_counter()
        u_out[...], b_out[...] = ctx.state_download()  # back to host arrays
        h2h.append(time.perf_counter() - th)
        times.append(t1 - t0)
        stats = ctx.solver_stats(reset=True)
    # one more solve, untimed, with the library's per-kind CUDA-event accounting: where the time goes
    ctx.state_upload(wl.u, wl.beta, wl.u_prev)
    ctx.profile_enable(True)
    ctx.profile_read(reset=True)
    ctx.newton_solve(rtol=rtol, maxit=maxit)
    prof = ctx.profile_read(reset=True)
    ctx.profile_enable(False)
    ctx.close()
    profile = {k: {"ms": round(ms, 3), "launches": n} for k, (ms, n) in prof.items() if n}
    return {"metric": NEWTON_METRIC.replace("1e-8", f"{rtol:g}"), "value": float(np.median(times)),
            "unit": "s", "higher_is_better": False, "precision": PREC_NAMES[prec],
            "host_to_host_s": float(np.median(h2h)),
            "newton_iterations": int(its), "linear_solves": int(stats[0]),
            "krylov_iterations": int(stats[1]), "final_rel": float(hist[-1] / hist[0]),
            "krylov": "GMRES(150), block ILU(0) right preconditioner, inexact Newton",
            "repeats": repeats, "times": [round(t, 4) for t in times],
            "profile": profile, "profile_note": "one further solve with per-kind CUDA events on the "
            "library's streams (ms summed over the solve; 'precond' is the ILU(0) factorisation and "
            "its sweeps)"}


def warmstart_study(vms, ctx, wl, args, dev):
    """Backward-Euler steps from rest: record args.ws_train steps (previous-step start), train the
    network, then run the next args.ws_eval steps twice from the same state: previous-step start
    and learned start; Newton to the same absolute target (1e-8 of the previous-step start's
    residual) in both. A failed Newton solve ends that run and is reported."""
    import torch
    from paper_0809_4802_gb300 import transient as tr

    def log(s):
        print(f"warm-start study: step {s.step} newton {s.newton_iterations} krylov {s.krylov_iterations} "
              f"{s.seconds:.2f} s {s.error}", file=sys.stderr, flush=True)

    def summary(st):
        ok = [s for s in st if s.newton_iterations >= 0]
        return {"steps": len(ok), "failed_steps": len(st) - len(ok),
                "newton_iterations": int(sum(s.newton_iterations for s in ok)),
                "krylov_iterations": int(sum(s.krylov_iterations for s in ok)),
                "wall_s": float(sum(s.seconds for s in st)),
                "newton_per_step": [s.newton_iterations for s in st],
                "errors": [s.error for s in st if s.error],
                "start_residual_ratio_mean": (float(np.mean([s.start_residual / s.reference_residual for s in ok]))
                                              if ok else None)}

    ctx.set_graph(False)
    ctx.state_upload(wl.u, wl.beta, wl.u_prev)
    rec = tr.Recorder()
    t0 = time.perf_counter()
    recorded = tr.run_steps(vms, ctx, args.ws_train, rtol=1e-8, record=rec, log=log)
    t_record = time.perf_counter() - t0
    out = {"steps_recorded": args.ws_train, "record_wall_s": t_record, "recording": summary(recorded)}
    if any(s.newton_iterations < 0 for s in recorded):
        out["note"] = "a Newton solve of the recorded steps failed; no network trained"
        return out
    u, beta = ctx.state_download()
    up = ctx.state_download_prev()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ws = tr.WarmStart(vms, dev.index or 0, seed=7)
    loss = ws.fit(rec, epochs=args.ws_epochs, batch=4096, lr=2e-3)
    torch.cuda.synchronize(dev)
    t_train = time.perf_counter() - t0
    base = tr.run_steps(vms, ctx, args.ws_eval, rtol=1e-8, first_step=args.ws_train, log=log)
    ctx.state_upload(u, beta, up)
    learned = tr.run_steps(vms, ctx, args.ws_eval, rtol=1e-8, warm=ws, first_step=args.ws_train, log=log)
    ws.mlp.close()
    out.update({"steps_evaluated": args.ws_eval, "train_wall_s": t_train, "train_epochs": args.ws_epochs,
                "final_loss": loss, "previous_step_start": summary(base), "learned_start": summary(learned),
                "newton_iterations_saved": summary(base)["newton_iterations"] - summary(learned)["newton_iterations"],
                "note": "warm start applied to the velocity; Newton to the same absolute target"})
    return out


def workload_config(name, wl, prec, batch=None):
    c = {"workload": name, "elements": wl.mesh.n_elems, "nodes": wl.mesh.n_nodes,
         "reynolds": round(1.0 / wl.nu, 3), "dt": wl.dt, "precision": PREC_NAMES[prec],
         "quad_points": 27, "l2": "flushed between timed steps (256 MB write)"}
    if batch is not None:
        edges = [int(round(w.mesh.n_elems ** (1 / 3))) for w in batch.members]
        c.update(instances=len(batch.members), reynolds="per instance, U[100, 1000]",
                 edge_counts={str(k): edges.count(k) for k in sorted(set(edges))})
    return c


def measured_peaks(vms, dev_index):
    """FP64 and FP32 FMA throughput of this GPU, measured by the library's probe kernel (best of
    three launches each; FP32 is the better of scalar and packed FMA), with the SM clock sampled
    during the probe."""
    with ClockSampler(dev_index) as clk:
        fp64 = vms.fma_throughput(dev_index, 0)
        fp32 = max(vms.fma_throughput(dev_index, 1), vms.fma_throughput(dev_index, 2))
    c = clk.summary()
    return {"fp64_tflops": fp64, "fp32_tflops": fp32, "sm_mhz": c.get("sm_mhz"),
            "source": "measured: vms_fma_throughput (independent FMA chains, CUDA events)"}


def timed_assembly(ctx, stream, steps, flush, barrier, dev):
    """CUDA-event time (ms, summed) of `steps` assemblies with device-resident inputs, the L2
    flushed before each; the library's launch counts over the same region."""
    import torch
    ctx.profile_read(reset=True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    barrier()
    for k in range(steps):
        flush.zero_()
        starts[k].record(stream)
        ctx.assemble()
        ends[k].record(stream)
    barrier()
    counts = ctx.profile_read(reset=True)
    return sum(s.elapsed_time(e) for s, e in zip(starts, ends)), int(sum(v[1] for v in counts.values()))


def kernel_times(ctx, steps, flush):
    """Per-kernel-kind milliseconds per launch, from the library's own CUDA events around each
    launch on the stream it is launched on (residual: the context's stream; tangent: its second
    stream), over `steps` assemblies."""
    ctx.profile_enable(True)
    ctx.profile_read(reset=True)   # launch counts of earlier, untimed calls must not enter the mean
    for _ in range(steps):
        flush.zero_()
        ctx.assemble()
    prof = ctx.profile_read(reset=True)
    ctx.profile_enable(False)
    return {k: v[0] / v[1] for k, v in prof.items() if v[1] > 0}


def roofline_entries(kern, E, prec, tet, peaks, workload):
    """One roofline entry per element kernel: algorithmic flops per launch / its event time."""
    out = []
    if tet:
        ms = kern["tangent"]
        fpe = EXECUTED_FLOPS["tet"]
        out.append({"bound": "alu", "kernel": "tet_assembly", "pipe": "fp64", "unit": "TFLOP/s",
                    "flops_per_element": fpe, "flops": "executed (ncu opcode counts; no algorithmic count is stated for the tetrahedron)",
                    "ms": ms, "achieved": fpe * E / (ms * 1e-3) / 1e12, "peak": peaks["fp64_tflops"],
                    "traffic": NCU_TRAFFIC_BYTES.get(("tangent", workload))})
    else:
        if "fused" in kern:
            # one launch holds both element kernels: its FP64 (residual) and FP32 (tangent) work
            # are each set against their own pipe's peak over the launch's duration
            ms = kern["fused"]
            for name, pipe, part in (("residual", "fp64", "FP64 residual work"),
                                     ("tangent", "fp32", "FP32 tangent work")):
                fpe = ALG_FLOPS[name]
                out.append({"bound": "alu", "kernel": "fused_assembly", "pipe": pipe, "unit": "TFLOP/s",
                            "part": part, "flops_per_element": fpe,
                            "executed_flops_per_element": EXECUTED_FLOPS["fused_fp64"] if pipe == "fp64" else None,
                            "ms": ms, "achieved": fpe * E / (ms * 1e-3) / 1e12,
                            "peak": peaks["fp64_tflops"] if pipe == "fp64" else peaks["fp32_tflops"],
                            "traffic": NCU_TRAFFIC_BYTES.get(("fused", workload))})
        for name, pipe in (("residual", "fp64"), ("tangent", "fp32" if prec != 0 else "fp64")):
            if name not in kern:
                continue
            ms = kern[name]
            fpe = ALG_FLOPS[name]
            exe = EXECUTED_FLOPS.get(name if name == "residual" else ("tangent_fp64" if prec == 0 else ""))
            out.append({"bound": "alu", "kernel": name, "pipe": pipe, "unit": "TFLOP/s",
                        "flops_per_element": fpe, "executed_flops_per_element": exe,
                        "ms": ms, "achieved": fpe * E / (ms * 1e-3) / 1e12,
                        "peak": peaks["fp64_tflops"] if pipe == "fp64" else peaks["fp32_tflops"],
                        "traffic": NCU_TRAFFIC_BYTES.get((name, workload))})
    for r in out:
        r["frac"] = r["achieved"] / r["peak"]
        r["ms"] = round(r["ms"], 4)
        r["peak_source"] = peaks["source"]
    return out


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
        prec = {"mixed": 1, "fp64": 0, "tc_bf16": 2, "tc_tf32": 3}[args.precision]
    mesh = wl.mesh
    E = mesh.n_elems
    tet = mesh.conn.shape[1] == 4
    stream = torch.cuda.current_stream(dev)
    peaks = measured_peaks(vms, local)

    def make_ctx(p):
        c = vms.Context(local, p)
        c.set_stream(stream.cuda_stream)
        c.mesh_upload(mesh.xyz, mesh.conn, wl.bc.dofs, wl.bc.vals)
        c.set_params(wl.nu, dt=wl.dt, scatter_mode=args.scatter)
        if batch is not None:
            c.set_element_viscosity(batch.nu_e)
            c.set_instances(batch.node_offsets, batch.elem_offsets)
        c.state_upload(wl.u, wl.beta, wl.u_prev)
        return c

    ctx = make_ctx(prec)
    tuning = None
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
    with ClockSampler(local) as clk:
        ms, gpu_launches = timed_assembly(ctx, stream, args.steps, flush, barrier, dev)
    ms = max_over_ranks(ms)
    value = ws * E * args.steps / (ms / 1000.0)

    # ---- the other kernel schedule of the mixed step (two kernels on two streams), for reference ----
    schedules = None
    if prec == 1 and not tet and batch is None and args.scatter == 0:
        ctx.set_tuning(schedule=vms.SCHEDULE_TWO_STREAMS)
        for _ in range(2):
            ctx.assemble()
        ms_two, _ = timed_assembly(ctx, stream, args.steps, flush, barrier, dev)
        ctx.set_tuning(schedule=vms.SCHEDULE_FUSED)
        ctx.assemble()
        schedules = {"fused_ms_per_step": ms / args.steps, "two_streams_ms_per_step": ms_two / args.steps}

    # ---- per-kernel times (events inside the library, on each kernel's stream) ----
    kern = kernel_times(ctx, args.steps, flush)
    entries = roofline_entries(kern, E, prec, tet, peaks, args.workload)
    # the dominant kernel: the largest share of the step's device time (the ncu launch list): the
    # fused residual + tangent kernel in mixed precision (its FP64 part, the binding pipe; with two
    # kernels on two streams the FP64 residual), the tangent in FP64, the single assembly kernel of
    # the tetrahedron. Every kernel's own entry is in `kernels`.
    kinds = [r["kernel"] for r in entries]
    dom_name = ("tet_assembly" if tet else "tangent" if prec == 0 else
                "fused_assembly" if "fused_assembly" in kinds else "residual")
    roofline = dict(next(r for r in entries if r["kernel"] == dom_name))
    roofline["kernels"] = entries
    roofline["kernel_ms"] = {k: round(v, 4) for k, v in kern.items()}
    roofline["concurrent"] = (
        "one persistent kernel runs the residual (FP64) and the tangent (FP32) warps side by side; "
        "its time is its own launch-to-completion in the step" if "fused" in kern else
        "one kernel per element pass" if tet else
        "residual (context stream) and tangent (second stream) overlap in the step; each time is "
        "that kernel's own launch-to-completion in the step")

    # ---- end to end through the C-ABI: host state in, assembled system (values + rhs) out ----
    u_host = torch.from_numpy(np.ascontiguousarray(wl.u)).pin_memory()
    beta_host = torch.from_numpy(np.ascontiguousarray(wl.beta)).pin_memory()
    u_prev_host = (torch.from_numpy(np.ascontiguousarray(wl.u_prev)).pin_memory()
                   if wl.u_prev is not None else None)
    view = ctx.csr()
    vals_host = torch.empty(view.nnz, dtype=torch.float32 if view.values_dtype == 1 else torch.float64).pin_memory()
    rhs_host = torch.empty(view.n_rows, dtype=torch.float64).pin_memory()
    # a pipeline of K steps: the download of step k (device snapshot, then a copy stream) runs
    # beside the upload and assembly of step k + 1; the timed region ends when the last
    # download has landed in host memory
    ctx.assemble()
    ctx.csr_download_async(values=vals_host, rhs=rhs_host)   # untimed: allocates the staging buffer
    ctx.csr_download_wait()
    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize(dev)
    # host clock per loop step and per call (the assembly call returns when its kernels are done;
    # the download call first waits for the previous step's copy to the host)
    host_ms, asm_ms, dl_ms = np.zeros(args.steps), np.zeros(args.steps), np.zeros(args.steps)
    e_start.record(stream)
    for k in range(args.steps):
        t_k = time.perf_counter()
        flush.zero_()
        ctx.state_upload(u_host, beta_host, u_prev_host)
        t_a = time.perf_counter()
        ctx.assemble()
        t_d = time.perf_counter()
        ctx.csr_download_async(values=vals_host, rhs=rhs_host)
        t_e = time.perf_counter()
        host_ms[k], asm_ms[k], dl_ms[k] = (t_e - t_k) * 1e3, (t_d - t_a) * 1e3, (t_e - t_d) * 1e3
    ctx.csr_download_wait()
    e_end.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    e_ms = max_over_ranks(e_start.elapsed_time(e_end))
    e2e = {"value": ws * E * args.steps / (e_ms / 1000.0), "unit": UNIT,
           "h2d_bytes_per_step": int(u_host.numel() * 8 + beta_host.numel() * 8
                                     + (u_prev_host.numel() * 8 if u_prev_host is not None else 0)),
           "d2h_bytes_per_step": int(vals_host.numel() * vals_host.element_size() + rhs_host.numel() * 8),
           "path": "per step: vms_state_upload (pinned host) + vms_assemble_newton_schur + "
                   "vms_csr_download_async (CSR values and right-hand side to pinned host, overlapping "
                   "the next step); the timed region ends after vms_csr_download_wait of the last step",
           "host_ms_per_step": {name: {"p50": round(float(np.median(v)), 3),
                                       "p99": round(float(np.percentile(v, 99)), 3),
                                       "max": round(float(v.max()), 3)}
                                for name, v in (("step", host_ms), ("assemble_call", asm_ms),
                                                ("download_call", dl_ms))}}
    ctx.close()
    del vals_host

    # ---- the same mesh in the other precision (FP64 beside mixed) ----
    other = None
    if not args.skip_other_precision:
        oprec = 1 if prec == 0 else 0
        c2 = make_ctx(oprec)
        for _ in range(2):
            c2.assemble()
        k2 = max(3, min(args.steps, 10))
        ms2, _ = timed_assembly(c2, stream, k2, flush, barrier, dev)
        kern2 = kernel_times(c2, 2, flush)
        other = {"precision": PREC_NAMES[oprec], "steps": k2,
                 "value": E * k2 / (max_over_ranks(ms2) / 1000.0), "unit": UNIT,
                 "ms_per_step": ms2 / k2,
                 "roofline": roofline_entries(kern2, E, oprec, tet, peaks, args.workload)}
        c2.close()

    # ---- the tensor-core modes of the tangent's contractions on the same mesh (hexahedra) ----
    tensor_core = None
    if prec == 1 and not tet and batch is None and not args.skip_other_precision:
        tensor_core = {}
        for tp in (2, 3):
            c3 = make_ctx(tp)
            for _ in range(2):
                c3.assemble()
            k3 = max(3, min(args.steps, 10))
            ms3, _ = timed_assembly(c3, stream, k3, flush, barrier, dev)
            kern3 = kernel_times(c3, 2, flush)
            tensor_core[PREC_NAMES[tp]] = {
                "value": E * k3 / (max_over_ranks(ms3) / 1000.0), "unit": UNIT, "steps": k3,
                "ms_per_step": ms3 / k3, "tangent_ms": round(kern3.get("tangent", 0.0), 4),
                "residual_ms": round(kern3.get("residual", 0.0), 4),
                "schedule": "residual and tensor-core tangent kernels on two streams"}
            c3.close()

    # ---- wall time per Newton solve: the 32^3 jittered cavity (mixed and plain FP64, to 1e-8)
    # and the 8^3 cavity (FP64, to 1e-10); the large workloads' solves take minutes each ----
    newton = None
    if args.newton == "on" or (args.newton == "auto" and WORKLOADS[args.workload].get("kind") != "warmstart"
                               and batch is None):
        nw = args.workload if (args.workload.startswith("cavity") or args.workload.startswith("tetcavity")) \
            else "cavity32_re400_mixed"
        nwl, nprec = make_workload(nw)
        newton = newton_timing(vms, nwl, nprec, local, stream.cuda_stream)
        newton["workload"] = nw
        o = newton_timing(vms, nwl, 1 - nprec, local, stream.cuda_stream)
        newton["other_precision"] = {k: o.get(k) for k in ("precision", "value", "host_to_host_s", "newton_iterations",
                                                           "krylov_iterations", "final_rel", "failed")}
        small, _ = make_workload("cavity8_re100_fp64")
        newton["cavity8_re100_fp64_to_1e-10"] = {
            k: v for k, v in newton_timing(vms, small, 0, local, stream.cuda_stream, rtol=1e-10,
                                           repeats=3).items()
            if k in ("value", "host_to_host_s", "unit", "newton_iterations", "krylov_iterations", "final_rel")}
        if newton["value"] is not None:
            newton["value"] = max_over_ranks(newton["value"])

    # ---- transient: learned warm start against the previous-step start ----
    warm = None
    if WORKLOADS[args.workload].get("kind") == "warmstart":
        ctx = make_ctx(prec)
        warm = warmstart_study(vms, ctx, wl, args, dev)
        ctx.close()

    # ---- batch: one linear solve per instance (the first inexact-Newton system, eta = 1e-2) ----
    per_instance = None
    if batch is not None:
        ctx = make_ctx(prec)
        ctx.set_preconditioner(vms.PRECOND_ILU0_FALLBACK)
        ctx.assemble()
        times, iters, iters_all, fails, direct, direct_ms = [], [], [], 0, 0, []
        for i in range(len(batch.members)):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            try:
                it, _ = ctx.solve_instance(i, rtol=1e-2, maxit=3000, restart=150, update=False)
                iters.append(it)
            except vms.VmsError:
                it = None
                fails += 1
            times.append(time.perf_counter() - t0)
            iters_all.append(it)
            if it is not None and it >= 3000:   # the Krylov attempt stopped at maxit: fallback solve
                direct += 1
                direct_ms.append(times[-1] * 1e3)
        ctx.close()
        ms_i = np.array(times) * 1e3
        per_instance = {"metric": "per-instance linear solve time (first Newton system, rtol 1e-2)",
                        "unit": "ms", "instances": len(times), "failures": fails,
                        "median": float(np.median(ms_i)), "p90": float(np.percentile(ms_i, 90)),
                        "max": float(ms_i.max()), "total": float(ms_i.sum()),
                        "krylov_iterations_median": float(np.median(iters)) if iters else None,
                        "fallback_solves": direct,
                        "fallback_ms": [round(t, 1) for t in direct_ms],
                        "slowest": [{"instance": int(k), "nodes": int(batch.node_offsets[k + 1] - batch.node_offsets[k]),
                                     "krylov_iterations": iters_all[k], "ms": round(float(ms_i[k]), 1)}
                                    for k in np.argsort(ms_i)[::-1][:4]],
                        "note": "instance 0's time includes the ILU(0) factorisation of the whole merged matrix",
                        "solver": "FP32 GMRES(150) + FP64 refinement, block ILU(0) (FP64-eliminated, FP32 sweeps); "
                                  "a solve that reaches maxit is repeated by a banded LU with partial pivoting "
                                  "(FP64, on the device) (VMS_PRECOND_ILU0_FALLBACK)"}

    cpu = None
    if rank == 0 and not args.skip_cpu_baseline:
        src = batch.members[0] if batch is not None else wl
        ob = oracle_baseline(src, target_s=args.cpu_seconds)
        what = "the first instance" if batch is not None else args.workload
        cpu = {"value": ob["one_core"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": (f"first {ob['elements']} elements of {what}: numpy FP64 oracle assembly "
                          f"(element kernels, condensation, CSR assembly, Dirichlet rows), "
                          f"{ob['one_core_s']:.1f} s on one core of {ob['cpu']}"),
               "all_cores": {"value": ob["all_cores"], "cores": ob["cores"], "seconds": ob["all_cores_s"],
                             "how": "the same elements in 4 chunks per core on spawned worker processes, "
                                    "partial systems summed"},
               "cpu": ob["cpu"]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec != 0 else "f64", "data": "synthetic",
            "config": workload_config(args.workload, wl, prec, batch),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "other_precision": other, "schedules": schedules, "tensor_core": tensor_core,
            "newton": newton,
            "scatter": "colour" if args.scatter == 1 else "atomic",
            "tuning": tuning, "graph": bool(batch is not None or args.graph),
            "per_instance_solve": per_instance, "warm_start": warm,
            "peaks": peaks, "gpu_launches": gpu_launches, "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--precision", choices=["mixed", "fp64", "tc_bf16", "tc_tf32"], default=None)
    ap.add_argument("--scatter", type=int, choices=[0, 1], default=0)
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--skip-other-precision", action="store_true",
                    help="do not time the same mesh in the other precision mode")
    ap.add_argument("--cpu-seconds", type=float, default=8.0)
    ap.add_argument("--ref-sample", type=int, default=8192)
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
