"""Backward-Euler time stepping with the Newton-Schur solver (Remark of Section 4.1: the transient
term; Section 4.2: Newton) and the learned warm start.

Step n -> n+1 on a context whose state holds u^n and u^{n-1}:
  1. features of u^n, d = u^n - u^{n-1} and the 1-ring mean of d (vms_node_features), if a
     network is used or the step is recorded for training;
  2. u_prev <- u^n (vms_shift_time); the reference residual r_ref is the residual at u^n;
  3. start: u^n (previous-step start) or u^n + network(features) (vms_apply_increment);
  4. Newton until ||R|| <= rtol * r_ref (vms_newton_solve_to): the same target for every start;
  5. if recorded: the training target u^{n+1} - u^n (vms_node_increment).
Every arithmetic step runs in the library's kernels; this module only sequences the calls and
keeps the recorded device buffers.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class StepStats:
    step: int
    newton_iterations: int
    krylov_iterations: int
    start_residual: float     # ||R|| at the starting point of Newton
    reference_residual: float  # ||R|| at the previous-step start
    seconds: float
    error: str = ""            # the library's error message of a failed Newton solve


@dataclass
class Recorder:
    X: list = field(default_factory=list)   # device float32 (n_nodes, 12) per recorded step
    D: list = field(default_factory=list)   # device float32 (n_nodes, 4)


class WarmStart:
    """The network and the feature / target scales it was trained with.

    By default (apply_pressure=False) the network is trained with zero pressure targets and the
    warm start moves the velocity only, keeping the previous step's pressure: on distorted meshes
    the step-to-step pressure increments are dominated by the near-null pressure modes of the
    condensed system (RMS 357 against 0.03 for the velocity on a jittered 6^3 vortex box), which
    no network predicts and which would corrupt the start."""

    def __init__(self, vms, device: int = 0, seed: int = 7, stream=None, apply_pressure=False):
        self.apply_pressure = apply_pressure
        from . import inputs
        self.vms = vms
        self.mlp = vms.Mlp(device)
        if stream is not None:
            self.mlp.set_stream(stream)
        self.mlp.set_params(inputs.mlp_init(seed))
        self.scale_in = np.ones(12, np.float32)
        self.scale_out = np.ones(4, np.float32)

    def fit(self, rec: Recorder, epochs: int = 30, batch: int = 1024, lr: float = 2e-3,
            seed: int = 11):
        """Set the scales from the recorded data (column RMS, floored) and train with Adam on
        shuffled minibatches of nodes from every recorded step. Returns the final loss."""
        import torch
        Xs = torch.cat(rec.X)   # device copies of the recorded steps, scaled in place below
        Ds = torch.cat(rec.D)
        sx = np.maximum(self.mlp.column_rms(Xs), 1e-6).astype(np.float32)
        sd = np.maximum(self.mlp.column_rms(Ds), 1e-9).astype(np.float32)
        mul_d = 1.0 / sd
        if not self.apply_pressure:
            sd[3] = 0.0      # the start keeps the previous step's pressure
            mul_d[3] = 0.0   # and the network is trained on zero pressure targets
        self.scale_in = sx
        self.scale_out = sd
        self.mlp.scale_columns(Xs, 1.0 / sx, Xs)
        self.mlp.scale_columns(Ds, mul_d, Ds)
        n = Xs.shape[0]
        rng = np.random.Generator(np.random.PCG64(seed))
        for _ in range(epochs):
            perm = torch.from_numpy(rng.permutation(n).astype(np.int32)).to(Xs.device)
            for b0 in range(0, n, batch):
                rows = perm[b0:b0 + batch]
                self.mlp.grad(Xs, Ds, rows=rows, want=False)
                self.mlp.adam(lr)
        loss, _ = self.mlp.grad(Xs, Ds)
        return loss


def run_steps(vms, ctx, n_steps: int, rtol: float = 1e-8, warm: WarmStart | None = None,
              record: Recorder | None = None, maxit: int = 20, first_step: int = 0, log=None):
    """Advance n_steps backward-Euler steps; returns a StepStats per step. A step whose Newton
    solve fails ends the run: its StepStats has newton_iterations = -1 and it is the last one.
    `log`, if given, is called with each step's StepStats."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    n = ctx.n_nodes
    X = torch.empty((n, 12), dtype=torch.float32, device=dev)
    Y = torch.empty((n, 4), dtype=torch.float32, device=dev)
    out = []
    for k in range(n_steps):
        t0 = time.perf_counter()
        if warm is not None or record is not None:
            ctx.node_features(X, None if warm is None else warm.scale_in)
            if record is not None:
                record.X.append(X.clone())
        ctx.shift_time()
        r_ref = ctx.residual()
        if warm is not None:
            warm.mlp.forward(X, Y)
            ctx.apply_increment(Y, warm.scale_out)
        r_start = ctx.residual()
        ctx.solver_stats(reset=True)
        try:
            its, hist = ctx.newton_solve_to(rtol * r_ref, maxit=maxit)
        except vms.VmsError as err:
            _, kits = ctx.solver_stats(reset=True)
            torch.cuda.synchronize(dev)
            out.append(StepStats(first_step + k + 1, -1, kits, r_start, r_ref, time.perf_counter() - t0,
                                 str(err)))
            if log is not None:
                log(out[-1])
            break
        _, kits = ctx.solver_stats(reset=True)
        if record is not None:
            ctx.node_increment(Y)
            record.D.append(Y.clone())
        torch.cuda.synchronize(dev)
        out.append(StepStats(first_step + k + 1, its, kits, r_start, r_ref, time.perf_counter() - t0))
        if log is not None:
            log(out[-1])
    return out
