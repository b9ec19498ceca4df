"""Parity at the full sizes of the step channel, the channel past a cube, the batch of 64 cavities
and the 39^3 tetrahedral cavity, on sampled outputs, through the C-ABI.

Each mesh is assembled at full size in mixed precision, the mode of its benchmark line, with a
random flow state, so that the convective and fine-scale terms are exercised. Three windows of
elements (the first, the last, one at random) are compared block by block with the FP64 oracle.
Sampled CSR rows and right-hand-side entries are compared with the oracle's assembly of the
elements that touch those rows; a row receives contributions from no other element.

Tolerances, relative to the largest entry of the compared block, as in test_gpu_assembly and
test_gpu_tet:
  hexahedra, mixed: 1e-5 for S_e, r_e and the FP32 CSR values; 1e-10 for the FP64 residual R_cp;
  tetrahedra: 1e-10 for S_e, r_e and R_cp (FP64 in both modes); 1e-6 for the FP32 CSR values.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle import Params
from paper_0809_4802_gb300 import inputs

pytestmark = pytest.mark.gpu

MIXED = 1


@pytest.fixture(scope="module")
def vms():
    from paper_0809_4802_gb300 import build, vms as v
    build.build()
    v.load_library()
    return v


def relerr(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def random_state(wl, seed, scale=0.5):
    """Uniform random velocities and pressures with the workload's Dirichlet values imposed, and
    random bubble coefficients."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(-scale, scale, (wl.mesh.n_nodes, 4))
    inputs.impose(u, wl.bc)
    beta = rng.uniform(-0.05, 0.05, (wl.mesh.n_elems, 3))
    return u, beta, rng


def oracle_blocks(conn, xyz, u, beta, p, u_prev=None):
    X, U, _, Up = oracle.gather(conn, xyz, u, beta, u_prev)
    blocks = oracle.pack_element(oracle.element_kernel(X, U, beta, p, Up))
    S, r, _, _ = oracle.condense(*blocks)
    return S, r, blocks[4]


def sampled_csr_rows(ctx, rows, n_dofs):
    """The assembled CSR rows `rows` (and their right-hand sides) copied from the device."""
    import torch
    rowptr, colidx, vals, rhs = ctx.csr_device()
    rp = rowptr.cpu().numpy().astype(np.int64)
    lens = rp[rows + 1] - rp[rows]
    idx = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows])
    it = torch.as_tensor(idx, device=colidx.device)
    cols = colidx[it].cpu().numpy()
    v = vals[it].cpu().numpy().astype(np.float64)
    b = rhs[torch.as_tensor(rows, device=rhs.device)].cpu().numpy()
    indptr = np.concatenate([[0], np.cumsum(lens)])
    return sp.csr_matrix((v, cols, indptr), shape=(rows.size, n_dofs)), b


def check_windows(ctx, mesh, u, beta, p, rng, tol_s, tol_r=1e-10, u_prev=None, nu_e=None):
    E = mesh.n_elems
    for first in (0, E - 37, int(rng.integers(0, E - 64))):
        n = 37 if first == E - 37 else 64
        el = np.arange(first, first + n)
        got = ctx.element_matrices(first, n)
        if nu_e is None:
            S, r, Rcp = oracle_blocks(mesh.conn[el], mesh.xyz, u, beta[el], p, u_prev)
        else:  # per-element viscosity: group the window by value
            S = np.empty_like(got["S"]); r = np.empty_like(got["r"]); Rcp = np.empty_like(got["Rcp"])
            for nu in np.unique(nu_e[el]):
                sel = np.nonzero(nu_e[el] == nu)[0]
                S[sel], r[sel], Rcp[sel] = oracle_blocks(mesh.conn[el[sel]], mesh.xyz, u,
                                                         beta[el[sel]], Params(nu=float(nu)))
        assert relerr(got["S"], S) < tol_s, ("S", first)
        assert relerr(got["r"], r) < tol_s, ("r", first)
        assert relerr(got["Rcp"], Rcp) < tol_r, ("Rcp", first)


def check_rows(ctx, mesh, bc, u, beta, p, rng, tol, u_prev=None, nu_e=None, count=40):
    nodes = rng.choice(mesh.n_nodes, count, replace=False)
    touch = np.nonzero(np.isin(mesh.conn, nodes).any(axis=1))[0]
    if nu_e is None:
        S, r, _ = oracle_blocks(mesh.conn[touch], mesh.xyz, u, beta[touch], p, u_prev)
    else:
        S = np.empty((touch.size, 32, 32)); r = np.empty((touch.size, 32))
        for nu in np.unique(nu_e[touch]):
            sel = np.nonzero(nu_e[touch] == nu)[0]
            S[sel], r[sel], _ = oracle_blocks(mesh.conn[touch[sel]], mesh.xyz, u, beta[touch[sel]],
                                              Params(nu=float(nu)))
    A, rhs = oracle.assemble(mesh.conn[touch], mesh.n_nodes, S, r)
    A, rhs = oracle.apply_dirichlet(A, rhs, bc.dofs)
    rows = np.sort((4 * nodes[:, None] + np.arange(4)[None, :]).ravel())
    G, g = sampled_csr_rows(ctx, rows, A.shape[1])
    Ar = A.tocsr()[rows]
    diff = abs(G - Ar).max()
    assert diff / max(abs(Ar).max(), 1e-300) < tol
    assert relerr(g, rhs[rows]) < tol


def hex_context(vms, wl, u, beta, p, u_prev=None):
    ctx = vms.Context(0, MIXED)
    ctx.mesh_upload(wl.mesh.xyz, wl.mesh.conn, wl.bc.dofs, wl.bc.vals)
    ctx.set_params(p.nu, p.visc_factor, p.dt, p.f, p.bubble_scale, p.quad_order, 0)
    ctx.state_upload(np.ascontiguousarray(u), np.ascontiguousarray(beta),
                     None if u_prev is None else np.ascontiguousarray(u_prev))
    return ctx


def test_step_channel_full_size_sampled(vms):
    """Backward-facing step, h = 1/13: 518,492 hexahedra, Re 800, mixed."""
    wl = inputs.bfs_workload(13, re=800.0, jitter_frac=0.1, seed=1003)
    assert wl.mesh.n_elems == 518_492
    u, beta, rng = random_state(wl, 31)
    p = Params(nu=wl.nu)
    ctx = hex_context(vms, wl, u, beta, p)
    ctx.assemble()
    check_windows(ctx, wl.mesh, u, beta, p, rng, 1e-5)
    check_rows(ctx, wl.mesh, wl.bc, u, beta, p, rng, 1e-5)
    ctx.close()


def test_channel_past_cube_full_size_sampled(vms):
    """Channel past a cube, 300 x 56 x 56 lattice: 937,860 hexahedra, Re 1000, one backward-Euler
    step (dt 0.01) from a perturbed previous state, mixed."""
    wl = inputs.channel_workload(300, 56, re=1000.0, dt=0.01, seed=1005)
    assert wl.mesh.n_elems == 937_860
    u, beta, rng = random_state(wl, 32)
    u_prev = u + rng.uniform(-0.05, 0.05, u.shape)
    p = Params(nu=wl.nu, dt=wl.dt)
    ctx = hex_context(vms, wl, u, beta, p, u_prev)
    ctx.assemble()
    check_windows(ctx, wl.mesh, u, beta, p, rng, 1e-5, u_prev=u_prev)
    check_rows(ctx, wl.mesh, wl.bc, u, beta, p, rng, 1e-5, u_prev=u_prev)
    ctx.close()


@pytest.mark.parametrize("schedule", [0, 1], ids=["fused", "two_streams"])
def test_batch64_full_size_sampled(vms, schedule):
    """The 64-cavity batch (edges 8-48, Re 100-1000 per instance) in the benchmark's launch
    configurations: CUDA-graph replay of the fused kernel, and of the two kernels with 4 tangent
    warps per block and 64 residual threads."""
    b = inputs.batched_workload(64, seed=1004)
    w = b.work
    ctx = vms.Context(0, MIXED)
    ctx.mesh_upload(w.mesh.xyz, w.mesh.conn, w.bc.dofs, w.bc.vals)
    ctx.set_params(w.nu)
    ctx.set_element_viscosity(b.nu_e)
    ctx.set_instances(b.node_offsets, b.elem_offsets)
    ctx.state_upload(w.u, w.beta)
    ctx.set_tuning(tangent_warps=4, residual_threads=64, schedule=schedule)
    ctx.set_graph(True)
    ctx.assemble()
    ctx.assemble()  # the second call replays the captured graph
    rng = np.random.default_rng(33)
    check_windows(ctx, w.mesh, w.u, w.beta, None, rng, 1e-5, nu_e=b.nu_e)
    check_rows(ctx, w.mesh, w.bc, w.u, w.beta, None, rng, 1e-5, nu_e=b.nu_e)
    ctx.close()


def test_tet_cavity39_full_size_sampled(vms):
    """Kuhn tetrahedra of the jittered 39^3 cavity: 355,914 tetrahedra, Re 400, mixed."""
    wl = inputs.tet_cavity_workload(39, re=400.0, jitter_frac=0.15, state="random", seed=1002)
    assert wl.mesh.n_elems == 355_914
    rng = np.random.default_rng(34)
    u = wl.u
    beta = rng.uniform(-0.05, 0.05, (wl.mesh.n_elems, 3))
    p = Params(nu=wl.nu, element="tet")
    ctx = hex_context(vms, wl, u, beta, p)
    ctx.assemble()
    check_windows(ctx, wl.mesh, u, beta, p, rng, 1e-10)
    check_rows(ctx, wl.mesh, wl.bc, u, beta, p, rng, 1e-6)
    ctx.close()
