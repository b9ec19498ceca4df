"""Batches of independent problems in one mesh: per-element viscosity, instance solves, the CUDA
graph of the assembly and the autotuner, through the C-ABI, against the FP64 oracle.

Each instance of a merged mesh must give the system the oracle gives for that instance alone,
with that instance's viscosity (FP64 1e-10, mixed 1e-5 relative to the largest entry, as in
test_gpu_assembly); the graph replay and every tuning must reproduce the plain assembly (bit for
bit with the colour-serialised scatter, whose summation order is fixed).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from oracle import Params
from paper_0809_4802_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 1: 1e-5}


@pytest.fixture(scope="module")
def vms():
    from paper_0809_4802_gb300 import build, vms as v
    build.build()
    v.load_library()
    return v


def relerr(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def small_batch():
    # four jittered cavities of uneven size (2^3, 3^3, 4^3, 3^3 elements) and Reynolds numbers
    parts = [inputs.cavity_workload(n, re, jitter_frac=0.15, state="random", seed=50 + i)
             for i, (n, re) in enumerate([(2, 150.0), (3, 900.0), (4, 420.0), (3, 100.0)])]
    rng = np.random.default_rng(5)
    for w in parts:
        w.beta = rng.uniform(-0.1, 0.1, w.beta.shape)
    return inputs.merge_workloads(parts)


@pytest.fixture(scope="module")
def regular_batch():
    # three distorted boxes (nodes jittered by up to a quarter of a cell, velocity fixed on the
    # bottom face only, different viscosities): regular systems, unlike the jittered cavities,
    # whose near-null pressure modes make the FP32 matrix inconsistent with the FP64 right-hand
    # side at the 1e-3 level
    parts = []
    for i, (n, nu) in enumerate([(2, 0.05), (3, 0.02), (2, 0.005)]):
        mesh = inputs.cavity_mesh(n)
        rng = np.random.default_rng(70 + i)
        mesh.xyz += rng.uniform(-0.25, 0.25, mesh.xyz.shape) / n
        bottom = np.nonzero(mesh.node_ijk[:, 2] == 0)[0]
        dofs = np.sort(np.concatenate([4 * bottom + c for c in range(3)]))
        u = rng.uniform(-0.5, 0.5, (mesh.n_nodes, 4))
        u.reshape(-1)[dofs] = 0.0
        parts.append(inputs.Workload(mesh=mesh, bc=inputs.Dirichlet(dofs=dofs, vals=np.zeros(dofs.size)),
                                     u=u, beta=rng.uniform(-0.2, 0.2, (mesh.n_elems, 3)), nu=nu))
    return inputs.merge_workloads(parts)


def batch_context(vms, b, prec, scatter=0):
    w = b.work
    ctx = vms.Context(0, prec)
    ctx.mesh_upload(w.mesh.xyz, w.mesh.conn, w.bc.dofs, w.bc.vals)
    ctx.set_params(w.nu, scatter_mode=scatter)
    ctx.set_element_viscosity(b.nu_e)
    ctx.set_instances(b.node_offsets, b.elem_offsets)
    ctx.state_upload(w.u, w.beta)
    return ctx


def oracle_instance_system(part):
    m = part.mesh
    X, U, _, _ = oracle.gather(m.conn, m.xyz, part.u, part.beta)
    k = oracle.element_kernel(X, U, part.beta, Params(nu=part.nu))
    S, r, _, _ = oracle.condense(*oracle.pack_element(k))
    A, rhs = oracle.assemble(m.conn, m.n_nodes, S, r)
    return oracle.apply_dirichlet(A, rhs, part.bc.dofs)


@pytest.mark.parametrize("prec", [0, 1])
def test_each_instance_block_matches_oracle(vms, small_batch, prec):
    """The merged CSR system is block diagonal and each diagonal block (with its right-hand side)
    is the oracle's system of that instance with its own viscosity."""
    b = small_batch
    ctx = batch_context(vms, b, prec)
    ctx.assemble()
    rowptr, colidx, vals, rhs = ctx.csr_host()
    G = sp.csr_matrix((vals.astype(np.float64), colidx, rowptr)).tocsr()
    for i, part in enumerate(b.members):
        r0, r1 = 4 * b.node_offsets[i], 4 * b.node_offsets[i + 1]
        rows = G[r0:r1]
        assert rows[:, :r0].nnz == 0 or np.abs(rows[:, :r0].data).max() == 0.0
        assert rows[:, r1:].nnz == 0 or np.abs(rows[:, r1:].data).max() == 0.0
        A, rref = oracle_instance_system(part)
        assert relerr(rows[:, r0:r1].toarray(), A.toarray()) <= TOL[prec], i
        assert relerr(rhs[r0:r1], rref) <= (1e-10 if prec == 0 else 1e-5), i
    ctx.close()


def test_graph_replay_reproduces_the_assembly(vms, small_batch):
    """With the colour-serialised scatter the graph replay (and a second replay) give the same
    bits as the plain assembly."""
    ctx = batch_context(vms, small_batch, 1, scatter=1)
    ctx.assemble()
    plain = [a.copy() for a in ctx.csr_host()[2:]]
    ctx.set_graph(True)
    for _ in range(2):
        ctx.assemble()
        vals, rhs = ctx.csr_host()[2:]
        np.testing.assert_array_equal(vals, plain[0])
        np.testing.assert_array_equal(rhs, plain[1])
    # a parameter change invalidates the graph: the next replay uses the new viscosity
    ctx.set_element_viscosity(2.0 * small_batch.nu_e)
    ctx.assemble()
    vals2 = ctx.csr_host()[2]
    assert np.abs(vals2 - plain[0]).max() > 0.0
    ctx.set_graph(False)
    ctx.assemble()
    np.testing.assert_array_equal(ctx.csr_host()[2], vals2)
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_direct_fallback_solves_each_instance(vms, regular_batch, prec):
    """With VMS_PRECOND_ILU0_FALLBACK a Krylov solve stopped at maxit (here after one iteration)
    is replaced by the banded direct solve of that instance's diagonal block: the increment
    satisfies the block to rounding level, matches a direct solve of it, and leaves the other
    instances unchanged."""
    b = regular_batch
    ctx = batch_context(vms, b, prec)
    ctx.set_preconditioner(vms.PRECOND_ILU0_FALLBACK)
    ctx.assemble()
    rowptr, colidx, vals, rhs = ctx.csr_host()
    G = sp.csr_matrix((vals.astype(np.float64), colidx, rowptr)).tocsr()
    u0, _ = ctx.state_download()
    for i in range(len(b.members)):
        it, rel = ctx.solve_instance(i, rtol=1e-11, maxit=1, restart=1, update=True)
        assert rel <= 1e-11 and it == 1
        u1, _ = ctx.state_download()
        n0, n1 = b.node_offsets[i], b.node_offsets[i + 1]
        np.testing.assert_array_equal(u1[:n0], u0[:n0])
        np.testing.assert_array_equal(u1[n1:], u0[n1:])
        blk = G[4 * n0:4 * n1, 4 * n0:4 * n1]
        r = rhs[4 * n0:4 * n1]
        du = (u1[n0:n1] - u0[n0:n1]).reshape(-1)
        assert np.linalg.norm(blk @ du + r) <= 1e-11 * np.linalg.norm(r)
        assert relerr(du, spla.spsolve(blk.tocsc(), -r)) <= 1e-8
        u0 = u1
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_instance_solves_update_only_their_instance(vms, regular_batch, prec):
    """vms_solve_instance solves one diagonal block (to 1e-10) and updates only that instance's
    state: its increment satisfies the assembled block and matches a direct solve of it, its
    bubble increments are the oracle's recovery from that increment, and nothing outside the
    instance moves."""
    b = regular_batch
    ctx = batch_context(vms, b, prec)
    ctx.assemble()
    rowptr, colidx, vals, rhs = ctx.csr_host()
    G = sp.csr_matrix((vals.astype(np.float64), colidx, rowptr)).tocsr()
    u0, beta0 = ctx.state_download()
    for i, part in enumerate(b.members):
        it, rel = ctx.solve_instance(i, rtol=1e-10, maxit=3000, restart=200, update=True)
        assert rel <= 1e-10 and it > 0
        u1, beta1 = ctx.state_download()
        n0, n1 = b.node_offsets[i], b.node_offsets[i + 1]
        e0, e1 = b.elem_offsets[i], b.elem_offsets[i + 1]
        np.testing.assert_array_equal(u1[:n0], u0[:n0])
        np.testing.assert_array_equal(u1[n1:], u0[n1:])
        np.testing.assert_array_equal(beta1[:e0], beta0[:e0])
        np.testing.assert_array_equal(beta1[e1:], beta0[e1:])
        blk = G[4 * n0:4 * n1, 4 * n0:4 * n1]
        r = rhs[4 * n0:4 * n1]
        du = (u1[n0:n1] - u0[n0:n1]).reshape(-1)
        assert np.linalg.norm(blk @ du + r) <= 2e-10 * np.linalg.norm(r)
        ref = spla.spsolve(blk.tocsc(), -r)
        assert relerr(du, ref) <= 1e-5
        m = part.mesh
        X, U, _, _ = oracle.gather(m.conn, m.xyz, part.u, part.beta)
        _, _, Xk, y = oracle.condense(*oracle.pack_element(oracle.element_kernel(X, U, part.beta, Params(nu=part.nu))))
        dbeta_ref = oracle.fine_recovery(m.conn, du, Xk, y)
        # mixed: the recovery uses the FP32 K_fc (relative error ~5e-7) and its two terms,
        # K_ff^-1 R_f and K_ff^-1 K_fc du, partly cancel at nu = 0.005
        assert relerr(beta1[e0:e1] - beta0[e0:e1], dbeta_ref) <= (1e-9 if prec == 0 else 5e-5)
        u0, beta0 = u1, beta1
    # an updated instance's block (and so the whole system) is stale until the next assembly
    for call in (lambda: ctx.solve_instance(0), lambda: ctx.solve(rtol=1e-6)):
        with pytest.raises(vms.VmsError) as ei:
            call()
        assert ei.value.code == vms.ERR_STATE
    ctx.assemble()
    it, rel = ctx.solve_instance(0, rtol=1e-6, maxit=3000, restart=200, update=False)
    assert rel <= 1e-6
    ctx.close()


def test_autotune_picks_an_offered_tuning_and_keeps_results(vms, small_batch):
    ctx = batch_context(vms, small_batch, 1, scatter=1)
    ctx.assemble()
    ref = [a.copy() for a in ctx.csr_host()[2:]]
    best = ctx.autotune(repeats=2)
    if best["schedule"] == vms.SCHEDULE_FUSED:   # one persistent launch, atomic scatter
        assert (best["tangent_warps"], best["residual_threads"], best["scatter_mode"]) == (0, 0, 0)
    else:
        assert best["schedule"] == vms.SCHEDULE_TWO_STREAMS
        assert best["tangent_warps"] in (2, 4, 8)
        assert best["residual_threads"] in (32, 64)
        assert best["scatter_mode"] in (0, 1)
    assert best["ms"] > 0.0
    assert ctx.get_tuning() == {**best, "ms": ctx.get_tuning()["ms"]}
    ctx.assemble()
    vals, rhs = ctx.csr_host()[2:]
    assert relerr(vals, ref[0]) <= 1e-6 and relerr(rhs, ref[1]) <= 1e-6
    # every offered tuning with the colour scatter reproduces the default bits
    for tw in (2, 4, 8):
        for rt in (32, 64):
            ctx.set_tuning(tw, rt, 1, vms.SCHEDULE_TWO_STREAMS)
            ctx.assemble()
            vals, rhs = ctx.csr_host()[2:]
            np.testing.assert_array_equal(vals, ref[0])
            np.testing.assert_array_equal(rhs, ref[1])
    for bad in ((3, 64, 1, 0), (4, 64, 1, 2)):
        with pytest.raises(vms.VmsError) as ei:
            ctx.set_tuning(*bad)
        assert ei.value.code == vms.ERR_INVALID_ARG
    ctx.close()


def test_instances_must_not_share_nodes(vms, small_batch):
    b = small_batch
    ctx = vms.Context(0, 0)
    w = b.work
    ctx.mesh_upload(w.mesh.xyz, w.mesh.conn, w.bc.dofs, w.bc.vals)
    bad = b.node_offsets.copy()
    bad[1] += 1  # the first instance would own a node of the second
    with pytest.raises(vms.VmsError) as ei:
        ctx.set_instances(bad, b.elem_offsets)
    assert ei.value.code == vms.ERR_INVALID_ARG
    with pytest.raises(vms.VmsError):
        ctx.solve_instance(0)
    ctx.close()
