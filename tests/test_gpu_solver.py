"""GPU Krylov solve, fine-scale recovery and Newton-Schur iteration against the FP64 oracle.

Velocities are unique and compared directly. On uniform cavities the pressure is unique only up to
the singular pressure modes of the single-bubble hexahedron, so there the GPU pressure is checked
through the oracle's residual evaluated at the GPU state.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from oracle import Params
from paper_0809_4802_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vms():
    from paper_0809_4802_gb300 import build, vms as v
    build.build()
    v.load_library()
    return v


def distorted_problem(n, seed, frac=0.25):
    mesh = inputs.cavity_mesh(n)
    rng = np.random.default_rng(seed)
    mesh.xyz += rng.uniform(-frac, frac, mesh.xyz.shape) / n
    bottom = np.nonzero(mesh.node_ijk[:, 2] == 0)[0]
    dofs = np.sort(np.concatenate([4 * bottom + c for c in range(3)]))
    bc = inputs.Dirichlet(dofs=dofs, vals=np.zeros(dofs.size))
    u = rng.uniform(-0.5, 0.5, (mesh.n_nodes, 4))
    u.reshape(-1)[dofs] = 0.0
    beta = rng.uniform(-0.2, 0.2, (mesh.n_elems, 3))
    return mesh, bc, u, beta


@pytest.mark.parametrize("precond", [0, 1], ids=["ilu0", "bjacobi"])
@pytest.mark.parametrize("prec,restart", [(0, 110), (0, 50), (1, 110), (1, 50)])
def test_solve_and_recovery_match_direct_solution(vms, prec, restart, precond):
    """2^3 distorted traction-free problem (108 unknowns): unrestarted GMRES (restart 110) and
    GMRES(50) with restarts both reach 1e-10 with either preconditioner; the solution matches a
    direct solve."""
    mesh, bc, u, beta = distorted_problem(2, 11)
    p = Params(nu=0.05)
    ctx = vms.Context(0, prec)
    ctx.set_preconditioner(precond)
    ctx.mesh_upload(mesh.xyz, mesh.conn, bc.dofs, bc.vals)
    ctx.set_params(p.nu)
    ctx.state_upload(u, beta)
    ctx.assemble()
    rowptr, colidx, vals, rhs = ctx.csr_host()
    G = sp.csr_matrix((vals.astype(np.float64), colidx, rowptr))
    du_ref = spla.spsolve(G.tocsc(), -rhs)
    it, rel = ctx.solve(rtol=1e-10, maxit=3000, restart=restart, update=True)
    assert rel <= 1e-10 and it > 0
    u2, beta2 = ctx.state_download()
    du = (u2 - u).reshape(-1)
    # the true residual of the assembled system, then the solution itself (condition number of
    # this system is about 1e6)
    assert np.linalg.norm(G @ du + rhs) <= 2e-10 * np.linalg.norm(rhs)
    assert np.abs(du - du_ref).max() <= 1e-5 * np.abs(du_ref).max()
    # fine-scale recovery from the oracle's element blocks and the GPU increment
    X, U, _, _ = oracle.gather(mesh.conn, mesh.xyz, u, beta)
    _, _, Xk, y = oracle.condense(*oracle.pack_element(oracle.element_kernel(X, U, beta, p)))
    dbeta_ref = oracle.fine_recovery(mesh.conn, du, Xk, y)
    tol = 1e-9 if prec == 0 else 1e-5
    assert np.abs((beta2 - beta) - dbeta_ref).max() <= tol * np.abs(dbeta_ref).max()
    ctx.close()


def test_krylov_maxit_is_reported_and_state_kept(vms):
    mesh, bc, u, beta = distorted_problem(2, 12)
    ctx = vms.Context(0, 0)
    ctx.mesh_upload(mesh.xyz, mesh.conn, bc.dofs, bc.vals)
    ctx.set_params(0.05)
    ctx.state_upload(u, beta)
    ctx.assemble()
    with pytest.raises(vms.VmsError) as ei:
        ctx.solve(rtol=1e-14, maxit=3, restart=3, update=True)
    assert ei.value.code == vms.ERR_KRYLOV_MAXIT
    u2, b2 = ctx.state_download()
    np.testing.assert_array_equal(u2, u)
    np.testing.assert_array_equal(b2, beta)
    ctx.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-8)])
def test_newton_cavity8_matches_oracle(vms, prec, tol):
    """The 8^3 lid-driven cavity at Re 100 from the seeded noisy start (Newton-Schur, Sections 4.2
    and 5) converges on the GPU; velocities agree with the oracle's converged solution and the
    oracle's own residual at the GPU state is below the tolerance."""
    wl = inputs.cavity_workload(8, re=100.0, state="noise", seed=1001)
    p = Params(nu=wl.nu)
    ctx = vms.Context(0, prec)
    ctx.mesh_upload(wl.mesh.xyz, wl.mesh.conn, wl.bc.dofs, wl.bc.vals)
    ctx.set_params(wl.nu)
    ctx.state_upload(wl.u, wl.beta)
    its, hist = ctx.newton_solve(rtol=tol, maxit=12)
    assert hist[-1] <= tol * hist[0]
    assert its <= (6 if prec == 0 else 8), hist
    u, beta = ctx.state_download()
    uo, bo, norms = oracle.newton_solve(wl.mesh.xyz, wl.mesh.conn, wl.u, wl.beta, wl.bc.dofs, p,
                                        tol=1e-12, maxit=15)
    assert abs(hist[0] - norms[0]) <= 1e-12 * norms[0]
    vel_tol = 1e-8 if prec == 0 else 1e-6
    assert np.abs(u[:, :3] - uo[:, :3]).max() <= vel_tol
    X, U, _, _ = oracle.gather(wl.mesh.conn, wl.mesh.xyz, u, beta)
    k = oracle.element_kernel(X, U, beta, p, with_tangent=False)
    R = oracle.residual_vector(wl.mesh.conn, wl.mesh.n_nodes, k, wl.bc.dofs)
    assert np.linalg.norm(R) <= 10 * tol * norms[0]
    ctx.close()


def one_element_problem(constrained_face_z, seed=13):
    """One distorted hexahedron with the velocity fixed on the face z = constrained_face_z."""
    mesh = inputs.cavity_mesh(1)
    rng = np.random.default_rng(seed)
    mesh.xyz += rng.uniform(-0.25, 0.25, mesh.xyz.shape)
    face = np.nonzero(mesh.node_ijk[:, 2] == constrained_face_z)[0]
    dofs = np.sort(np.concatenate([4 * face + c for c in range(3)]))
    bc = inputs.Dirichlet(dofs=dofs, vals=np.zeros(dofs.size))
    u = rng.uniform(-0.5, 0.5, (mesh.n_nodes, 4))
    u.reshape(-1)[dofs] = 0.0
    beta = rng.uniform(-0.2, 0.2, (mesh.n_elems, 3))
    return mesh, bc, u, beta


@pytest.mark.parametrize("prec", [0, 1])
def test_ilu0_of_a_full_pattern_is_exact(vms, prec):
    """On a one-element mesh every node neighbours every other, so the block pattern is full and
    ILU(0) is the exact block LU factorisation: right-preconditioned GMRES converges at once.
    (Velocity fixed on the top face, so the first nodes eliminated carry all four unknowns and
    every pivot block is well conditioned: condition numbers 2 to 5e4.)"""
    mesh, bc, u, beta = one_element_problem(1)
    ctx = vms.Context(0, prec)
    ctx.set_preconditioner(vms.PRECOND_ILU0)
    ctx.mesh_upload(mesh.xyz, mesh.conn, bc.dofs, bc.vals)
    ctx.set_params(0.05)
    ctx.state_upload(u, beta)
    ctx.assemble()
    it, rel = ctx.solve(rtol=1e-10, maxit=20, restart=20, update=False)
    # FP64: one iteration (a second at most, for rounding: the system's condition number is 4e5);
    # mixed: each FP64 refinement pass of the FP32 inner solve takes one or two iterations
    assert it <= (2 if prec == 0 else 10) and rel <= 1e-10, (it, rel)
    ctx.close()


def test_ilu0_zero_pivot_is_reported_and_context_stays_usable(vms):
    """With the velocity fixed on the bottom face instead, the four bottom nodes come first in the
    node order and only their pressures remain: the Schur complement of their pressure block is
    singular, so block LU without pivoting meets a zero pivot at the fourth node. The solve
    reports VMS_ERR_ZERO_PIVOT, leaves the state unchanged, and the same context then solves the
    system with block-Jacobi preconditioning."""
    mesh, bc, u, beta = one_element_problem(0)
    ctx = vms.Context(0, 0)
    ctx.set_preconditioner(vms.PRECOND_ILU0)
    ctx.mesh_upload(mesh.xyz, mesh.conn, bc.dofs, bc.vals)
    ctx.set_params(0.05)
    ctx.state_upload(u, beta)
    ctx.assemble()
    with pytest.raises(vms.VmsError) as ei:
        ctx.solve(rtol=1e-10, maxit=20, restart=20, update=True)
    assert ei.value.code == vms.ERR_ZERO_PIVOT
    u2, b2 = ctx.state_download()
    np.testing.assert_array_equal(u2, u)
    np.testing.assert_array_equal(b2, beta)
    ctx.set_preconditioner(vms.PRECOND_BLOCK_JACOBI)
    it, rel = ctx.solve(rtol=1e-10, maxit=200, restart=50, update=False)
    assert rel <= 1e-10
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_zero_pivot_falls_back_to_the_pivoted_direct_solve(vms, prec):
    """The one-element system whose block LU without pivoting meets a zero pivot: with
    VMS_PRECOND_ILU0_FALLBACK the banded LU with partial pivoting solves it directly."""
    mesh, bc, u, beta = one_element_problem(0)
    ctx = vms.Context(0, prec)
    ctx.set_preconditioner(vms.PRECOND_ILU0_FALLBACK)
    ctx.mesh_upload(mesh.xyz, mesh.conn, bc.dofs, bc.vals)
    ctx.set_params(0.05)
    ctx.state_upload(u, beta)
    ctx.assemble()
    rowptr, colidx, vals, rhs = ctx.csr_host()
    G = sp.csr_matrix((vals.astype(np.float64), colidx, rowptr))
    it, rel = ctx.solve(rtol=1e-10, maxit=20, restart=20, update=True)
    assert rel <= 1e-12
    du = (ctx.state_download()[0] - u).reshape(-1)
    assert np.linalg.norm(G @ du + rhs) <= 1e-12 * np.linalg.norm(rhs)
    du_ref = spla.spsolve(G.tocsc(), -rhs)
    assert np.abs(du - du_ref).max() <= 1e-9 * np.abs(du_ref).max()
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_direct_solve_in_a_bandwidth_reducing_order(vms, prec):
    """An elongated distorted box (12 x 3 x 3 cells, numbered x fastest, so a node couples to nodes
    66 numbers away): the banded direct fallback orders it by reverse Cuthill-McKee from the far
    end face (bandwidth about a third of that) and its solution still satisfies the system to
    rounding level and matches a direct solve."""
    mesh = inputs.box_mesh(12, 3, 3, hi=(4.0, 1.0, 1.0))
    rng = np.random.default_rng(17)
    mesh.xyz += rng.uniform(-0.08, 0.08, mesh.xyz.shape)
    x0 = np.nonzero(mesh.node_ijk[:, 0] == 0)[0]
    dofs = np.sort(np.concatenate([4 * x0 + c for c in range(3)]))
    u = rng.uniform(-0.5, 0.5, (mesh.n_nodes, 4))
    u.reshape(-1)[dofs] = 0.0
    beta = rng.uniform(-0.2, 0.2, (mesh.n_elems, 3))
    ctx = vms.Context(0, prec)
    ctx.set_preconditioner(vms.PRECOND_ILU0_FALLBACK)
    ctx.mesh_upload(mesh.xyz, mesh.conn, dofs, np.zeros(dofs.size))
    ctx.set_params(0.05)
    ctx.state_upload(u, beta)
    ctx.assemble()
    rowptr, colidx, vals, rhs = ctx.csr_host()
    G = sp.csr_matrix((vals.astype(np.float64), colidx, rowptr))
    it, rel = ctx.solve(rtol=1e-11, maxit=1, restart=1, update=True)   # one Krylov step, then direct
    assert it == 1 and rel <= 1e-11
    du = (ctx.state_download()[0] - u).reshape(-1)
    assert np.linalg.norm(G @ du + rhs) <= 1e-11 * np.linalg.norm(rhs)
    du_ref = spla.spsolve(G.tocsc(), -rhs)
    assert np.abs(du - du_ref).max() <= 1e-8 * np.abs(du_ref).max()
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_ilu0_beats_block_jacobi_on_cavity(vms, prec):
    """12^3 lid-driven cavity at Re 400 from the noisy start: both preconditioners give solutions
    with the requested residual, and ILU(0) needs several times fewer GMRES(50) iterations."""
    wl = inputs.cavity_workload(12, re=400.0, state="noise", seed=1001)
    out = {}
    for precond in (vms.PRECOND_ILU0, vms.PRECOND_BLOCK_JACOBI):
        ctx = vms.Context(0, prec)
        ctx.set_preconditioner(precond)
        ctx.mesh_upload(wl.mesh.xyz, wl.mesh.conn, wl.bc.dofs, wl.bc.vals)
        ctx.set_params(wl.nu)
        ctx.state_upload(wl.u, wl.beta)
        ctx.assemble()
        rowptr, colidx, vals, rhs = ctx.csr_host()
        G = sp.csr_matrix((vals.astype(np.float64), colidx, rowptr))
        it, rel = ctx.solve(rtol=1e-6, maxit=5000, restart=50, update=True)
        u2, _ = ctx.state_download()
        du = (u2 - wl.u).reshape(-1)
        du[wl.bc.dofs] = 0.0
        assert np.linalg.norm(G @ du + rhs) <= 2e-6 * np.linalg.norm(rhs)
        out[precond] = it
        ctx.close()
    assert 3 * out[vms.PRECOND_ILU0] <= out[vms.PRECOND_BLOCK_JACOBI], out


@pytest.mark.parametrize("prec", [0, 1])
def test_ilu0_row_with_more_than_16_lower_blocks(vms, prec):
    """The 2^3 distorted problem renumbered so that the centre node comes last: its row has 26
    lower neighbour blocks, more than the two-lanes-per-block layout of the FP64 sweeps takes, so
    that row is solved with one lane per block. The solve still matches a direct solution."""
    mesh, bc, u, beta = distorted_problem(2, 11)
    order = np.arange(mesh.n_nodes)
    centre = int(np.nonzero(np.all(mesh.node_ijk == 1, axis=1))[0][0])
    order[[centre, mesh.n_nodes - 1]] = order[[mesh.n_nodes - 1, centre]]
    new_of_old = np.empty_like(order)
    new_of_old[order] = np.arange(mesh.n_nodes)
    xyz = np.ascontiguousarray(mesh.xyz[order])
    conn = np.ascontiguousarray(new_of_old[mesh.conn].astype(np.int32))
    dofs = np.sort(4 * new_of_old[bc.dofs // 4] + bc.dofs % 4)
    u2 = np.ascontiguousarray(u[order])
    ctx = vms.Context(0, prec)
    ctx.set_preconditioner(vms.PRECOND_ILU0)
    ctx.mesh_upload(xyz, conn, dofs, np.zeros(dofs.size))
    ctx.set_params(0.05)
    ctx.state_upload(u2, beta)
    ctx.assemble()
    rowptr, colidx, vals, rhs = ctx.csr_host()
    last = 4 * (mesh.n_nodes - 1)
    assert np.all(colidx[rowptr[last]:rowptr[last + 1]] // 4 <= mesh.n_nodes - 1)
    assert (rowptr[last + 1] - rowptr[last]) // 4 == 27   # 26 lower blocks and the diagonal
    G = sp.csr_matrix((vals.astype(np.float64), colidx, rowptr))
    du_ref = spla.spsolve(G.tocsc(), -rhs)
    it, rel = ctx.solve(rtol=1e-10, maxit=3000, restart=110, update=True)
    assert rel <= 1e-10 and it > 0
    du = (ctx.state_download()[0] - u2).reshape(-1)
    assert np.linalg.norm(G @ du + rhs) <= 2e-10 * np.linalg.norm(rhs)
    assert np.abs(du - du_ref).max() <= 1e-5 * np.abs(du_ref).max()
    ctx.close()


def test_fallback_solves_a_system_whose_ilu0_is_unstable():
    """A coarse high-Reynolds cavity (12^3, Re 719, random state, one of the batch's instances):
    its ILU(0) factor is unstable (CPU study: |M^-1 v| / |A^-1 v| ~ 1e7 and more) and GMRES with it
    stalls. Block Jacobi with GMRES(480) reaches the batch's per-instance target of 1e-2;
    VMS_PRECOND_ILU0_FALLBACK ends the stagnating ILU(0) attempt early and solves the system
    directly (banded LU with partial pivoting, FP64), and the solution's residual, taken on the host with the downloaded CSR matrix, is at rounding
    level."""
    from paper_0809_4802_gb300 import build, vms
    build.build()
    vms.load_library()
    wl = inputs.cavity_workload(12, 719.1888472918997, jitter_frac=0.15, state="random", seed=1021)
    ctx = vms.Context(0, vms.PREC_MIXED)
    ctx.mesh_upload(wl.mesh.xyz, wl.mesh.conn, wl.bc.dofs, wl.bc.vals)
    ctx.set_params(wl.nu)
    ctx.state_upload(wl.u, wl.beta)
    ctx.assemble()
    with pytest.raises(vms.VmsError) as ei:
        ctx.solve(rtol=1e-2, maxit=3000, restart=150, update=False)
    assert ei.value.code == vms.ERR_KRYLOV_MAXIT
    ctx.set_preconditioner(vms.PRECOND_BLOCK_JACOBI)
    it, rel = ctx.solve(rtol=1e-2, maxit=3000, restart=480, update=False)
    assert rel <= 1e-2
    rowptr, colidx, vals, rhs = ctx.csr_host()
    G = sp.csr_matrix((vals.astype(np.float64), colidx, rowptr))
    u0 = ctx.state_download()[0]
    ctx.set_preconditioner(vms.PRECOND_ILU0_FALLBACK)
    it, rel = ctx.solve(rtol=1e-2, maxit=3000, restart=150, update=True)
    # the ILU(0) attempt ends early (its cycles' rate would not reach 1e-2 within maxit), then the
    # direct solve's residual
    assert 0 < it < 3000 and rel <= 1e-9, (it, rel)
    du = (ctx.state_download()[0] - u0).reshape(-1)
    du[wl.bc.dofs] = 0.0   # the update also imposes the boundary values
    assert np.linalg.norm(G @ du + rhs) <= 1e-9 * np.linalg.norm(rhs)
    du_ref = spla.spsolve(G.tocsc(), -rhs)
    print("band solve: rel", rel, "forward", np.abs(du - du_ref).max() / np.abs(du_ref).max())
    ctx.set_preconditioner(vms.PRECOND_ILU0)
    ctx.close()
