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


@pytest.mark.parametrize("prec,restart", [(0, 110), (0, 50), (1, 110), (1, 50)])
def test_solve_and_recovery_match_direct_solution(vms, prec, restart):
    """2^3 distorted traction-free problem (108 unknowns): unrestarted GMRES (restart 110) and
    GMRES(50) with restarts both reach 1e-10; the solution matches a direct solve."""
    mesh, bc, u, beta = distorted_problem(2, 11)
    p = Params(nu=0.05)
    ctx = vms.Context(0, prec)
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
