"""Solve-level pins of the FP64 oracle (Sections 4.2 and 5 of the paper)."""
import numpy as np
import pytest

import oracle
from oracle import Params
from paper_0809_4802_gb300 import inputs


def condensed_step(mesh, u, beta, bc, p):
    X, U, _, _ = oracle.gather(mesh.conn, mesh.xyz, u, beta)
    k = oracle.element_kernel(X, U, beta, p)
    blocks = oracle.pack_element(k)
    S, r, Xk, y = oracle.condense(*blocks)
    A, rhs = oracle.assemble(mesh.conn, mesh.n_nodes, S, r)
    A, rhs = oracle.apply_dirichlet(A, rhs, bc.dofs)
    du = np.linalg.solve(A.toarray(), -rhs)
    dbeta = oracle.fine_recovery(mesh.conn, du, Xk, y)
    return du, dbeta, blocks


def uncondensed_step(mesh, blocks, bc):
    K, R = oracle.uncondensed_system(mesh.conn, mesh.n_nodes, *blocks, bc.dofs)
    dz = np.linalg.solve(K, -R)
    nc = 4 * mesh.n_nodes
    return dz[:nc], dz[nc:].reshape(-1, 3)


def distorted_problem(n, seed, frac=0.25):
    """Every node (boundary ones too) moved by U[-frac h, frac h]; velocity fixed on z = 0 only,
    traction-free elsewhere. Unlike the uniform cavity, this system has no singular pressure
    modes, so solutions can be compared directly."""
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


@pytest.mark.parametrize("n,seed", [(2, 3), (3, 4)])
def test_schur_step_equals_uncondensed_step(n, seed):
    """Block Gauss elimination is exact (Section 5): the condensed solve followed by fine-scale
    recovery reproduces the solve of the full coarse+fine system of Eq. NewtonUpdate2."""
    mesh, bc, u, beta = distorted_problem(n, seed)
    p = Params(nu=0.05)
    du, dbeta, blocks = condensed_step(mesh, u, beta, bc, p)
    K, R = oracle.uncondensed_system(mesh.conn, mesh.n_nodes, *blocks, bc.dofs)
    dz = np.concatenate([du, dbeta.reshape(-1)])
    assert np.linalg.norm(K @ dz + R) <= 1e-12 * np.linalg.norm(R)
    du2, dbeta2 = uncondensed_step(mesh, blocks, bc)
    np.testing.assert_allclose(du, du2, atol=1e-8 * np.abs(du2).max())
    np.testing.assert_allclose(dbeta, dbeta2, atol=1e-8 * np.abs(dbeta2).max())


def test_newton_schur_iterates_equal_newton_raphson():
    """The paper reports identical Newton-Schur and Newton-Raphson results (Section 6.1). Three
    iterations of each from the same start agree to rounding."""
    mesh, bc, u0, beta0 = distorted_problem(2, 8)
    p = Params(nu=0.05)
    u1, b1 = u0.copy(), beta0.copy()
    u2, b2 = u0.copy(), beta0.copy()
    for _ in range(3):
        du, db, _ = condensed_step(mesh, u1, b1, bc, p)
        u1 += du.reshape(-1, 4); b1 += db
        X, U, _, _ = oracle.gather(mesh.conn, mesh.xyz, u2, b2)
        blocks = oracle.pack_element(oracle.element_kernel(X, U, b2, p))
        du, db = uncondensed_step(mesh, blocks, bc)
        u2 += du.reshape(-1, 4); b2 += db
    np.testing.assert_allclose(u1, u2, atol=1e-9)
    np.testing.assert_allclose(b1, b2, atol=1e-9)


def test_uniform_cavity_null_space_is_pressure_only_and_consistent():
    """On a uniform hexahedral cavity with every wall velocity prescribed, one bubble per element
    does not penalise every equal-order pressure mode: the condensed matrix keeps a four-dimensional
    null space of pure pressure modes. The condensed residual is orthogonal to the left null space,
    so the Newton system stays consistent and Krylov solves remain well posed."""
    wl = inputs.cavity_workload(4, re=100.0, state="noise", seed=1001)
    p = Params(nu=wl.nu)
    X, U, _, _ = oracle.gather(wl.mesh.conn, wl.mesh.xyz, wl.u, wl.beta)
    S, r, _, _ = oracle.condense(*oracle.pack_element(oracle.element_kernel(X, U, wl.beta, p)))
    A, rhs = oracle.assemble(wl.mesh.conn, wl.mesh.n_nodes, S, r)
    A, rhs = oracle.apply_dirichlet(A, rhs, wl.bc.dofs)
    Uu, sv, Vt = np.linalg.svd(A.toarray())
    k = int(np.sum(sv < 1e-12 * sv[0]))
    assert k == 4, sv[-6:]
    right = Vt[-k:].reshape(k, -1, 4)
    assert np.abs(right[:, :, :3]).max() < 1e-10          # pressure only
    left = Uu[:, -k:]
    assert np.abs(left.T @ rhs).max() < 1e-12 * np.linalg.norm(rhs)


def test_dirichlet_rows_and_columns():
    wl = inputs.cavity_workload(2, re=10.0, state="random", seed=1)
    p = Params(nu=wl.nu)
    X, U, _, _ = oracle.gather(wl.mesh.conn, wl.mesh.xyz, wl.u, wl.beta)
    S, r, _, _ = oracle.condense(*oracle.pack_element(oracle.element_kernel(X, U, wl.beta, p)))
    A, rhs = oracle.assemble(wl.mesh.conn, wl.mesh.n_nodes, S, r)
    A, rhs = oracle.apply_dirichlet(A, rhs, wl.bc.dofs)
    D = A.toarray()
    d = wl.bc.dofs
    np.testing.assert_array_equal(D[d][:, d], np.eye(d.size))
    free = np.setdiff1d(np.arange(D.shape[0]), d)
    assert np.all(D[np.ix_(d, free)] == 0) and np.all(D[np.ix_(free, d)] == 0)
    assert np.all(rhs[d] == 0)


@pytest.mark.slow
def test_newton_quadratic_convergence_cavity_8():
    """Consistent linearisation gives quadratic convergence (Section 1, Section 4.2): the 8^3
    lid-driven cavity at Re = 100 from a noisy start converges to 1e-10 relative, and in the
    asymptotic range r_{k+1} / r_k^2 stays bounded."""
    wl = inputs.cavity_workload(8, re=100.0, state="noise", seed=1001)
    p = Params(nu=wl.nu)
    u, beta, norms = oracle.newton_solve(wl.mesh.xyz, wl.mesh.conn, wl.u, wl.beta, wl.bc.dofs, p,
                                         tol=1e-10, maxit=15)
    rel = np.array(norms) / norms[0]
    assert rel[-1] < 1e-10, rel
    assert len(norms) <= 10, rel
    # quadratic rate: once below 1e-2, each step at least squares the error (up to a constant)
    tail = [k for k in range(len(rel) - 1) if rel[k] < 1e-2 and rel[k + 1] > 1e-14]
    assert tail, rel
    for k in tail:
        assert rel[k + 1] <= 50.0 * rel[k] ** 2 + 1e-13, rel
    # converged fine scale satisfies R_f = 0 on every element, and the Dirichlet values held
    X, U, _, _ = oracle.gather(wl.mesh.conn, wl.mesh.xyz, u, beta)
    k = oracle.element_kernel(X, U, beta, p, with_tangent=False)
    assert np.abs(k["Rf"]).max() < 1e-9 * norms[0]
    np.testing.assert_array_equal(u.reshape(-1)[wl.bc.dofs], wl.bc.vals)
