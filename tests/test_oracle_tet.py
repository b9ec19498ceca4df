"""Pins of the oracle's tetrahedral P1 + bubble element (oracle/vms.py, element="tet") against
facts that do not come from the oracle: the exact integrals of barycentric monomials over a
tetrahedron, the P1 identities, the bubble's values, finite differences of the residual,
constant-state patch tests, the uncondensed system, and Newton's quadratic convergence.
"""
from math import factorial

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
from oracle import Params
from paper_0809_4802_gb300 import inputs


def monomial_integral(a):
    """int over the reference tetrahedron of prod lambda_i^a_i = prod a_i! 3! / (|a|+3)! / 6."""
    return np.prod([factorial(k) for k in a]) * factorial(3) / factorial(sum(a) + 3) / 6.0


@pytest.mark.parametrize("n", [2, 3, 4])
def test_tet_rule_is_exact_to_degree_2n_minus_1(n):
    pts, wts = oracle.tet_rule(n)
    lam, _ = oracle.p1_basis(pts)
    assert wts.sum() == pytest.approx(1.0 / 6.0, rel=1e-14)
    assert np.all(wts > 0) and np.all(lam > 0)
    for deg in range(2 * n):
        for a0 in range(deg + 1):
            for a1 in range(deg + 1 - a0):
                for a2 in range(deg + 1 - a0 - a1):
                    a = (a0, a1, a2, deg - a0 - a1 - a2)
                    got = np.sum(wts * np.prod(lam ** np.array(a)[None, :], axis=1))
                    assert got == pytest.approx(monomial_integral(a), rel=1e-12, abs=1e-16), a
    # and not beyond: lambda_1^(2n) is integrated with an error
    a = (0, 2 * n, 0, 0)
    got = np.sum(wts * lam[:, 1] ** (2 * n))
    assert abs(got - monomial_integral(a)) > 1e-12 * monomial_integral(a)


def test_p1_basis_and_bubble():
    rng = np.random.default_rng(1)
    xi = rng.dirichlet(np.ones(4), size=50)[:, 1:]
    N, dN = oracle.p1_basis(xi)
    np.testing.assert_allclose(N.sum(axis=1), 1.0, atol=1e-15)
    np.testing.assert_allclose(N @ oracle.TET_CORNERS, xi, atol=1e-15)   # linear reproduction
    np.testing.assert_allclose(dN.sum(axis=1), 0.0, atol=1e-15)
    b, db = oracle.tet_bubble(np.array([[0.25, 0.25, 0.25]]))
    assert b[0] == pytest.approx(1.0) and np.abs(db).max() < 1e-14   # maximum at the centroid
    face = np.array([[0.2, 0.3, 0.0], [0.0, 0.4, 0.1], [0.3, 0.0, 0.5], [0.3, 0.3, 0.4]])
    np.testing.assert_allclose(oracle.tet_bubble(face)[0], 0.0, atol=1e-15)
    h = 1e-6
    b0, d0 = oracle.tet_bubble(xi)
    for al in range(3):
        e = np.zeros(3); e[al] = h
        fd = (oracle.tet_bubble(xi + e)[0] - oracle.tet_bubble(xi - e)[0]) / (2 * h)
        np.testing.assert_allclose(d0[:, al], fd, rtol=1e-7, atol=1e-9)


def random_tets(n, seed):
    rng = np.random.default_rng(seed)
    X = oracle.TET_CORNERS[None] * rng.uniform(0.5, 1.5, (n, 1, 1)) + rng.uniform(-0.2, 0.2, (n, 4, 3))
    vol = np.einsum("ei,ei->e", X[:, 1] - X[:, 0], np.cross(X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]))
    X[vol < 0] = X[vol < 0][:, [0, 2, 1, 3]]
    U = rng.uniform(-1, 1, (n, 4, 4))
    beta = rng.uniform(-0.5, 0.5, (n, 3))
    return X, U, beta


@pytest.mark.parametrize("dt", [0.0, 0.1])
def test_tet_tangent_matches_central_differences(dt):
    X, U, beta = random_tets(3, 2)
    Up = U + np.random.default_rng(3).uniform(-0.1, 0.1, U.shape)
    p = Params(nu=0.03, dt=dt, f=(0.2, -0.1, 0.4), element="tet")
    k = oracle.element_kernel(X, U, beta, p, Up)
    Kcc, Kcf, Kfc, Kff, Rcp, Rf = oracle.pack_element(k)
    h = 1e-6
    for c in range(16):
        a, comp = divmod(c, 4)
        Upl, Umi = U.copy(), U.copy()
        Upl[:, a, comp] += h
        Umi[:, a, comp] -= h
        rp = oracle.pack_residual(oracle.element_kernel(X, Upl, beta, p, Up, with_tangent=False))
        rm = oracle.pack_residual(oracle.element_kernel(X, Umi, beta, p, Up, with_tangent=False))
        np.testing.assert_allclose(Kcc[:, :, c], (rp[0] - rm[0]) / (2 * h), rtol=1e-6, atol=1e-8)
        np.testing.assert_allclose(Kfc[:, :, c], (rp[1] - rm[1]) / (2 * h), rtol=1e-6, atol=1e-8)
    for m in range(3):
        bp, bm = beta.copy(), beta.copy()
        bp[:, m] += h
        bm[:, m] -= h
        rp = oracle.pack_residual(oracle.element_kernel(X, U, bp, p, Up, with_tangent=False))
        rm = oracle.pack_residual(oracle.element_kernel(X, U, bm, p, Up, with_tangent=False))
        np.testing.assert_allclose(Kcf[:, :, m], (rp[0] - rm[0]) / (2 * h), rtol=1e-6, atol=1e-8)
        np.testing.assert_allclose(Kff[:, :, m], (rp[1] - rm[1]) / (2 * h), rtol=1e-6, atol=1e-8)


def test_constant_states_pass_the_patch_test():
    """A constant velocity and pressure with no bubble and no force is an exact steady solution:
    the assembled coarse residual vanishes at interior nodes (the element contributions
    -p int g_a cancel around every interior node) and so does every R_f (int d = 0)."""
    wl = inputs.tet_cavity_workload(3, 100.0, jitter_frac=0.2, seed=4)
    m = wl.mesh
    u = np.tile([0.3, -0.2, 0.5, 1.7], (m.n_nodes, 1))
    X, U, _, _ = oracle.gather(m.conn, m.xyz, u, np.zeros((m.n_elems, 3)))
    k = oracle.element_kernel(X, U, np.zeros((m.n_elems, 3)), Params(nu=0.01, element="tet"),
                              with_tangent=False)
    R = oracle.assemble_vector(m.conn, m.n_nodes, oracle.pack_residual(k)[0]).reshape(-1, 4)
    inner = np.all((m.node_ijk > 0) & (m.node_ijk < 3), axis=1)
    assert np.abs(R[inner]).max() < 1e-13
    assert np.abs(k["Rf"]).max() < 1e-13


def test_tet_condensed_system_equals_uncondensed():
    """Solving the condensed system and recovering the bubbles reproduces the solution of the
    uncondensed mixed system (Section 5), on a small distorted tetrahedral mesh."""
    wl = inputs.tet_cavity_workload(2, 50.0, jitter_frac=0.2, state="random", seed=5)
    m = wl.mesh
    beta = np.random.default_rng(6).uniform(-0.2, 0.2, (m.n_elems, 3))
    p = Params(nu=wl.nu, element="tet")
    X, U, _, _ = oracle.gather(m.conn, m.xyz, wl.u, beta)
    k = oracle.element_kernel(X, U, beta, p)
    blocks = oracle.pack_element(k)
    S, r, Xk, y = oracle.condense(*blocks)
    A, rhs = oracle.assemble(m.conn, m.n_nodes, S, r)
    A, rhs = oracle.apply_dirichlet(A, rhs, wl.bc.dofs)
    du = spla.spsolve(A.tocsc(), -rhs)
    dbeta = oracle.fine_recovery(m.conn, du, Xk, y)
    K, R = oracle.uncondensed_system(m.conn, m.n_nodes, *blocks, wl.bc.dofs)
    full = np.linalg.solve(K, -R)
    np.testing.assert_allclose(du, full[:4 * m.n_nodes], rtol=0, atol=1e-9 * np.abs(full).max())
    np.testing.assert_allclose(dbeta.ravel(), full[4 * m.n_nodes:], rtol=0,
                               atol=1e-9 * np.abs(full).max())


def test_tet_newton_converges_quadratically_on_the_cavity():
    wl = inputs.tet_cavity_workload(4, 100.0, state="noise", seed=1001)
    u, beta, norms = oracle.newton_solve(wl.mesh.xyz, wl.mesh.conn, wl.u, wl.beta, wl.bc.dofs,
                                         Params(nu=wl.nu, element="tet"), tol=1e-12, maxit=12)
    r = np.array(norms) / norms[0]
    assert r[-1] <= 1e-12 and len(r) <= 7, r
    # quadratic once close: each ratio below the square of the previous one times a constant
    k = int(np.argmax(r < 1e-2))
    for i in range(k, len(r) - 1):
        if r[i + 1] > 1e-13:
            assert r[i + 1] <= 50 * r[i] ** 2, r
