"""GPU parity of the tetrahedral P1 + bubble element against the FP64 oracle, through the C-ABI.

The tetrahedral kernel computes in FP64 in both precision modes, so its element blocks agree with
the oracle to 1e-10 of the block's largest entry in both; in mixed precision the assembled CSR
values are stored in FP32 (1e-6). Quadrature orders 2 (8 points), 3 (27) and 4 (64, more points
than lanes) are covered; meshes are the Kuhn tetrahedra of jittered lattices.
"""
import numpy as np
import pytest
import scipy.sparse as sp

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


def relerr(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def case(name):
    rng = np.random.default_rng(21)
    if name == "cavity":
        wl = inputs.tet_cavity_workload(3, 400.0, jitter_frac=0.2, state="random", seed=22)
        beta = rng.uniform(-0.1, 0.1, (wl.mesh.n_elems, 3))
        return wl.mesh, wl.bc, wl.u, beta, Params(nu=wl.nu, element="tet"), None
    if name == "box_transient":
        # 5x4x3 lattice minus a 2x2x3 block (jittered), Kuhn tetrahedra: 288 elements
        hexm = inputs.box_mesh(5, 4, 3, hi=(1.25, 1.0, 0.75), jitter_frac=0.2, seed=23,
                               hole=((1, 3), (0, 2), (0, 3)))
        m = inputs.tet_mesh_from_lattice(hexm)
        bc = inputs.wall_bc(hexm, (0.2, 0.0, -0.1))
        u = rng.uniform(-1, 1, (m.n_nodes, 4))
        inputs.impose(u, bc)
        u_prev = u + rng.uniform(-0.05, 0.05, u.shape)
        beta = rng.uniform(-0.2, 0.2, (m.n_elems, 3))
        return m, bc, u, beta, Params(nu=0.004, dt=0.01, f=(0.1, -0.3, 1.0), element="tet"), u_prev
    raise KeyError(name)


def upload(ctx, mesh, bc, u, beta, p, u_prev=None, scatter=0):
    ctx.mesh_upload(mesh.xyz, mesh.conn, bc.dofs, bc.vals)
    ctx.set_params(p.nu, p.visc_factor, p.dt, p.f, p.bubble_scale, p.quad_order, scatter)
    ctx.state_upload(np.ascontiguousarray(u), np.ascontiguousarray(beta),
                     None if u_prev is None else np.ascontiguousarray(u_prev))


def oracle_blocks(mesh, u, beta, p, u_prev=None):
    X, U, _, Up = oracle.gather(mesh.conn, mesh.xyz, u, beta, u_prev)
    k = oracle.element_kernel(X, U, beta, p, Up)
    Kcc, Kcf, Kfc, Kff, Rcp, Rf = oracle.pack_element(k)
    S, r, _, _ = oracle.condense(Kcc, Kcf, Kfc, Kff, Rcp, Rf)
    return dict(S=S, r=r, Kcc=Kcc, Kcf=Kcf, Kfc=Kfc, Kff=Kff, Rcp=Rcp, Rf=Rf)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["cavity", "box_transient"])
def test_tet_element_blocks_match_oracle(vms, prec, name):
    mesh, bc, u, beta, p, u_prev = case(name)
    ctx = vms.Context(0, prec)
    upload(ctx, mesh, bc, u, beta, p, u_prev)
    got = ctx.element_matrices(0, mesh.n_elems)
    ref = oracle_blocks(mesh, u, beta, p, u_prev)
    for key in ("Kcc", "Kcf", "Kfc", "Kff", "S", "r", "Rcp", "Rf"):
        assert relerr(got[key], ref[key]) <= 1e-10, (key, relerr(got[key], ref[key]))
    ctx.close()


@pytest.mark.parametrize("qo", [2, 4])
def test_tet_quadrature_orders(vms, qo):
    mesh, bc, u, beta, p, u_prev = case("box_transient")
    p.quad_order = qo
    ctx = vms.Context(0, 0)
    upload(ctx, mesh, bc, u, beta, p, u_prev)
    got = ctx.element_matrices(0, mesh.n_elems)
    ref = oracle_blocks(mesh, u, beta, p, u_prev)
    for key in ("S", "r", "Kff"):
        assert relerr(got[key], ref[key]) <= 1e-10, (qo, key)
    ctx.close()


@pytest.mark.parametrize("prec,scatter", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_tet_assembled_system_matches_oracle(vms, prec, scatter):
    mesh, bc, u, beta, p, u_prev = case("box_transient")
    ctx = vms.Context(0, prec)
    upload(ctx, mesh, bc, u, beta, p, u_prev, scatter)
    ctx.assemble()
    rowptr, colidx, vals, rhs = ctx.csr_host()
    G = sp.csr_matrix((vals.astype(np.float64), colidx, rowptr))
    ref = oracle_blocks(mesh, u, beta, p, u_prev)
    A, rref = oracle.assemble(mesh.conn, mesh.n_nodes, ref["S"], ref["r"])
    A, rref = oracle.apply_dirichlet(A, rref, bc.dofs)
    tol = 1e-10 if prec == 0 else 1e-6
    assert relerr(G.toarray(), A.toarray()) <= tol
    assert relerr(rhs, rref) <= 1e-10
    ctx.close()


def test_tet_residual_matches_oracle(vms):
    mesh, bc, u, beta, p, u_prev = case("box_transient")
    ctx = vms.Context(0, 0)
    upload(ctx, mesh, bc, u, beta, p, u_prev)
    norm, R = ctx.residual(want_vector=True)
    X, U, _, Up = oracle.gather(mesh.conn, mesh.xyz, ctx.state_download()[0], beta, u_prev)
    k = oracle.element_kernel(X, U, beta, p, Up, with_tangent=False)
    Rref = oracle.residual_vector(mesh.conn, mesh.n_nodes, k, bc.dofs)
    assert relerr(R, Rref) <= 1e-10
    assert abs(norm - np.linalg.norm(Rref)) <= 1e-10 * np.linalg.norm(Rref)
    ctx.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-8)])
def test_tet_newton_cavity_matches_oracle(vms, prec, tol):
    """Newton-Schur on the 4^3 tetrahedral lid-driven cavity at Re 100 (the element has no
    spurious pressure modes, so velocity and pressure are both compared with the oracle)."""
    wl = inputs.tet_cavity_workload(4, 100.0, state="noise", seed=1001)
    p = Params(nu=wl.nu, element="tet")
    ctx = vms.Context(0, prec)
    ctx.mesh_upload(wl.mesh.xyz, wl.mesh.conn, wl.bc.dofs, wl.bc.vals)
    ctx.set_params(wl.nu)
    ctx.state_upload(wl.u, wl.beta)
    its, hist = ctx.newton_solve(rtol=tol, maxit=12)
    assert hist[-1] <= tol * hist[0] and its <= 8, hist
    u, beta = ctx.state_download()
    uo, bo, norms = oracle.newton_solve(wl.mesh.xyz, wl.mesh.conn, wl.u, wl.beta, wl.bc.dofs, p,
                                        tol=1e-12, maxit=15)
    assert abs(hist[0] - norms[0]) <= 1e-12 * norms[0]
    err_tol = 1e-7 if prec == 0 else 1e-5
    assert relerr(u, uo) <= err_tol, relerr(u, uo)
    ctx.close()
