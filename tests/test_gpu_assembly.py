"""GPU parity of the Newton-Schur assembly against the FP64 oracle, through the C-ABI.

Tolerances (relative to the largest entry of the oracle's block):
  FP64 mode: 1e-10 for every element block, S_e, r_e and the assembled CSR system;
  mixed mode: 1e-5 for the FP32 tangent blocks and S_e, r_e; 1e-10 for the FP64 residuals.
The CSR pattern (rowptr, colidx) is integer work and must match exactly.
"""
import numpy as np
import pytest
import scipy.sparse as sp

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


def upload(ctx, mesh, bc, u, beta, params: Params, u_prev=None, scatter=0):
    ctx.mesh_upload(mesh.xyz, mesh.conn, bc.dofs, bc.vals)
    ctx.set_params(params.nu, params.visc_factor, params.dt, params.f, params.bubble_scale,
                   params.quad_order, scatter)
    ctx.state_upload(np.ascontiguousarray(u), np.ascontiguousarray(beta),
                     None if u_prev is None else np.ascontiguousarray(u_prev))


def oracle_blocks(mesh, u, beta, p, u_prev=None, elems=None):
    conn = mesh.conn if elems is None else mesh.conn[elems]
    b = beta if elems is None else beta[elems]
    X, U, _, Up = oracle.gather(conn, mesh.xyz, u, b, u_prev)
    k = oracle.element_kernel(X, U, b, p, Up)
    Kcc, Kcf, Kfc, Kff, Rcp, Rf = oracle.pack_element(k)
    S, r, _, _ = oracle.condense(Kcc, Kcf, Kfc, Kff, Rcp, Rf)
    return dict(S=S, r=r, Kcc=Kcc, Kcf=Kcf, Kfc=Kfc, Kff=Kff, Rcp=Rcp, Rf=Rf)


def case_mesh(name):
    rng = np.random.default_rng(17)
    if name == "cavity8":
        wl = inputs.cavity_workload(8, re=100.0, state="noise", seed=1001)
        beta = rng.uniform(-0.1, 0.1, (wl.mesh.n_elems, 3))
        return wl.mesh, wl.bc, wl.u, beta, Params(nu=wl.nu), None
    if name == "box_hole_transient":
        # 9x7x5 lattice minus a 3x2x5 block: 285 elements, not a multiple of the warps per block
        m = inputs.box_mesh(9, 7, 5, hi=(1.8, 1.4, 1.0), jitter_frac=0.2, seed=3,
                            hole=((2, 5), (0, 2), (0, 5)))
        bc = inputs.wall_bc(m, (0.2, 0.0, -0.1))
        u = rng.uniform(-1, 1, (m.n_nodes, 4))
        inputs.impose(u, bc)
        u_prev = u + rng.uniform(-0.05, 0.05, u.shape)
        beta = rng.uniform(-0.2, 0.2, (m.n_elems, 3))
        return m, bc, u, beta, Params(nu=0.004, dt=0.01, f=(0.1, -0.3, 1.0)), u_prev
    raise KeyError(name)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["cavity8", "box_hole_transient"])
def test_element_blocks_match_oracle(vms, prec, name):
    mesh, bc, u, beta, p, u_prev = case_mesh(name)
    ctx = vms.Context(0, prec)
    upload(ctx, mesh, bc, u, beta, p, u_prev)
    got = ctx.element_matrices(0, mesh.n_elems)
    ref = oracle_blocks(mesh, u, beta, p, u_prev)
    tol = TOL[prec]
    for key in ("Kcc", "Kcf", "Kfc", "Kff", "S", "r"):
        assert relerr(got[key], ref[key]) < tol, (key, relerr(got[key], ref[key]))
    for key in ("Rcp", "Rf"):   # FP64 residual in both modes
        assert relerr(got[key], ref[key]) < 1e-10, (key, relerr(got[key], ref[key]))
    ctx.close()


@pytest.mark.parametrize("qo", [2, 4])
def test_quadrature_orders(vms, qo):
    mesh, bc, u, beta, p, _ = case_mesh("cavity8")
    p.quad_order = qo
    ctx = vms.Context(0, 0)
    upload(ctx, mesh, bc, u, beta, p)
    got = ctx.element_matrices(5, 40)
    ref = oracle_blocks(mesh, u, beta, p, elems=np.arange(5, 45))
    for key in ("S", "r", "Rcp", "Rf"):
        assert relerr(got[key], ref[key]) < 1e-10, key
    ctx.close()


def oracle_system(mesh, bc, u, beta, p, u_prev=None):
    ref = oracle_blocks(mesh, u, beta, p, u_prev)
    A, rhs = oracle.assemble(mesh.conn, mesh.n_nodes, ref["S"], ref["r"])
    pattern = A.copy()
    A, rhs = oracle.apply_dirichlet(A, rhs, bc.dofs)
    return pattern, A, rhs


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("scatter", [0, 1])
@pytest.mark.parametrize("name", ["cavity8", "box_hole_transient"])
def test_assembled_csr_matches_oracle(vms, prec, scatter, name):
    mesh, bc, u, beta, p, u_prev = case_mesh(name)
    ctx = vms.Context(0, prec)
    upload(ctx, mesh, bc, u, beta, p, u_prev, scatter)
    view = ctx.assemble()
    rowptr, colidx, vals, rhs = ctx.csr_host()
    pattern, A, rhs_ref = oracle_system(mesh, bc, u, beta, p, u_prev)
    pattern.sort_indices()
    np.testing.assert_array_equal(rowptr, pattern.indptr)
    np.testing.assert_array_equal(colidx, pattern.indices)
    G = sp.csr_matrix((vals.astype(np.float64), colidx, rowptr), shape=A.shape)
    assert relerr(G.toarray(), A.toarray()) < TOL[prec]
    assert relerr(rhs, rhs_ref) < TOL[prec]
    assert view.n_rows == 4 * mesh.n_nodes and view.nnz == pattern.nnz
    ctx.close()


def test_colour_scatter_is_deterministic(vms):
    mesh, bc, u, beta, p, _ = case_mesh("cavity8")
    ctx = vms.Context(0, 0)
    upload(ctx, mesh, bc, u, beta, p, scatter=1)
    ctx.assemble()
    v1 = ctx.csr_host()[2].copy()
    ctx.assemble()
    v2 = ctx.csr_host()[2]
    assert np.array_equal(v1, v2)
    assert ctx.csr().n_colours == 8
    ctx.close()


@pytest.mark.parametrize("name", ["cavity8", "box_hole_transient"])
def test_residual_matches_oracle(vms, name):
    mesh, bc, u, beta, p, u_prev = case_mesh(name)
    ctx = vms.Context(0, 1)
    upload(ctx, mesh, bc, u, beta, p, u_prev)
    norm, R = ctx.residual(want_vector=True)
    X, U, _, Up = oracle.gather(mesh.conn, mesh.xyz, u, beta, u_prev)
    k = oracle.element_kernel(X, U, beta, p, Up, with_tangent=False)
    Rref = oracle.residual_vector(mesh.conn, mesh.n_nodes, k, bc.dofs)
    assert relerr(R, Rref) < 1e-12
    assert abs(norm - np.linalg.norm(Rref)) < 1e-12 * np.linalg.norm(Rref)
    ctx.close()


def test_apply_matches_scipy(vms):
    import torch
    mesh, bc, u, beta, p, _ = case_mesh("cavity8")
    ctx = vms.Context(0, 0)
    upload(ctx, mesh, bc, u, beta, p)
    ctx.assemble()
    rowptr, colidx, vals, _ = ctx.csr_host()
    G = sp.csr_matrix((vals, colidx, rowptr))
    x = np.random.default_rng(2).standard_normal(G.shape[0])
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    ctx.apply(xd, yd)
    torch.cuda.synchronize()
    assert relerr(yd.cpu().numpy(), G @ x) < 1e-13
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_cavity32_sampled(vms, prec):
    """The 32^3 jittered cavity at Re 400 with a random state (32,768 elements), assembled in the
    configuration the benchmark times; sampled elements and sampled CSR rows against the oracle."""
    wl = inputs.cavity_workload(32, re=400.0, jitter_frac=0.15, state="random", seed=1002)
    mesh, bc = wl.mesh, wl.bc
    rng = np.random.default_rng(5)
    beta = np.zeros((mesh.n_elems, 3))
    p = Params(nu=wl.nu)
    ctx = vms.Context(0, prec)
    upload(ctx, mesh, bc, wl.u, beta, p)
    ctx.assemble()
    rowptr, colidx, vals, rhs = ctx.csr_host()
    # sampled element blocks (first, last, random)
    for first in (0, mesh.n_elems - 37, int(rng.integers(0, mesh.n_elems - 64))):
        n = 37 if first == mesh.n_elems - 37 else 64
        got = ctx.element_matrices(first, n)
        ref = oracle_blocks(mesh, wl.u, beta, p, elems=np.arange(first, first + n))
        for key in ("S", "r"):
            assert relerr(got[key], ref[key]) < TOL[prec], key
        assert relerr(got["Rcp"], ref["Rcp"]) < 1e-10
    # sampled rows: every row of node n receives contributions only from elements touching n
    nodes = rng.choice(mesh.n_nodes, 40, replace=False)
    touch = np.nonzero(np.isin(mesh.conn, nodes).any(axis=1))[0]
    ref = oracle_blocks(mesh, wl.u, beta, p, elems=touch)
    A, r = oracle.assemble(mesh.conn[touch], mesh.n_nodes, ref["S"], ref["r"])
    A, r = oracle.apply_dirichlet(A, r, bc.dofs)
    G = sp.csr_matrix((vals.astype(np.float64), colidx, rowptr), shape=A.shape)
    rows = (4 * nodes[:, None] + np.arange(4)[None, :]).ravel()
    Gr, Ar = G[rows].toarray(), A[rows].toarray()
    assert relerr(Gr, Ar) < TOL[prec]
    assert relerr(rhs[rows], r[rows]) < TOL[prec]
    ctx.close()


def test_error_paths(vms):
    mesh, bc, u, beta, p, _ = case_mesh("cavity8")
    ctx = vms.Context(0, 0)
    with pytest.raises(vms.VmsError) as ei:
        ctx.assemble()
    assert ei.value.code == vms.ERR_STATE
    upload(ctx, mesh, bc, u, beta, p)
    with pytest.raises(vms.VmsError) as ei:
        ctx.element_matrices(mesh.n_elems - 1, 5)
    assert ei.value.code == vms.ERR_INVALID_ARG
    # a NaN in the state is reported, not propagated silently
    bad = u.copy(); bad[300, 3] = np.nan
    ctx.state_upload(bad, beta)
    with pytest.raises(vms.VmsError) as ei:
        ctx.residual()
    assert ei.value.code == vms.ERR_NAN
    # an inverted element: mirror one element's nodes through its centre
    m2 = inputs.cavity_mesh(3)
    conn = m2.conn.copy()
    conn[4] = conn[4][[1, 0, 3, 2, 5, 4, 7, 6]]
    with pytest.raises(ValueError):
        ctx.mesh_upload(m2.xyz, conn[:, :7].copy(), bc.dofs[:0], bc.vals[:0])
    bad_conn = conn.copy(); bad_conn[0, 0] = m2.n_nodes
    with pytest.raises(vms.VmsError) as ei:
        ctx.mesh_upload(m2.xyz, bad_conn, np.zeros(0, np.int64), np.zeros(0))
    assert ei.value.code == vms.ERR_INVALID_ARG
    ctx.mesh_upload(m2.xyz, conn, np.zeros(0, np.int64), np.zeros(0))
    ctx.state_upload(np.zeros((m2.n_nodes, 4)))
    with pytest.raises(vms.VmsError) as ei:
        ctx.assemble()
    assert ei.value.code == vms.ERR_NEG_JACOBIAN
    ctx.close()
