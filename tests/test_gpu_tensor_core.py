"""The tensor-core modes of the tangent's basis contractions against the FP64 oracle, through the
C-ABI (element blocks, the assembled CSR system, and the full-size step channel on sampled
windows).

Bounds, relative to the largest entry of the oracle's block (the errors measured on a GB300 are
about a fifth of them):
  VMS_PREC_MIXED_TC_TF32 (TF32 high/low operands, three products): 1e-5 for the tangent blocks,
      S_e, r_e and the FP32 CSR values, as in the FP32 mixed mode (measured 2e-7 .. 1e-6);
  VMS_PREC_MIXED_TC_BF16 (BF16 operands, one product): 1e-2 for the blocks computed by the
      contractions (K_cc, K_cf, K_fc), S_e, r_e and the CSR values (measured 1e-3 .. 4e-3);
  both: K_ff (CUDA cores, FP32 sums) at 1e-5 and the FP64 residual at 1e-10.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from oracle import Params
from paper_0809_4802_gb300 import inputs

pytestmark = pytest.mark.gpu

TC_BF16, TC_TF32 = 2, 3
TOL = {TC_TF32: 1e-5, TC_BF16: 1e-2}


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
    rng = np.random.default_rng(17)
    if name == "cavity8":
        wl = inputs.cavity_workload(8, re=100.0, state="noise", seed=1001)
        beta = rng.uniform(-0.1, 0.1, (wl.mesh.n_elems, 3))
        return wl.mesh, wl.bc, wl.u, beta, Params(nu=wl.nu), None
    # 9x7x5 lattice minus a 3x2x5 block: 285 elements (not a multiple of the warps per block),
    # transient with a body force
    m = inputs.box_mesh(9, 7, 5, hi=(1.8, 1.4, 1.0), jitter_frac=0.2, seed=3,
                        hole=((2, 5), (0, 2), (0, 5)))
    bc = inputs.wall_bc(m, (0.2, 0.0, -0.1))
    u = rng.uniform(-1, 1, (m.n_nodes, 4))
    inputs.impose(u, bc)
    u_prev = u + rng.uniform(-0.05, 0.05, u.shape)
    beta = rng.uniform(-0.2, 0.2, (m.n_elems, 3))
    return m, bc, u, beta, Params(nu=0.004, dt=0.01, f=(0.1, -0.3, 1.0)), u_prev


def context(vms, prec, mesh, bc, u, beta, p, u_prev=None):
    ctx = vms.Context(0, prec)
    ctx.mesh_upload(mesh.xyz, mesh.conn, bc.dofs, bc.vals)
    ctx.set_params(p.nu, p.visc_factor, p.dt, p.f, p.bubble_scale, p.quad_order, 0)
    ctx.state_upload(np.ascontiguousarray(u), np.ascontiguousarray(beta),
                     None if u_prev is None else np.ascontiguousarray(u_prev))
    return ctx


def oracle_blocks(conn, xyz, u, beta, p, u_prev=None):
    X, U, _, Up = oracle.gather(conn, xyz, u, beta, u_prev)
    Kcc, Kcf, Kfc, Kff, Rcp, Rf = oracle.pack_element(oracle.element_kernel(X, U, beta, p, Up))
    S, r, _, _ = oracle.condense(Kcc, Kcf, Kfc, Kff, Rcp, Rf)
    return dict(S=S, r=r, Kcc=Kcc, Kcf=Kcf, Kfc=Kfc, Kff=Kff, Rcp=Rcp, Rf=Rf)


@pytest.mark.parametrize("prec", [TC_TF32, TC_BF16], ids=["tf32x3", "bf16"])
@pytest.mark.parametrize("name", ["cavity8", "box_hole_transient"])
def test_tensor_core_element_blocks_match_oracle(vms, prec, name):
    mesh, bc, u, beta, p, u_prev = case(name)
    ctx = context(vms, prec, mesh, bc, u, beta, p, u_prev)
    got = ctx.element_matrices(0, mesh.n_elems)
    ref = oracle_blocks(mesh.conn, mesh.xyz, u, beta, p, u_prev)
    for key in ("Kcc", "Kcf", "Kfc", "S", "r"):
        assert relerr(got[key], ref[key]) < TOL[prec], (key, relerr(got[key], ref[key]))
    assert relerr(got["Kff"], ref["Kff"]) < 1e-5
    for key in ("Rcp", "Rf"):
        assert relerr(got[key], ref[key]) < 1e-10, key
    # the BF16 bound is not loose for nothing: the error is well above FP32 rounding
    if prec == TC_BF16:
        assert relerr(got["Kcc"], ref["Kcc"]) > 1e-5
    ctx.close()


@pytest.mark.parametrize("prec", [TC_TF32, TC_BF16], ids=["tf32x3", "bf16"])
def test_tensor_core_assembled_system_matches_oracle(vms, prec):
    mesh, bc, u, beta, p, u_prev = case("box_hole_transient")
    ctx = context(vms, prec, mesh, bc, u, beta, p, u_prev)
    ctx.assemble()
    rowptr, colidx, vals, rhs = ctx.csr_host()
    ref = oracle_blocks(mesh.conn, mesh.xyz, u, beta, p, u_prev)
    A, r = oracle.assemble(mesh.conn, mesh.n_nodes, ref["S"], ref["r"])
    pattern = A.tocsr().copy()
    pattern.sort_indices()
    A, r = oracle.apply_dirichlet(A, r, bc.dofs)
    np.testing.assert_array_equal(rowptr, pattern.indptr)      # integer work: exact
    np.testing.assert_array_equal(colidx, pattern.indices)
    G = sp.csr_matrix((vals.astype(np.float64), colidx, rowptr), shape=A.shape)
    assert abs(G - A).max() / abs(A).max() < TOL[prec]
    assert relerr(rhs, r) < TOL[prec]
    ctx.close()


def test_tensor_core_modes_need_at_most_27_points(vms):
    mesh, bc, u, beta, p, _ = case("cavity8")
    ctx = vms.Context(0, TC_TF32)
    ctx.mesh_upload(mesh.xyz, mesh.conn, bc.dofs, bc.vals)
    with pytest.raises(vms.VmsError) as ei:
        ctx.set_params(p.nu, quad_order=4)
    assert ei.value.code == vms.ERR_UNSUPPORTED
    ctx.set_params(p.nu, quad_order=2)   # 8 points: the padding of the contractions' K dimension
    ctx.state_upload(u, beta)
    got = ctx.element_matrices(0, 40)
    ref = oracle_blocks(mesh.conn[:40], mesh.xyz, u, beta[:40], Params(nu=p.nu, quad_order=2))
    assert relerr(got["S"], ref["S"]) < 1e-5
    ctx.close()


@pytest.mark.parametrize("prec", [TC_TF32, TC_BF16], ids=["tf32x3", "bf16"])
def test_step_channel_full_size_tensor_core_sampled(vms, prec):
    """The backward-facing step at full size (518,492 hexahedra, Re 800, random state) in the
    tensor-core modes: three windows of elements against the oracle."""
    wl = inputs.bfs_workload(13, re=800.0, jitter_frac=0.1, seed=1003)
    rng = np.random.default_rng(31)
    u = rng.uniform(-0.5, 0.5, (wl.mesh.n_nodes, 4))
    inputs.impose(u, wl.bc)
    beta = rng.uniform(-0.05, 0.05, (wl.mesh.n_elems, 3))
    p = Params(nu=wl.nu)
    ctx = context(vms, prec, wl.mesh, wl.bc, u, beta, p)
    ctx.assemble()
    E = wl.mesh.n_elems
    for first in (0, E - 37, int(rng.integers(0, E - 64))):
        n = 37 if first == E - 37 else 64
        got = ctx.element_matrices(first, n)
        ref = oracle_blocks(wl.mesh.conn[first:first + n], wl.mesh.xyz, u, beta[first:first + n], p)
        assert relerr(got["S"], ref["S"]) < TOL[prec], ("S", first)
        assert relerr(got["r"], ref["r"]) < TOL[prec], ("r", first)
        assert relerr(got["Rcp"], ref["Rcp"]) < 1e-10, ("Rcp", first)
    ctx.close()
