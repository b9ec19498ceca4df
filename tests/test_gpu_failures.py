"""Failure detection of the GPU path, without a GPU fault: every failure is made on the host (an
iteration limit, a state, a wait limit) and must come back as a status code with the context
still usable.

  VMS_ERR_TIMEOUT          the ILU(0) kernels' device-side waits are bounded; a wait limit of one
                           poll makes them give up, the solve reports it and leaves the state
                           unchanged, and the same context solves once the default limit is back
  VMS_ERR_NEWTON_DIVERGED  Newton with an iteration limit it cannot meet
  VMS_ERR_SINGULAR_KFF     a bubble block K_ff whose determinant underflows to zero
"""
import numpy as np
import pytest

from paper_0809_4802_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vms():
    from paper_0809_4802_gb300 import build, vms as v
    build.build()
    v.load_library()
    return v


def cavity_ctx(vms, prec, n=8):
    wl = inputs.cavity_workload(n, re=100.0, state="noise", seed=1001)
    ctx = vms.Context(0, prec)
    ctx.mesh_upload(wl.mesh.xyz, wl.mesh.conn, wl.bc.dofs, wl.bc.vals)
    ctx.set_params(wl.nu)
    ctx.state_upload(wl.u, wl.beta)
    return ctx, wl


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_wait_limit_timeout_is_reported_and_context_recovers(vms, prec):
    """With one poll per wait the factorisation's row hand-overs and the sweeps' dependencies cannot
    all be met in time: the solve returns VMS_ERR_TIMEOUT with the state unchanged. Restoring the
    default limit, the same context solves the same system."""
    ctx, wl = cavity_ctx(vms, prec)
    u0, b0 = ctx.state_download()
    ctx.assemble()
    ctx.set_wait_limit(1)
    with pytest.raises(vms.VmsError) as ei:
        ctx.solve(rtol=1e-8, maxit=200, restart=50, update=True)
    assert ei.value.code == vms.ERR_TIMEOUT
    u1, b1 = ctx.state_download()
    np.testing.assert_array_equal(u1, u0)
    np.testing.assert_array_equal(b1, b0)
    ctx.set_wait_limit(0)
    it, rel = ctx.solve(rtol=1e-6, maxit=3000, restart=150, update=True)
    assert rel <= 1e-6 and it > 0
    with pytest.raises(vms.VmsError) as ei:
        ctx.set_wait_limit(-1)
    assert ei.value.code == vms.ERR_INVALID_ARG
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_newton_iteration_limit_reports_divergence(vms, prec):
    """One Newton step cannot reach 1e-10 from the noisy start of the 8^3 cavity: the driver
    reports VMS_ERR_NEWTON_DIVERGED after one step, and the state it leaves solves on."""
    ctx, wl = cavity_ctx(vms, prec)
    r0 = ctx.residual()
    with pytest.raises(vms.VmsError) as ei:
        ctx.newton_solve(rtol=1e-10, maxit=1)
    assert ei.value.code == vms.ERR_NEWTON_DIVERGED
    assert ctx.residual() < r0          # the one step was taken
    it, hist = ctx.newton_solve(rtol=1e-8 * r0 / ctx.residual(), maxit=20)
    assert hist[-1] <= 1e-8 * r0 * 1.0001
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_singular_bubble_block_is_reported(vms, prec):
    """At rest (v = 0, beta = 0) K_ff = nut int(d.d) I; with nu = 1e-120 its determinant
    (~1e-360) underflows to exactly zero in FP64, and its entries to zero in FP32: the assembly
    reports VMS_ERR_SINGULAR_KFF. The same context assembles once nu is physical again."""
    mesh = inputs.cavity_mesh(3)
    bottom = np.nonzero(mesh.node_ijk[:, 2] == 0)[0]
    dofs = np.sort(np.concatenate([4 * bottom + c for c in range(3)]))
    ctx = vms.Context(0, prec)
    ctx.mesh_upload(mesh.xyz, mesh.conn, dofs, np.zeros(dofs.size))
    ctx.set_params(1e-120)
    ctx.state_upload(np.zeros((mesh.n_nodes, 4)), np.zeros((mesh.n_elems, 3)))
    with pytest.raises(vms.VmsError) as ei:
        ctx.assemble()
    assert ei.value.code == vms.ERR_SINGULAR_KFF
    ctx.set_params(0.01)
    ctx.assemble()
    ctx.close()
