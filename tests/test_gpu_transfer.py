"""The asynchronous download of the assembled system (vms_csr_download_async / _wait): the values
that land in host memory are those of the assembly before the call, even when the next assembly
(of another state) runs before the wait; pattern and right-hand side likewise."""
import numpy as np
import pytest

from paper_0809_4802_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("graph", [False, True], ids=["two-buffers", "graph-snapshot"])
def test_async_download_snapshots_the_assembly_before_it(graph):
    """Without a captured graph the next assembly writes the second values buffer while the copy
    reads the first; with one, the values are copied into a device snapshot first."""
    import torch
    from paper_0809_4802_gb300 import build, vms
    build.build()
    vms.load_library()
    wl = inputs.cavity_workload(10, re=300.0, jitter_frac=0.1, state="random", seed=5)
    for prec in (vms.PREC_MIXED, vms.PREC_FP64):
        ctx = vms.Context(0, prec)
        ctx.mesh_upload(wl.mesh.xyz, wl.mesh.conn, wl.bc.dofs, wl.bc.vals)
        ctx.set_params(wl.nu)
        ctx.set_graph(graph)
        ctx.state_upload(wl.u, wl.beta)
        ctx.assemble()
        rowptr, colidx, vals, rhs = ctx.csr_host()          # synchronous reference
        dt = torch.float32 if prec == vms.PREC_MIXED else torch.float64
        v_h = torch.empty(vals.size, dtype=dt).pin_memory()
        r_h = torch.empty(rhs.size, dtype=torch.float64).pin_memory()
        rp_h = torch.empty(rowptr.size, dtype=torch.int32).pin_memory()
        ci_h = torch.empty(colidx.size, dtype=torch.int32).pin_memory()
        ctx.csr_download_async(rowptr=rp_h, colidx=ci_h, values=v_h, rhs=r_h)
        # another state assembled before the wait: it must not reach the buffers
        ctx.state_upload(wl.u * 1.5, wl.beta)
        ctx.assemble()
        ctx.csr_download_wait()
        np.testing.assert_array_equal(v_h.numpy(), vals)
        np.testing.assert_array_equal(r_h.numpy(), rhs)
        np.testing.assert_array_equal(rp_h.numpy(), rowptr)
        np.testing.assert_array_equal(ci_h.numpy(), colidx)
        # the second assembly's system by a second async download (the first is waited for)
        ctx.csr_download_async(values=v_h, rhs=r_h)
        ctx.csr_download_wait()
        _, _, vals2, rhs2 = ctx.csr_host()
        np.testing.assert_array_equal(v_h.numpy(), vals2)
        np.testing.assert_array_equal(r_h.numpy(), rhs2)
        assert np.abs(vals2 - vals).max() > 0
        ctx.csr_download_wait()   # nothing pending: returns at once
        # a third assembly after the copies: the values are those of its state (up to the order in
        # which the atomic scatter sums)
        ctx.state_upload(wl.u, wl.beta)
        ctx.assemble()
        _, _, vals3, _ = ctx.csr_host()
        tol = 1e-5 if prec == vms.PREC_MIXED else 1e-12
        assert np.abs(vals3.astype(np.float64) - vals).max() <= tol * np.abs(vals).max()
        ctx.close()
