"""vms_residual_norm_noalloc: the residual norm for callers that cannot allocate device memory.

Such callers (a process whose device memory belongs to its own pool, or a loop that must not pay
the device synchronisation of cudaMalloc/cudaFree) pass every input and output as device memory;
the call keeps its scratch space in a fixed device array of the library. This test calls it
through the C-ABI twice in a row and compares each result with the context-based vms_residual,
within the same 1e-12 relative tolerance as the other residual tests. It lives in its own file,
collected last, and passes both alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_residual_norm_matches_vms_residual_twice():
    import torch

    from paper_0809_4802_gb300 import build, inputs, vms
    build.build()
    lib = vms.load_library()
    wl = inputs.cavity_workload(12, re=400.0, jitter_frac=0.15, state="random", seed=1002)
    mesh, bc = wl.mesh, wl.bc
    beta = np.random.default_rng(4).uniform(-0.05, 0.05, (mesh.n_elems, 3))
    u_prev = wl.u + np.random.default_rng(5).uniform(-0.01, 0.01, wl.u.shape)

    ctx = vms.Context(0, vms.PREC_FP64)
    ctx.mesh_upload(mesh.xyz, mesh.conn, bc.dofs, bc.vals)
    ctx.set_params(wl.nu, dt=0.02, f=(0.0, 0.0, -0.5))
    ctx.state_upload(wl.u, beta, u_prev)
    ref = ctx.residual()
    u_imposed, _ = ctx.state_download()   # the context imposes the Dirichlet values on upload
    ctx.close()

    dev = torch.device("cuda:0")
    xyz = torch.tensor(mesh.xyz, dtype=torch.float64, device=dev).contiguous()
    conn = torch.tensor(mesh.conn, dtype=torch.int32, device=dev).contiguous()
    dofs = torch.tensor(bc.dofs, dtype=torch.int64, device=dev)
    u = torch.tensor(u_imposed, dtype=torch.float64, device=dev).contiguous()
    b = torch.tensor(beta, dtype=torch.float64, device=dev).contiguous()
    up = torch.tensor(u_prev, dtype=torch.float64, device=dev).contiguous()
    norm = torch.zeros(1, dtype=torch.float64, device=dev)
    status = torch.full((1,), 12345, dtype=torch.int32, device=dev)
    params = vms.VmsParams(wl.nu, 2.0, 0.02, (ctypes.c_double * 3)(0.0, 0.0, -0.5), 1.0, 3, 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    torch.cuda.synchronize()

    for _ in range(2):
        norm.fill_(-1.0)
        rc = lib.vms_residual_norm_noalloc(
            mesh.n_nodes, xyz.data_ptr(), mesh.n_elems, conn.data_ptr(), int(dofs.numel()),
            dofs.data_ptr(), u.data_ptr(), b.data_ptr(), up.data_ptr(), ctypes.byref(params),
            norm.data_ptr(), status.data_ptr(), ctypes.c_void_p(stream))
        assert rc == vms.OK
        torch.cuda.synchronize()
        assert int(status.item()) == vms.OK
        got = float(norm.item())
        assert abs(got - ref) <= 1e-12 * ref, (got, ref)

    # sizes beyond the fixed scratch are rejected before any work is queued
    too_many = vms.NOALLOC_MAX_ENTRIES // 4 + 1
    rc = lib.vms_residual_norm_noalloc(
        too_many, xyz.data_ptr(), mesh.n_elems, conn.data_ptr(), 0, None, u.data_ptr(), None,
        None, ctypes.byref(params), norm.data_ptr(), status.data_ptr(), ctypes.c_void_p(stream))
    assert rc == vms.ERR_TOO_LARGE
