"""vms_residual_norm_noalloc: the residual norm for callers that cannot allocate device memory.

Such callers (a process whose device memory belongs to its own pool, or a loop that must not pay
the device synchronisation of cudaMalloc/cudaFree) pass every input and output as device memory;
the call keeps its scratch space in a fixed device array of the library. These tests call it
through the C-ABI twice in a row and compare each result with the context-based vms_residual,
within the same 1e-12 relative tolerance as the other residual tests, for steady and transient
parameters with and without a body force and with u_prev omitted; they also check the status
words it writes (an index outside the mesh, a non-finite state) and the size limit. They live in
their own file, collected last, and pass both alone in a fresh process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CASES = [  # (dt, body force, pass u_prev)
    (0.0, (0.0, 0.0, 0.0), True),
    (0.02, (0.0, 0.0, 0.0), True),
    (0.02, (0.0, 0.0, -0.5), True),
    (0.02, (0.3, 0.0, 0.0), False),
]


@pytest.fixture(scope="module")
def setup():
    import torch

    from paper_0809_4802_gb300 import build, inputs, vms
    build.build()
    lib = vms.load_library()
    wl = inputs.cavity_workload(12, re=400.0, jitter_frac=0.15, state="random", seed=1002)
    beta = np.random.default_rng(4).uniform(-0.05, 0.05, (wl.mesh.n_elems, 3))
    u_prev = wl.u + np.random.default_rng(5).uniform(-0.01, 0.01, wl.u.shape)
    dev = torch.device("cuda:0")
    t = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev).contiguous()  # noqa: E731
    d = dict(torch=torch, vms=vms, lib=lib, wl=wl, beta=beta, u_prev=u_prev, dev=dev,
             xyz=t(wl.mesh.xyz, torch.float64), conn=t(wl.mesh.conn, torch.int32),
             dofs=t(wl.bc.dofs, torch.int64), b=t(beta, torch.float64),
             up=t(u_prev, torch.float64),
             norm=torch.zeros(1, dtype=torch.float64, device=dev),
             status=torch.full((1,), 12345, dtype=torch.int32, device=dev),
             stream=torch.cuda.current_stream(dev).cuda_stream)
    return d


def reference_norm(d, dt, f, with_prev):
    vms, wl = d["vms"], d["wl"]
    ctx = vms.Context(0, vms.PREC_FP64)
    ctx.mesh_upload(wl.mesh.xyz, wl.mesh.conn, wl.bc.dofs, wl.bc.vals)
    ctx.set_params(wl.nu, dt=dt, f=f)
    ctx.state_upload(wl.u, d["beta"], d["u_prev"] if with_prev else None)
    ref = ctx.residual()
    u_imposed, _ = ctx.state_download()   # the context imposes the Dirichlet values on upload
    ctx.close()
    return ref, u_imposed


def call(d, u, dt, f, up, dofs=None, n_nodes=None):
    vms, wl = d["vms"], d["wl"]
    params = vms.VmsParams(wl.nu, 2.0, dt, (ctypes.c_double * 3)(*f), 1.0, 3, 0)
    dofs = d["dofs"] if dofs is None else dofs
    return d["lib"].vms_residual_norm_noalloc(
        wl.mesh.n_nodes if n_nodes is None else n_nodes, d["xyz"].data_ptr(), wl.mesh.n_elems,
        d["conn"].data_ptr(), int(dofs.numel()), dofs.data_ptr(), u.data_ptr(),
        d["b"].data_ptr(), None if up is None else up.data_ptr(), ctypes.byref(params),
        d["norm"].data_ptr(), d["status"].data_ptr(), ctypes.c_void_p(d["stream"]))


@pytest.mark.parametrize("dt,f,with_prev", CASES)
def test_noalloc_residual_norm_matches_vms_residual_twice(setup, dt, f, with_prev):
    d = setup
    torch, vms = d["torch"], d["vms"]
    ref, u_imposed = reference_norm(d, dt, f, with_prev)
    u = torch.tensor(u_imposed, dtype=torch.float64, device=d["dev"]).contiguous()
    torch.cuda.synchronize()
    for _ in range(2):
        d["norm"].fill_(-1.0)
        d["status"].fill_(12345)
        rc = call(d, u, dt, f, d["up"] if with_prev else None)
        assert rc == vms.OK
        torch.cuda.synchronize()
        assert int(d["status"].item()) == vms.OK
        got = float(d["norm"].item())
        assert abs(got - ref) <= 1e-12 * ref, (got, ref)


def test_noalloc_status_words_and_size_limit(setup):
    d = setup
    torch, vms, wl = d["torch"], d["vms"], d["wl"]
    _, u_imposed = reference_norm(d, 0.0, (0.0, 0.0, 0.0), True)
    u = torch.tensor(u_imposed, dtype=torch.float64, device=d["dev"]).contiguous()

    # a constrained dof outside the mesh: skipped and reported, the norm is still finite
    bad = torch.cat([d["dofs"], torch.tensor([4 * wl.mesh.n_nodes + 7], dtype=torch.int64,
                                             device=d["dev"])])
    assert call(d, u, 0.0, (0.0, 0.0, 0.0), None, dofs=bad) == vms.OK
    torch.cuda.synchronize()
    assert int(d["status"].item()) == vms.ERR_INVALID_ARG
    assert np.isfinite(float(d["norm"].item()))

    # a non-finite state value
    un = u.clone()
    un[wl.mesh.n_nodes // 2, 0] = float("nan")
    assert call(d, un, 0.0, (0.0, 0.0, 0.0), None) == vms.OK
    torch.cuda.synchronize()
    assert int(d["status"].item()) == vms.ERR_NAN

    # the next call starts from a cleared scratch array: OK again
    assert call(d, u, 0.0, (0.0, 0.0, 0.0), None) == vms.OK
    torch.cuda.synchronize()
    assert int(d["status"].item()) == vms.OK

    # sizes beyond the fixed scratch are rejected before any work is queued
    assert call(d, u, 0.0, (0.0, 0.0, 0.0), None,
                n_nodes=vms.NOALLOC_MAX_ENTRIES // 4 + 1) == vms.ERR_TOO_LARGE
