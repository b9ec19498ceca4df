"""The learned warm start on the GPU: the network's forward pass, gradient and Adam step against the
FP64 oracle (oracle/warmstart.py) with the same BF16 weights, the node features against the
oracle's 1-ring mean, and the gain of the trained network over the previous-step start on a
transient cavity (Newton converges to the same absolute target from both starts).

Tolerances: the kernels accumulate in FP32 over at most 128 terms and use FP32 tanh; the 128-wide
contractions run on BF16 tensor cores with the FP32 activations split into three BF16 terms
(forward, D W2^T) or two (H1^T D, three products), about 2^-24 and 2^-16 of each term; outputs
1e-5 of the largest output, gradients 1e-4 of each block's largest entry, Adam 1e-6.
"""
import numpy as np
import pytest

from oracle import warmstart as ows
from paper_0809_4802_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_0809_4802_gb300 import build, vms
    build.build()
    vms.load_library()
    return vms, torch, torch.device("cuda:0")


def params(seed=3):
    p = inputs.mlp_init(seed).astype(np.float64)
    rng = np.random.default_rng(seed)
    q = ows.unpack(p)
    for b in ("b1", "b2", "b3"):
        q[b] = rng.uniform(-0.3, 0.3, q[b].shape)
    return ows.pack(q).astype(np.float32)


def blocks_relerr(g, ref):
    gb, rb = ows.unpack(g), ows.unpack(ref)
    return {k: float(np.abs(gb[k] - rb[k]).max() / max(np.abs(rb[k]).max(), 1e-30)) for k in rb}


def test_forward_matches_oracle_and_weights_are_bf16(env):
    vms, torch, dev = env
    mlp = vms.Mlp(0)
    p = params(3)
    mlp.set_params(p)
    stored = mlp.get_params(stored=True)
    ref = ows.stored(p)
    np.testing.assert_array_equal(stored.astype(np.float64), ows.pack(ref))   # BF16 rounding, exact
    np.testing.assert_array_equal(mlp.get_params(stored=False), p)
    n = 1000   # 15 full tiles of 64 rows and a ragged one
    X = np.random.default_rng(1).normal(size=(n, ows.N_IN)).astype(np.float32)
    Xd = torch.from_numpy(X).to(dev)
    Yd = torch.empty((n, ows.N_OUT), dtype=torch.float32, device=dev)
    mlp.forward(Xd, Yd)
    y_ref, _ = ows.forward(ref, X.astype(np.float64))
    y = Yd.cpu().numpy()
    assert np.abs(y - y_ref).max() <= 1e-5 * np.abs(y_ref).max()
    mlp.close()


def test_gradient_and_loss_match_oracle(env):
    vms, torch, dev = env
    mlp = vms.Mlp(0)
    p = params(4)
    mlp.set_params(p)
    rng = np.random.default_rng(2)
    X = rng.normal(size=(1000, ows.N_IN)).astype(np.float32)
    T = rng.normal(size=(1000, ows.N_OUT)).astype(np.float32)
    rows = rng.permutation(1000)[:777].astype(np.int32)   # ragged, through an index list
    loss, g = mlp.grad(torch.from_numpy(X).to(dev), torch.from_numpy(T).to(dev),
                       rows=torch.from_numpy(rows).to(dev))
    lref, gref = ows.loss_and_grad(ows.stored(p), X[rows].astype(np.float64), T[rows].astype(np.float64))
    assert abs(loss - lref) <= 1e-5 * lref
    err = blocks_relerr(g.astype(np.float64), ows.pack(gref))
    assert max(err.values()) <= 1e-4, err
    # and over the first n rows without an index list
    loss2, g2 = mlp.grad(torch.from_numpy(X).to(dev), torch.from_numpy(T).to(dev), n=130)
    lref2, gref2 = ows.loss_and_grad(ows.stored(p), X[:130].astype(np.float64), T[:130].astype(np.float64))
    assert abs(loss2 - lref2) <= 1e-5 * lref2
    assert max(blocks_relerr(g2.astype(np.float64), ows.pack(gref2)).values()) <= 1e-4
    mlp.close()


def test_adam_steps_match_oracle(env):
    vms, torch, dev = env
    mlp = vms.Mlp(0)
    p = params(5)
    mlp.set_params(p)
    rng = np.random.default_rng(3)
    X = torch.from_numpy(rng.normal(size=(300, ows.N_IN)).astype(np.float32)).to(dev)
    T = torch.from_numpy(rng.normal(size=(300, ows.N_OUT)).astype(np.float32)).to(dev)
    w, m, v = p.astype(np.float64), np.zeros(ows.N_PARAMS), np.zeros(ows.N_PARAMS)
    for t in (1, 2, 3):
        _, g = mlp.grad(X, T)
        mlp.adam(1e-3)
        w, m, v = ows.adam_step(w, g.astype(np.float64), m, v, t, 1e-3)
        got = mlp.get_params(stored=False).astype(np.float64)
        assert np.abs(got - w).max() <= 1e-6, t
        np.testing.assert_array_equal(mlp.get_params(stored=True).astype(np.float64),
                                      ows.pack(ows.stored(got)))
    mlp.close()


def test_training_reduces_the_loss(env):
    vms, torch, dev = env
    mlp = vms.Mlp(0)
    mlp.set_params(inputs.mlp_init(6))
    rng = np.random.default_rng(4)
    X = rng.normal(size=(4096, ows.N_IN)).astype(np.float32)
    T = (0.5 * X[:, :4] - 0.3 * X[:, 4:8] + 0.2 * np.tanh(X[:, 8:12])).astype(np.float32)
    Xd, Td = torch.from_numpy(X).to(dev), torch.from_numpy(T).to(dev)
    l0, _ = mlp.grad(Xd, Td)
    for it in range(300):
        rows = torch.from_numpy(rng.permutation(4096)[:512].astype(np.int32)).to(dev)
        mlp.grad(Xd, Td, rows=rows, want=False)
        mlp.adam(3e-3)
    l1, _ = mlp.grad(Xd, Td)
    assert l1 < 0.05 * l0, (l0, l1)
    mlp.close()


def test_node_features_increment_and_shift(env):
    vms, torch, dev = env
    wl = inputs.cavity_workload(4, re=100.0, jitter_frac=0.1, state="random", seed=9)
    u_prev = wl.u + np.random.default_rng(8).normal(scale=0.1, size=wl.u.shape)
    ctx = vms.Context(0, 0)
    ctx.mesh_upload(wl.mesh.xyz, wl.mesh.conn, wl.bc.dofs, wl.bc.vals)
    ctx.set_params(wl.nu, dt=0.05)
    ctx.state_upload(wl.u, wl.beta, u_prev)
    n = wl.mesh.n_nodes
    X = torch.empty((n, 12), dtype=torch.float32, device=dev)
    scale = np.linspace(0.5, 2.0, 12).astype(np.float32)
    ctx.node_features(X, scale)
    ref = ows.features(wl.mesh.conn, wl.u, u_prev, scale)
    assert np.abs(X.cpu().numpy() - ref).max() <= 1e-6 * np.abs(ref).max()
    D = torch.empty((n, 4), dtype=torch.float32, device=dev)
    ctx.node_increment(D)
    assert np.abs(D.cpu().numpy() - (wl.u - u_prev)).max() <= 1e-6 * np.abs(wl.u - u_prev).max()
    # u += D moves the state back to u_prev except where Dirichlet values are imposed
    D.neg_()
    ctx.apply_increment(D)
    u2, _ = ctx.state_download()
    free = np.ones(4 * n, bool)
    free[wl.bc.dofs] = False
    assert np.abs(u2.reshape(-1)[free] - u_prev.reshape(-1)[free]).max() <= 1e-6
    np.testing.assert_array_equal(u2.reshape(-1)[wl.bc.dofs], wl.bc.vals)
    # shift_time: u_prev <- u (the increment is then zero)
    ctx.shift_time()
    ctx.node_increment(D)
    assert float(D.abs().max()) == 0.0
    ctx.close()


def test_trained_warm_start_beats_previous_step_start(env):
    """Decaying vortex in a closed 6^3 box (jittered 0.1 h, Re 200, dt 0.02, FP64): 14 recorded
    steps train the network; on steps 15-22 the predicted start has a much smaller residual than
    the previous-step start and Newton needs no more iterations to reach the same absolute
    target (1e-8 of the previous-step start's residual)."""
    vms, torch, dev = env
    from paper_0809_4802_gb300 import transient as tr

    def fresh():
        wl = inputs.vortex_box_workload(6, re=200.0, dt=0.02, jitter_frac=0.1)
        ctx = vms.Context(0, 0)
        ctx.mesh_upload(wl.mesh.xyz, wl.mesh.conn, wl.bc.dofs, wl.bc.vals)
        ctx.set_params(wl.nu, dt=wl.dt)
        ctx.state_upload(wl.u, wl.beta, wl.u_prev)
        return ctx

    ctx = fresh()
    rec = tr.Recorder()
    tr.run_steps(vms, ctx, 14, rtol=1e-8, record=rec)
    base = tr.run_steps(vms, ctx, 8, rtol=1e-8, first_step=14)
    ctx.close()
    ws = tr.WarmStart(vms, 0, seed=7)
    loss = ws.fit(rec, epochs=300, batch=512, lr=2e-3)
    ctx = fresh()
    tr.run_steps(vms, ctx, 14, rtol=1e-8)
    warm = tr.run_steps(vms, ctx, 8, rtol=1e-8, warm=ws, first_step=14)
    ctx.close()
    ratio = np.mean([s.start_residual / s.reference_residual for s in warm])
    it_base = sum(s.newton_iterations for s in base)
    it_warm = sum(s.newton_iterations for s in warm)
    assert ratio < 0.5, (ratio, loss)
    assert it_warm <= it_base, (it_warm, it_base)


def test_column_rms_and_scaling(env):
    """The training-data scaling kernels: per-column RMS (FP64 sums) and column multipliers, on a
    row count that is not a multiple of the block size."""
    vms, torch, dev = env
    mlp = vms.Mlp(0)
    rng = np.random.default_rng(5)
    X = (rng.normal(size=(3001, 12)) * np.logspace(-3, 2, 12)).astype(np.float32)
    Xd = torch.from_numpy(X).to(dev)
    rms = mlp.column_rms(Xd)
    ref = np.sqrt((X.astype(np.float64) ** 2).mean(axis=0))
    np.testing.assert_allclose(rms, ref, rtol=1e-12)
    mul = (1.0 / ref).astype(np.float32)
    mul[3] = 0.0
    Yd = torch.empty_like(Xd)
    mlp.scale_columns(Xd, mul, Yd)
    np.testing.assert_array_equal(Yd.cpu().numpy(), X * mul)   # one FP32 product per entry
    mlp.scale_columns(Xd, mul, Xd)                              # in place
    np.testing.assert_array_equal(Xd.cpu().numpy(), X * mul)
    with pytest.raises(vms.VmsError):
        mlp.column_rms(torch.zeros((4, 17), dtype=torch.float32, device=dev))
    mlp.close()
