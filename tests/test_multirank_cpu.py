"""Multi-rank path on CPU (gloo, world size 2), launched by torchrun as the benchmark would be.

The paper partitions the mesh into blocks and exchanges only the contributions to shared nodes at
assembly (Section 6); fine-scale unknowns stay local (Section 5). The halo sum over two ranks must
reproduce the single-process assembled residual on every owned row, and the distributed norm the
global one."""
import json
import os
import socket
import subprocess
import sys

import numpy as np

import oracle
from oracle import Params
from paper_0809_4802_gb300 import inputs, partition

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_partition_covers_every_element_once_and_owns_every_node_once():
    mesh = inputs.cavity_mesh(5)
    for n in (1, 2, 3, 7):
        parts = partition.build_parts(mesh.conn, mesh.n_nodes, n)
        el = np.concatenate([p.elems for p in parts])
        assert np.array_equal(np.sort(el), np.arange(mesh.n_elems))
        owned = np.concatenate([p.nodes[p.owned] for p in parts])
        assert np.array_equal(np.sort(owned), np.arange(mesh.n_nodes))
        for p in parts:
            for s, rows in p.send.items():
                assert np.all(p.owner[rows] == s)
                assert parts[s].recv[p.rank].size == rows.size


def test_halo_sum_two_gloo_ranks(tmp_path):
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={free_port()}",
           os.path.join(ROOT, "tests", "multirank_worker.py"), str(tmp_path)]
    p = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-3000:]
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    # reference: one process, all elements
    wl = inputs.cavity_workload(6, re=200.0, jitter_frac=0.15, state="random", seed=11)
    mesh = wl.mesh
    beta = np.random.default_rng(3).uniform(-0.05, 0.05, (mesh.n_elems, 3))
    X, U, _, _ = oracle.gather(mesh.conn, mesh.xyz, wl.u, beta)
    k = oracle.element_kernel(X, U, beta, Params(nu=wl.nu), with_tangent=False)
    R = oracle.residual_vector(mesh.conn, mesh.n_nodes, k, wl.bc.dofs)
    Rc = R[: 4 * mesh.n_nodes].reshape(-1, 4)
    seen = np.zeros(mesh.n_nodes, bool)
    for r in res:
        nodes = np.array(r["nodes"], dtype=np.int64)
        np.testing.assert_allclose(np.array(r["rows"]), Rc[nodes], atol=1e-13 * np.abs(Rc).max())
        assert not seen[nodes].any()
        seen[nodes] = True
        assert r["worst"] == 2.5                # max over the two ranks
    # the interface nodes belong to rank 0 (lowest rank): rank 1 sends, rank 0 sends nothing
    assert res[0]["n_send"] == {} and res[1]["n_send"].get("0", 0) > 0
    assert seen.all()
    assert abs(res[0]["norm2"] - np.sum(R ** 2)) <= 1e-12 * np.sum(R ** 2)
    assert res[0]["norm2"] == res[1]["norm2"]
