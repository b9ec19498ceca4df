"""The once-per-mesh host work of the library (row a0: CSR pattern, element -> CSR block map,
element colouring, Dirichlet bookkeeping), built from `csrc/pattern.cpp` into a small driver and
run on the CPU. Integer work, so every check is exact:

- rowptr and colidx equal the sparsity of the oracle's assembly of the same mesh (Section 5: the
  assembled operator sums the element matrices; with all-ones element matrices nothing cancels);
- every block-map entry addresses entry (4 n_a, 4 n_b) of its element's block (a, b), and the
  whole block sits where the layout rule puts it;
- no two elements of one colour share a node, and the colour lists cover every element once;
- the Dirichlet mask has bit 4a + c set exactly for constrained element dofs, and each constrained
  dof's diagonal position holds its diagonal;
- malformed meshes are refused with a message.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_0809_4802_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("pattern") / "pattern_driver")
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"), "-I", CUDA_INC,
                    os.path.join(ROOT, "tests", "pattern_driver.cpp"),
                    os.path.join(ROOT, "paper_0809_4802_gb300", "csrc", "pattern.cpp"), "-o", exe],
                   check=True, capture_output=True)
    return exe


def run(exe, n_nodes, conn, dir_dofs):
    conn = np.asarray(conn, dtype=np.int64)
    dir_dofs = np.asarray(dir_dofs, dtype=np.int64)
    text = f"{n_nodes} {conn.shape[0]} {conn.shape[1]} {dir_dofs.size}\n"
    text += " ".join(map(str, conn.ravel())) + "\n" + " ".join(map(str, dir_dofs)) + "\n"
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout
    res = {}
    for line in out.splitlines():
        key, *rest = line.split()
        if key == "error":
            return {"error": " ".join(rest)}
        if key == "n_colours":
            res[key] = int(rest[0])
        else:
            res[key] = np.array(rest[1:], dtype=np.int64)
            assert res[key].size == int(rest[0])
    return res


def meshes():
    cav = inputs.cavity_workload(3, re=100.0, state="noise", seed=1)
    hole = inputs.box_mesh(5, 4, 3, jitter_frac=0.1, seed=2, hole=((1, 3), (0, 2), (0, 3)))
    hole_bc = inputs.wall_bc(hole, (0.1, 0.0, 0.0))
    tet = inputs.tet_cavity_workload(2, 100.0, state="noise", seed=3)
    return [("cavity3", cav.mesh, cav.bc.dofs), ("box_with_hole", hole, hole_bc.dofs),
            ("tet_cavity2", tet.mesh, tet.bc.dofs)]


@pytest.mark.parametrize("name,mesh,dofs", meshes(), ids=lambda x: x if isinstance(x, str) else "")
def test_pattern_matches_the_oracle_assembly(driver, name, mesh, dofs):
    P = run(driver, mesh.n_nodes, mesh.conn, dofs)
    E, npe = mesh.conn.shape
    nc = 4 * npe
    A, _ = oracle.assemble(mesh.conn, mesh.n_nodes, np.ones((E, nc, nc)), np.zeros((E, nc)))
    A = A.tocsr()
    A.sort_indices()
    np.testing.assert_array_equal(P["rowptr"], A.indptr)
    np.testing.assert_array_equal(P["colidx"], A.indices)
    rowptr, colidx = P["rowptr"], P["colidx"]

    # block map: block (a, b) of element e starts at entry (4 n_a, 4 n_b), rows 4 n_a + i at
    # offsets i * rowlen[n_a], columns 4 n_b + k at offsets k
    blk = P["blk"].reshape(E, npe, npe)
    for e in range(E):
        for a in range(npe):
            na = mesh.conn[e, a]
            for b in range(npe):
                nb = mesh.conn[e, b]
                v = blk[e, a, b]
                for i in range(4):
                    for k in range(4):
                        pos = v + i * P["rowlen"][na] + k
                        assert rowptr[4 * na + i] <= pos < rowptr[4 * na + i + 1]
                        assert colidx[pos] == 4 * nb + k

    # colouring: the colour lists cover every element once; one colour never repeats a node
    order, start = P["colour_order"], P["colour_start"]
    assert start[0] == 0 and start[-1] == E and P["n_colours"] == start.size - 1
    np.testing.assert_array_equal(np.sort(order), np.arange(E))
    for c in range(P["n_colours"]):
        els = order[start[c]:start[c + 1]]
        assert np.all(P["colour"][els] == c)
        nodes = mesh.conn[els].ravel()
        assert np.unique(nodes).size == nodes.size

    # Dirichlet bookkeeping
    dset = set(int(d) for d in dofs)
    for e in range(E):
        want = 0
        for a in range(npe):
            for c in range(4):
                if 4 * mesh.conn[e, a] + c in dset:
                    want |= 1 << (4 * a + c)
        assert P["dir_mask"][e] == want
    for d, pos in zip(dofs, P["diag_pos"]):
        assert rowptr[d] <= pos < rowptr[d + 1] and colidx[pos] == d


def test_malformed_meshes_are_refused(driver):
    assert "out of range" in run(driver, 4, [[0, 1, 2, 4]], [])["error"]
    assert "repeated node" in run(driver, 4, [[0, 1, 1, 3]], [])["error"]
    assert "4 or 8 nodes" in run(driver, 6, [[0, 1, 2, 3, 4, 5]], [])["error"]
