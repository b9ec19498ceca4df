"""The host-side node order of the banded direct fallback (`csrc/band_order.cpp`), built into a
small driver and run on the CPU. It returns the order of smallest bandwidth among the graph's own
numbering and two reverse Cuthill-McKee orders. Checked: the result is a permutation whose
bandwidth is the one reported and never above the graph's own; a path and a ring numbered at
random come out with bandwidth 1 and 2 (the least possible); a cube lattice numbered line by line
keeps that numbering (its own order is already the best of the three); an elongated lattice comes
out ordered by cross-sections; disconnected graphs are ordered part by part.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_0809_4802_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("needs g++")
    exe = str(tmp_path_factory.mktemp("bandorder") / "band_order_driver")
    subprocess.run([gxx, "-std=c++17", "-O2", os.path.join(ROOT, "tests", "band_order_driver.cpp"),
                    os.path.join(ROOT, "paper_0809_4802_gb300", "csrc", "band_order.cpp"), "-o", exe],
                   check=True, capture_output=True)
    return exe


def run(exe, graphs):
    """graphs: list of (nodes, list of neighbour arrays). Returns [(bw, perm)]."""
    lines = []
    for n, nbrs in graphs:
        start = np.zeros(n + 1, np.int64)
        start[1:] = np.cumsum([len(x) for x in nbrs])
        adj = np.concatenate([np.asarray(x, np.int64) for x in nbrs]) if n else np.zeros(0, np.int64)
        lines.append(f"{n} {len(adj)}")
        lines.append(" ".join(map(str, start)))
        lines.append(" ".join(map(str, adj)))
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True).stdout.split("\n")
    res = []
    for line in out[:len(graphs)]:
        tok = line.split()
        res.append((int(tok[0]), np.array(tok[1:], np.int64)))
    return res


def bandwidth(nbrs, perm):
    bw = 0
    for a, x in enumerate(nbrs):
        if len(x):
            bw = max(bw, int(np.abs(perm[a] - perm[np.asarray(x)]).max()))
    return bw


def from_edges(n, edges):
    nbrs = [set() for _ in range(n)]
    for a, b in edges:
        if a != b:
            nbrs[a].add(b)
            nbrs[b].add(a)
    return [sorted(x) for x in nbrs]


def mesh_graph(m):
    edges = set()
    for e in m.conn:
        for a in e:
            for b in e:
                if a < b:
                    edges.add((int(a), int(b)))
    return from_edges(m.n_nodes, edges)


def check(nbrs, bw, perm):
    n = len(nbrs)
    assert sorted(perm.tolist()) == list(range(n))
    assert bw == bandwidth(nbrs, perm)
    assert bw <= bandwidth(nbrs, np.arange(n))


def test_path_and_ring_numbered_at_random(driver):
    rng = np.random.default_rng(3)
    n = 40
    lab = rng.permutation(n)
    path = from_edges(n, [(lab[k], lab[k + 1]) for k in range(n - 1)])
    ring = from_edges(n, [(lab[k], lab[(k + 1) % n]) for k in range(n)])
    (bp, pp), (br, pr) = run(driver, [(n, path), (n, ring)])
    check(path, bp, pp)
    check(ring, br, pr)
    assert bp == 1 and br == 2


def test_lattices(driver):
    cube = mesh_graph(inputs.cavity_mesh(6))          # 7^3 nodes numbered x fastest
    box = mesh_graph(inputs.box_mesh(24, 4, 4))       # 25 x 5 x 5, x fastest
    (bc, pc), (bb, pb) = run(driver, [(len(cube), cube), (len(box), box)])
    check(cube, bc, pc)
    check(box, bb, pb)
    assert bc == 7 * 7 + 7 + 1 and np.array_equal(pc, np.arange(len(cube)))
    # own numbering: 25 * 5 + 25 + 1 = 151; by cross-sections (5 x 5 nodes) about two of them
    assert bandwidth(box, np.arange(len(box))) == 151 and bb <= 2 * 25 + 5


def test_disconnected_and_isolated_nodes(driver):
    rng = np.random.default_rng(9)
    n = 30
    lab = rng.permutation(n)
    edges = [(lab[k], lab[k + 1]) for k in range(9)] + [(lab[k], lab[k + 1]) for k in range(12, 25)]
    g = from_edges(n, edges)                          # two paths and five isolated nodes
    ((b, p),) = run(driver, [(n, g)])
    check(g, b, p)
    assert b == 1


def test_random_graphs(driver):
    rng = np.random.default_rng(21)
    graphs = []
    for n in (1, 2, 17, 120):
        m = rng.integers(0, 3 * n + 1)
        edges = [tuple(rng.integers(0, n, 2)) for _ in range(m)]
        graphs.append((n, from_edges(n, edges)))
    for (n, g), (b, p) in zip(graphs, run(driver, graphs)):
        check(g, b, p)
