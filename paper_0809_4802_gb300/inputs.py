"""Seeded synthetic inputs: hexahedral lattice meshes, Dirichlet sets and flow states.

This module holds no arithmetic of the variational multiscale method. It only lays out node
coordinates, element connectivity, the lists of constrained degrees of freedom and their values,
and seeded random initial states. Both the CUDA path and the FP64 oracle consume its arrays.

Conventions shared by everything that reads these arrays:

* Local node order of a hexahedron (reference corners, xi/eta/zeta):
  (-,-,-) (+,-,-) (+,+,-) (-,+,-) (-,-,+) (+,-,+) (+,+,+) (-,+,+).
* Coarse degrees of freedom are node-major: global dof ``4*node + c`` with c = 0,1,2 the
  velocity components and c = 3 the pressure.
* Fine (bubble) unknowns are three per element, internal to it (Section 3.3 of the paper).

The workloads mirror the paper's 3D problems (Section 6: the lid-driven cavity of
Fig. "3DCavity", a step channel and a channel with an obstacle standing in for the jet problem,
whose geometry only exists in a missing figure).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Local corner signs of the 8-node hexahedron, in the node order stated above.
HEX_CORNERS = np.array(
    [[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
     [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=np.int64)


@dataclass
class Mesh:
    """An unstructured hexahedral mesh (stored explicitly even when it came from a lattice)."""
    xyz: np.ndarray            # (n_nodes, 3) float64
    conn: np.ndarray           # (n_elems, 8) int32, local order above
    name: str = ""
    # lattice bookkeeping (element lattice indices), used only by generators and colouring hints
    elem_ijk: np.ndarray | None = None   # (n_elems, 3) int64
    node_ijk: np.ndarray | None = None   # (n_nodes, 3) int64
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.conn.shape[0])

    @property
    def n_coarse_dof(self) -> int:
        return 4 * self.n_nodes

    @property
    def n_fine_dof(self) -> int:
        return 3 * self.n_elems


@dataclass
class Dirichlet:
    """Constrained global dofs (4*node+c) and their prescribed values."""
    dofs: np.ndarray   # (n_dir,) int64, sorted, unique
    vals: np.ndarray   # (n_dir,) float64


@dataclass
class Workload:
    mesh: Mesh
    bc: Dirichlet
    u: np.ndarray          # (n_nodes, 4) float64 nodal (v, p), Dirichlet values already imposed
    beta: np.ndarray       # (n_elems, 3) float64 bubble coefficients
    nu: float
    dt: float = 0.0        # 0 -> steady
    u_prev: np.ndarray | None = None   # (n_nodes, 4) previous time step (transient only)
    name: str = ""


# ----------------------------------------------------------------------------------------------
# lattice construction
# ----------------------------------------------------------------------------------------------

def _lattice(nx: int, ny: int, nz: int, lo, hi, keep_elem=None) -> Mesh:
    """Box [lo, hi] split into nx*ny*nz hexahedra; ``keep_elem(i,j,k)->bool`` removes elements.

    Node and element orderings are lexicographic with i fastest. Nodes used by no kept element
    are dropped and the rest renumbered in the same order.
    """
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    ei, ej, ek = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    eijk = np.stack([ei.ravel(order="F"), ej.ravel(order="F"), ek.ravel(order="F")], axis=1)
    if keep_elem is not None:
        mask = keep_elem(eijk[:, 0], eijk[:, 1], eijk[:, 2])
        eijk = eijk[mask]
    ox = HEX_CORNERS.clip(0, 1)  # (8,3) offsets 0/1
    nijk = eijk[:, None, :] + ox[None, :, :]                   # (E,8,3)
    lin = nijk[..., 0] + (nx + 1) * (nijk[..., 1] + (ny + 1) * nijk[..., 2])
    used = np.unique(lin.ravel())
    remap = -np.ones((nx + 1) * (ny + 1) * (nz + 1), dtype=np.int64)
    remap[used] = np.arange(used.size)
    conn = remap[lin].astype(np.int32)
    ni = used % (nx + 1)
    nj = (used // (nx + 1)) % (ny + 1)
    nk = used // ((nx + 1) * (ny + 1))
    node_ijk = np.stack([ni, nj, nk], axis=1)
    h = (hi - lo) / np.array([nx, ny, nz], float)
    xyz = lo[None, :] + node_ijk * h[None, :]
    return Mesh(xyz=xyz, conn=conn, elem_ijk=eijk, node_ijk=node_ijk,
                meta={"dims": (nx, ny, nz), "h": h, "lo": lo, "hi": hi})


def box_mesh(nx: int, ny: int, nz: int, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
             jitter_frac: float = 0.0, seed: int = 0, hole=None) -> Mesh:
    """Lattice of nx*ny*nz hexahedra on the box [lo, hi]; `hole` = ((i0,i1),(j0,j1),(k0,k1))
    removes the elements with lattice indices in those half-open ranges."""
    keep = None
    if hole is not None:
        (i0, i1), (j0, j1), (k0, k1) = hole
        keep = lambda i, j, k: ~((i >= i0) & (i < i1) & (j >= j0) & (j < j1) & (k >= k0) & (k < k1))  # noqa: E731
    m = _lattice(nx, ny, nz, lo, hi, keep_elem=keep)
    m.name = f"box{nx}x{ny}x{nz}"
    if jitter_frac > 0:
        jitter(m, jitter_frac, np.random.Generator(np.random.PCG64(seed)))
    return m


def wall_bc(mesh: Mesh, values=(0.0, 0.0, 0.0), pin_pressure_node: int | None = None) -> Dirichlet:
    """Every velocity component prescribed on every boundary node; optionally one pressure pin."""
    walls = np.nonzero(boundary_nodes(mesh))[0]
    dofs = [4 * walls + c for c in range(3)]
    vals = [np.full(walls.size, float(values[c])) for c in range(3)]
    if pin_pressure_node is not None:
        dofs.append(np.array([4 * pin_pressure_node + 3]))
        vals.append(np.zeros(1))
    return _dirichlet(dofs, vals)


def boundary_nodes(mesh: Mesh) -> np.ndarray:
    """Boolean mask of nodes on the domain boundary (fewer than 8 incident hexahedra)."""
    count = np.bincount(mesh.conn.ravel().astype(np.int64), minlength=mesh.n_nodes)
    return count < 8


def jitter(mesh: Mesh, frac: float, rng: np.random.Generator) -> None:
    """Move every interior node by U[-frac*h, frac*h] per coordinate (in place)."""
    if frac <= 0:
        return
    h = np.asarray(mesh.meta["h"], float)
    inner = ~boundary_nodes(mesh)
    d = rng.uniform(-frac, frac, size=(int(inner.sum()), 3)) * h[None, :]
    mesh.xyz[inner] += d


def element_colours(mesh: Mesh) -> np.ndarray:
    """8-colouring of lattice elements by index parity: same-colour elements share no node."""
    e = mesh.elem_ijk
    return ((e[:, 0] & 1) | ((e[:, 1] & 1) << 1) | ((e[:, 2] & 1) << 2)).astype(np.int32)


def _dirichlet(dofs: list, vals: list) -> Dirichlet:
    d = np.concatenate(dofs).astype(np.int64)
    v = np.concatenate(vals).astype(np.float64)
    # later entries take precedence for duplicated dofs
    _, last = np.unique(d[::-1], return_index=True)
    keep = (d.size - 1 - last)
    keep.sort()
    d, v = d[keep], v[keep]
    o = np.argsort(d, kind="stable")
    return Dirichlet(dofs=d[o], vals=v[o])


def impose(u: np.ndarray, bc: Dirichlet) -> np.ndarray:
    flat = u.reshape(-1)
    flat[bc.dofs] = bc.vals
    return u


# ----------------------------------------------------------------------------------------------
# lid-driven cavity (Fig. "3DCavity": unit cube, lid u=(1,0,0) at z=1, no-slip elsewhere,
# pressure prescribed zero at one node at the centre)
# ----------------------------------------------------------------------------------------------

def cavity_mesh(n: int, jitter_frac: float = 0.0, seed: int = 0) -> Mesh:
    m = _lattice(n, n, n, (0, 0, 0), (1, 1, 1))
    m.name = f"cavity{n}"
    if jitter_frac > 0:
        jitter(m, jitter_frac, np.random.Generator(np.random.PCG64(seed)))
    return m


def cavity_bc(mesh: Mesh, lid_speed: float = 1.0) -> Dirichlet:
    n = mesh.meta["dims"][0]
    ijk = mesh.node_ijk
    on_wall = boundary_nodes(mesh)
    walls = np.nonzero(on_wall)[0]
    lid = np.nonzero(ijk[:, 2] == n)[0]
    dofs = [4 * walls + c for c in range(3)]
    vals = [np.zeros(walls.size) for _ in range(3)]
    # lid nodes take precedence on the z=1 edges ("leaky lid")
    dofs += [4 * lid + 0, 4 * lid + 1, 4 * lid + 2]
    vals += [np.full(lid.size, lid_speed), np.zeros(lid.size), np.zeros(lid.size)]
    centre = np.nonzero((ijk[:, 0] == n // 2) & (ijk[:, 1] == n // 2) & (ijk[:, 2] == n // 2))[0]
    dofs.append(4 * centre + 3)
    vals.append(np.zeros(centre.size))
    return _dirichlet(dofs, vals)


def cavity_workload(n: int, re: float, *, jitter_frac: float = 0.0, state: str = "noise",
                    seed: int = 1001) -> Workload:
    """state='noise': v ~ U[-0.05,0.05] at interior nodes, p = 0 (steady cavity, 8^3 case).
    state='random': v ~ U[-0.5,0.5], p ~ N(0, sigma=0.1) at all nodes (32^3 case)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mesh = cavity_mesh(n)
    if jitter_frac > 0:
        jitter(mesh, jitter_frac, rng)
    bc = cavity_bc(mesh)
    u = np.zeros((mesh.n_nodes, 4))
    if state == "noise":
        inner = ~boundary_nodes(mesh)
        u[inner, :3] = rng.uniform(-0.05, 0.05, size=(int(inner.sum()), 3))
    elif state == "random":
        u[:, :3] = rng.uniform(-0.5, 0.5, size=(mesh.n_nodes, 3))
        u[:, 3] = rng.normal(0.0, 0.1, size=mesh.n_nodes)
    elif state != "zero":
        raise ValueError(state)
    impose(u, bc)
    beta = np.zeros((mesh.n_elems, 3))
    return Workload(mesh=mesh, bc=bc, u=u, beta=beta, nu=1.0 / re, name=f"cavity{n}_re{re:g}")


# ----------------------------------------------------------------------------------------------
# backward-facing step: [0,30]x[0,2]x[0,4] minus [0,1]x[0,1]x[0,4], inflow on x=0 above the step
# ----------------------------------------------------------------------------------------------

def bfs_mesh(per_unit: int = 13, jitter_frac: float = 0.1, seed: int = 1003) -> Mesh:
    nx, ny, nz = 30 * per_unit, 2 * per_unit, 4 * per_unit
    s = per_unit
    m = _lattice(nx, ny, nz, (0, 0, 0), (30, 2, 4), keep_elem=lambda i, j, k: ~((i < s) & (j < s)))
    m.name = f"bfs_h1/{per_unit}"
    m.meta["step"] = s
    if jitter_frac > 0:
        jitter(m, jitter_frac, np.random.Generator(np.random.PCG64(seed)))
    return m


def bfs_workload(per_unit: int = 13, re: float = 800.0, jitter_frac: float = 0.1,
                 seed: int = 1003) -> Workload:
    mesh = bfs_mesh(per_unit, jitter_frac, seed)
    x = mesh.xyz
    onb = boundary_nodes(mesh)
    outflow = np.isclose(x[:, 0], 30.0)
    inflow = np.isclose(x[:, 0], 0.0) & (x[:, 1] >= 1.0 - 1e-12)
    walls = np.nonzero(onb & ~outflow & ~inflow)[0]
    inl = np.nonzero(inflow)[0]
    y, z = x[inl, 1], x[inl, 2]
    ux = np.clip((y - 1.0) * (2.0 - y), 0, None) * z * (4.0 - z)
    dofs = [4 * walls + c for c in range(3)] + [4 * inl + c for c in range(3)]
    vals = [np.zeros(walls.size)] * 3 + [ux, np.zeros(inl.size), np.zeros(inl.size)]
    bc = _dirichlet(dofs, vals)
    u = np.zeros((mesh.n_nodes, 4))
    impose(u, bc)
    return Workload(mesh=mesh, bc=bc, u=u, beta=np.zeros((mesh.n_elems, 3)), nu=1.0 / re,
                    name=f"bfs_re{re:g}")


# ----------------------------------------------------------------------------------------------
# channel past a cube: [0,20]x[0,4]x[0,4] minus [4,5]x[1.5,2.5]^2, transient
# ----------------------------------------------------------------------------------------------

def channel_mesh(nx: int = 300, nyz: int = 56) -> Mesh:
    hx = 20.0 / nx
    hy = 4.0 / nyz
    i0, i1 = int(round(4.0 / hx)), int(round(5.0 / hx))
    j0, j1 = int(round(1.5 / hy)), int(round(2.5 / hy))
    m = _lattice(nx, nyz, nyz, (0, 0, 0), (20, 4, 4),
                 keep_elem=lambda i, j, k: ~((i >= i0) & (i < i1) & (j >= j0) & (j < j1)
                                             & (k >= j0) & (k < j1)))
    m.name = f"channel{nx}x{nyz}"
    return m


def channel_workload(nx: int = 300, nyz: int = 56, re: float = 1000.0, dt: float = 0.01,
                     seed: int = 1005) -> Workload:
    mesh = channel_mesh(nx, nyz)
    x = mesh.xyz
    onb = boundary_nodes(mesh)
    outflow = np.isclose(x[:, 0], 20.0)
    inflow = np.isclose(x[:, 0], 0.0)
    walls = np.nonzero(onb & ~outflow & ~inflow)[0]
    inl = np.nonzero(inflow)[0]
    y, z = x[inl, 1], x[inl, 2]
    ux = y * (4.0 - y) * z * (4.0 - z) / 16.0
    dofs = [4 * walls + c for c in range(3)] + [4 * inl + c for c in range(3)]
    vals = [np.zeros(walls.size)] * 3 + [ux, np.zeros(inl.size), np.zeros(inl.size)]
    bc = _dirichlet(dofs, vals)
    u = np.zeros((mesh.n_nodes, 4))
    impose(u, bc)
    return Workload(mesh=mesh, bc=bc, u=u, beta=np.zeros((mesh.n_elems, 3)), nu=1.0 / re,
                    dt=dt, u_prev=u.copy(), name=f"channel_re{re:g}")


# ----------------------------------------------------------------------------------------------
# random single elements / small states for unit tests
# ----------------------------------------------------------------------------------------------

def random_elements(n_elems: int, seed: int, distort: float = 0.15, h: float = 1.0):
    """Independent jittered hexahedra around the reference cube scaled by h/2, random states.

    Returns X (E,8,3), U (E,8,4), beta (E,3), Uprev (E,8,4)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = 0.5 * h * HEX_CORNERS.astype(float)
    X = base[None] + rng.uniform(-distort, distort, size=(n_elems, 8, 3)) * h
    X += rng.uniform(-2, 2, size=(n_elems, 1, 3))
    U = rng.uniform(-1, 1, size=(n_elems, 8, 4))
    beta = rng.uniform(-0.5, 0.5, size=(n_elems, 3))
    Uprev = U + rng.uniform(-0.1, 0.1, size=U.shape)
    return X, U, beta, Uprev


def batched_cavities(count: int = 64, seed: int = 1004, edges=(8, 12, 16, 24, 32, 48)):
    """Edge counts and Reynolds numbers of a batch of independent cavity problems."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = rng.choice(np.array(edges), size=count)
    res = rng.uniform(100.0, 1000.0, size=count)
    return [(int(n), float(r)) for n, r in zip(ns, res)]


@dataclass
class Batch:
    """Independent problems merged into one mesh (instance i owns nodes node_offsets[i]:...[i+1]
    and elements elem_offsets[i]:...[i+1]); nu_e is each element's viscosity."""
    work: Workload
    node_offsets: np.ndarray
    elem_offsets: np.ndarray
    nu_e: np.ndarray
    members: list


def merge_workloads(parts: list) -> Batch:
    """Concatenate workloads into one mesh: node numbers, connectivity and constrained dofs are
    shifted by each instance's node offset."""
    n_off = np.concatenate([[0], np.cumsum([w.mesh.n_nodes for w in parts])]).astype(np.int64)
    e_off = np.concatenate([[0], np.cumsum([w.mesh.n_elems for w in parts])]).astype(np.int64)
    xyz = np.concatenate([w.mesh.xyz for w in parts])
    conn = np.concatenate([w.mesh.conn.astype(np.int64) + n_off[i] for i, w in enumerate(parts)])
    ijk = np.concatenate([w.mesh.node_ijk for w in parts])
    eijk = np.concatenate([w.mesh.elem_ijk for w in parts])
    mesh = Mesh(xyz=xyz, conn=conn.astype(np.int32), elem_ijk=eijk, node_ijk=ijk,
                meta={"instances": len(parts)})
    mesh.name = f"batch{len(parts)}"
    dofs = np.concatenate([w.bc.dofs + 4 * n_off[i] for i, w in enumerate(parts)])
    vals = np.concatenate([w.bc.vals for w in parts])
    nu_e = np.concatenate([np.full(w.mesh.n_elems, w.nu) for w in parts])
    work = Workload(mesh=mesh, bc=Dirichlet(dofs=dofs.astype(np.int64), vals=vals),
                    u=np.concatenate([w.u for w in parts]),
                    beta=np.concatenate([w.beta for w in parts]), nu=float(parts[0].nu),
                    name=mesh.name)
    return Batch(work=work, node_offsets=n_off, elem_offsets=e_off, nu_e=nu_e, members=parts)


def batched_workload(count: int = 64, seed: int = 1004, edges=(8, 12, 16, 24, 32, 48),
                     jitter_frac: float = 0.15) -> Batch:
    """A serving-style mix: `count` lid-driven cavities with edge counts drawn from `edges` and
    Re ~ U[100, 1000], each with its own seeded jittered mesh and random state (as the 32^3
    cavity)."""
    parts = [cavity_workload(n, re, jitter_frac=jitter_frac, state="random", seed=seed + 1 + i)
             for i, (n, re) in enumerate(batched_cavities(count, seed, edges))]
    return merge_workloads(parts)


# ----------------------------------------------------------------------------------------------
# initial parameters of the warm-start network (random numbers the method draws, passed in)
# ----------------------------------------------------------------------------------------------

def mlp_init(seed: int = 7, n_in: int = 12, width: int = 128, n_out: int = 4) -> np.ndarray:
    """Flat FP32 parameter vector (W1, b1, W2, b2, W3, b3; row-major): weights uniform in
    +-sqrt(6 / (fan_in + fan_out)) (Glorot), biases zero."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for fi, fo in ((n_in, width), (width, width), (width, n_out)):
        a = np.sqrt(6.0 / (fi + fo))
        parts += [rng.uniform(-a, a, fi * fo), np.zeros(fo)]
    return np.concatenate(parts).astype(np.float32)


# ----------------------------------------------------------------------------------------------
# decaying vortex in a closed box (a smooth transient for the warm start): no-slip on every wall,
# pressure pinned at the centre, initial velocity f(z) (d psi/dy, -d psi/dx, 0) with
# psi = sin^2(pi x) sin^2(pi y) and f(z) = sin(pi z): divergence-free and zero on the walls
# ----------------------------------------------------------------------------------------------

def vortex_box_workload(n: int, re: float = 200.0, dt: float = 0.02, jitter_frac: float = 0.0,
                        seed: int = 1006, amplitude: float = 1.0) -> Workload:
    rng = np.random.Generator(np.random.PCG64(seed))
    mesh = cavity_mesh(n)
    if jitter_frac > 0:
        jitter(mesh, jitter_frac, rng)
    ijk = mesh.node_ijk
    centre = np.nonzero((ijk[:, 0] == n // 2) & (ijk[:, 1] == n // 2) & (ijk[:, 2] == n // 2))[0]
    bc = wall_bc(mesh, (0.0, 0.0, 0.0), pin_pressure_node=int(centre[0]))
    x, y, z = mesh.xyz[:, 0], mesh.xyz[:, 1], mesh.xyz[:, 2]
    pi = np.pi
    dpsi_dy = np.sin(pi * x) ** 2 * 2 * pi * np.sin(pi * y) * np.cos(pi * y)
    dpsi_dx = 2 * pi * np.sin(pi * x) * np.cos(pi * x) * np.sin(pi * y) ** 2
    f = np.sin(pi * z)
    u = np.zeros((mesh.n_nodes, 4))
    u[:, 0] = amplitude * f * dpsi_dy
    u[:, 1] = -amplitude * f * dpsi_dx
    impose(u, bc)
    return Workload(mesh=mesh, bc=bc, u=u, beta=np.zeros((mesh.n_elems, 3)), nu=1.0 / re, dt=dt,
                    u_prev=u.copy(), name=f"vortex{n}_re{re:g}")


# ----------------------------------------------------------------------------------------------
# tetrahedral meshes: every lattice hexahedron split into the 6 tetrahedra along its main diagonal
# (Kuhn subdivision: the paths 000 -> 111 along the three axes in every order), which is
# conforming across neighbouring cubes
# ----------------------------------------------------------------------------------------------

def tet_mesh_from_lattice(hexm: Mesh) -> Mesh:
    """Split a lattice hexahedral mesh into tetrahedra (6 per hexahedron), positively oriented."""
    # local hex corner of offset (dx, dy, dz) in the order of HEX_CORNERS
    off = HEX_CORNERS.clip(0, 1).astype(int)
    local = {tuple(o): a for a, o in enumerate(off)}
    paths = []
    for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        p = np.zeros(3, int)
        verts = [local[tuple(p)]]
        for ax in perm:
            p = p.copy()
            p[ax] = 1
            verts.append(local[tuple(p)])
        paths.append(verts)
    conn = np.concatenate([hexm.conn[:, v] for v in paths], axis=0)
    x = hexm.xyz[conn]
    vol = np.einsum("ei,ei->e", x[:, 1] - x[:, 0], np.cross(x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]))
    neg = vol < 0
    conn[neg] = conn[neg][:, [0, 2, 1, 3]]
    m = Mesh(xyz=hexm.xyz.copy(), conn=np.ascontiguousarray(conn, dtype=np.int32), node_ijk=hexm.node_ijk,
             meta=dict(hexm.meta, element="tet"))
    m.name = hexm.name + "_tet"
    return m


def tet_cavity_workload(n: int, re: float, *, jitter_frac: float = 0.0, state: str = "noise",
                        seed: int = 1001) -> Workload:
    """The lid-driven cavity of cavity_workload on the Kuhn tetrahedral mesh of the n^3 lattice
    (6 n^3 tetrahedra, (n+1)^3 nodes): same boundary conditions, pressure pin and states."""
    rng = np.random.Generator(np.random.PCG64(seed))
    hexm = cavity_mesh(n)
    if jitter_frac > 0:
        jitter(hexm, jitter_frac, rng)
    bc = cavity_bc(hexm)
    u = np.zeros((hexm.n_nodes, 4))
    if state == "noise":
        inner = ~boundary_nodes(hexm)
        u[inner, :3] = rng.uniform(-0.05, 0.05, size=(int(inner.sum()), 3))
    elif state == "random":
        u[:, :3] = rng.uniform(-0.5, 0.5, size=(hexm.n_nodes, 3))
        u[:, 3] = rng.normal(0.0, 0.1, size=hexm.n_nodes)
    elif state != "zero":
        raise ValueError(state)
    impose(u, bc)
    mesh = tet_mesh_from_lattice(hexm)
    return Workload(mesh=mesh, bc=bc, u=u, beta=np.zeros((mesh.n_elems, 3)), nu=1.0 / re,
                    name=f"tetcavity{n}_re{re:g}")
