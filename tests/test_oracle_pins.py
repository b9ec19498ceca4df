"""Pins of the FP64 oracle against facts fixed by the mathematics, not by the oracle itself.

Each test names the passage of the paper it checks and the closed form or invariant it uses.
"""
import numpy as np
import pytest

import oracle
from oracle import Params
from paper_0809_4802_gb300 import inputs

CORNERS = inputs.HEX_CORNERS.astype(float)


def affine_cube(h, origin=(0.3, -0.2, 1.1)):
    return (np.asarray(origin)[None, :] + 0.5 * h * (CORNERS + 1.0))[None]


def q1_laplacian_cube(h):
    """Closed form of int grad N_a . grad N_b on a cube of side h (hand-derived):
    h/12 * [4 on the diagonal, 0 for edge neighbours, -1 for face and body diagonals]."""
    K = np.zeros((8, 8))
    for a in range(8):
        for b in range(8):
            nd = int(np.sum(CORNERS[a] != CORNERS[b]))
            K[a, b] = {0: 4.0, 1: 0.0, 2: -1.0, 3: -1.0}[nd] * h / 12.0
    return K


def q1_grad_mass_cube(h):
    """int dN_a/dx_i N_b on a cube of side h: h^2 s_ai (3+s_aj s_bj)(3+s_ak s_bk)/288."""
    G = np.zeros((8, 3, 8))
    for a in range(8):
        for b in range(8):
            sig = CORNERS[a] * CORNERS[b]
            for i in range(3):
                j, k = [d for d in range(3) if d != i]
                G[a, i, b] = h * h * CORNERS[a, i] * (3 + sig[j]) * (3 + sig[k]) / 288.0
    return G


# ----------------------------------------------------------------------------------------------
# reference element (Section 3.3, Eq. DefineBubbles3; Section 4.1 shape-function notation)
# ----------------------------------------------------------------------------------------------

def test_q1_basis_partition_and_nodality():
    rng = np.random.default_rng(0)
    xi = rng.uniform(-1, 1, size=(50, 3))
    N, dN = oracle.q1_basis(xi)
    np.testing.assert_allclose(N.sum(axis=1), 1.0, atol=1e-15)
    np.testing.assert_allclose(dN.sum(axis=1), 0.0, atol=1e-15)
    Nc, _ = oracle.q1_basis(CORNERS)
    np.testing.assert_allclose(Nc, np.eye(8), atol=1e-15)
    # derivative against a difference quotient of the textbook polynomial
    eps = 1e-6
    for al in range(3):
        e = np.zeros(3); e[al] = eps
        Np, _ = oracle.q1_basis(xi + e); Nm, _ = oracle.q1_basis(xi - e)
        np.testing.assert_allclose((Np - Nm) / (2 * eps), dN[:, :, al], atol=1e-9)


def test_bubble_vanishes_on_faces():
    """Eq. SC_Fine_Scale_Vanish: the fine scale is zero on every element face."""
    rng = np.random.default_rng(1)
    for face_dim in range(3):
        for s in (-1.0, 1.0):
            xi = rng.uniform(-1, 1, size=(20, 3)); xi[:, face_dim] = s
            b, _ = oracle.bubble(xi)
            np.testing.assert_allclose(b, 0.0, atol=1e-15)
    b0, db0 = oracle.bubble(np.zeros((1, 3)), scale=2.5)
    assert b0[0] == 2.5 and np.all(db0 == 0.0)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_gauss_rule_exact_for_degree_2n_minus_1(n):
    pts, w = oracle.gauss_rule(n)

    def exact(p):  # int_{-1}^{1} x^p dx
        return 2.0 / (p + 1) if p % 2 == 0 else 0.0

    for p in range(2 * n):
        for q in (0, 2, 2 * n - 1):
            val = np.sum(w * pts[:, 0] ** p * pts[:, 1] ** q)
            assert abs(val - exact(p) * exact(q) * 2.0) < 1e-14


# ----------------------------------------------------------------------------------------------
# closed forms on an affine cube (Section 4.1 residuals, Section 5 condensation)
# ----------------------------------------------------------------------------------------------

@pytest.mark.parametrize("h", [1.0, 0.37])
@pytest.mark.parametrize("qo", [3, 4])
def test_affine_cube_elementary_integrals(h, qo):
    """volume h^3, int b = 8h^3/27, int |grad b|^2 = 1024h/225, int b dN_a/dx_k = 2h^2 s_ak/27."""
    X = affine_cube(h)
    I = oracle.elementary_integrals(X, qo)
    assert abs(I["vol"][0] - h ** 3) < 1e-15 * 10
    assert abs(I["b"][0] - 8 * h ** 3 / 27) < 1e-14
    assert abs(I["dd"][0] - 1024 * h / 225) < 1e-13
    np.testing.assert_allclose(I["b_g"][0], 2 * h * h * CORNERS / 27, atol=1e-14)
    np.testing.assert_allclose(I["N_d"][0], -2 * h * h * CORNERS / 27, atol=1e-14)


@pytest.mark.parametrize("seed", [0, 1])
def test_integration_by_parts_on_distorted_hexes(seed):
    """int N_a grad b = - int b grad N_a because b = 0 on the element boundary (Eq.
    SC_Fine_Scale_Vanish). With the cofactor (Piola) identity both integrands are polynomials of
    degree <= 5 per direction, so the 3-point rule is exact on trilinear hexahedra. A transposed
    inverse Jacobian breaks this identity on distorted elements."""
    X, _, _, _ = inputs.random_elements(16, seed, distort=0.2)
    I = oracle.elementary_integrals(X, 3)
    np.testing.assert_allclose(I["N_d"], -I["b_g"], atol=1e-14 * np.abs(I["b_g"]).max() * 10)


def test_affine_volume_is_determinant():
    rng = np.random.default_rng(3)
    A = np.eye(3) + 0.3 * rng.standard_normal((3, 3))
    if np.linalg.det(A) < 0:
        A[:, 0] *= -1
    X = (CORNERS @ A.T + rng.standard_normal(3))[None]
    I = oracle.elementary_integrals(X, 3)
    assert abs(I["vol"][0] - 8 * np.linalg.det(A)) < 1e-13


@pytest.mark.parametrize("h,nu", [(1.0, 0.5), (0.25, 0.01)])
def test_stokes_limit_condensed_matrix_closed_form(h, nu):
    """Stokes limit (vhat = 0, beta = 0, steady, no force) on an affine cube: the condensed element
    matrix is fully closed form. K_vf = 0 (int grad N_a . grad b = 0 on a cube), so
      S_vv = nut * Q1 Laplacian (x) I3,   S_vp = K_vp = -int g_ai N_b,   S_pv = S_vp^T,
      S_pp = -K_pf K_ff^-1 K_fp = -(25 h^3 / (20736 nut)) s_a . s_b   (Section 5, Eq. SchurUpdate)."""
    X = affine_cube(h)
    p = Params(nu=nu)
    k = oracle.element_kernel(X, np.zeros((1, 8, 4)), np.zeros((1, 3)), p)
    S, r, _, _ = oracle.condense(*oracle.pack_element(k))
    S = S[0].reshape(8, 4, 8, 4)
    nut = 2 * nu
    Lap = q1_laplacian_cube(h)
    G = q1_grad_mass_cube(h)
    exp_vv = nut * np.einsum("ab,ik->aibk", Lap, np.eye(3))
    scale = np.abs(S).max()
    np.testing.assert_allclose(S[:, :3, :, :3], exp_vv, atol=1e-13 * scale)
    np.testing.assert_allclose(S[:, :3, :, 3], -G, atol=1e-13 * scale)
    np.testing.assert_allclose(S[:, 3, :, :3], -G.transpose(2, 0, 1), atol=1e-13 * scale)
    exp_pp = -(25 * h ** 3 / (20736 * nut)) * CORNERS @ CORNERS.T
    np.testing.assert_allclose(S[:, 3, :, 3], exp_pp, atol=1e-13 * scale)
    np.testing.assert_allclose(r, 0.0, atol=0)
    # the eliminated block is the bubble's Dirichlet energy
    np.testing.assert_allclose(k["Kff"][0], nut * 1024 * h / 225 * np.eye(3), rtol=1e-14)


def test_transient_terms_closed_form():
    """Backward-Euler Remark of Section 4.1: only the coarse velocity carries the rate term, in R_c
    through the Q1 mass matrix (diagonal h^3/27) and in R_f through int b N_b (sum 8h^3/27)."""
    h, dt = 0.5, 0.02
    X = affine_cube(h)
    p = Params(nu=0.0, dt=dt)
    k = oracle.element_kernel(X, np.zeros((1, 8, 4)), np.zeros((1, 3)), p, Uprev=np.zeros((1, 8, 4)))
    M = np.array([[np.prod(3 + CORNERS[a] * CORNERS[b]) for b in range(8)] for a in range(8)]) * h ** 3 / 1728
    np.testing.assert_allclose(k["Kvv"][0, :, 0, :, 0], M / dt, rtol=1e-13)
    np.testing.assert_allclose(k["Kvv"][0, :, 0, :, 1], 0.0, atol=1e-15)
    np.testing.assert_allclose(k["Kfv"][0, 1, :, 1].sum(), 8 * h ** 3 / 27 / dt, rtol=1e-13)
    np.testing.assert_allclose(k["Kvf"][0], 0.0, atol=1e-15)      # no fine-scale mass
    np.testing.assert_allclose(k["Kff"][0], 0.0, atol=1e-15)


# ----------------------------------------------------------------------------------------------
# patch tests on a uniform lattice (Section 4.1 residual vectors, assembled)
# ----------------------------------------------------------------------------------------------

def test_linear_velocity_patch():
    """v = A x + c (A not symmetric), p constant, beta = 0 on a uniform lattice of spacing h.
    Q1 reproduces v exactly, so L = A and conv = A v (linear). At interior nodes the viscous and
    pressure terms cancel (int over the patch of grad N_a = 0) and, by symmetry of N_a,
      R_c[a] = h^3 A v(x_a),   R_p[a] = -h^3 tr A;   per element R_f = (8h^3/27) A v(x_centre)
    because int b grad b = 0 and b (A v) has degree 3 per direction. conv = A^T v would fail."""
    n = 3
    mesh = inputs.cavity_mesh(n)
    h = 1.0 / n
    rng = np.random.default_rng(7)
    A = rng.standard_normal((3, 3)); c = rng.standard_normal(3)
    u = np.zeros((mesh.n_nodes, 4))
    u[:, :3] = mesh.xyz @ A.T + c
    u[:, 3] = 0.77
    X, U, beta, _ = oracle.gather(mesh.conn, mesh.xyz, u, np.zeros((mesh.n_elems, 3)))
    k = oracle.element_kernel(X, U, beta, Params(nu=0.37), with_tangent=False)
    Rcp, Rf = oracle.pack_residual(k)
    R = oracle.assemble_vector(mesh.conn, mesh.n_nodes, Rcp).reshape(-1, 4)
    inner = ~inputs.boundary_nodes(mesh)
    x = mesh.xyz[inner]
    np.testing.assert_allclose(R[inner, :3], h ** 3 * (x @ A.T + c) @ A.T, atol=1e-14)
    np.testing.assert_allclose(R[inner, 3], -h ** 3 * np.trace(A), atol=1e-14)
    xc = mesh.xyz[mesh.conn].mean(axis=1)
    np.testing.assert_allclose(Rf, 8 * h ** 3 / 27 * (xc @ A.T + c) @ A.T, atol=1e-14)


def test_constant_state_patch_on_jittered_mesh():
    """Constant v and p with beta = 0: L = 0, so interior R_c = -p int grad N_a = 0, R_p = 0 and
    R_f = -p int grad b = 0 on every element, whatever the (valid) element shapes."""
    mesh = inputs.cavity_mesh(4, jitter_frac=0.2, seed=5)
    u = np.zeros((mesh.n_nodes, 4)); u[:, :3] = [0.3, -1.2, 0.5]; u[:, 3] = 2.0
    X, U, beta, _ = oracle.gather(mesh.conn, mesh.xyz, u, np.zeros((mesh.n_elems, 3)))
    k = oracle.element_kernel(X, U, beta, Params(nu=0.1), with_tangent=False)
    rc, _ = oracle.pack_residual(k)
    R = oracle.assemble_vector(mesh.conn, mesh.n_nodes, rc).reshape(-1, 4)
    inner = ~inputs.boundary_nodes(mesh)
    np.testing.assert_allclose(R[inner], 0.0, atol=1e-14)
    np.testing.assert_allclose(k["Rf"], 0.0, atol=1e-14)


# ----------------------------------------------------------------------------------------------
# consistency of the tangent (Section 4.2, Eq. NewtonUpdate2: the tangent is the exact derivative)
# ----------------------------------------------------------------------------------------------

def packed_residual(X, U, beta, p, Up):
    k = oracle.element_kernel(X, U, beta, p, Up, with_tangent=False)
    E = X.shape[0]
    rc = np.concatenate([k["Rc"], k["Rp"][:, :, None]], axis=2).reshape(E, 32)
    return np.concatenate([rc, k["Rf"]], axis=1)


def packed_tangent(k):
    Kcc, Kcf, Kfc, Kff, _, _ = oracle.pack_element(k)
    top = np.concatenate([Kcc, Kcf], axis=2)
    bot = np.concatenate([Kfc, Kff], axis=2)
    return np.concatenate([top, bot], axis=1)


@pytest.mark.parametrize("dt,f", [(0.0, (0, 0, 0)), (0.05, (0.3, -0.1, 2.0))])
def test_tangent_matches_central_differences(dt, f):
    X, U, beta, Up = inputs.random_elements(5, seed=11, distort=0.15)
    p = Params(nu=0.013, dt=dt, f=f)
    K = packed_tangent(oracle.element_kernel(X, U, beta, p, Up))
    eps = 1e-6
    E = X.shape[0]
    Kfd = np.zeros((E, 35, 35))
    for j in range(35):
        Uplus, Umin = U.copy(), U.copy(); bplus, bmin = beta.copy(), beta.copy()
        if j < 32:
            Uplus[:, j // 4, j % 4] += eps; Umin[:, j // 4, j % 4] -= eps
        else:
            bplus[:, j - 32] += eps; bmin[:, j - 32] -= eps
        Kfd[:, :, j] = (packed_residual(X, Uplus, bplus, p, Up) - packed_residual(X, Umin, bmin, p, Up)) / (2 * eps)
    err = np.abs(Kfd - K).max() / np.abs(K).max()
    assert err < 1e-8, err


# ----------------------------------------------------------------------------------------------
# invariances
# ----------------------------------------------------------------------------------------------

def test_condensed_system_invariant_under_bubble_scaling():
    """The bubble's normalisation is not stated (Section 3.3). Scaling b by c with beta -> beta/c
    leaves the fine velocity, hence S_e and r_e, unchanged."""
    X, U, beta, _ = inputs.random_elements(4, seed=2)
    p1 = Params(nu=0.05)
    c = 2.7
    p2 = Params(nu=0.05, bubble_scale=c)
    S1, r1, _, _ = oracle.condense(*oracle.pack_element(oracle.element_kernel(X, U, beta, p1)))
    S2, r2, _, _ = oracle.condense(*oracle.pack_element(oracle.element_kernel(X, U, beta / c, p2)))
    np.testing.assert_allclose(S2, S1, atol=1e-12 * np.abs(S1).max())
    np.testing.assert_allclose(r2, r1, atol=1e-12 * np.abs(r1).max())


def test_rotation_covariance():
    """Rotating mesh, velocities and beta by Q rotates the momentum residuals and conjugates the
    tangent; the continuity residual is invariant."""
    X, U, beta, _ = inputs.random_elements(3, seed=4)
    rng = np.random.default_rng(9)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    p = Params(nu=0.03)
    k = oracle.element_kernel(X, U, beta, p)
    Xr = X @ Q.T
    Ur = U.copy(); Ur[:, :, :3] = U[:, :, :3] @ Q.T
    kr = oracle.element_kernel(Xr, Ur, beta @ Q.T, p)
    np.testing.assert_allclose(kr["Rc"], k["Rc"] @ Q.T, atol=1e-13)
    np.testing.assert_allclose(kr["Rp"], k["Rp"], atol=1e-13)
    np.testing.assert_allclose(kr["Rf"], k["Rf"] @ Q.T, atol=1e-13)
    T = np.zeros((35, 35))
    for a in range(8):
        T[4 * a:4 * a + 3, 4 * a:4 * a + 3] = Q
        T[4 * a + 3, 4 * a + 3] = 1.0
    T[32:, 32:] = Q
    K, Kr = packed_tangent(k), packed_tangent(kr)
    np.testing.assert_allclose(Kr, T @ K @ T.T, atol=1e-12 * np.abs(K).max())


# ----------------------------------------------------------------------------------------------
# bookkeeping against Table 1 of the paper (fine DOF = 3 per element)
# ----------------------------------------------------------------------------------------------

def test_table1_dof_bookkeeping():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_mesh_sizes.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for name, coarse, fine, total in rows:
        coarse, fine, total = int(coarse), int(fine), int(total)
        assert fine % 3 == 0, name          # three bubble unknowns per element
        assert coarse + fine == total, name
    m = inputs.cavity_mesh(8)
    assert m.n_fine_dof == 3 * 512 and m.n_coarse_dof == 4 * 729


def test_workload_sizes():
    assert (inputs.cavity_mesh(8).n_elems, inputs.cavity_mesh(8).n_nodes) == (512, 729)
    m = inputs.cavity_mesh(32)
    assert (m.n_elems, m.n_nodes) == (32768, 35937)
    b = inputs.bfs_mesh(13, jitter_frac=0.0)
    assert (b.n_elems, b.n_nodes) == (518492, 550564)
    c = inputs.channel_mesh(300, 56)
    assert (c.n_elems, c.n_nodes) == (937860, 975583)
