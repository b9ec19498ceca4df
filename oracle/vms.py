"""Plain FP64 oracle: element residual, consistent tangent, Schur condensation, assembly, Newton.

Test infrastructure only (see the package docstring). Loops run over quadrature points; every
operation inside is vectorised over elements only, with the formula written as printed.

Notation (per quadrature point q of element e):
  w_q          Gauss weight,  omega = w_q * det J
  N_a, dN_a    trilinear shape functions and their reference derivatives (a = 0..7)
  J[i,al]      = dx_i/dxi_al = sum_a x_{a,i} dN_a/dxi_al
  g[a,j]       = dN_a/dx_j   = sum_al dN_a/dxi_al (J^-1)[al,j]
  b, d[j]      bubble and its physical gradient (Eq. DefineBubbles3: v' = b beta)
  v            = sum_a N_a vhat_a + b beta          (Eq. SC_Decompose_v)
  L[i,j]       = dv_i/dx_j = sum_a vhat_{a,i} g[a,j] + beta_i d[j]
  p            = sum_a N_a phat_a                    (no fine pressure, Section 3.1)
  conv_i       = sum_j v_j L[i,j]                    ((v . grad) v)
  nut          = visc_factor * nu                    (the "2 nu" of Eq. SC_CoarseScale_Momentum)
  tau          = 1/dt for backward Euler, 0 when steady (Remark in Section 4.1)
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# Reference corners in the local node order (-,-,-) (+,-,-) (+,+,-) (-,+,-) (-,-,+) (+,-,+)
# (+,+,+) (-,+,+). Written out here, not imported, so the oracle stands alone.
CORNERS = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                    [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=np.float64)


@dataclass
class Params:
    nu: float                   # kinematic viscosity (Eq. SC_Equilibrium)
    visc_factor: float = 2.0    # weak-form viscous coefficient nut = visc_factor*nu (Eq. SC_CoarseScale_Momentum)
    dt: float = 0.0             # backward-Euler step; 0 = steady
    f: tuple = (0.0, 0.0, 0.0)  # body force b (constant)
    quad_order: int = 3         # Gauss points per direction
    bubble_scale: float = 1.0   # b = bubble_scale * (1-xi^2)(1-eta^2)(1-zeta^2) (hexahedron)
    element: str = "hex"        # "hex": Q1 + one bubble; "tet": P1 + one bubble (MINI-type)

    @property
    def nut(self) -> float:
        return self.visc_factor * self.nu

    @property
    def tau(self) -> float:
        return 0.0 if self.dt == 0.0 else 1.0 / self.dt


class NegativeJacobian(ValueError):
    pass


# ----------------------------------------------------------------------------------------------
# reference element (Section 3.3 and Section 4.1's DN / J notation, here for the trilinear hex)
# ----------------------------------------------------------------------------------------------

def gauss_rule(n: int):
    """Tensor-product Gauss-Legendre rule on [-1,1]^3: points (nq,3), weights (nq,)."""
    x, w = np.polynomial.legendre.leggauss(n)
    pts, wts = [], []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                pts.append((x[i], x[j], x[k]))
                wts.append(w[i] * w[j] * w[k])
    return np.array(pts), np.array(wts)


def q1_basis(xi: np.ndarray):
    """N_a(xi) = 1/8 prod_d (1 + s_{a,d} xi_d) and dN_a/dxi_al, for points xi (nq,3).

    Returns N (nq,8) and dN (nq,8,3)."""
    xi = np.atleast_2d(xi)
    fac = 1.0 + CORNERS[None, :, :] * xi[:, None, :]          # (nq,8,3)
    N = fac.prod(axis=2) / 8.0
    dN = np.empty(fac.shape)
    for al in range(3):
        others = [d for d in range(3) if d != al]
        dN[:, :, al] = CORNERS[None, :, al] * fac[:, :, others[0]] * fac[:, :, others[1]] / 8.0
    return N, dN


def bubble(xi: np.ndarray, scale: float = 1.0):
    """b(xi) = scale * prod_d (1 - xi_d^2), zero on every face of the element (Eq.
    SC_Fine_Scale_Vanish), and its reference gradient. Returns b (nq,), db (nq,3)."""
    xi = np.atleast_2d(xi)
    fac = 1.0 - xi ** 2
    b = scale * fac.prod(axis=1)
    db = np.empty(xi.shape)
    for al in range(3):
        others = [d for d in range(3) if d != al]
        db[:, al] = scale * (-2.0 * xi[:, al]) * fac[:, others[0]] * fac[:, others[1]]
    return b, db


# ----------------------------------------------------------------------------------------------
# reference tetrahedron: vertices (0,0,0), (1,0,0), (0,1,0), (0,0,1); barycentric coordinates
# lambda = (1 - xi - eta - zeta, xi, eta, zeta); P1 shape functions N_a = lambda_a; the bubble
# b = 256 lambda_0 lambda_1 lambda_2 lambda_3 (zero on every face, 1 at the centroid)
# ----------------------------------------------------------------------------------------------

TET_CORNERS = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
TET_DLAMBDA = np.array([[-1, -1, -1], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)


def tet_rule(n: int):
    """Conical-product (collapsed Gauss) rule on the reference tetrahedron with n points per
    direction: xi = u, eta = v (1 - u), zeta = w (1 - u)(1 - v) with Gauss-Jacobi points in u
    (weight (1-u)^2), v (weight (1-v)) and Gauss-Legendre points in w, all on [0, 1]; exact for
    polynomials of total degree 2n - 1. Returns points (n^3, 3) and weights (sum 1/6)."""
    from scipy.special import roots_jacobi
    def on01(x, w, a):   # Gauss-Jacobi on [-1,1] with weight (1-x)^a -> [0,1] with (1-u)^a
        return (x + 1.0) / 2.0, w / 2.0 ** (a + 1)
    ux, uw = on01(*roots_jacobi(n, 2.0, 0.0), 2)
    vx, vw = on01(*roots_jacobi(n, 1.0, 0.0), 1)
    wx, ww = on01(*roots_jacobi(n, 0.0, 0.0), 0)
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                u, v, w = ux[i], vx[j], wx[k]
                pts.append((u, v * (1.0 - u), w * (1.0 - u) * (1.0 - v)))
                wts.append(uw[i] * vw[j] * ww[k])
    return np.array(pts), np.array(wts)


def p1_basis(xi: np.ndarray):
    """N_a = lambda_a and the constant reference gradients. Returns N (nq,4), dN (nq,4,3)."""
    xi = np.atleast_2d(xi)
    lam = np.stack([1.0 - xi.sum(axis=1), xi[:, 0], xi[:, 1], xi[:, 2]], axis=1)
    dN = np.broadcast_to(TET_DLAMBDA, (xi.shape[0], 4, 3)).copy()
    return lam, dN


def tet_bubble(xi: np.ndarray, scale: float = 1.0):
    """b = scale * 256 prod_a lambda_a and its reference gradient. Returns b (nq,), db (nq,3)."""
    lam, _ = p1_basis(xi)
    b = scale * 256.0 * lam.prod(axis=1)
    db = np.zeros((lam.shape[0], 3))
    for a in range(4):
        others = np.prod(lam[:, [c for c in range(4) if c != a]], axis=1)
        db += scale * 256.0 * others[:, None] * TET_DLAMBDA[a][None, :]
    return b, db


def element_basis(params):
    """Quadrature points, weights, shape functions and bubble of the element kind in params."""
    if params.element == "tet":
        pts, wts = tet_rule(params.quad_order)
        N, dN = p1_basis(pts)
        b, db = tet_bubble(pts, params.bubble_scale)
    else:
        pts, wts = gauss_rule(params.quad_order)
        N, dN = q1_basis(pts)
        b, db = bubble(pts, params.bubble_scale)
    return pts, wts, N, dN, b, db


# ----------------------------------------------------------------------------------------------
# element residual and consistent tangent (Section 4.1 Eqs. SC_Coarse_Resid_Vec, _Vec_2,
# SC_Fine_Resid_Vec and the transient Remark; Section 4.2 Eq. NewtonUpdate2)
# ----------------------------------------------------------------------------------------------

def _qp_fields(Xe, V, P, beta, N, dN, b, db):
    """Geometry and fields at one quadrature point, for all elements at once."""
    J = np.einsum("eai,ak->eik", Xe, dN)             # J[e,i,al] = dx_i/dxi_al
    detJ = np.linalg.det(J)
    if np.any(detJ <= 0.0):
        raise NegativeJacobian(f"det J <= 0 in {int(np.sum(detJ <= 0))} element(s)")
    Jinv = np.linalg.inv(J)                          # Jinv[e,al,j] = dxi_al/dx_j
    g = np.einsum("ak,ekj->eaj", dN, Jinv)           # dN_a/dx_j
    d = np.einsum("k,ekj->ej", db, Jinv)             # db/dx_j
    vbar = np.einsum("a,eai->ei", N, V)
    v = vbar + b * beta
    L = np.einsum("eai,eaj->eij", V, g) + np.einsum("ei,ej->eij", beta, d)
    p = np.einsum("a,ea->e", N, P)
    conv = np.einsum("ej,eij->ei", v, L)
    return detJ, g, d, v, L, p, conv


def element_kernel(X, U, beta, params: Params, Uprev=None, with_tangent=True):
    """Element residuals R_c (E,8,3), R_p (E,8), R_f (E,3) and, if asked, the consistent tangent
    blocks of Eq. NewtonUpdate2 for every element.

    X (E,8,3) nodal coordinates, U (E,8,4) nodal (v, p), beta (E,3), Uprev (E,8,4) previous step.

    Residuals (Section 4.1), integrated with the Gauss rule of params.quad_order:
      R_c[a,i] = int N_a conv_i + nut sum_j g_aj L_ij - g_ai p - N_a f_i + tau N_a (vbar - vbar_n)_i
      R_p[a]   = - int N_a tr L
      R_f[i]   = int b conv_i + nut sum_j d_j L_ij - d_i p - b f_i + tau b (vbar - vbar_n)_i
    The transient terms act on the coarse velocity only, in both R_c and R_f (Remark, Sec. 4.1).

    Tangent blocks, the exact derivatives of the residuals above with respect to vhat_{b,k},
    phat_b and beta_k (c_b = v.g_b, c_d = v.d):
      K_vv[a,i,b,k] = int N_a (N_b L_ik + d_ik c_b) + nut d_ik g_a.g_b + tau d_ik N_a N_b
      K_vp[a,i,b]   = - int g_ai N_b            K_pv[a,b,k] = - int N_a g_bk       K_pp = 0
      K_vf[a,i,k]   = int N_a (b L_ik + d_ik c_d) + nut d_ik g_a.d
      K_pf[a,k]     = - int N_a d_k
      K_fv[i,b,k]   = int b (N_b L_ik + d_ik c_b) + nut d_ik d.g_b + tau d_ik b N_b
      K_fp[i,b]     = - int d_i N_b
      K_ff[i,k]     = int b (b L_ik + d_ik c_d) + nut d_ik d.d
    """
    X = np.asarray(X, np.float64)
    U = np.asarray(U, np.float64)
    beta = np.asarray(beta, np.float64)
    E = X.shape[0]
    V, P = U[:, :, :3], U[:, :, 3]
    nut, tau = params.nut, params.tau
    f = np.asarray(params.f, np.float64)
    dV = None
    if tau != 0.0:
        if Uprev is None:
            raise ValueError("transient step needs the previous velocity")
        dV = V - np.asarray(Uprev, np.float64)[:, :, :3]
    pts, wts, Nq, dNq, bq, dbq = element_basis(params)
    I3 = np.eye(3)
    na = X.shape[1]   # nodes per element: 8 (hexahedron) or 4 (tetrahedron)

    Rc = np.zeros((E, na, 3)); Rp = np.zeros((E, na)); Rf = np.zeros((E, 3))
    if with_tangent:
        Kvv = np.zeros((E, na, 3, na, 3)); Kvp = np.zeros((E, na, 3, na)); Kpv = np.zeros((E, na, na, 3))
        Kvf = np.zeros((E, na, 3, 3)); Kpf = np.zeros((E, na, 3))
        Kfv = np.zeros((E, 3, na, 3)); Kfp = np.zeros((E, 3, na)); Kff = np.zeros((E, 3, 3))

    for q in range(pts.shape[0]):
        N, dN, b, db = Nq[q], dNq[q], bq[q], dbq[q]
        detJ, g, d, v, L, p, conv = _qp_fields(X, V, P, beta, N, dN, b, db)
        om = wts[q] * detJ                               # (E,)
        trL = np.einsum("eii->e", L)
        src = -f[None, :] * np.ones((E, 1))              # - f_i
        if dV is not None:
            src = src + tau * np.einsum("a,eai->ei", N, dV)   # + tau (vbar - vbar_n)_i

        # residuals
        Rc += om[:, None, None] * (
            N[None, :, None] * conv[:, None, :]
            + nut * np.einsum("eaj,eij->eai", g, L)
            - g * p[:, None, None]
            + N[None, :, None] * src[:, None, :])
        Rp += om[:, None] * (-N[None, :] * trL[:, None])
        Rf += om[:, None] * (
            b * conv + nut * np.einsum("ej,eij->ei", d, L) - d * p[:, None] + b * src)

        if not with_tangent:
            continue
        cb = np.einsum("ej,ebj->eb", v, g)               # v . g_b
        cd = np.einsum("ej,ej->e", v, d)                 # v . d
        gg = np.einsum("eaj,ebj->eab", g, g)             # g_a . g_b
        gd = np.einsum("eaj,ej->ea", g, d)               # g_a . d
        dd = np.einsum("ej,ej->e", d, d)                 # d . d
        NN = np.outer(N, N)                              # N_a N_b

        Kvv += om[:, None, None, None, None] * (
            NN[None, :, None, :, None] * L[:, None, :, None, :]
            + I3[None, None, :, None, :] * (
                N[None, :, None, None, None] * cb[:, None, None, :, None]
                + nut * gg[:, :, None, :, None]
                + tau * NN[None, :, None, :, None]))
        Kvp += om[:, None, None, None] * (-g[:, :, :, None] * N[None, None, None, :])
        Kpv += om[:, None, None, None] * (-N[None, :, None, None] * g[:, None, :, :])
        Kvf += om[:, None, None, None] * (
            N[None, :, None, None] * (b * L[:, None, :, :]
                                      + I3[None, None] * cd[:, None, None, None])
            + nut * I3[None, None] * gd[:, :, None, None])
        Kpf += om[:, None, None] * (-N[None, :, None] * d[:, None, :])
        Kfv += om[:, None, None, None] * (
            b * (N[None, None, :, None] * L[:, :, None, :]
                 + I3[None, :, None, :] * cb[:, None, :, None])
            + nut * I3[None, :, None, :] * np.einsum("ej,ebj->eb", d, g)[:, None, :, None]
            + tau * I3[None, :, None, :] * (b * N)[None, None, :, None])
        Kfp += om[:, None, None] * (-d[:, :, None] * N[None, None, :])
        Kff += om[:, None, None] * (
            b * (b * L + I3[None] * cd[:, None, None]) + nut * I3[None] * dd[:, None, None])

    out = {"Rc": Rc, "Rp": Rp, "Rf": Rf}
    if with_tangent:
        out.update(Kvv=Kvv, Kvp=Kvp, Kpv=Kpv, Kvf=Kvf, Kpf=Kpf, Kfv=Kfv, Kfp=Kfp, Kff=Kff)
    return out


def element_residual_only(X, U, beta, params: Params, Uprev=None):
    return element_kernel(X, U, beta, params, Uprev, with_tangent=False)


def elementary_integrals(X, quad_order=3, bubble_scale=1.0):
    """Integrals of basis products over each element, through the same geometry code as
    element_kernel: volume, int b, int |grad b|^2, int N_a d_k and int b g_ak (E,8,3)."""
    X = np.asarray(X, np.float64)
    E = X.shape[0]
    pts, wts = gauss_rule(quad_order)
    Nq, dNq = q1_basis(pts)
    bq, dbq = bubble(pts, bubble_scale)
    zV = np.zeros((E, 8, 3)); zP = np.zeros((E, 8)); zb = np.zeros((E, 3))
    out = {"vol": np.zeros(E), "b": np.zeros(E), "dd": np.zeros(E),
           "N_d": np.zeros((E, 8, 3)), "b_g": np.zeros((E, 8, 3))}
    for q in range(pts.shape[0]):
        detJ, g, d, _, _, _, _ = _qp_fields(X, zV, zP, zb, Nq[q], dNq[q], bq[q], dbq[q])
        om = wts[q] * detJ
        out["vol"] += om
        out["b"] += om * bq[q]
        out["dd"] += om * np.einsum("ej,ej->e", d, d)
        out["N_d"] += om[:, None, None] * Nq[q][None, :, None] * d[:, None, :]
        out["b_g"] += om[:, None, None] * bq[q] * g
    return out


def pack_element(k):
    """Pack the blocks in node-major coarse order (dof 4a+c, c=3 pressure); n = 4 * nodes per
    element (32 for the hexahedron, 16 for the tetrahedron).

    Returns Kcc (E,n,n), Kcf (E,n,3), Kfc (E,3,n), Kff (E,3,3), Rcp (E,n), Rf (E,3)."""
    E, na = k["Rc"].shape[0], k["Rc"].shape[1]
    nc = 4 * na
    Kcc = np.zeros((E, na, 4, na, 4))
    Kcc[:, :, :3, :, :3] = k["Kvv"]
    Kcc[:, :, :3, :, 3] = k["Kvp"]
    Kcc[:, :, 3, :, :3] = k["Kpv"]
    Kcf = np.zeros((E, na, 4, 3))
    Kcf[:, :, :3, :] = k["Kvf"]
    Kcf[:, :, 3, :] = k["Kpf"]
    Kfc = np.zeros((E, 3, na, 4))
    Kfc[:, :, :, :3] = k["Kfv"]
    Kfc[:, :, :, 3] = k["Kfp"]
    Rcp = np.zeros((E, na, 4))
    Rcp[:, :, :3] = k["Rc"]
    Rcp[:, :, 3] = k["Rp"]
    return (Kcc.reshape(E, nc, nc), Kcf.reshape(E, nc, 3), Kfc.reshape(E, 3, nc),
            k["Kff"].copy(), Rcp.reshape(E, nc), k["Rf"].copy())


def pack_residual(k):
    """Residuals in node-major coarse order: Rcp (E,4 na) with dof 4a+c, and Rf (E,3)."""
    E, na = k["Rc"].shape[0], k["Rc"].shape[1]
    Rcp = np.concatenate([k["Rc"], k["Rp"][:, :, None]], axis=2).reshape(E, 4 * na)
    return Rcp, k["Rf"].copy()


def condense(Kcc, Kcf, Kfc, Kff, Rcp, Rf):
    """Block Gauss elimination of the three bubble unknowns (Section 5, Eq. SchurUpdate):
      S_e = K_cc - K_cf K_ff^-1 K_fc,     r_e = R_cp - K_cf K_ff^-1 R_f.
    Returns S (E,n,n), r (E,n), KffinvKfc (E,3,n), KffinvRf (E,3)."""
    X = np.linalg.solve(Kff, Kfc)                    # K_ff^-1 K_fc
    y = np.linalg.solve(Kff, Rf[:, :, None])[:, :, 0]
    S = Kcc - Kcf @ X
    r = Rcp - np.einsum("eck,ek->ec", Kcf, y)
    return S, r, X, y


# ----------------------------------------------------------------------------------------------
# global assembly (the assembly operator A_e of Section 5) and Dirichlet conditions
# ----------------------------------------------------------------------------------------------

def element_dofs(conn):
    conn = np.asarray(conn, np.int64)
    return (4 * conn[:, :, None] + np.arange(4)[None, None, :]).reshape(conn.shape[0], 4 * conn.shape[1])


def gather(conn, xyz, u, beta, u_prev=None):
    X = xyz[conn]
    U = u[conn]
    Up = None if u_prev is None else u_prev[conn]
    return X, U, beta, Up


def assemble(conn, n_nodes, S, r):
    """Sum element matrices and vectors into the global coarse system (CSR, duplicates summed)."""
    dofs = element_dofs(conn)
    E = dofs.shape[0]
    nc = dofs.shape[1]
    rows = np.repeat(dofs, nc, axis=1).reshape(-1)
    cols = np.tile(dofs, (1, nc)).reshape(-1)
    n = 4 * n_nodes
    A = sp.coo_matrix((S.reshape(-1), (rows, cols)), shape=(n, n)).tocsr()
    A.sum_duplicates()
    rhs = np.zeros(n)
    np.add.at(rhs, dofs.reshape(-1), r.reshape(-1))
    return A, rhs


def assemble_vector(conn, n_nodes, Rcp):
    """Sum element coarse vectors (E,32) into a global vector of 4*n_nodes entries."""
    out = np.zeros(4 * n_nodes)
    np.add.at(out, element_dofs(conn).reshape(-1), np.asarray(Rcp).reshape(-1))
    return out


def apply_dirichlet(A, rhs, dofs):
    """Constrained dofs get increment 0: their rows and columns are zeroed, the diagonal set to 1
    and the right-hand-side entry set to 0 (the prescribed values already sit in the state)."""
    dofs = np.asarray(dofs, np.int64)
    n = A.shape[0]
    keep = np.ones(n)
    keep[dofs] = 0.0
    D = sp.diags(keep)
    A = D @ sp.csr_matrix(A) @ D + sp.diags(1.0 - keep)
    rhs = rhs.copy()
    rhs[dofs] = 0.0
    return sp.csr_matrix(A), rhs


def residual_vector(conn, n_nodes, k, dir_dofs):
    """Full nonlinear residual: assembled [R_c; R_p] on free dofs and every element's R_f."""
    dofs = element_dofs(conn)
    Rcp = np.zeros(4 * n_nodes)
    E = conn.shape[0]
    rc = np.concatenate([k["Rc"], k["Rp"][:, :, None]], axis=2).reshape(E, dofs.shape[1])
    np.add.at(Rcp, dofs.reshape(-1), rc.reshape(-1))
    Rcp[np.asarray(dir_dofs, np.int64)] = 0.0
    return np.concatenate([Rcp, k["Rf"].reshape(-1)])


def fine_recovery(conn, du, X_kfc, y_rf):
    """Delta beta_e = K_ff^-1 (-R_f - K_fc Delta u_e)  (Section 5, after Eq. SchurUpdate)."""
    due = du[element_dofs(conn)]                     # (E,4 na)
    return -y_rf - np.einsum("eic,ec->ei", X_kfc, due)


def newton_solve(mesh_xyz, conn, u0, beta0, dir_dofs, params: Params, tol=1e-10, maxit=20,
                 u_prev=None, linear_solver=None, history=None):
    """Newton-Schur iteration (Section 4.2 update equations, Section 5 condensation and fine
    recovery): assemble S and r, solve S du = -r with Dirichlet rows, recover d beta per element,
    update, until ||R|| / ||R^0|| < tol. Returns (u, beta, residual norms)."""
    u = np.array(u0, np.float64, copy=True)
    beta = np.array(beta0, np.float64, copy=True)
    n_nodes = u.shape[0]
    norms = []
    for it in range(maxit + 1):
        X, U, _, Up = gather(conn, mesh_xyz, u, beta, u_prev)
        k = element_kernel(X, U, beta, params, Up)
        R = residual_vector(conn, n_nodes, k, dir_dofs)
        norms.append(float(np.linalg.norm(R)))
        if history is not None:
            history.append((u.copy(), beta.copy()))
        if norms[-1] <= tol * norms[0] or it == maxit:
            break
        Kcc, Kcf, Kfc, Kff, Rcp, Rf = pack_element(k)
        S, r, Xk, y = condense(Kcc, Kcf, Kfc, Kff, Rcp, Rf)
        A, rhs = assemble(conn, n_nodes, S, r)
        A, rhs = apply_dirichlet(A, rhs, dir_dofs)
        du = (linear_solver or spla.spsolve)(A.tocsc(), -rhs)
        dbeta = fine_recovery(conn, du, Xk, y)
        u += du.reshape(n_nodes, 4)
        beta += dbeta
    return u, beta, norms


# ----------------------------------------------------------------------------------------------
# the uncondensed mixed system (Eq. NewtonUpdate2 with coarse and fine unknowns side by side),
# used to pin the exactness of the Schur form
# ----------------------------------------------------------------------------------------------

def uncondensed_system(conn, n_nodes, Kcc, Kcf, Kfc, Kff, Rcp, Rf, dir_dofs):
    """Dense global matrix over [4*n_nodes coarse dofs, 3*n_elems fine dofs] with Dirichlet rows
    and columns of the constrained coarse dofs replaced by identity; returns (K, R)."""
    E = conn.shape[0]
    nc = 4 * n_nodes
    n = nc + 3 * E
    K = np.zeros((n, n))
    R = np.zeros(n)
    dofs = element_dofs(conn)
    for e in range(E):
        c = dofs[e]
        fdofs = nc + 3 * e + np.arange(3)
        K[np.ix_(c, c)] += Kcc[e]
        K[np.ix_(c, fdofs)] += Kcf[e]
        K[np.ix_(fdofs, c)] += Kfc[e]
        K[np.ix_(fdofs, fdofs)] += Kff[e]
        R[c] += Rcp[e]
        R[fdofs] += Rf[e]
    d = np.asarray(dir_dofs, np.int64)
    K[d, :] = 0.0
    K[:, d] = 0.0
    K[d, d] = 1.0
    R[d] = 0.0
    return K, R
