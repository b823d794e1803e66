"""Exact discrete solution of the generalized Stokes system and its diagnostics.

The system (Eq. Saddle_point_A_BT_B, extended with a pressure load g):
    A U - B^T P = F,     B U = g,
has a pressure determined up to a constant (B^T 1 = 0 since int div v = 0 on
H^1_0). The constant is fixed by int p_h = (M_Q 1)^T P = 0 through a bordered
system with one Lagrange multiplier s:
    [ A    -B^T   0 ] [U]   [F]
    [ B     0     m ] [P] = [g],   m = M_Q 1.
    [ 0     m^T   0 ] [s]   [0]
If sum(g) = 0 the multiplier is zero at the solution, so (U, P) solves the
original system. SuperLU (a library routine) is the factorisation.

The augmented-Lagrangian form (Eqs. LA_problem, def_of_Alambda) has the same
solution (U, P) when its right-hand side is F + gamma mu B^T M_Q^{-1} g, so
one direct solve serves every gamma.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .assemble import StokesSystem
from .quadrature import reference_tet_rule
from .reference_element import p2_eval


def bordered_matrix(sys_: StokesSystem) -> sp.csr_matrix:
    m = sys_.MQ1[:, None]
    nv = sys_.A.shape[0]
    z = sp.csr_matrix((nv, 1))
    K = sp.bmat([[sys_.A, -sys_.B.T, z],
                 [sys_.B, None, sp.csr_matrix(m)],
                 [None, sp.csr_matrix(m.T), None]], format="csc")
    return K


def direct_solve(sys_: StokesSystem, F: np.ndarray, g: np.ndarray | None = None):
    """(U, P) of the saddle system with int p_h = 0, by sparse LU."""
    nv, npr = sys_.A.shape[0], sys_.B.shape[0]
    if g is None:
        g = np.zeros(npr)
    rhs = np.concatenate([F, g, [0.0]])
    x = spla.splu(bordered_matrix(sys_), permc_spec="COLAMD").solve(rhs)
    return x[:nv], x[nv:nv + npr]


def schur_cg_solve(sys_: StokesSystem, F: np.ndarray, g: np.ndarray | None = None,
                   tol: float = 1e-14, maxiter: int = 500):
    """(U, P) by conjugate gradients on the pressure Schur complement with exact
    inner solves (Sec. 2.3, Method 1 with every inverse applied exactly).

    A^{-1} is a sparse LU factorisation of A (a library routine), so S = B A^{-1} B^T
    is applied to rounding accuracy; the outer CG is preconditioned by the
    Cahouet-Chabard operator C^Lambda = dt^{-1} (B Lambda_V^{-1} B^T)^+ + mu M_Q^{-1}
    (Eqs. Schur_complement_preconditioners), also applied with sparse LU. The
    pressure iterates are kept orthogonal to the constants; the final P is
    shifted so that int p_h = 0. This is the oracle for meshes too large for
    the bordered direct solve; it is pinned against it on small meshes.
    """
    nv, npr = sys_.A.shape[0], sys_.B.shape[0]
    if g is None:
        g = np.zeros(npr)
    luA = spla.splu(sys_.A.tocsc(), permc_spec="MMD_AT_PLUS_A",
                    options=dict(SymmetricMode=True), diag_pivot_thresh=0.0)
    B = sys_.B
    T = (B @ sp.diags(1.0 / sys_.Lam) @ B.T).tocsr()
    ones = np.ones((npr, 1))
    luT = spla.splu(sp.bmat([[T, sp.csr_matrix(ones)], [sp.csr_matrix(ones.T), None]],
                            format="csc"), permc_spec="MMD_AT_PLUS_A")
    luM = spla.splu(sys_.MQ.tocsc())

    def S(p):
        return B @ luA.solve(B.T @ p)

    def C(r):
        r = r - r.mean()
        z = luT.solve(np.concatenate([r, [0.0]]))[:npr]
        return z / sys_.dt + sys_.mu * luM.solve(r)

    def proj(r):
        return r - r.mean()

    # S P = g - B A^{-1} F
    rhs = proj(g - B @ luA.solve(F))
    P = np.zeros(npr)
    r = rhs.copy()
    nr0 = np.linalg.norm(rhs)
    if nr0 == 0.0:
        U = luA.solve(F)
        return U, P
    z = C(r)
    d = z.copy()
    rz = r @ z
    for _ in range(maxiter):
        q = S(d)
        alpha = rz / (d @ q)
        P += alpha * d
        r = proj(r - alpha * q)
        if np.linalg.norm(r) <= tol * nr0:
            break
        z = C(r)
        rz_new = r @ z
        d = z + (rz_new / rz) * d
        rz = rz_new
    P -= (sys_.MQ1 @ P) / sys_.MQ1.sum()
    U = luA.solve(F + B.T @ P)
    return U, P


def oracle_solve(sys_: StokesSystem, F: np.ndarray, g: np.ndarray | None = None):
    """The oracle's exact discrete solution: bordered LU on small meshes, exact-inverse
    Schur CG above that (both to rounding-level residuals)."""
    if sys_.mesh.n <= 5:
        return direct_solve(sys_, F, g)
    return schur_cg_solve(sys_, F, g)


def dense_solve(sys_: StokesSystem, F: np.ndarray, g: np.ndarray | None = None):
    """Same bordered system by dense LU (numpy) - brute force for tiny meshes."""
    nv, npr = sys_.A.shape[0], sys_.B.shape[0]
    if g is None:
        g = np.zeros(npr)
    K = bordered_matrix(sys_).toarray()
    x = np.linalg.solve(K, np.concatenate([F, g, [0.0]]))
    return x[:nv], x[nv:nv + npr]


def residual(sys_: StokesSystem, U, P, F, g=None):
    """Full-system residual [F - A U + B^T P ; g - B U]."""
    if g is None:
        g = np.zeros(sys_.B.shape[0])
    return np.concatenate([F - sys_.A @ U + sys_.B.T @ P, g - sys_.B @ U])


def relative_residual(sys_: StokesSystem, U, P, F, g=None) -> float:
    if g is None:
        g = np.zeros(sys_.B.shape[0])
    r = residual(sys_, U, P, F, g)
    return float(np.linalg.norm(r) / np.linalg.norm(np.concatenate([F, g])))


def l2_errors(sys_: StokesSystem, U_nodal: np.ndarray, P: np.ndarray, exact, q: int = 6):
    """Relative L2 errors ||u - u_h|| / ||u|| and ||p - p_h|| / ||p|| by quadrature."""
    mesh = sys_.mesh
    lam, w = reference_tet_rule(q)                      # (Q,4), (Q,)
    phi = p2_eval(lam)                                  # (Q,10)
    X = np.einsum("qi,tic->tqc", lam, mesh.coords)      # (T,Q,3)
    vol = np.abs(sys_.det) / 6.0
    wts = 6.0 * vol[:, None] * w[None, :]               # (T,Q)
    uh = np.einsum("qa,tac->tqc", phi, U_nodal[mesh.tet_p2])
    ph = np.einsum("qi,ti->tq", lam, P[mesh.tet_vertices])
    Xf = X.reshape(-1, 3)
    ue = exact.velocity(Xf).reshape(uh.shape)
    pe = exact.pressure(Xf).reshape(ph.shape)
    eu = np.sqrt(np.sum(wts[..., None] * (ue - uh) ** 2) / np.sum(wts[..., None] * ue ** 2))
    ep = np.sqrt(np.sum(wts * (pe - ph) ** 2) / np.sum(wts * pe ** 2))
    return float(eu), float(ep)
