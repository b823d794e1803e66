"""P2 (velocity) and P1 (pressure) Lagrange elements on an affine tetrahedron.

Every P2 basis function is written as a homogeneous quadratic form in the
barycentric coordinates, phi_a = lam^T Q_a lam, using sum(lam) = 1:

* vertex i:     lam_i (2 lam_i - 1) = lam_i^2 - sum_{j != i} lam_i lam_j
* edge (i, j):  4 lam_i lam_j

Integrals of barycentric monomials over a tetrahedron K are exact:
    int_K lam^alpha dx = |K| * 3! * prod(alpha_k!) / (|alpha| + 3)!

The matrices follow the paper's definitions (Sec. 2.2, "Discrete problem";
Sec. 3.2, L_V and D; Sec. 4.1, L_Q and Lambda_V):
    M_V,ij = int phi_i . phi_j,      M_Q,kl = int psi_k psi_l,
    E_V = int 2 eps(phi_i) : eps(phi_j),   L_V,ij = int grad phi_i : grad phi_j,
    D_ij = int div phi_i div phi_j,  B_kj = int psi_k div phi_j,
    L_Q,kl = int grad psi_k . grad psi_l,  Lambda_V,ii = int |phi_i|.
"""

from __future__ import annotations

import itertools
from math import factorial

import numpy as np

# local P2 node order: 4 vertices, then the 6 edges in this order
LOCAL_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


def p2_quadratic_forms() -> np.ndarray:
    """Q[a] (4x4 symmetric) with phi_a(lam) = lam^T Q[a] lam, a = 0..9."""
    Q = np.zeros((10, 4, 4))
    for i in range(4):
        Q[i, i, i] = 1.0
        for j in range(4):
            if j != i:
                Q[i, i, j] -= 0.5
                Q[i, j, i] -= 0.5
    for e, (i, j) in enumerate(LOCAL_EDGES):
        Q[4 + e, i, j] = 2.0
        Q[4 + e, j, i] = 2.0
    return Q


def monomial_integral(alpha) -> float:
    """int_K prod lam_k^alpha_k dx / |K| = 3! prod(alpha!) / (|alpha|+3)!."""
    num = 6.0
    for a in alpha:
        num *= factorial(a)
    return num / factorial(sum(alpha) + 3)


def _barycentric_moment_tensor(order: int) -> np.ndarray:
    """T[i1..i_order] = int_K lam_i1 ... lam_i_order dx / |K|."""
    T = np.zeros((4,) * order)
    for idx in itertools.product(range(4), repeat=order):
        alpha = [idx.count(k) for k in range(4)]
        T[idx] = monomial_integral(alpha)
    return T


MOMENT2 = _barycentric_moment_tensor(2)  # (1 + delta_ij) / 20
MOMENT4 = _barycentric_moment_tensor(4)


def p2_reference_mass() -> np.ndarray:
    """10x10 matrix Mref with int_K phi_a phi_b = |K| Mref[a,b]."""
    Q = p2_quadratic_forms()
    return np.einsum("aij,bkl,ijkl->ab", Q, Q, MOMENT4)


P2_MASS_REF = p2_reference_mass()


def tet_geometry(X: np.ndarray):
    """For tets with vertex coordinates X (..., 4, 3): (|K|, det J, grad lam (...,4,3)).

    J has columns x1-x0, x2-x0, x3-x0; lam_{1..3} = J^{-1}(x - x0), so the rows of
    J^{-1} are grad lam_1..3 and grad lam_0 = -(sum of the others).
    """
    J = np.stack([X[..., 1, :] - X[..., 0, :], X[..., 2, :] - X[..., 0, :],
                  X[..., 3, :] - X[..., 0, :]], axis=-1)
    det = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    G = np.empty(X.shape[:-2] + (4, 3))
    G[..., 1:, :] = Jinv
    G[..., 0, :] = -Jinv.sum(axis=-2)
    return np.abs(det) / 6.0, det, G


def p2_gradient_coefficients(G: np.ndarray) -> np.ndarray:
    """W (..., 10, 4, 3) with grad phi_a = sum_i lam_i W[a, i, :].

    grad(lam^T Q lam) = 2 sum_{i,j} Q_ij lam_i grad lam_j (Q symmetric).
    """
    Q = p2_quadratic_forms()
    return 2.0 * np.einsum("aij,...jc->...aic", Q, G)


def p2_gradient_products(vol: np.ndarray, G: np.ndarray) -> np.ndarray:
    """H (..., 10, 10, 3, 3): H[a,b,c,d] = int_K d_c phi_a d_d phi_b."""
    W = p2_gradient_coefficients(G)
    return vol[..., None, None, None, None] * np.einsum(
        "...aic,ik,...bkd->...abcd", W, MOMENT2, W)


def element_matrices(X: np.ndarray) -> dict:
    """All element matrices for tets with vertex coordinates X (..., 4, 3).

    Returns a dict of arrays (leading dims of X kept):
      mass    (10,10)        int phi_a phi_b                       (scalar P2)
      lap     (10,10)        int grad phi_a . grad phi_b           (scalar P2)
      strain  (10,3,10,3)    int 2 eps(phi_a e_c) : eps(phi_b e_d)
      graddiv (10,3,10,3)    int d_c phi_a d_d phi_b   (= D on (a,c),(b,d))
      div     (4,10,3)       int psi_k d_c phi_a       (B, row = P1 vertex k)
      pmass   (4,4)          int psi_k psi_l
      plap    (4,4)          int grad psi_k . grad psi_l
      lumped  (10,)          int |phi_a|
      vol, det
    """
    vol, det, G = tet_geometry(X)
    H = p2_gradient_products(vol, G)
    lap = np.einsum("...abcc->...ab", H)
    eye3 = np.eye(3)
    # 2 eps(u):eps(v) = grad u : grad v + grad u : (grad v)^T; for u = phi_a e_c and
    # v = phi_b e_d this is delta_cd grad phi_a . grad phi_b + d_d phi_a d_c phi_b.
    strain = (np.einsum("...ab,cd->...acbd", lap, eye3)
              + np.einsum("...abdc->...acbd", H))
    graddiv = np.einsum("...abcd->...acbd", H)
    W = p2_gradient_coefficients(G)
    div = vol[..., None, None, None] * np.einsum("ki,...aic->...kac", MOMENT2, W)
    pmass = vol[..., None, None] * MOMENT2
    plap = vol[..., None, None] * np.einsum("...kc,...lc->...kl", G, G)
    mass = vol[..., None, None] * P2_MASS_REF
    lumped = vol[..., None] * LUMPED_REF
    return dict(mass=mass, lap=lap, strain=strain, graddiv=graddiv, div=div,
                pmass=pmass, plap=plap, lumped=lumped, vol=vol, det=det)


# int_K |lam (2 lam - 1)| = 3|K|/32 and int_K 4 lam_i lam_j = |K|/5.  One
# barycentric coordinate of a uniform point in K has density 3 (1 - t)^2 on
# [0, 1]; splitting the vertex integrand at t = 1/2, where it changes sign,
# gives 7/320 + 23/320 = 3/32.  (Sec. 4.1: the absolute value is needed
# because P2 vertex functions integrate to -|K|/20.)
LUMPED_REF = np.array([3.0 / 32.0] * 4 + [1.0 / 5.0] * 6)


def p2_eval(lam: np.ndarray) -> np.ndarray:
    """phi_a at barycentric points lam (..., 4) -> (..., 10)."""
    Q = p2_quadratic_forms()
    return np.einsum("...i,aij,...j->...a", lam, Q, lam)


def p2_eval_grad(lam: np.ndarray, G: np.ndarray) -> np.ndarray:
    """grad phi_a at barycentric points lam (P, 4) on one tet with grad lam G (4,3)
    -> (P, 10, 3)."""
    W = p2_gradient_coefficients(G)  # (10, 4, 3)
    return np.einsum("pi,aic->pac", lam, W)
