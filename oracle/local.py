"""Residual rows of the saddle system from the elements around chosen nodes.

For meshes too large for a global assembly in numpy, the oracle evaluates
selected rows of r = [F - A U + B^T P ; g - B U] (Eq. Saddle_point_A_BT_B with
A = M_V/dt + mu E_V, F = M_V f_h) using only the tetrahedra that contain the
chosen nodes, plus the exact norm ||F|| from a vectorised element loop. Each
row is a sum of element contributions, so this is the same definition as
oracle.assemble restricted to a few rows; it is pinned against the global
assembly on small meshes (tests/test_oracle_local.py).
"""

from __future__ import annotations

import numpy as np

from .mesh import KuhnMesh
from .quadrature import reference_tet_rule
from .reference_element import (MOMENT2, P2_MASS_REF, element_matrices, p2_eval,
                                p2_gradient_coefficients, tet_geometry)


def node_to_tets(mesh: KuhnMesh, nodes: np.ndarray, vertex: bool = False):
    """For each requested node: array of (tet, local index) pairs containing it."""
    table = mesh.tet_vertices if vertex else mesh.tet_p2
    flat = table.ravel()
    order = np.argsort(flat, kind="stable")
    sorted_ids = flat[order]
    out = []
    for nd in nodes:
        lo = np.searchsorted(sorted_ids, nd, side="left")
        hi = np.searchsorted(sorted_ids, nd, side="right")
        pos = order[lo:hi]
        out.append((pos // table.shape[1], pos % table.shape[1]))
    return out


def velocity_residual_rows(mesh: KuhnMesh, mu: float, dt: float, f_nodal, u_nodal, p, nodes):
    """r_i = F_i - (A U)_i + (B^T P)_i at interior P2 nodes `nodes`; returns (len, 3)."""
    res = np.zeros((len(nodes), 3))
    for row, (tets, loc) in enumerate(node_to_tets(mesh, nodes)):
        X = mesh.coords[tets]
        em = element_matrices(X)
        for t in range(len(tets)):
            a = loc[t]
            gl = mesh.tet_p2[tets[t]]
            fl = f_nodal[gl]                     # (10, 3)
            ul = u_nodal[gl]                     # (10, 3), zero on the boundary
            pl = p[mesh.tet_vertices[tets[t]]]   # (4,)
            M = em["mass"][t]                    # (10, 10)
            Es = em["strain"][t]                 # (10, 3, 10, 3)
            Bt = em["div"][t]                    # (4, 10, 3)
            F_loc = M[a] @ fl                    # (3,)
            AU = M[a] @ ul / dt + mu * np.einsum("cbd,bd->c", Es[a], ul)
            BtP = np.einsum("k,kc->c", pl, Bt[:, a, :])
            res[row] += F_loc - AU + BtP
    return res


def pressure_residual_rows(mesh: KuhnMesh, u_nodal, g, vertices):
    """r_k = g_k - (B U)_k at P1 vertices `vertices`."""
    res = np.array([g[v] if g is not None else 0.0 for v in vertices], dtype=float)
    for row, (tets, loc) in enumerate(node_to_tets(mesh, vertices, vertex=True)):
        X = mesh.coords[tets]
        em = element_matrices(X)
        for t in range(len(tets)):
            k = loc[t]
            ul = u_nodal[mesh.tet_p2[tets[t]]]
            res[row] -= np.einsum("ac,ac->", em["div"][t][k], ul)
    return res


def load_norm(mesh: KuhnMesh, f_nodal, chunk: int = 20000) -> float:
    """||F||_2 of F = M_V f_h on interior rows, by a vectorised element loop."""
    F = np.zeros((mesh.n_p2, 3))
    for s in range(0, mesh.n_tets, chunk):
        X = mesh.coords[s:s + chunk]
        J = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=-1)
        vol = np.abs(np.linalg.det(J)) / 6.0             # element mass = |K| * P2_MASS_REF
        gl = mesh.tet_p2[s:s + chunk]
        contrib = vol[:, None, None] * np.einsum("ab,tbc->tac", P2_MASS_REF, f_nodal[gl])
        for c in range(3):
            F[:, c] += np.bincount(gl.ravel(), weights=contrib[:, :, c].ravel(), minlength=mesh.n_p2)
    return float(np.linalg.norm(F[mesh.interior]))


def _chunk_geometry(mesh: KuhnMesh, s: int, e: int):
    """|K| and the gradient coefficients W (T, 10, 4, 3) of tets s..e-1:
    grad phi_a = sum_i lam_i W[a, i, :] on each tet."""
    vol, _, G = tet_geometry(mesh.coords[s:e])
    return vol, p2_gradient_coefficients(G)


def full_residual(mesh: KuhnMesh, mu: float, dt: float, f_nodal, cases, chunk: int = 50000):
    """Every row of r = [F - A U + B^T P ; g - B U] for several (u, p, g).

    A = M_V/dt + mu E_V and B_kj = int psi_k div phi_j are the operators of the
    saddle system (Sec. 2.2, Eq. Saddle_point_A_BT_B), F = M_V f_h. Each row
    is a sum of element contributions, evaluated here tet by tet in vectorised
    chunks without forming any global matrix, from the gradients of the P2
    functions (linear on an affine tet) and the exact barycentric moments:
      int_K 2 eps(u_h) : eps(phi_a e_c) = |K| sum_{i,d} W[a,i,d] (Q[i,d,c] + Q[i,c,d]),
      Q[i,d,e] = sum_k M2[i,k] sum_b W[b,k,d] u_b,e   (M2[i,k] = int lam_i lam_k / |K|),
      int_K psi_k div(u_h)       = |K| sum_i M2[k,i] sum_d Q'[i,d,d],
      int_K p_h div(phi_a e_c)   = |K| sum_i (sum_k p_k M2[k,i]) W[a,i,c].
    `f_nodal` (n_p2, 3) is one force for all cases or a list with one per
    case; `cases` is a list of (u_nodal (n_p2, 3) with
    zero boundary rows, p (n_p1,), g (n_p1,) or None). Returns a list of
    (rF (n_interior, 3), rg (n_p1,)) and ||[F; g]|| per case.
    """
    npv, npp = mesh.n_p2, mesh.n_p1
    forces = list(f_nodal) if isinstance(f_nodal, (list, tuple)) else [f_nodal] * len(cases)
    assert len(forces) == len(cases)
    R = [np.zeros((npv, 3)) for _ in cases]
    Fs = [np.zeros((npv, 3)) for _ in cases]
    BU = [np.zeros(npp) for _ in cases]
    for s in range(0, mesh.n_tets, chunk):
        e = min(s + chunk, mesh.n_tets)
        vol, W = _chunk_geometry(mesh, s, e)
        gl = mesh.tet_p2[s:e]                       # (T, 10)
        gv = mesh.tet_vertices[s:e]                 # (T, 4)
        T = e - s
        Wf = W.reshape(T, 10, 12)                                        # (a, (i, d))
        for j, (u_nodal, p, _) in enumerate(cases):
            fl = np.einsum("ab,tbc->tac", P2_MASS_REF, forces[j][gl], optimize=True) * vol[:, None, None]
            ul = u_nodal[gl]                                             # (T, 10, 3)
            # gradu[k, d, e]: d_d u_e = sum_k lam_k gradu[k, d, e]
            gradu = np.matmul(np.swapaxes(Wf, 1, 2), ul).reshape(T, 4, 3, 3)
            Q = np.einsum("ik,tkde->tide", MOMENT2, gradu, optimize=True)
            S2 = (Q + np.swapaxes(Q, 2, 3)).reshape(T, 12, 3)            # ((i, d), c)
            strain = np.matmul(Wf, S2) * vol[:, None, None]
            mass = np.einsum("ab,tbc->tac", P2_MASS_REF, ul, optimize=True) * vol[:, None, None]
            au = mass / dt + mu * strain
            pm = p[gv] @ MOMENT2                                         # (T, 4), M2 symmetric
            btp = np.einsum("ti,taic->tac", pm, W, optimize=True) * vol[:, None, None]
            divu = np.einsum("tidd->ti", Q)                              # int lam_i div u_h / |K|
            bu = divu * vol[:, None]
            loc = fl - au + btp                                          # F - A U + B^T P
            for c in range(3):
                R[j][:, c] += np.bincount(gl.ravel(), weights=loc[:, :, c].ravel(), minlength=npv)
                Fs[j][:, c] += np.bincount(gl.ravel(), weights=fl[:, :, c].ravel(), minlength=npv)
            BU[j] += np.bincount(gv.ravel(), weights=bu.ravel(), minlength=npp)
    inner = mesh.interior
    out = []
    for j, (_, _, g) in enumerate(cases):
        gg = np.zeros(npp) if g is None else np.asarray(g, dtype=float)
        rF = R[j][inner]
        rg = gg - BU[j]
        norm = float(np.sqrt(np.sum(Fs[j][inner] ** 2) + np.sum(gg ** 2)))
        out.append((rF, rg, norm))
    return out


def relative_residuals(mesh: KuhnMesh, mu: float, dt: float, f_nodal, cases, chunk: int = 50000):
    """||[F - A U + B^T P; g - B U]||_2 / ||[F; g]||_2 per case (see full_residual)."""
    res = []
    for rF, rg, norm in full_residual(mesh, mu, dt, f_nodal, cases, chunk):
        res.append(float(np.sqrt(np.sum(rF ** 2) + np.sum(rg ** 2)) / norm))
    return res


def l2_errors_chunked(mesh: KuhnMesh, u_nodal, p, exact, q: int = 4, chunk: int = 20000):
    """Relative L2 errors ||u - u_h|| / ||u||, ||p - p_h|| / ||p|| by the conical
    Gauss rule with q points per direction, tet by tet in chunks (the same
    definition as oracle.solve.l2_errors, for meshes too large to assemble)."""
    lam, w = reference_tet_rule(q)
    phi = p2_eval(lam)
    num_u = den_u = num_p = den_p = 0.0
    for s in range(0, mesh.n_tets, chunk):
        e = min(s + chunk, mesh.n_tets)
        X = mesh.coords[s:e]
        vol, _, _ = tet_geometry(X)
        wts = 6.0 * vol[:, None] * w[None, :]
        Xq = np.einsum("qi,tic->tqc", lam, X).reshape(-1, 3)
        uh = np.einsum("qa,tac->tqc", phi, u_nodal[mesh.tet_p2[s:e]])
        ph = np.einsum("qi,ti->tq", lam, p[mesh.tet_vertices[s:e]])
        ue = exact.velocity(Xq).reshape(uh.shape)
        pe = exact.pressure(Xq).reshape(ph.shape)
        num_u += float(np.sum(wts[..., None] * (ue - uh) ** 2))
        den_u += float(np.sum(wts[..., None] * ue ** 2))
        num_p += float(np.sum(wts * (pe - ph) ** 2))
        den_p += float(np.sum(wts * pe ** 2))
    return float(np.sqrt(num_u / den_u)), float(np.sqrt(num_p / den_p))
