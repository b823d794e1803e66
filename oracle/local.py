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
from .reference_element import P2_MASS_REF, element_matrices


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
