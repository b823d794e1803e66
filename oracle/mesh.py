"""Kuhn (Freudenthal) tetrahedral mesh of the unit cube and its DOF numbering.

Cube (i, j, k) with base corner b is split into six tetrahedra, one per
permutation pi of the axes: vertices b, b + e_pi0, b + e_pi0 + e_pi1,
b + (1,1,1). The split is conforming across cubes and self-similar under
2x refinement. (It stands in for the paper's unstructured triangle meshes,
Sec. 3.1 and Sec. 5.2, which are not available.)

Numbering (shared layouts, not arithmetic): vertices lexicographic with x
fastest on the (n+1)^3 grid; P2 nodes on the (2n+1)^3 half-grid with the node
of an edge at the sum of its endpoints' integer coordinates.
"""

from __future__ import annotations

import itertools

import numpy as np

PERMUTATIONS = tuple(itertools.permutations(range(3)))


def kuhn_tets(n: int) -> np.ndarray:
    """Integer vertex coordinates of all tets: shape (6 n^3, 4, 3)."""
    c = np.arange(n)
    K, J, I = np.meshgrid(c, c, c, indexing="ij")
    base = np.stack([I.ravel(), J.ravel(), K.ravel()], axis=1)  # (n^3, 3)
    tets = []
    for p in PERMUTATIONS:
        e0 = np.eye(3, dtype=int)[p[0]]
        e1 = np.eye(3, dtype=int)[p[1]]
        corners = np.stack([np.zeros(3, int), e0, e0 + e1, np.ones(3, int)])
        tets.append(base[:, None, :] + corners[None, :, :])
    # order: cube-major, then permutation
    return np.stack(tets, axis=1).reshape(-1, 4, 3)


def vertex_id(ijk: np.ndarray, n: int) -> np.ndarray:
    nv = n + 1
    return ijk[..., 0] + nv * (ijk[..., 1] + nv * ijk[..., 2])


def p2_id(q: np.ndarray, n: int) -> np.ndarray:
    """Global P2 node id of half-grid coordinates q (..., 3)."""
    N = 2 * n + 1
    return q[..., 0] + N * (q[..., 1] + N * q[..., 2])


def p2_element_nodes(tets: np.ndarray, n: int) -> np.ndarray:
    """Global P2 node ids of the 10 local nodes (4 vertices, 6 edges) per tet."""
    from .reference_element import LOCAL_EDGES
    q = [2 * tets[:, a, :] for a in range(4)]
    q += [tets[:, i, :] + tets[:, j, :] for (i, j) in LOCAL_EDGES]
    return np.stack([p2_id(x, n) for x in q], axis=1)


def p2_interior_mask(n: int) -> np.ndarray:
    N = 2 * n + 1
    q = np.arange(N)
    K, J, I = np.meshgrid(q, q, q, indexing="ij")
    inner = lambda a: (a > 0) & (a < N - 1)  # noqa: E731
    return (inner(I) & inner(J) & inner(K)).ravel()


class KuhnMesh:
    """Topology + geometry of a (possibly jittered) Kuhn mesh."""

    def __init__(self, n: int, vertices: np.ndarray):
        self.n = n
        self.vertices = np.asarray(vertices, dtype=np.float64)
        assert self.vertices.shape == ((n + 1) ** 3, 3)
        self.tets_ijk = kuhn_tets(n)
        self.tet_vertices = vertex_id(self.tets_ijk, n)            # (T, 4)
        self.tet_p2 = p2_element_nodes(self.tets_ijk, n)           # (T, 10)
        self.coords = self.vertices[self.tet_vertices]             # (T, 4, 3)
        self.n_p2 = (2 * n + 1) ** 3
        self.n_p1 = (n + 1) ** 3
        mask = p2_interior_mask(n)
        self.interior = np.nonzero(mask)[0]
        self.p2_to_interior = -np.ones(self.n_p2, dtype=np.int64)
        self.p2_to_interior[self.interior] = np.arange(self.interior.size)
        # reference orientation of each tet (sign of det J on the unjittered grid)
        ref = self.tets_ijk.astype(np.float64)
        J = np.stack([ref[:, 1] - ref[:, 0], ref[:, 2] - ref[:, 0], ref[:, 3] - ref[:, 0]], -1)
        self.ref_sign = np.sign(np.linalg.det(J))

    @property
    def n_tets(self) -> int:
        return self.tet_vertices.shape[0]

    def p2_coords(self) -> np.ndarray:
        """Coordinates of all P2 nodes (vertices and straight-edge midpoints)."""
        X = np.zeros((self.n_p2, 3))
        from .reference_element import LOCAL_EDGES
        for a in range(4):
            X[self.tet_p2[:, a]] = self.coords[:, a]
        for e, (i, j) in enumerate(LOCAL_EDGES):
            X[self.tet_p2[:, 4 + e]] = 0.5 * (self.coords[:, i] + self.coords[:, j])
        return X
