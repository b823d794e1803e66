"""Global FP64 matrices of the P2-P1 generalized Stokes problem (plain COO sums).

Follows the paper's definitions (Sec. 2.2 "Discrete problem"):
    A_ij = M_V,ij / dt + mu E_V,ij,    B_kj = b(phi_j, psi_k) = int psi_k div phi_j,
with homogeneous Dirichlet velocity on the whole boundary (Sec. 3.1: V = H^1_0),
so boundary velocity rows and columns are removed. The pressure space is all P1
nodes (the constant is fixed separately, by int p_h = 0).

Velocity DOFs of the reduced system: 3*k + c for the k-th interior P2 node
(lexicographic order) and component c. Also provides the preconditioner
matrices of Sec. 3.2, Eqs. for A~_lambda,1..3 (L_V, D), Sec. 4.1 (L_Q,
Lambda_V, eps M_Q + L_Q).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import KuhnMesh
from .reference_element import element_matrices


def _coo(rows, cols, vals, shape):
    return sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=shape).tocsr()


class StokesSystem:
    """Assembled P2-P1 operators on one Kuhn mesh for given (mu, dt)."""

    def __init__(self, mesh: KuhnMesh, mu: float, dt: float, gamma: float = 0.0):
        self.mesh, self.mu, self.dt, self.gamma = mesh, float(mu), float(dt), float(gamma)
        em = element_matrices(mesh.coords)
        self.det = em["det"]
        inverted = np.sign(self.det) != mesh.ref_sign
        if np.any(inverted) or np.any(em["vol"] <= 0):
            raise ValueError(f"{int(inverted.sum())} inverted tetrahedra in the jittered mesh")
        T = mesh.n_tets
        nodes = mesh.tet_p2                                  # (T, 10)
        npv, npp = mesh.n_p2, mesh.n_p1
        # scalar P2 on all nodes
        r = np.repeat(nodes[:, :, None], 10, axis=2)
        c = np.repeat(nodes[:, None, :], 10, axis=1)
        self.mass_all = _coo(r, c, em["mass"], (npv, npv))
        self.lap_all = _coo(r, c, em["lap"], (npv, npv))
        # vector P2 (3 components interleaved) on all nodes
        vd = (3 * nodes[:, :, None] + np.arange(3)[None, None, :]).reshape(T, 30)
        rv = np.repeat(vd[:, :, None], 30, axis=2)
        cv = np.repeat(vd[:, None, :], 30, axis=1)
        self.strain_all = _coo(rv, cv, em["strain"].reshape(T, 30, 30), (3 * npv, 3 * npv))
        self.graddiv_all = _coo(rv, cv, em["graddiv"].reshape(T, 30, 30), (3 * npv, 3 * npv))
        # B: P1 rows x vector P2 columns
        pv = mesh.tet_vertices                               # (T, 4)
        rb = np.repeat(pv[:, :, None], 30, axis=2)
        cb = np.repeat(vd[:, None, :], 4, axis=1)
        self.B_all = _coo(rb, cb, em["div"].reshape(T, 4, 30), (npp, 3 * npv))
        rp = np.repeat(pv[:, :, None], 4, axis=2)
        cp = np.repeat(pv[:, None, :], 4, axis=1)
        self.MQ = _coo(rp, cp, em["pmass"], (npp, npp))
        self.LQ = _coo(rp, cp, em["plap"], (npp, npp))
        self.lumped_all = np.bincount(nodes.ravel(), weights=em["lumped"].ravel(), minlength=npv)

        # restriction to interior velocity DOFs
        inner = mesh.interior
        self.n_inner = inner.size
        vin = (3 * inner[:, None] + np.arange(3)[None, :]).ravel()
        self.vel_dofs = vin
        self.Ms = self.mass_all[inner][:, inner].tocsr()          # scalar M_V
        self.Ls = self.lap_all[inner][:, inner].tocsr()           # scalar L_V
        self.M_rows_all = self.mass_all[inner].tocsr()            # for F = M_V f
        self.E = self.strain_all[vin][:, vin].tocsr()             # E_V
        self.D = self.graddiv_all[vin][:, vin].tocsr()            # grad-div D
        I3 = sp.identity(3, format="csr")
        self.Mv = sp.kron(self.Ms, I3, format="csr")              # vector M_V
        self.Lv = sp.kron(self.Ls, I3, format="csr")              # vector L_V
        self.A = (self.Mv / self.dt + self.mu * self.E).tocsr()   # A = M_V/dt + mu E_V
        self.B = self.B_all[:, vin].tocsr()
        self.lumped = self.lumped_all[inner]                      # Lambda_V per node
        self.Lam = np.repeat(self.lumped, 3)                      # per velocity DOF
        # scalar A~_3 = M/dt + mu L (Eq. precond_A_plus_lambda_D_3, per component)
        self.A3s = (self.Ms / self.dt + self.mu * self.Ls).tocsr()
        self.MQ1 = np.asarray(self.MQ.sum(axis=1)).ravel()        # int psi_k

    # -- right-hand sides -------------------------------------------------
    def load(self, f_nodal: np.ndarray) -> np.ndarray:
        """F = M_V f_h on interior rows, f_h the P2 interpolant of the nodal force."""
        f_nodal = np.asarray(f_nodal, dtype=np.float64).reshape(-1, 3)
        return (self.M_rows_all @ f_nodal).ravel()

    # -- layouts -----------------------------------------------------------
    def expand_velocity(self, U: np.ndarray) -> np.ndarray:
        """Reduced velocity vector -> (n_p2, 3) nodal field with zero boundary."""
        out = np.zeros((self.mesh.n_p2, 3))
        out[self.mesh.interior] = np.asarray(U).reshape(-1, 3)
        return out

    def restrict_velocity(self, u_nodal: np.ndarray) -> np.ndarray:
        return np.asarray(u_nodal).reshape(-1, 3)[self.mesh.interior].ravel()
