"""Dense (tiny-mesh) Schur complements and Cahouet-Chabard preconditioners.

Plain definitions for pinning, with explicit dense inverses:
* S = B A^{-1} B^T (Sec. 2.3, Method 1),
* A_lambda = A + lambda mu B^T M_Q^{-1} B and S_lambda = B A_lambda^{-1} B^T
  (Eqs. def_of_Alambda, def_Schur_LA_problem),
* C_lambda, C^Lambda_lambda, C^Delta_lambda (Eqs.
  Schur_complement_preconditioners):
      dt^{-1} (B M_V^{-1} B^T)^+ + mu (1+lambda) M_Q^{-1}, and the same with
      Lambda_V or L_Q in place of B M_V^{-1} B^T.
The pressure operators annihilate constants (B^T 1 = 0); "^+" is the
Moore-Penrose pseudo-inverse, i.e. the inverse on the Euclidean complement of
the constants.
"""

from __future__ import annotations

import numpy as np

from .assemble import StokesSystem


def dense(m):
    return m.toarray() if hasattr(m, "toarray") else np.asarray(m)


def schur(sys_: StokesSystem, lam: float = 0.0) -> np.ndarray:
    A = dense(sys_.A)
    B = dense(sys_.B)
    if lam != 0.0:
        A = A + lam * sys_.mu * B.T @ np.linalg.solve(dense(sys_.MQ), B)
    return B @ np.linalg.solve(A, B.T)


def preconditioner(sys_: StokesSystem, kind: str, lam: float = 0.0) -> np.ndarray:
    """Dense C for kind in {'mass' (C), 'lumped' (C^Lambda), 'laplace' (C^Delta)}."""
    B = dense(sys_.B)
    MQinv = np.linalg.inv(dense(sys_.MQ))
    if kind == "mass":
        T = B @ np.linalg.solve(dense(sys_.Mv), B.T)
    elif kind == "lumped":
        T = B @ (B.T / sys_.Lam[:, None])
    elif kind == "laplace":
        T = dense(sys_.LQ)
    else:
        raise ValueError(kind)
    return np.linalg.pinv(T, rcond=1e-12, hermitian=True) / sys_.dt + sys_.mu * (1 + lam) * MQinv


def mean_zero_basis(m: int) -> np.ndarray:
    """Orthonormal basis of the Euclidean complement of the constants."""
    Qm, _ = np.linalg.qr(np.eye(m) - np.ones((m, m)) / m)
    return Qm[:, : m - 1]


def preconditioned_spectrum(C: np.ndarray, S: np.ndarray) -> np.ndarray:
    """Eigenvalues of C S on the complement of its kernel (the constants)."""
    Z = mean_zero_basis(S.shape[0])
    Sh = Z.T @ S @ Z
    # C S restricted: generalised problem Sh x = theta (Z^T C Z)^{-1} x; C SPD.
    Ch = Z.T @ C @ Z
    L = np.linalg.cholesky(Ch)
    ev = np.linalg.eigvalsh(L.T @ Sh @ L)
    return np.sort(ev)
