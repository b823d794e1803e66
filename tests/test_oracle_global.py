"""Pins for the oracle's global matrices and exact solution (CPU only).

Checks that do not restate the oracle's own formulas: invariants of the
assembled operators, polynomial exactness, the identity E_V = L_V + D on
H^1_0 (Sec. 3.2), symmetry/definiteness, brute-force dense solves, the
paper's convergence rates (velocity O(h^3), pressure O(h^2); Sec. 3.3 tables),
the augmented-Lagrangian identity (Proposition "Augmented Lagrangian") and the
Cahouet-Chabard limits (Sec. 4.1).
"""

import json
import os

import numpy as np
import pytest

import workload as wl
from oracle.assemble import StokesSystem
from oracle.mesh import KuhnMesh
from oracle.operators import dense, preconditioned_spectrum, preconditioner, schur
from oracle.solve import (dense_solve, direct_solve, l2_errors, relative_residual,
                          schur_cg_solve)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def build(n, mu=1e-2, dt=1e-2, jitter=0.2, seed=7, gamma=0.0):
    V = wl.kuhn_vertices(n, jitter, seed)
    return StokesSystem(KuhnMesh(n, V), mu, dt, gamma)


@pytest.fixture(scope="module")
def sys3():
    return build(3)


def test_counts_match_layout():
    s = build(4)
    assert s.mesh.n_tets == 6 * 4 ** 3
    assert s.mesh.n_p2 == 9 ** 3 and s.mesh.n_p1 == 5 ** 3
    assert s.n_inner == 7 ** 3
    assert wl.num_dofs(8) == 14739 + 729        # config-1 DOF count
    # every P2 node of the half grid is used by some tet
    assert np.unique(s.mesh.tet_p2).size == s.mesh.n_p2


def test_geometry_invariants(sys3):
    s = sys3
    one = np.ones(s.mesh.n_p2)
    assert abs(one @ s.mass_all @ one - 1.0) < 1e-13          # |Omega| = 1
    assert np.abs(s.lap_all @ one).max() < 1e-12               # L_V 1 = 0
    p1 = np.ones(s.mesh.n_p1)
    assert np.abs(s.LQ @ p1).max() < 1e-12                     # L_Q 1 = 0
    assert abs(p1 @ s.MQ @ p1 - 1.0) < 1e-13
    assert abs(s.lumped_all.sum() - (4 * 3 / 32 + 6 / 5) * 1.0) < 1e-12  # sum over tets
    # B^T 1 = 0 on interior velocity DOFs (int div v = 0 for v in H^1_0)
    assert np.abs(s.B.T @ p1).max() < 1e-13


def test_polynomial_exactness_of_divergence(sys3):
    """For a quadratic field u, B_all I2(u) = M_Q I1(div u) exactly."""
    s = sys3
    rng = np.random.default_rng(3)
    C = rng.standard_normal((3, 10))

    def u(X):
        x, y, z = X.T
        mons = np.stack([np.ones_like(x), x, y, z, x * x, y * y, z * z, x * y, y * z, x * z])
        return (C @ mons).T

    def divu(X):
        x, y, z = X.T
        dx = C[0, 1] + 2 * C[0, 4] * x + C[0, 7] * y + C[0, 9] * z
        dy = C[1, 2] + 2 * C[1, 5] * y + C[1, 7] * x + C[1, 8] * z
        dz = C[2, 3] + 2 * C[2, 6] * z + C[2, 8] * y + C[2, 9] * x
        return dx + dy + dz

    lhs = s.B_all @ u(s.mesh.p2_coords()).ravel()
    rhs = s.MQ @ divu(s.mesh.vertices)
    assert np.allclose(lhs, rhs, atol=1e-13)


def test_strain_equals_laplacian_plus_graddiv(sys3):
    """E_V = L_V + D on interior DOFs (integration by parts on H^1_0, Sec. 3.2)."""
    s = sys3
    diff = (s.E - s.Lv - s.D)
    assert abs(diff).max() < 1e-12 * abs(s.E).max()
    # ... but not on the full space (the boundary terms do not vanish there)
    full = s.strain_all - s.graddiv_all
    assert abs(full).max() > 1e-3


def test_symmetry_and_definiteness(sys3):
    s = sys3
    A = dense(s.A)
    assert np.allclose(A, A.T, atol=1e-12 * np.abs(A).max())
    assert np.linalg.eigvalsh(A).min() > 0
    S = schur(s)
    assert np.allclose(S, S.T, atol=1e-12 * np.abs(S).max())
    ev = np.linalg.eigvalsh(S)
    assert abs(ev[0]) < 1e-10 * ev[-1] and ev[1] > 1e-8 * ev[-1]   # kernel = constants


def test_schur_cg_oracle_matches_bordered_lu():
    s = build(4, mu=1e-2, dt=1e-3, seed=3)
    F = s.load(wl.random_force(4, seed=2))
    g = wl.random_pressure_load(4, seed=5)
    U1, P1 = direct_solve(s, F, g)
    U2, P2 = schur_cg_solve(s, F, g)
    assert np.linalg.norm(U1 - U2) < 1e-11 * np.linalg.norm(U1)
    assert np.linalg.norm(P1 - P2) < 1e-11 * np.linalg.norm(P1)
    assert relative_residual(s, U2, P2, F, g) < 1e-12


@pytest.mark.parametrize("n", [2, 3])
def test_direct_solve_matches_dense_brute_force(n):
    s = build(n, mu=0.3, dt=0.05)
    f = wl.random_force(n, seed=11)
    F = s.load(f)
    g = wl.random_pressure_load(n, seed=12)
    U1, P1 = direct_solve(s, F, g)
    U2, P2 = dense_solve(s, F, g)
    assert np.allclose(U1, U2, rtol=1e-10, atol=1e-12 * np.abs(U2).max())
    assert np.allclose(P1, P2, rtol=1e-10, atol=1e-12 * np.abs(P2).max())
    assert relative_residual(s, U1, P1, F, g) < 1e-13
    assert abs(s.MQ1 @ P1) < 1e-12 * np.abs(P1).max()          # int p_h = 0
    assert np.abs(s.B @ U1 - g).max() < 1e-12 * np.abs(g).max()


def test_manufactured_convergence_rates():
    """Velocity L2 error O(h^3), pressure O(h^2) (Sec. 3.3, Tables vel_pb_*)."""
    facts = json.load(open(os.path.join(GOLDEN, "paper_facts.json")))
    eu, ep, hs = [], [], []
    for n in (4, 8):
        V = wl.kuhn_vertices(n, 0.0, 1)
        s = StokesSystem(KuhnMesh(n, V), mu=1.0, dt=1.0)
        ms = wl.Manufactured(seed=1)
        ms.m[:] = 1
        f = ms.body_force(s.mesh.p2_coords(), 1.0, 1.0)
        U, P = schur_cg_solve(s, s.load(f))
        a, b = l2_errors(s, s.expand_velocity(U), P, ms)
        eu.append(a)
        ep.append(b)
        hs.append(1.0 / n)
    ru = np.log(eu[-2] / eu[-1]) / np.log(2.0)
    rp = np.log(ep[-2] / ep[-1]) / np.log(2.0)
    assert ru > facts["p2_velocity_l2_rate"] - 0.35, (eu, ru)
    assert rp > facts["p1_pressure_l2_rate"] - 0.35, (ep, rp)


def test_augmented_lagrangian_identity():
    """S_rho^+ = S^+ + rho Pi M_Q^{-1} Pi (Prop. 'Augmented Lagrangian', rho = lambda mu)."""
    s = build(2, mu=0.7, dt=0.1)
    lam = 3.0
    rho = lam * s.mu
    S = schur(s)
    Sr = schur(s, lam)
    m = S.shape[0]
    Pi = np.eye(m) - np.ones((m, m)) / m
    lhs = np.linalg.pinv(Sr, rcond=1e-12, hermitian=True)
    rhs = np.linalg.pinv(S, rcond=1e-12, hermitian=True) + rho * Pi @ np.linalg.inv(dense(s.MQ)) @ Pi
    assert np.allclose(lhs, rhs, rtol=1e-8, atol=1e-9 * np.abs(rhs).max())


def test_cahouet_chabard_limits():
    """S -> dt B M_V^{-1} B^T as mu dt / h^2 -> 0 and mu S -> B E_V^{-1} B^T as
    mu dt / h^2 -> infinity (Sec. 4.1); C^Lambda keeps the preconditioned
    spectrum bounded across the whole range."""
    n = 2
    small = build(n, mu=1e-8, dt=1e-2)
    T0 = dense(small.B) @ np.linalg.solve(dense(small.Mv), dense(small.B).T)
    S0 = schur(small)
    assert np.abs(S0 / small.dt - T0).max() < 1e-4 * np.abs(T0).max()
    big = build(n, mu=1e6, dt=1.0)
    Tinf = dense(big.B) @ np.linalg.solve(dense(big.E), dense(big.B).T)
    Sinf = schur(big)
    assert np.abs(big.mu * Sinf - Tinf).max() < 1e-4 * np.abs(Tinf).max()
    # preconditioned condition numbers stay bounded over 12 decades of mu dt/h^2
    for kind in ("mass", "lumped"):
        conds = []
        for mu in 10.0 ** np.arange(-8, 5, 2):
            s = build(n, mu=mu, dt=1e-2)
            ev = preconditioned_spectrum(preconditioner(s, kind), schur(s))
            conds.append(ev[-1] / ev[0])
        assert max(conds) < 30, (kind, conds)
    # C (with M_V) is exact in the mu -> 0 limit
    ev = preconditioned_spectrum(preconditioner(small, "mass"), S0)
    assert ev[-1] / ev[0] < 1 + 1e-3


def test_pressure_laplacian_preconditioner_bounds():
    """C^Delta_lambda = dt^{-1} L_Q^+ + mu (1+lambda) M_Q^{-1} (Eqs.
    Schur_complement_preconditioners, pressure-Laplacian form) against bounds
    that follow from the continuous operators, not from its own formula:
    * (div v, q) = -(v, grad q) for v in H^1_0 gives q^T B M_V^{-1} B^T q <=
      q^T L_Q q, so in the limit mu dt / h^2 -> 0 (S -> dt B M_V^{-1} B^T) every
      eigenvalue of C^Delta S is <= 1;
    * ||div v||^2 <= ||eps(v)||^2 = v^T E_V v / 2 on H^1_0 gives
      M_Q^{-1} B E_V^{-1} B^T <= 1/2, so as mu dt / h^2 -> infinity
      (mu S -> B E_V^{-1} B^T) the eigenvalues are <= 1/2;
    * S <= both limits, hence lambda_max(C^Delta S) <= 3/2 for every mu, dt;
    * with the augmented Lagrangian, S_lambda^+ = S^+ + lambda mu M_Q^{-1}, so as
      lambda -> infinity C^Delta_lambda S_lambda -> (1+lambda)/lambda -> 1.
    A wrong dt or mu scaling, a missing (1+lambda) or M_Q in place of M_Q^{-1}
    breaks one of these. On the unjittered Kuhn mesh the interior rows of L_Q
    are h times the 7-point finite-difference Laplacian (a closed form)."""
    for n in (2, 3):
        for mu in 10.0 ** np.arange(-8, 7, 2):
            s = build(n, mu=mu, dt=1e-2)
            ev = preconditioned_spectrum(preconditioner(s, "laplace"), schur(s))
            assert ev[0] > 0 and ev[-1] <= 1.5 + 1e-10, (n, mu, ev[-1])
            if mu <= 1e-6:
                assert ev[-1] <= 1.0 + 1e-6, (n, mu, ev[-1])
            if mu >= 1e4:
                assert ev[-1] <= 0.5 + 1e-6, (n, mu, ev[-1])
    s = build(2, mu=0.3, dt=1e-2)
    ev = preconditioned_spectrum(preconditioner(s, "laplace", 1e6), schur(s, 1e6))
    assert abs(ev[0] - 1) < 1e-4 and abs(ev[-1] - 1) < 1e-4, (ev[0], ev[-1])
    # closed form of L_Q on the unjittered Kuhn mesh
    n = 3
    s = build(n, jitter=0.0)
    LQ = dense(s.LQ)
    h, nv = 1.0 / n, n + 1
    for (i, j, k) in ((1, 1, 1), (2, 1, 2), (1, 2, 2)):
        v = i + nv * (j + nv * k)
        ref = np.zeros(nv ** 3)
        ref[v] = 6 * h
        for d in (1, nv, nv * nv):
            ref[v - d] = ref[v + d] = -h
        assert np.abs(LQ[v] - ref).max() < 1e-13
