"""Pins for the oracle's element integrals (CPU only).

Each closed-form element matrix is checked against an independent route:
quadrature with the conical Gauss rule, basis gradients from central finite
differences in physical coordinates (exact for quadratics up to rounding),
barycentric coordinates from a 4x4 linear solve rather than the inverse
Jacobian, and the strain tensor formed explicitly as 2 eps(u):eps(v).
"""

import numpy as np
import pytest

from oracle.quadrature import reference_tet_rule
from oracle.reference_element import (LOCAL_EDGES, LUMPED_REF, P2_MASS_REF,
                                      element_matrices, monomial_integral, p2_eval)

RNG = np.random.default_rng(12345)


def random_tet():
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    X = X + 0.25 * RNG.standard_normal((4, 3))
    if np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], -1)) < 0:
        X[[1, 2]] = X[[2, 1]]
    return X


def barycentric(X, x):
    """lam with sum lam = 1 and sum lam_i X_i = x, by a plain 4x4 solve."""
    M = np.vstack([np.ones(4), X.T])
    return np.linalg.solve(M, np.concatenate([[1.0], x]))


def grad_fd(fun, x, h=1e-3):
    g = []
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        g.append((fun(x + e) - fun(x - e)) / (2 * h))
    return np.stack(g, axis=-1)


def quad_points(X, q=5):
    lam, w = reference_tet_rule(q)
    vol = abs(np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], -1))) / 6
    return lam @ X, 6 * vol * w, vol


def test_nodal_basis_and_partition_of_unity():
    nodes = [np.eye(4)[i] for i in range(4)]
    nodes += [0.5 * (np.eye(4)[i] + np.eye(4)[j]) for i, j in LOCAL_EDGES]
    V = p2_eval(np.array(nodes))
    assert np.allclose(V, np.eye(10), atol=1e-15)
    lam = RNG.dirichlet(np.ones(4), size=50)
    assert np.allclose(p2_eval(lam).sum(axis=1), 1.0, atol=1e-14)


def test_monomial_integral_against_quadrature():
    lam, w = reference_tet_rule(6)
    for alpha in [(0, 0, 0, 0), (1, 0, 0, 0), (2, 1, 0, 0), (1, 1, 1, 1), (0, 2, 0, 2), (3, 0, 1, 0)]:
        quad = np.sum(w * np.prod(lam ** np.array(alpha), axis=1)) * 6  # |K_ref| = 1/6
        assert abs(quad - monomial_integral(alpha)) < 1e-14


def test_p2_mass_reference():
    lam, w = reference_tet_rule(5)
    phi = p2_eval(lam)
    Mq = 6 * np.einsum("q,qa,qb->ab", w, phi, phi)
    assert np.allclose(Mq, P2_MASS_REF, atol=1e-15, rtol=1e-13)
    # row sums: int phi_vertex = -|K|/20, int phi_edge = |K|/5; total |K|
    rs = P2_MASS_REF.sum(axis=1)
    assert np.allclose(rs[:4], -1 / 20) and np.allclose(rs[4:], 1 / 5)
    assert abs(P2_MASS_REF.sum() - 1.0) < 1e-14


@pytest.mark.parametrize("trial", range(3))
def test_element_matrices_against_fd_quadrature(trial):
    X = random_tet()
    em = element_matrices(X[None])
    pts, wts, vol = quad_points(X)
    assert abs(em["vol"][0] - vol) < 1e-14

    def phi_at(x):
        return p2_eval(barycentric(X, x)[None])[0]

    gphi = np.stack([grad_fd(phi_at, x) for x in pts])           # (Q,10,3)
    lam = np.stack([barycentric(X, x) for x in pts])              # (Q,4)
    glam = grad_fd(lambda x: barycentric(X, x), pts[0])           # (4,3), constant
    phi = p2_eval(lam)
    tol = dict(rtol=1e-8, atol=1e-9 * np.abs(em["lap"]).max())
    # mass, Laplacian
    assert np.allclose(np.einsum("q,qa,qb->ab", wts, phi, phi), em["mass"][0], rtol=1e-12, atol=1e-15)
    assert np.allclose(np.einsum("q,qac,qbc->ab", wts, gphi, gphi), em["lap"][0], **tol)
    # strain: 2 eps(phi_a e_c) : eps(phi_b e_d) built from explicit tensors
    S = np.zeros((10, 3, 10, 3))
    for a in range(10):
        for c in range(3):
            Gu = np.zeros((len(pts), 3, 3))
            Gu[:, c, :] = gphi[:, a, :]                      # grad(phi_a e_c), row c
            eu = 0.5 * (Gu + Gu.transpose(0, 2, 1))
            for b in range(10):
                for d in range(3):
                    Gv = np.zeros((len(pts), 3, 3))
                    Gv[:, d, :] = gphi[:, b, :]
                    ev = 0.5 * (Gv + Gv.transpose(0, 2, 1))
                    S[a, c, b, d] = np.sum(wts * 2 * np.einsum("qij,qij->q", eu, ev))
    assert np.allclose(S, em["strain"][0], **tol)
    # grad-div: div(phi_a e_c) = d_c phi_a
    Dq = np.einsum("q,qac,qbd->acbd", wts, gphi, gphi)
    assert np.allclose(Dq, em["graddiv"][0], **tol)
    # divergence: int psi_k d_c phi_a, psi_k = lam_k
    Bq = np.einsum("q,qk,qac->kac", wts, lam, gphi)
    assert np.allclose(Bq, em["div"][0], rtol=1e-8, atol=1e-9 * np.abs(Bq).max())
    # P1 mass / Laplacian
    assert np.allclose(np.einsum("q,qk,ql->kl", wts, lam, lam), em["pmass"][0], rtol=1e-12)
    assert np.allclose(vol * glam @ glam.T, em["plap"][0], rtol=1e-8)


def test_lumped_velocity_mass_constants():
    """int |phi_a| over the reference tet (|K| = 1/6), split where the vertex
    function changes sign (Sec. 4.1: the absolute value matters)."""
    lam, w = reference_tet_rule(8, u_split=0.5)   # lam_1 = u: kink of vertex 1 at 1/2
    for a in range(10):
        # permute barycentric coordinates so that node a plays vertex 1's role
        perm = list(range(4))
        if a < 4:
            perm[a], perm[1] = perm[1], perm[a]
        lp = lam[:, perm]
        val = 6 * np.sum(w * np.abs(p2_eval(lp)[:, a]))
        assert abs(val - LUMPED_REF[a]) < 1e-13, (a, val)
    # the signed vertex integral is negative, which is why the lumping uses |phi|
    assert abs(6 * np.sum(w * p2_eval(lam)[:, 1]) + 1 / 20) < 1e-14


def test_jacobi_scaled_mass_intervals():
    """Chebyshev-Jacobi on M_Q and M_V needs sigma(D^{-1} M). For affine
    tetrahedra M_K = |K| M_ref, so the element pencil (M_K, diag M_K) has
    shape-independent eigenvalues: P1 {1/2, 1/2, 1/2, 5/2} (Wathen 1987) and
    for P2 extremes 1/4 and 4.34747. Wathen's element argument then bounds the
    assembled, Dirichlet-restricted D^{-1} M; checked here on a jittered mesh."""
    import scipy.linalg as sla
    import workload as wl
    from oracle.assemble import StokesSystem
    from oracle.mesh import KuhnMesh
    from oracle.reference_element import element_matrices
    rng = np.random.default_rng(4)
    X = rng.standard_normal((3, 4, 3))
    em = element_matrices(X)
    for t in range(3):
        for M, lo, hi in ((em["mass"][t], 0.25, 4.347467), (em["pmass"][t], 0.5, 2.5)):
            w = sla.eigh(M, np.diag(np.diag(M)), eigvals_only=True)
            assert abs(w[0] - lo) < 1e-9 and abs(w[-1] - hi) < 1e-6, w
    sysm = StokesSystem(KuhnMesh(3, wl.kuhn_vertices(3, 0.2, 1)), 1.0, 1.0)
    Mv = sysm.Mv.toarray()[::3, ::3]                       # one velocity component
    w = sla.eigh(Mv, np.diag(np.diag(Mv)), eigvals_only=True)
    assert w[0] >= 0.25 - 1e-12 and w[-1] <= 4.3475, (w[0], w[-1])
    Mq = sysm.MQ.toarray()
    w = sla.eigh(Mq, np.diag(np.diag(Mq)), eigvals_only=True)
    assert w[0] >= 0.5 - 1e-12 and w[-1] <= 2.5 + 1e-12
