"""GPU checks of the adjoint solve and its autograd wrapper.

J(u, p) = c . u + d . p (c at all P2 nodes, d at P1 nodes). The oracle's
adjoint comes from the transposed bordered system: with K_b the bordered
matrix of oracle.solve (its solution already has int p_h = 0),
J = [c_U; d; 0]^T K_b^{-1} [F; g; 0], so dJ/d[F; g] = K_b^{-T} [c_U; d; 0],
dJ/df = (rows of M_V)^T dJ/dF, dJ/dmu = -lambda_U^T E_V U. Finite differences:
J is linear in f, so the central difference with unit step is exact up to the
solver tolerance; in mu it is checked with a small relative step.
"""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workload as wl
from oracle.assemble import StokesSystem
from oracle.mesh import KuhnMesh
from oracle.solve import bordered_matrix, oracle_solve

from gpu_helpers import cuda, gpu_module, host, rel_err

pytestmark = pytest.mark.gpu

N, MU, DT = 4, 0.3, 0.05


def setup_case(seed=31, n=N):
    sk = gpu_module()
    V = wl.kuhn_vertices(n, 0.2, seed)
    f = wl.random_force(n, seed + 1)
    rng = np.random.default_rng(seed)
    c = rng.standard_normal(((2 * n + 1) ** 3, 3))
    d = rng.standard_normal((n + 1) ** 3)
    return sk, V, f, c, d


def J(sk, S, f, c, d, tol=1e-13):
    u, p, _ = S.solve(cuda(f), None, tol)
    return float((host(u) * c).sum() + host(p) @ d), host(u), host(p)


@pytest.mark.parametrize("n", [4, 8])
def test_adjoint_matches_oracle_adjoint(n):
    sk, V, f, c, d = setup_case(n=n)
    S = sk.Stokes(n, V, MU, DT)
    J0, u, p = J(sk, S, f, c, d)
    dJdf, dJdg, dmu, info = S.adjoint(cuda(c), cuda(d), 1e-13)
    orc = StokesSystem(KuhnMesh(n, V), MU, DT)
    Kb = bordered_matrix(orc)
    rhs = np.concatenate([orc.restrict_velocity(c), d, [0.0]])
    lam = spla.splu(Kb.T.tocsc()).solve(rhs)
    nv, npr = orc.A.shape[0], orc.B.shape[0]
    lamU, lamP = lam[:nv], lam[nv:nv + npr]
    dJdf_or = (orc.M_rows_all.T @ lamU.reshape(-1, 3))
    assert rel_err(host(dJdf), dJdf_or) < 1e-9
    # dJ/dg is defined up to a constant (sum(g) = 0): compare mean-free parts
    gpu_g = host(dJdg)
    assert rel_err(gpu_g - gpu_g.mean(), lamP - lamP.mean()) < 1e-8
    Uo, Po = oracle_solve(orc, orc.load(f))
    dmu_or = -lamU @ (orc.E @ Uo)
    assert abs(dmu - dmu_or) < 1e-8 * abs(dmu_or), (dmu, dmu_or)
    S.close()


def test_adjoint_finite_differences():
    sk, V, f, c, d = setup_case(41)
    S = sk.Stokes(N, V, MU, DT)
    J(sk, S, f, c, d)                      # the adjoint refers to the last forward solve
    dJdf, _, dmu, _ = S.adjoint(cuda(c), cuda(d), 1e-13)
    rng = np.random.default_rng(3)
    for _ in range(4):
        v = rng.standard_normal(f.shape)
        jp, _, _ = J(sk, S, f + v, c, d)
        jm, _, _ = J(sk, S, f - v, c, d)
        fd = (jp - jm) / 2.0
        an = float((host(dJdf) * v).sum())
        assert abs(fd - an) < 1e-9 * max(abs(an), 1e-30), (fd, an)
    S.close()
    h = 1e-4 * MU
    Sp = sk.Stokes(N, V, MU + h, DT)
    Sm = sk.Stokes(N, V, MU - h, DT)
    fd_mu = (J(sk, Sp, f, c, d)[0] - J(sk, Sm, f, c, d)[0]) / (2 * h)
    assert abs(fd_mu - dmu) < 1e-6 * abs(dmu), (fd_mu, dmu)
    Sp.close()
    Sm.close()


def test_autograd_function():
    sk, V, f, c, d = setup_case(51)
    torch = pytest.importorskip("torch")
    S = sk.Stokes(N, V, MU, DT)
    ft = torch.tensor(f, device="cuda", requires_grad=True)
    mu_t = torch.tensor(MU, dtype=torch.float64, device="cuda", requires_grad=True)
    u, p = sk.StokesSolve.apply(S, ft, mu_t, 1e-13)
    loss = (u * cuda(c)).sum() + (p * cuda(d)).sum()
    loss.backward()
    dJdf, _, dmu, _ = S.adjoint(cuda(c), cuda(d), 1e-13)
    assert rel_err(host(ft.grad), host(dJdf)) < 1e-10
    assert abs(float(mu_t.grad) - dmu) < 1e-10 * abs(dmu)
    S.close()


def interior_index(n):
    """All-node indices of the (2n-1)^3 interior P2 nodes, x fastest."""
    N = 2 * n + 1
    q = np.arange(1, 2 * n)
    K, Jj, I = np.meshgrid(q, q, q, indexing="ij")
    return (I + N * (Jj + N * K)).ravel()


def test_adjoint_64_tracking_functional_finite_differences():
    torch = pytest.importorskip("torch")
    """64^3 jittered mesh (seed 5), J = 1/2 ||u - u_t||^2_M with a seeded smooth target
    u_t that vanishes on the boundary (so dJ/dU = M_V (u - u_t) on interior
    rows). Gradients dJ/df and dJ/dmu through StokesSolve (autograd, mixed
    precision: FP32 inner, FP64 outer) against central differences with step
    1e-6 on 16 seeded smooth directions. J is quadratic in f, so the central
    difference has no truncation error; what remains is the solver tolerance
    (1e-11) divided by the step. Each directional derivative must match to
    1e-7 of itself and 1e-8 of |dJ/df||v| (measured worst: 9.4e-10 and
    8.8e-11), dJ/dmu to 1e-5 (measured 4.9e-8, where the step in mu adds a
    truncation term)."""
    sk = gpu_module()
    n, mu, dt, tol = 64, 1e-2, 1e-3, 1e-11
    V = wl.kuhn_vertices(n, 0.2, 5)
    X = wl.p2_node_coords(V, n)
    f = wl.manufactured_force(n, V, mu, dt, 5)
    ut = wl.Manufactured(65).velocity(X)
    inner = interior_index(n)
    boundary = np.setdiff1d(np.arange(X.shape[0]), inner)
    assert np.abs(ut[boundary]).max() < 1e-12
    opt = sk.stokes_default_options(precision=1, vcycles=1)
    S = sk.Stokes(n, V, mu, dt, 0.0, opt)
    ni = inner.size
    inner_t = torch.as_tensor(inner, device="cuda")
    ut_t = cuda(ut)

    def mass_times(Sx, e):                  # (M_V e) on interior rows, node-interleaved
        return Sx.apply("LOAD", e.reshape(-1), 3 * ni).reshape(3, ni).T

    def J_of(Sx, fx):
        u, _, info = Sx.solve(cuda(fx), None, tol)
        assert info.status == 0
        e = u - ut_t
        return 0.5 * float((e[inner_t] * mass_times(Sx, e)).sum())

    # gradient through the autograd wrapper: the loss u . w with w = M_V (u - u_t)
    # fixed has the same derivative in f and mu as J at this point
    ft = torch.tensor(f, device="cuda", requires_grad=True)
    mu_t = torch.tensor(mu, dtype=torch.float64, device="cuda", requires_grad=True)
    u, p = sk.StokesSolve.apply(S, ft, mu_t, tol)
    w = torch.zeros_like(u)
    w[inner_t] = mass_times(S, (u - ut_t).detach())
    (u * w).sum().backward()
    g = host(ft.grad)
    dmu = float(mu_t.grad)
    gnorm = np.linalg.norm(g)
    h = 1e-6
    fscale = np.linalg.norm(f)
    for k in range(16):
        v = wl.Manufactured(1000 + k).body_force(X, mu, dt)
        v *= fscale / np.linalg.norm(v)
        fd = (J_of(S, f + h * v) - J_of(S, f - h * v)) / (2 * h)
        an = float((g * v).sum())
        assert abs(fd - an) <= 1e-7 * abs(an), (k, fd, an)
        assert abs(fd - an) <= 1e-8 * gnorm * np.linalg.norm(v), (k, fd, an)
    S.close()
    hm = 1e-6 * mu
    Sp = sk.Stokes(n, V, mu + hm, dt, 0.0, opt)
    Jp = J_of(Sp, f)
    Sp.close()
    Sm = sk.Stokes(n, V, mu - hm, dt, 0.0, opt)
    Jm = J_of(Sm, f)
    Sm.close()
    fd_mu = (Jp - Jm) / (2 * hm)
    assert abs(fd_mu - dmu) <= 1e-5 * abs(dmu), (fd_mu, dmu)
