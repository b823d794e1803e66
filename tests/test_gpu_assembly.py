"""GPU parity: element-coloured assembly and sparse operators vs the oracle.

Matrices are exported through the C ABI and compared entrywise with the
oracle's independent COO assembly (FP64, relative to the largest entry);
products are compared on seeded random vectors.
"""

import numpy as np
import pytest

import workload as wl
from oracle.assemble import StokesSystem
from oracle.mesh import KuhnMesh

from gpu_helpers import aos, coarse_vertices, cuda, gpu_module, host, rel_err, soa, to_scipy

pytestmark = pytest.mark.gpu

CASES = [(2, 0.0, 1), (4, 0.2, 3), (6, 0.2, 5)]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"n{c[0]}j{c[1]}")
def pair(request):
    sk = gpu_module()
    n, jit, seed = request.param
    V = wl.kuhn_vertices(n, jit, seed)
    mu, dt = 0.37, 0.011
    S = sk.Stokes(n, V, mu, dt, 0.0, sk.stokes_default_options(eps_pressure=1.0))
    orc = StokesSystem(KuhnMesh(n, V), mu, dt)
    yield sk, S, orc, V, n, mu, dt
    S.close()


def assert_same(Mg, Mo, tol=1e-12):
    Mg = Mg.tocsr()
    Mo = Mo.tocsr()
    scale = abs(Mo).max()
    diff = abs(Mg - Mo).max()
    assert diff <= tol * scale, (diff, scale)


def test_matrices_match_oracle(pair):
    sk, S, orc, V, n, mu, dt = pair
    rp, ci, v, shp = S.matrix("A")
    assert v.shape[1:] == (3, 3)
    assert_same(to_scipy(rp, ci, v, shp), orc.A)
    rp, ci, v, shp = S.matrix("A3")
    assert_same(to_scipy(rp, ci, v, shp), orc.A3s)
    rp, ci, v, shp = S.matrix("B")
    assert_same(to_scipy(rp, ci, v, shp), orc.B)
    rp, ci, v, shp = S.matrix("BT")
    assert_same(to_scipy(rp, ci, v, shp), orc.B.T)
    rp, ci, v, shp = S.matrix("MQ")
    assert_same(to_scipy(rp, ci, v, shp), orc.MQ)
    rp, ci, v, shp = S.matrix("LQ")
    assert_same(to_scipy(rp, ci, v, shp), orc.LQ)
    rp, ci, v, shp = S.matrix("KQ")
    assert_same(to_scipy(rp, ci, v, shp), orc.MQ + orc.LQ)
    _, _, lum, _ = S.matrix("LUMPED")
    assert np.allclose(lum, orc.lumped, rtol=1e-13, atol=0)


def test_pattern_is_structural(pair):
    """Column indices sorted, no duplicates, diagonal present, symmetric pattern."""
    sk, S, orc, V, n, mu, dt = pair
    for which in ("A3", "KQ"):
        rp, ci, v, shp = S.matrix(which)
        for r in range(shp[0]):
            row = ci[rp[r]:rp[r + 1]]
            assert np.all(np.diff(row) > 0)
            assert r in row
        M = to_scipy(rp, ci, v, shp)
        assert (abs(M - M.T) > 1e-14 * abs(M).max()).nnz == 0


def test_coarse_levels_match_oracle(pair):
    sk, S, orc, V, n, mu, dt = pair
    levels = S.sizes["levels"]
    Vl, nl = V, n
    for lvl in range(1, levels):
        Vl, nl = coarse_vertices(Vl, nl), nl // 2
        o = StokesSystem(KuhnMesh(nl, Vl), mu, dt)
        rp, ci, v, shp = S.matrix("A3", lvl)
        assert_same(to_scipy(rp, ci, v, shp), o.A3s)
        rp, ci, v, shp = S.matrix("KQ", lvl)
        assert_same(to_scipy(rp, ci, v, shp), o.MQ + o.LQ)


def test_operator_products(pair):
    sk, S, orc, V, n, mu, dt = pair
    rng = np.random.default_rng(7)
    nv, np_ = orc.A.shape[0], orc.B.shape[0]
    x = rng.standard_normal(nv)
    p = rng.standard_normal(np_)
    xs = cuda(soa(x))
    assert rel_err(aos(host(S.apply("A", xs, nv))), orc.A @ x) < 1e-13
    assert rel_err(aos(host(S.apply("A3", xs, nv))), (orc.A3s @ x.reshape(-1, 3)).ravel()) < 1e-13
    assert rel_err(host(S.apply("B", xs, np_)), orc.B @ x) < 1e-13
    assert rel_err(aos(host(S.apply("BT", cuda(p), nv))), orc.B.T @ p) < 1e-13
    assert rel_err(host(S.apply("MQ", cuda(p), np_)), orc.MQ @ p) < 1e-13
    assert rel_err(host(S.apply("LQ", cuda(p), np_)), orc.LQ @ p) < 1e-13
    assert rel_err(host(S.apply("KQ", cuda(p), np_)), (orc.MQ + orc.LQ) @ p) < 1e-13
    assert rel_err(aos(host(S.apply("LUMPED_INV", xs, nv))), x / orc.Lam) < 1e-14
    # load vector F = M_V f on interior rows from nodal f on all nodes
    f = rng.standard_normal((orc.mesh.n_p2, 3))
    assert rel_err(aos(host(S.apply("LOAD", cuda(f), nv))), orc.load(f)) < 1e-13


@pytest.mark.parametrize("fmt", [1, 2])
def test_operator_products_every_storage(fmt):
    """The same products with CSR everywhere (1) and stencil storage on every
    level (2): the stencil kernel's boundary and interior paths on small meshes."""
    sk = gpu_module()
    for n in (3, 4, 6, 9):
        V = wl.kuhn_vertices(n, 0.2, 40 + n)
        S = sk.Stokes(n, V, 0.2, 0.03, options=sk.stokes_default_options(format=fmt))
        orc = StokesSystem(KuhnMesh(n, V), 0.2, 0.03)
        rng = np.random.default_rng(n)
        x = rng.standard_normal(orc.A.shape[0])
        p = rng.standard_normal(orc.B.shape[0])
        nv, np_ = x.size, p.size
        assert rel_err(aos(host(S.apply("A3", cuda(soa(x)), nv))), (orc.A3s @ x.reshape(-1, 3)).ravel()) < 1e-13
        assert rel_err(host(S.apply("KQ", cuda(p), np_)), (orc.MQ + orc.LQ) @ p) < 1e-13
        assert rel_err(host(S.apply("MQ", cuda(p), np_)), orc.MQ @ p) < 1e-13
        assert rel_err(host(S.apply("LQ", cuda(p), np_)), orc.LQ @ p) < 1e-13
        S.close()


def test_augmented_operator_matches_definition():
    """A_gamma x = A x + gamma mu B^T M_Q^{-1} B x (Eq. def_of_Alambda); M_Q^{-1} by
    Chebyshev (24 steps on [1/2, 5/2], error below 0.382^24 ~ 1e-10)."""
    sk = gpu_module()
    n, gamma = 4, 3.0
    V = wl.kuhn_vertices(n, 0.2, 9)
    S = sk.Stokes(n, V, 0.5, 0.02, gamma)
    orc = StokesSystem(KuhnMesh(n, V), 0.5, 0.02)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(orc.A.shape[0])
    import scipy.sparse.linalg as spla
    ref = orc.A @ x + gamma * 0.5 * (orc.B.T @ spla.spsolve(orc.MQ.tocsc(), orc.B @ x))
    assert rel_err(aos(host(S.apply("AGAMMA", cuda(soa(x)), x.size))), ref) < 1e-8
    S.close()


def test_double_float_residual_product():
    """The mixed-precision refinement residual forms A U from FP32 hi/lo pairs
    with exact FP32 products and double-float sums. Each row must match the
    FP64 product within 1e-12 of sum_j |A_ij||x_j| (the error analysis gives
    ~k^2 2^-48 for k products per lane; a plain FP32 product misses by ~1e-7,
    so the bound discriminates)."""
    sk = gpu_module()
    n, mu, dt = 6, 0.05, 2e-3
    V = wl.kuhn_vertices(n, 0.2, 17)
    orc = StokesSystem(KuhnMesh(n, V), mu, dt)
    S = sk.Stokes(n, V, mu, dt, 0.0, sk.stokes_default_options(precision=1))
    x = np.random.default_rng(5).standard_normal(orc.A.shape[0])
    y = aos(host(S.apply("A_DF", cuda(soa(x)), x.size)))
    ref = orc.A @ x
    scale = abs(orc.A) @ abs(x)
    err = float(np.max(np.abs(y - ref) / scale))
    print("double-float product: max error / (|A||x|) =", err)
    assert err <= 1e-12
    S.close()
