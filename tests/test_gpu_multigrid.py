"""GPU checks of the multigrid components.

Transfers: on nested Kuhn meshes the coarse P2 (P1) space is contained in the
fine one, so prolongation must reproduce any global quadratic (linear) field
exactly at the fine nodes' logical positions, and restriction is its exact
transpose. V-cycles: symmetric (so usable in CG) and contracting at a rate
independent of h.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workload as wl
from oracle.assemble import StokesSystem
from oracle.mesh import KuhnMesh

from gpu_helpers import aos, coarse_vertices, cuda, gpu_module, host, rel_err, soa, to_scipy

pytestmark = pytest.mark.gpu


def logical_grid(n, interior_p2):
    if interior_p2:
        q = np.arange(1, 2 * n) / (2.0 * n)
    else:
        q = np.arange(n + 1) / float(n)
    K, J, I = np.meshgrid(q, q, q, indexing="ij")
    return np.stack([I.ravel(), J.ravel(), K.ravel()], 1)


def quad_field(X, C):
    x, y, z = X.T
    mons = np.stack([np.ones_like(x), x, y, z, x * x, y * y, z * z, x * y, y * z, x * z])
    return (C @ mons).T


@pytest.mark.parametrize("n", [8, 12])
def test_prolongation_exact_on_polynomials(n):
    """Coarse interior values of a quadratic q: the prolonged field equals q at every
    fine node whose coarse cube has only interior nodes (boundary coarse values
    are not unknowns, so elsewhere the interpolant differs from q)."""
    sk = gpu_module()
    S = sk.Stokes(n, wl.kuhn_vertices(n, 0.2, 1), 1.0, 0.01)
    rng = np.random.default_rng(n)
    C = rng.standard_normal((3, 10))
    nc = n // 2
    Xc = logical_grid(nc, True)
    Xf = logical_grid(n, True)
    ucoarse = quad_field(Xc, C)
    y = aos(host(S.apply("PROLONG_P2", cuda(soa(ucoarse)), Xf.shape[0] * 3, level=0))).reshape(-1, 3)
    ufine = quad_field(Xf, C)
    inside = np.all((Xf > 1.0 / nc) & (Xf < 1.0 - 1.0 / nc), axis=1)
    assert inside.sum() > 0
    assert np.abs(y[inside] - ufine[inside]).max() < 1e-12 * np.abs(ufine).max()
    # restriction is the transpose of prolongation
    a = rng.standard_normal(Xc.shape[0] * 3)
    b = rng.standard_normal(Xf.shape[0] * 3)
    Pa = host(S.apply("PROLONG_P2", cuda(a), b.size, level=0))
    Rb = host(S.apply("RESTRICT_P2", cuda(b), a.size, level=0))
    assert abs(Pa @ b - a @ Rb) < 1e-12 * abs(Pa @ b)
    # P1: linear fields are reproduced everywhere (all P1 nodes are unknowns)
    Xc1 = logical_grid(nc, False)
    Xf1 = logical_grid(n, False)
    L = rng.standard_normal(4)
    lin = lambda X: L[0] + X @ L[1:]  # noqa: E731
    y1 = host(S.apply("PROLONG_P1", cuda(lin(Xc1)), Xf1.shape[0], level=0))
    assert np.abs(y1 - lin(Xf1)).max() < 1e-12 * np.abs(lin(Xf1)).max()
    S.close()


def vcycle_stats(sk, n, mu, dt, which, seed=0):
    V = wl.kuhn_vertices(n, 0.2, 2)
    S = sk.Stokes(n, V, mu, dt, 0.0, sk.stokes_default_options(vcycles=1))
    orc = StokesSystem(KuhnMesh(n, V), mu, dt)
    rng = np.random.default_rng(seed)
    if which == "A3":
        A = orc.A3s
        apply = lambda r: host(S.apply("VCYCLE_A3", cuda(r), r.size))  # noqa: E731
        mat = lambda x: soa((A @ aos(x).reshape(-1, 3)).ravel())  # noqa: E731
        m = 3 * A.shape[0]
    else:
        A = (orc.MQ + orc.LQ).tocsr()
        apply = lambda r: host(S.apply("VCYCLE_KQ", cuda(r), r.size))  # noqa: E731
        mat = lambda x: A @ x  # noqa: E731
        m = A.shape[0]
    x = rng.standard_normal(m)
    y = rng.standard_normal(m)
    sym = abs(apply(x) @ y - x @ apply(y)) / abs(x @ apply(y))
    # error propagation e <- (I - V A) e: contraction over 8 cycles
    e = rng.standard_normal(m)
    n0 = np.sqrt(e @ mat(e))
    for _ in range(8):
        e = e - apply(mat(e))
    rate = (np.sqrt(e @ mat(e)) / n0) ** (1 / 8)
    S.close()
    return sym, rate


@pytest.mark.parametrize("mu,dt", [(1.0, 1e-3), (1e-2, 1e-3), (1e-4, 1e-3), (1.0, 1.0)])
def test_vcycle_symmetric_and_contracting(mu, dt):
    sk = gpu_module()
    rates = []
    for n in (8, 16):
        sym, rate = vcycle_stats(sk, n, mu, dt, "A3")
        assert sym < 1e-10
        assert rate < 0.5, (n, rate)
        rates.append(rate)
    assert rates[1] < rates[0] + 0.15        # no growth with refinement
    for n in (8, 16):
        sym, rate = vcycle_stats(sk, n, mu, dt, "KQ")
        assert sym < 1e-10 and rate < 0.5


@pytest.mark.parametrize("op", ["VCYCLE_A3", "VCYCLE_KQ"])
def test_graph_replay_matches_plain_launches(op):
    """The coarse levels run eagerly on the first V-cycle, are captured as a
    CUDA graph on the second and replayed afterwards; every call must give the
    same bits as plain launches (the reductions are deterministic)."""
    sk = gpu_module()
    n = 12
    V = wl.kuhn_vertices(n, 0.2, 5)
    outs = {}
    for graphs in (0, 1):
        S = sk.Stokes(n, V, 0.05, 1e-3, options=sk.stokes_default_options(graphs=graphs))
        size = 3 * S.sizes["n_inner"] if op == "VCYCLE_A3" else S.n_p1
        r = np.random.default_rng(2).standard_normal(size)
        # fixed buffers: the first call runs plainly, the second records the
        # whole-cycle graph, the third and fourth replay it
        x = cuda(r)
        y = torch.zeros(size, dtype=torch.float64, device="cuda")
        outs[graphs] = []
        for k in range(4):
            x.copy_(cuda(r * (k + 1)))
            sk.stokes_apply(S.ctx, sk.OP[op], x, y, 0)
            outs[graphs].append(host(y))
        S.close()
    for k in range(4):
        assert np.array_equal(outs[0][k], outs[1][k]), k


def test_solve_with_graphs_is_bitwise_identical():
    sk = gpu_module()
    n = 12
    V = wl.kuhn_vertices(n, 0.2, 6)
    f = wl.random_force(n, 7)
    res = []
    for graphs in (0, 1):
        for precision in (0, 1):
            S = sk.Stokes(n, V, 1e-2, 1e-3, options=sk.stokes_default_options(
                graphs=graphs, precision=precision, schur_inner_iters=2))
            u, p, info = S.solve(cuda(f), None, 1e-9)
            res.append((host(u), host(p), info.outer_iters))
            S.close()
    for a, b in ((0, 2), (1, 3)):
        assert np.array_equal(res[a][0], res[b][0]) and np.array_equal(res[a][1], res[b][1])
        assert res[a][2] == res[b][2]


@pytest.mark.parametrize("vel_prec,gamma", [(2, 0.0), (1, 1.0)])
def test_block_velocity_preconditioner(vel_prec, gamma):
    """A~_2 = A and A~_1 = A + gamma mu D (Sec. 5.1): the 3x3-block operator is
    re-assembled on every level (checked against the oracle on levels 0 and 1),
    and its block V-cycle is symmetric and contracting at h-independent rate."""
    sk = gpu_module()
    mu, dt = 0.05, 1e-3
    rates = []
    for n in (8, 16):
        V = wl.kuhn_vertices(n, 0.2, 2)
        S = sk.Stokes(n, V, mu, dt, gamma, sk.stokes_default_options(vcycles=1, vel_prec=vel_prec))
        orc = StokesSystem(KuhnMesh(n, V), mu, dt)
        ref = (orc.A + gamma * mu * orc.D).tocsr()
        rp, ci, v, shp = S.matrix("AV", 0)
        assert_same_bsr(to_scipy(rp, ci, v, shp), ref)
        if n == 8:
            Vc = coarse_vertices(V, n)
            oc = StokesSystem(KuhnMesh(n // 2, Vc), mu, dt)
            rp, ci, v, shp = S.matrix("AV", 1)
            assert_same_bsr(to_scipy(rp, ci, v, shp), (oc.A + gamma * mu * oc.D).tocsr())
        P = soa_perm(ref.shape[0])
        Ac = ref[P][:, P]                               # component-major ordering
        apply = lambda r: host(S.apply("VCYCLE_VEL", cuda(r), r.size))  # noqa: E731
        rng = np.random.default_rng(n)
        x, y = rng.standard_normal(Ac.shape[0]), rng.standard_normal(Ac.shape[0])
        sym = abs(apply(x) @ y - x @ apply(y)) / abs(x @ apply(y))
        assert sym < 1e-10, sym
        e = rng.standard_normal(Ac.shape[0])
        n0 = np.sqrt(e @ (Ac @ e))
        for _ in range(8):
            e = e - apply(Ac @ e)
        rate = (np.sqrt(e @ (Ac @ e)) / n0) ** (1 / 8)
        assert rate < 0.6, (n, rate)
        rates.append(rate)
        S.close()
    assert rates[1] < rates[0] + 0.15, rates


def soa_perm(m3):
    """Index map: component-major position -> node-interleaved position."""
    m = m3 // 3
    return (3 * np.arange(m)[None, :] + np.arange(3)[:, None]).ravel()


def assert_same_bsr(got, ref):
    d = (got - ref).tocsr()
    scale = abs(ref).max()
    assert (abs(d).max() if d.nnz else 0.0) <= 1e-12 * scale


@pytest.mark.parametrize("op", ["VCYCLE_A3", "VCYCLE_KQ"])
@pytest.mark.parametrize("n", [8, 16, 13])
def test_coarse_level_kernel_matches_separate_launches(op, n):
    """The levels below the finest run as one cooperative kernel (grid-wide
    barriers between the steps) or as one launch per step: the same steps and
    coefficients, so the V-cycles agree to rounding (the row sums are reduced
    in a different order); repeated calls reuse the kernel's fixed buffers."""
    sk = gpu_module()
    V = wl.kuhn_vertices(n, 0.2, 9)
    outs = {}
    for ck in (0, 1):
        S = sk.Stokes(n, V, 0.05, 1e-3, options=sk.stokes_default_options(coarse_kernel=ck, vcycles=1))
        assert S.sizes["levels"] >= 3
        size = 3 * S.sizes["n_inner"] if op == "VCYCLE_A3" else S.n_p1
        rng = np.random.default_rng(4)
        outs[ck] = []
        for k in range(3):
            r = rng.standard_normal(size)
            outs[ck].append(host(S.apply(op, cuda(r), size)))
        S.close()
    for k in range(3):
        assert rel_err(outs[1][k], outs[0][k]) < 1e-12, k
