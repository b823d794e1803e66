"""Edge cases of the GPU path: smallest and odd meshes, degenerate right-hand
sides, a one-level hierarchy, and the largest configuration."""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workload as wl
from oracle.assemble import StokesSystem
from oracle.mesh import KuhnMesh
from oracle.solve import oracle_solve

from gpu_helpers import aos, cuda, gpu_module, host, rel_err, soa

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [2, 3, 5, 7])
def test_small_and_odd_meshes_match_oracle(n):
    """n = 2 is the smallest mesh (27 interior P2 nodes); odd n cannot be halved,
    so the hierarchy has a single level solved by the dense coarse inverse."""
    sk = gpu_module()
    V = wl.kuhn_vertices(n, 0.2, 60 + n)
    f = wl.random_force(n, 70 + n)
    g = wl.random_pressure_load(n, 80 + n)
    orc = StokesSystem(KuhnMesh(n, V), 0.05, 0.02)
    Uo, Po = oracle_solve(orc, orc.load(f), g)
    S = sk.Stokes(n, V, 0.05, 0.02)
    u, p, info = S.solve(cuda(f), cuda(g), 1e-12)
    assert rel_err(orc.restrict_velocity(host(u)), Uo) < 1e-9
    assert rel_err(host(p), Po) < 1e-9
    S.close()


@pytest.mark.parametrize("n", [9, 11])
def test_non_nested_hierarchies_match_oracle(n):
    """Odd n coarsens to ceil(n/2) with logical-coordinate transfers (non-nested
    spaces, interpolated coarse geometry); the solution is unaffected."""
    sk = gpu_module()
    V = wl.kuhn_vertices(n, 0.2, 90 + n)
    f = wl.random_force(n, 91 + n)
    orc = StokesSystem(KuhnMesh(n, V), 0.02, 0.01)
    Uo, Po = oracle_solve(orc, orc.load(f))
    S = sk.Stokes(n, V, 0.02, 0.01, options=sk.stokes_default_options(vcycles=1))
    assert S.sizes["levels"] >= 3
    u, p, info = S.solve(cuda(f), None, 1e-12)
    assert rel_err(orc.restrict_velocity(host(u)), Uo) < 1e-9
    assert rel_err(host(p), Po) < 1e-9
    S.close()


def test_non_nested_vcycle_contracts():
    from test_gpu_multigrid import vcycle_stats
    sk = gpu_module()
    for n in (13, 15):
        sym, rate = vcycle_stats(sk, n, 1e-2, 1e-3, "A3")
        assert sym < 1e-10 and rate < 0.6, (n, rate)
        sym, rate = vcycle_stats(sk, n, 1e-2, 1e-3, "KQ")
        assert sym < 1e-10 and rate < 0.6, (n, rate)


def test_zero_rhs_and_loose_tolerance():
    sk = gpu_module()
    n = 4
    V = wl.kuhn_vertices(n, 0.2, 3)
    S = sk.Stokes(n, V, 0.1, 0.01)
    z = np.zeros(((2 * n + 1) ** 3, 3))
    u, p, info = S.solve(cuda(z), None, 1e-10)
    assert info.status == 0 and info.outer_iters == 0
    assert np.abs(host(u)).max() == 0 and np.abs(host(p)).max() == 0
    f = wl.random_force(n, 4)
    u, p, info = S.solve(cuda(f), None, 1.0)                   # tol >= 1: nothing to do
    assert info.status == 0 and info.outer_iters == 0 and np.abs(host(u)).max() == 0
    S.close()


def test_one_level_vcycle_is_exact_inverse():
    """With a single level the V-cycle is the dense coarse inverse of A~_3."""
    sk = gpu_module()
    n = 2
    V = wl.kuhn_vertices(n, 0.2, 8)
    S = sk.Stokes(n, V, 0.3, 0.02, options=sk.stokes_default_options(vcycles=1))
    orc = StokesSystem(KuhnMesh(n, V), 0.3, 0.02)
    r = np.random.default_rng(1).standard_normal(3 * orc.n_inner)
    z = aos(host(S.apply("VCYCLE_A3", cuda(soa(r)), r.size)))
    ref = spla.spsolve(orc.A3s.tocsc(), r.reshape(-1, 3))
    assert rel_err(z, ref.ravel()) < 1e-12
    S.close()


@pytest.fixture(scope="module")
def coupled96():
    n, mu, dt = 96, 1e-3, 1e-3
    V = wl.kuhn_vertices(n, 0.2, 3)
    return n, mu, dt, V, KuhnMesh(n, V), wl.manufactured_force(n, V, mu, dt, 3)


@pytest.mark.parametrize("gamma", [0.0, 1.0, 10.0])
def test_largest_configuration_coupled_96(coupled96, gamma):
    """96^3 jittered mesh (22.5 M DOFs), block-triangular FGMRES(30) on the
    coupled system with augmented Lagrangian gamma, mixed precision. Every
    row of the residual of the original saddle system (the augmented form has
    the same solution) is evaluated by the oracle's element loop and must meet
    the tolerance, in agreement with the GPU's own FP64 residual."""
    from oracle.local import relative_residuals
    sk = gpu_module()
    n, mu, dt, V, mesh, f = coupled96
    S = sk.Stokes(n, V, mu, dt, gamma, sk.stokes_default_options(precision=1, vcycles=1, method=1, block_lu=0))
    assert S.sizes["dofs"] == 21567171 + 912673
    u, p, info = S.solve(cuda(f), None, 1e-8)
    assert info.status == 0 and info.rel_residual <= 1e-8, info.as_dict()
    uh, ph = host(u), host(p)
    S.close()
    rel = relative_residuals(mesh, mu, dt, f, [(uh, ph, None)])[0]
    print(f"96^3 gamma={gamma:g}: oracle residual {rel:.3e}, GPU residual {info.rel_residual:.3e}")
    assert rel <= 1e-8 * (1 + 1e-6) and abs(rel - info.rel_residual) <= 1e-11, (rel, info.rel_residual)


def test_largest_configuration_manufactured_errors_96(coupled96):
    """Discretisation error of the GPU's 96^3 solution against the manufactured
    (u, p), next to the 48^3 solution of the same problem: velocity L2 error
    O(h^3) and pressure O(h^2) (Sec. 3.3) between the two meshes, evaluated by
    the oracle's chunked quadrature."""
    from oracle.local import l2_errors_chunked
    sk = gpu_module()
    n, mu, dt, V, mesh, f = coupled96
    errs = []
    for m, Vm, msh, fm in ((48, None, None, None), (n, V, mesh, f)):
        if Vm is None:
            Vm = wl.kuhn_vertices(m, 0.2, 3)
            msh = KuhnMesh(m, Vm)
            fm = wl.manufactured_force(m, Vm, mu, dt, 3)
        S = sk.Stokes(m, Vm, mu, dt, 0.0, sk.stokes_default_options(precision=1, vcycles=1, method=1, block_lu=0))
        u, p, info = S.solve(cuda(fm), None, 1e-10)
        assert info.status == 0
        uh, ph = host(u), host(p)
        S.close()
        errs.append(l2_errors_chunked(msh, uh, ph, wl.Manufactured(3), q=3))
    ru = np.log2(errs[0][0] / errs[1][0])
    rp = np.log2(errs[0][1] / errs[1][1])
    print(f"manufactured L2 errors 48^3 {errs[0]}, 96^3 {errs[1]}: rates velocity {ru:.2f}, pressure {rp:.2f}")
    assert ru > 2.65 and rp > 1.65, (errs, ru, rp)


def test_indefinite_smoother_reports_breakdown():
    """A Chebyshev smoothing interval far below the spectrum of D^{-1} A~_3
    ([0.01, 0.05] x lambda_max instead of [0.1, 1.1]) over-relaxes the high
    modes, so the V-cycle preconditioner is indefinite: the inner PCG meets
    r^T z <= 0, the device flags it, and the failed solve is reported as a
    Krylov breakdown rather than as a plain failure to converge."""
    sk = gpu_module()
    n = 8
    V = wl.kuhn_vertices(n, 0.2, 4)
    f = wl.random_force(n, 5)
    S = sk.Stokes(n, V, 0.1, 1e-2, options=sk.stokes_default_options(cheb_low=0.01, cheb_high=0.05,
                                                                      max_refine=2, max_inner=50, max_outer=20))
    with pytest.raises(sk.StokesError) as err:
        S.solve(cuda(f), None, 1e-10)
    assert err.value.status == -5, str(err.value)       # STOKES_ERR_BREAKDOWN
    S.close()
    # the default interval on the same problem converges
    S = sk.Stokes(n, V, 0.1, 1e-2)
    _, _, info = S.solve(cuda(f), None, 1e-10)
    assert info.status == 0
    S.close()


def test_bounded_device_wait_expires_and_context_stays_usable():
    """The cooperative coarse-level kernel separates its steps with grid-wide
    barriers whose waits are bounded. A barrier that nothing completes must
    give up (about a second), report STOKES_ERR_TIMEOUT, and leave the context
    usable: a solve with the cooperative kernel afterwards succeeds."""
    sk = gpu_module()
    n = 8
    V = wl.kuhn_vertices(n, 0.2, 4)
    S = sk.Stokes(n, V, 0.1, 1e-2, options=sk.stokes_default_options(coarse_kernel=1))
    st = sk._L.stokes_check_bounded_wait(S.ctx)
    assert st == -7, st                                   # STOKES_ERR_TIMEOUT
    f = wl.random_force(n, 5)
    _, _, info = S.solve(cuda(f), None, 1e-10)
    assert info.status == 0 and info.rel_residual <= 1e-10
    S.close()
