"""Several right-hand sides in one call (stokes_solve_multi): four systems in
lockstep (Method 2 FGMRES or Method 1 Schur CG), sharing every V-cycle,
mass-inverse, product and vector-kernel sweep. Each system is checked on its
own against the oracle's exact discrete solution and the oracle's residual of
the GPU answer."""

import numpy as np
import pytest

import workload as wl
from oracle.assemble import StokesSystem
from oracle.mesh import KuhnMesh
from oracle.solve import oracle_solve, relative_residual

from gpu_helpers import cuda, gpu_module, host, rel_err

pytestmark = pytest.mark.gpu


def multi_case(n, mu, dt, k, tol, seed=11, gamma=0.0, pressure_load=False, zero=(), scale=None, method=1, **opt):
    sk = gpu_module()
    V = wl.kuhn_vertices(n, 0.2, seed)
    orc = StokesSystem(KuhnMesh(n, V), mu, dt)
    fs = [wl.random_force(n, 100 * seed + j) for j in range(k)]
    for j in zero:
        fs[j] = np.zeros_like(fs[j])
    if scale:
        for j, a in scale.items():
            fs[j] = a * fs[j]
    gs = [wl.random_pressure_load(n, 200 * seed + j) for j in range(k)] if pressure_load else None
    S = sk.Stokes(n, V, mu, dt, gamma, sk.stokes_default_options(method=method, **opt))
    F = cuda(np.stack(fs))
    G = cuda(np.stack(gs)) if gs is not None else None
    U, P, infos = S.solve_multi(F, G, tol)
    U, P = host(U), host(P)
    # the same systems one at a time through stokes_solve
    single = []
    for j in range(k):
        u, p, inf = S.solve(cuda(fs[j]), cuda(gs[j]) if gs is not None else None, tol)
        single.append((host(u), host(p), inf.as_dict()))
    S.close()
    out = []
    for j in range(k):
        Fo = orc.load(fs[j])
        g = gs[j] if gs is not None else None
        Uo, Po = oracle_solve(orc, Fo, g)
        Ug = orc.restrict_velocity(U[j])
        info = infos[j].as_dict()
        out.append(dict(info=info, res=relative_residual(orc, Ug, P[j], Fo, g),
                        eu=rel_err(Ug, Uo), ep=rel_err(P[j], Po), mean=float(orc.MQ1 @ P[j]),
                        du=rel_err(U[j], single[j][0]), dp=rel_err(P[j], single[j][1]),
                        zero=not np.any(fs[j]) and (g is None or not np.any(g)), U=U[j], P=P[j]))
    return out


def test_four_systems_fp64_match_oracle():
    """Four N(0,1) forces with pressure loads, FP64, to 1e-12: each system
    within the 1e-9 parity bar of the oracle's exact solution."""
    res = multi_case(6, 1e-2, 1e-3, 4, 1e-12, pressure_load=True)
    for r in res:
        assert r["info"]["status"] == 0 and r["info"]["rel_residual"] <= 1e-12, r["info"]
        assert r["res"] <= 2e-12, r["res"]
        assert r["eu"] <= 1e-9 and r["ep"] <= 1e-9, (r["eu"], r["ep"])
        assert abs(r["mean"]) < 1e-12


def test_mixed_precision_lockstep_matches_single_solves():
    """Mixed precision to 1e-8: the lockstep systems meet the tolerance on the
    oracle's residual and agree with the one-system path to the accuracy both
    were asked for."""
    res = multi_case(8, 1e-3, 1e-3, 4, 1e-8, seed=12, precision=1, vcycles=1)
    for r in res:
        assert r["info"]["status"] == 0 and r["info"]["rel_residual"] <= 1e-8, r["info"]
        assert r["res"] <= 1e-8 * (1 + 1e-6), r["res"]
        assert r["eu"] < 1e-5 and r["ep"] < 1e-4, (r["eu"], r["ep"])
        assert r["du"] < 1e-5 and r["dp"] < 1e-4, (r["du"], r["dp"])


@pytest.mark.parametrize("k", [2, 3, 5])
def test_ragged_counts_padding_and_single_tail(k):
    """k = 2, 3 (one group padded with zero systems) and 5 (a group of four and
    one system through the one-system path)."""
    res = multi_case(5, 0.3, 1e-2, k, 1e-11, seed=13)
    assert len(res) == k
    for r in res:
        assert r["info"]["status"] == 0 and r["info"]["rel_residual"] <= 1e-11
        assert r["eu"] <= 1e-8 and r["ep"] <= 1e-8, (r["eu"], r["ep"])


def test_zero_and_scaled_systems_in_one_group():
    """A zero force gives the zero solution at once (no iterations) while the
    others iterate; a force scaled by 1e6 converges like its unscaled twin
    (each system's test is relative to its own right-hand side)."""
    res = multi_case(6, 1e-2, 1e-2, 4, 1e-10, seed=14, zero=(1,), scale={3: 1e6})
    assert res[1]["zero"]
    assert np.all(res[1]["U"] == 0) and np.all(res[1]["P"] == 0)
    assert res[1]["info"]["outer_iters"] == 0 and res[1]["info"]["status"] == 0
    for j in (0, 2, 3):
        r = res[j]
        assert r["info"]["status"] == 0 and r["info"]["rel_residual"] <= 1e-10
        assert r["eu"] <= 1e-7 and r["ep"] <= 1e-7, (j, r["eu"], r["ep"])


def test_augmented_lagrangian_and_block_triangular():
    """gamma = 10 with the block-triangular preconditioner (no left factor)."""
    res = multi_case(6, 1e-2, 1e-3, 4, 1e-11, seed=15, gamma=10.0, block_lu=0)
    for r in res:
        assert r["info"]["status"] == 0 and r["info"]["rel_residual"] <= 1e-11
        assert r["eu"] <= 1e-8 and r["ep"] <= 1e-8, (r["eu"], r["ep"])


def test_inner_cg_velocity_solves():
    """m2_inner_cg: the lockstep inner PCG (per-system convergence masks)."""
    res = multi_case(6, 1e-2, 1e-3, 4, 1e-11, seed=16, m2_inner_cg=1, inner_tol=1e-3)
    for r in res:
        assert r["info"]["status"] == 0 and r["info"]["rel_residual"] <= 1e-11
        assert r["eu"] <= 1e-8 and r["ep"] <= 1e-8, (r["eu"], r["ep"])


@pytest.mark.parametrize("gamma", [0.0, 1.0])
def test_schur_cg_lockstep_fp64_matches_oracle(gamma):
    """Method 1 (flexible Schur CG, lockstep inner PCG with per-system
    stopping) in FP64 to 1e-12 with pressure loads: each system within the
    1e-9 parity bar."""
    res = multi_case(6, 1e-2, 1e-3, 4, 1e-12, seed=17, gamma=gamma, pressure_load=True, method=0)
    for r in res:
        assert r["info"]["status"] == 0 and r["info"]["rel_residual"] <= 1e-12, r["info"]
        assert r["eu"] <= 1e-9 and r["ep"] <= 1e-9, (r["eu"], r["ep"])
        assert abs(r["mean"]) < 1e-12


def test_schur_cg_lockstep_mixed_with_zero_system():
    """Method 1, mixed precision to 1e-8, one zero force among four."""
    res = multi_case(8, 1e-3, 1e-3, 4, 1e-8, seed=18, zero=(2,), method=0, precision=1, vcycles=1)
    assert np.all(res[2]["U"] == 0) and np.all(res[2]["P"] == 0)
    for j in (0, 1, 3):
        r = res[j]
        assert r["info"]["status"] == 0 and r["info"]["rel_residual"] <= 1e-8, r["info"]
        assert r["res"] <= 1e-8 * (1 + 1e-6), r["res"]
        assert r["eu"] < 1e-5 and r["ep"] < 1e-4, (r["eu"], r["ep"])


@pytest.mark.parametrize("opt", [dict(format=1), dict(format=2), dict(vel_prec=1), dict(schur_prec=1),
                                 dict(schur_prec=2), dict(method=0, format=3)])
def test_lockstep_option_variants(opt):
    """The lockstep path under the storage formats (CSR/BSR3 only, stencils
    everywhere, BSR3 products), the block velocity V-cycle (one right-hand
    side per cycle), C^Delta and C_lambda with the velocity mass."""
    res = multi_case(5, 1e-2, 1e-3, 4, 1e-11, seed=19, **opt)
    for r in res:
        assert r["info"]["status"] == 0 and r["info"]["rel_residual"] <= 1e-11, r["info"]
        assert r["eu"] <= 1e-8 and r["ep"] <= 1e-8, (r["eu"], r["ep"])
