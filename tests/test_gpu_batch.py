"""Batched solves: uneven instances on concurrent streams, several right-hand
sides each, checked one by one against the oracle's exact solutions."""

import numpy as np
import pytest

import workload as wl
from oracle.assemble import StokesSystem
from oracle.mesh import KuhnMesh
from oracle.solve import oracle_solve

from gpu_helpers import cuda, gpu_module, host, rel_err

pytestmark = pytest.mark.gpu


def test_batch_of_uneven_instances_matches_oracle():
    sk = gpu_module()
    specs = [(5, 0.3, 1e-3), (6, 1e-3, 1e-2), (7, 1e-2, 1e-4), (8, 1.0, 1e-3)]
    inst, forces, Vs = [], [], []
    for i, (n, mu, dt) in enumerate(specs):
        V = wl.kuhn_vertices(n, 0.2, 500 + i)
        Vs.append(V)
        inst.append((n, V, mu, dt, 0.0))
        forces.append([wl.random_force(n, 600 + 10 * i + k) for k in range(3)])
    B = sk.StokesBatch(inst, sk.stokes_default_options(precision=1, vcycles=1))
    dev_forces = [[cuda(f) for f in fl] for fl in forces]
    outs, infos, ms = B.solve_all(dev_forces, tol=1e-10)
    assert ms > 0
    for i, (n, mu, dt) in enumerate(specs):
        orc = StokesSystem(KuhnMesh(n, Vs[i]), mu, dt)
        for k, f in enumerate(forces[i]):
            assert infos[i][k]["status"] == 0 and infos[i][k]["rel_residual"] <= 1e-10
            Uo, Po = oracle_solve(orc, orc.load(f))
            u, p = outs[i][k]
            assert rel_err(orc.restrict_velocity(host(u)), Uo) < 1e-7
            assert rel_err(host(p), Po) < 1e-6
    B.close()


def test_benchmark_batch_every_solution_checked_by_oracle():
    """The benchmark's uneven batch exactly as bench.py runs it: 32 seeded
    instances (n in 12..40, mu log-U[1e-4, 1], dt log-U[1e-4, 1e-2]), 4 N(0,1)
    body forces each, coupled FGMRES(30) + block-LU, mixed precision, one
    V-cycle, one context and stream per instance, the four forces of an
    instance in lockstep (stokes_solve_multi), solved concurrently to 1e-8.
    Every row of every one of the 128 residuals is evaluated by the oracle's
    element loop; the smallest instance (n = 12) is also compared with the
    oracle's exact discrete solution."""
    from oracle.local import relative_residuals
    from oracle.solve import schur_cg_solve
    sk = gpu_module()
    insts = wl.batched_instances(32, seed=4)
    verts = [i.vertices() for i in insts]
    spec = [(i.n, V, i.mu, i.dt, 0.0) for i, V in zip(insts, verts)]
    B = sk.StokesBatch(spec, sk.stokes_default_options(precision=1, vcycles=1, method=1))
    forces = [[wl.random_force(i.n, i.seed * 10 + k) for k in range(4)] for i in insts]
    outs, infos, ms = B.solve_all([[cuda(f) for f in fl] for fl in forces], tol=1e-8)
    sols = [[(host(u), host(p)) for (u, p) in o] for o in outs]
    B.close()
    worst = 0.0
    for i, inst in enumerate(insts):
        mesh = KuhnMesh(inst.n, verts[i])
        for k in range(4):
            assert infos[i][k]["status"] == 0 and infos[i][k]["rel_residual"] <= 1e-8, (i, k, infos[i][k])
        # one oracle pass per instance for its four right-hand sides (they share
        # the element geometry)
        rels = relative_residuals(mesh, inst.mu, inst.dt, forces[i], [(u, p, None) for (u, p) in sols[i]])
        for k, rel in enumerate(rels):
            assert rel <= 1e-8 * (1 + 1e-6), (i, k, rel)
            assert abs(rel - infos[i][k]["rel_residual"]) <= 1e-11, (i, k, rel, infos[i][k]["rel_residual"])
            worst = max(worst, rel)
    small = min(range(len(insts)), key=lambda j: insts[j].n)
    inst = insts[small]
    orc = StokesSystem(KuhnMesh(inst.n, verts[small]), inst.mu, inst.dt)
    Uo, Po = schur_cg_solve(orc, orc.load(forces[small][0]))
    u, p = sols[small][0]
    eu, ep = rel_err(orc.restrict_velocity(u), Uo), rel_err(p, Po)
    print(f"batch: worst oracle residual {worst:.3e}; n={inst.n} member vs exact solution: "
          f"velocity {eu:.2e}, pressure {ep:.2e}")
    assert eu < 1e-5 and ep < 1e-4, (eu, ep)
