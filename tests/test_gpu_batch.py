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
