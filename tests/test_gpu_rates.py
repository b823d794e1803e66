"""Manufactured-solution convergence of the GPU's own solutions.

The GPU solves the seeded manufactured problem (u = curl psi, p = d cos cos cos,
f = u/dt - mu Lap u + grad p) on jittered Kuhn meshes with n = 8, 16, 32, in
FP64 to 1e-12 and in mixed precision to 1e-8; the oracle measures the L2
errors of the GPU's (u_h, p_h) by quadrature. P2-P1 Taylor-Hood gives velocity
errors O(h^3) and pressure errors O(h^2) (Sec. 3.3, Tables vel_pb_exact and
vel_pb_2fvc: the error ratio per halving of h approaches 2^3 and 2^2).
"""

import json
import os

import numpy as np
import pytest

import workload as wl
from oracle.local import l2_errors_chunked
from oracle.mesh import KuhnMesh

from gpu_helpers import cuda, gpu_module, host

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-8)])
def test_gpu_solutions_converge_at_paper_rates(precision, tol):
    sk = gpu_module()
    facts = json.load(open(os.path.join(GOLDEN, "paper_facts.json")))
    mu, dt = 1.0, 1.0
    ms = wl.Manufactured(seed=1)
    ms.m[:] = 1
    errs = []
    for n in (8, 16, 32):
        V = wl.kuhn_vertices(n, 0.2, 1)
        f = ms.body_force(wl.p2_node_coords(V, n), mu, dt)
        S = sk.Stokes(n, V, mu, dt, 0.0, sk.stokes_default_options(precision=precision, vcycles=1))
        u, p, info = S.solve(cuda(f), None, tol)
        assert info.status == 0 and info.rel_residual <= tol
        errs.append(l2_errors_chunked(KuhnMesh(n, V), host(u), host(p), ms, q=4))
        S.close()
    eu, ep = np.array(errs).T
    ru, rp = np.log2(eu[:-1] / eu[1:]), np.log2(ep[:-1] / ep[1:])
    print(f"precision={precision}: velocity errors {eu}, rates {ru}; pressure errors {ep}, rates {rp}")
    assert np.all(ru > facts["p2_velocity_l2_rate"] - 0.35), ru
    assert np.all(rp > facts["p1_pressure_l2_rate"] - 0.35), rp
