"""Iteration counts flat in h: the preconditioned Schur CG (C^Lambda) and the
coupled FGMRES need a bounded number of outer iterations as the mesh is
refined (the paper's weak-scalability observation), for a fixed time step and
for a time step tied to the mesh size."""

import numpy as np
import pytest

import workload as wl

from gpu_helpers import cuda, gpu_module

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("dt_rule", ["fixed", "h"])
def test_outer_iterations_flat_in_h(method, dt_rule):
    sk = gpu_module()
    mu = 1e-2
    iters = []
    for n in (8, 16, 32):
        dt = 1e-3 if dt_rule == "fixed" else 1.0 / n
        V = wl.kuhn_vertices(n, 0.2, 1)
        f = wl.manufactured_force(n, V, mu, dt, 1)
        S = sk.Stokes(n, V, mu, dt, 0.0, sk.stokes_default_options(method=method))
        _, _, info = S.solve(cuda(f), None, 1e-8)
        assert info.status == 0, info.as_dict()
        iters.append(info.outer_iters)          # summed over defect-correction passes
        S.close()
    print("method", method, "dt", dt_rule, "outer iterations n=8,16,32:", iters)
    assert max(iters) <= 1.5 * min(iters) + 2, iters
    assert iters[-1] <= iters[-2] + 3, iters
