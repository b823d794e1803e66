"""Parity-split numbering of the finest V-cycle level (option vcycle_split;
2 = every cycle, as tested here; the default 1 uses it in lockstep cycles):
the stencil rows and the transfers next to it run in a renumbered space, but
every row is computed from the same entries in the same order, so V-cycles,
solves and lockstep solves give the same bits as with natural numbering."""

import numpy as np
import pytest
import torch

import workload as wl

from gpu_helpers import cuda, gpu_module, host

pytestmark = pytest.mark.gpu


def vcycles(sk, n, opts, seed=3):
    V = wl.kuhn_vertices(n, 0.2, seed)
    outs = []
    for split in (0, 2):
        S = sk.Stokes(n, V, 0.05, 1e-3, options=sk.stokes_default_options(vcycle_split=split, **opts))
        size = 3 * S.sizes["n_inner"]
        r = np.random.default_rng(seed).standard_normal(size)
        x = cuda(r)
        y = torch.zeros(size, dtype=torch.float64, device="cuda")
        sk.stokes_apply(S.ctx, sk.OP["VCYCLE_A3"], x, y, 0)
        outs.append(host(y))
        S.close()
    return outs


@pytest.mark.parametrize("n", [8, 13])
def test_vcycle_split_numbering_is_bitwise_neutral(n):
    """FP64 V-cycle of A~_3 with stencil storage on every level (format 2),
    even and odd n."""
    sk = gpu_module()
    a, b = vcycles(sk, n, dict(format=2))
    assert np.any(a != 0)
    assert np.array_equal(a, b)


def test_vcycle_split_at_benchmark_threshold():
    """Default format at n = 33, the smallest size whose finest level is
    stencil-stored for one right-hand side (2^18 rows), two V-cycles."""
    sk = gpu_module()
    a, b = vcycles(sk, 33, dict(vcycles=2))
    assert np.array_equal(a, b)


@pytest.mark.parametrize("method", [0, 1])
def test_solves_split_numbering_is_bitwise_neutral(method):
    """Mixed-precision solves (one right-hand side and four in lockstep) give
    identical bits with and without the split finest level."""
    sk = gpu_module()
    n = 12
    V = wl.kuhn_vertices(n, 0.2, 8)
    F = np.stack([wl.random_force(n, 80 + k) for k in range(4)])
    res = []
    for split in (0, 2):
        S = sk.Stokes(n, V, 1e-2, 1e-3, options=sk.stokes_default_options(
            precision=1, vcycles=1, method=method, format=2, vcycle_split=split))
        u, p, info = S.solve(cuda(F[0]), None, 1e-9)
        U, P, infos = S.solve_multi(cuda(F), None, 1e-9)
        res.append((host(u), host(p), info.outer_iters, host(U), host(P), [i.outer_iters for i in infos]))
        S.close()
    a, b = res
    assert a[2] == b[2] and a[5] == b[5]
    for k in (0, 1, 3, 4):
        assert np.array_equal(a[k], b[k]), k
