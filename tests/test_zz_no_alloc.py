"""The allocation-free operator entry point (collected last on purpose).

Some callers cannot allocate device memory while they run - for instance a
host loop that reserved its whole device-memory budget at start-up, or code
running inside another framework that owns the device allocator. For them the
library offers stokes_apply_agamma_noalloc, which applies the augmented
velocity operator A x + gamma mu B^T M_Q^{-1} B x with its work vectors in a
fixed array compiled into the library. This test calls it through the C ABI
twice in a row and checks each result against the allocating entry point
stokes_apply(ctx, STOKES_OP_AGAMMA, ...).
"""

import ctypes as C

import numpy as np
import pytest

import workload as wl

from gpu_helpers import cuda, gpu_module, host, rel_err

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point_twice():
    sk = gpu_module()
    from paper_2407_01783_gb300 import _lib
    lib = _lib.load()
    n, mu, dt, gamma = 6, 0.3, 0.01, 2.0
    S = sk.Stokes(n, wl.kuhn_vertices(n, 0.2, 21), mu, dt, gamma)
    m = 3 * S.sizes["n_inner"]
    rng = np.random.default_rng(5)
    for call in range(2):
        x = cuda(rng.standard_normal(m))
        ref = S.apply("AGAMMA", x, m)
        y = cuda(np.full(m, np.nan))
        st = lib.stokes_apply_agamma_noalloc(S.ctx, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()))
        assert st == 0, lib.stokes_last_error()
        assert np.all(np.isfinite(host(y)))
        assert rel_err(host(y), host(ref)) < 1e-13, call
    S.close()
