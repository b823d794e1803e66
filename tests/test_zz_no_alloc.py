"""The allocation-free operator entry point (collected last on purpose).

Some callers cannot allocate device memory while they run - for instance a
host loop that reserved its whole device-memory budget at start-up, or code
running inside another framework that owns the device allocator. For them the
library offers stokes_apply_agamma_noalloc, which applies the augmented
velocity operator A x + gamma mu B^T M_Q^{-1} B x with its work vectors in a
fixed array compiled into the library. This test calls it through the C ABI
twice in a row and checks each result against the allocating entry point
stokes_apply(ctx, STOKES_OP_AGAMMA, ...), and against the oracle's assembled
A + gamma mu B^T M_Q^{-1} B (Eq. def_of_Alambda), for gamma > 0 and gamma = 0.
"""

import ctypes as C

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workload as wl
from oracle.assemble import StokesSystem
from oracle.mesh import KuhnMesh

from gpu_helpers import aos, cuda, gpu_module, host, rel_err, soa

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("gamma", [2.0, 0.0])
def test_noalloc_matches_allocating_entry_point_and_oracle_twice(gamma):
    sk = gpu_module()
    from paper_2407_01783_gb300 import _lib
    lib = _lib.load()
    n, mu, dt = 6, 0.3, 0.01
    V = wl.kuhn_vertices(n, 0.2, 21)
    S = sk.Stokes(n, V, mu, dt, gamma)
    orc = StokesSystem(KuhnMesh(n, V), mu, dt)
    m = 3 * S.sizes["n_inner"]
    rng = np.random.default_rng(5)
    for call in range(2):
        xi = rng.standard_normal(m)                     # node-interleaved (oracle layout)
        x = cuda(soa(xi))
        ref = S.apply("AGAMMA", x, m)
        y = cuda(np.full(m, np.nan))
        st = lib.stokes_apply_agamma_noalloc(S.ctx, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()))
        assert st == 0, lib.stokes_last_error()
        yh = host(y)
        assert np.all(np.isfinite(yh))
        assert rel_err(yh, host(ref)) < 1e-13, call
        exact = orc.A @ xi
        if gamma > 0:
            exact = exact + gamma * mu * (orc.B.T @ spla.spsolve(orc.MQ.tocsc(), orc.B @ xi))
        # M_Q^{-1} by 24 Chebyshev steps on [1/2, 5/2]: error below 0.382^24 ~ 1e-10
        assert rel_err(aos(yh), exact) < 1e-8, call
    S.close()
