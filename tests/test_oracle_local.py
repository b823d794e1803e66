"""Pin the oracle's element-local residual rows against its global assembly (CPU)."""

import numpy as np

import workload as wl
from oracle.assemble import StokesSystem
from oracle.local import load_norm, pressure_residual_rows, velocity_residual_rows
from oracle.mesh import KuhnMesh
from oracle.solve import residual


def test_local_rows_equal_global_residual():
    n, mu, dt = 4, 0.2, 0.03
    V = wl.kuhn_vertices(n, 0.2, 5)
    mesh = KuhnMesh(n, V)
    s = StokesSystem(mesh, mu, dt)
    rng = np.random.default_rng(0)
    f = rng.standard_normal((mesh.n_p2, 3))
    U = rng.standard_normal(s.A.shape[0])
    P = rng.standard_normal(s.B.shape[0])
    g = wl.random_pressure_load(n, 3)
    r = residual(s, U, P, s.load(f), g)
    nv = s.A.shape[0]
    u_nodal = s.expand_velocity(U)
    picks = rng.choice(mesh.interior.size, 12, replace=False)
    loc = velocity_residual_rows(mesh, mu, dt, f, u_nodal, P, mesh.interior[picks])
    ref = r[:nv].reshape(-1, 3)[picks]
    assert np.allclose(loc, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
    verts = rng.choice(mesh.n_p1, 10, replace=False)
    locp = pressure_residual_rows(mesh, u_nodal, g, verts)
    assert np.allclose(locp, r[nv:][verts], rtol=1e-12, atol=1e-12 * np.abs(r[nv:]).max())
    assert abs(load_norm(mesh, f) - np.linalg.norm(s.load(f))) < 1e-12 * np.linalg.norm(s.load(f))
