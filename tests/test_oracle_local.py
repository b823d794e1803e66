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


def test_vectorised_full_residual_equals_global_residual():
    """oracle.local.full_residual (element gradients, no global matrices) gives
    every row of the globally assembled residual, for several cases at once."""
    from oracle.local import full_residual, relative_residuals
    n, mu, dt = 3, 0.07, 0.02
    V = wl.kuhn_vertices(n, 0.2, 9)
    mesh = KuhnMesh(n, V)
    s = StokesSystem(mesh, mu, dt)
    rng = np.random.default_rng(1)
    f = rng.standard_normal((mesh.n_p2, 3))
    cases, refs = [], []
    for k in range(3):
        U = rng.standard_normal(s.A.shape[0])
        P = rng.standard_normal(s.B.shape[0])
        g = wl.random_pressure_load(n, 10 + k) if k else None
        cases.append((s.expand_velocity(U), P, g))
        refs.append(residual(s, U, P, s.load(f), g))
    nv = s.A.shape[0]
    out = full_residual(mesh, mu, dt, f, cases, chunk=37)       # ragged chunks
    for (rF, rg, norm), ref, (_, _, g) in zip(out, refs, cases):
        scale = np.abs(ref).max()
        assert np.abs(rF.ravel() - ref[:nv]).max() < 1e-12 * scale
        assert np.abs(rg - ref[nv:]).max() < 1e-12 * scale
        gg = np.zeros(mesh.n_p1) if g is None else g
        assert abs(norm - np.linalg.norm(np.concatenate([s.load(f), gg]))) < 1e-12 * norm
    rel = relative_residuals(mesh, mu, dt, f, cases[:1])
    assert abs(rel[0] - np.linalg.norm(refs[0]) / np.linalg.norm(s.load(f))) < 1e-12


def test_full_residual_vanishes_at_exact_solution():
    """At the oracle's exact discrete solution every residual row is at rounding level."""
    from oracle.local import relative_residuals
    from oracle.solve import direct_solve
    n, mu, dt = 4, 0.3, 0.01
    V = wl.kuhn_vertices(n, 0.2, 2)
    mesh = KuhnMesh(n, V)
    s = StokesSystem(mesh, mu, dt)
    f = wl.random_force(n, 3)
    g = wl.random_pressure_load(n, 4)
    U, P = direct_solve(s, s.load(f), g)
    rel = relative_residuals(mesh, mu, dt, f, [(s.expand_velocity(U), P, g)])[0]
    assert rel < 1e-13, rel


def test_chunked_l2_errors_equal_global_definition():
    from oracle.local import l2_errors_chunked
    from oracle.solve import l2_errors, schur_cg_solve
    n = 4
    V = wl.kuhn_vertices(n, 0.2, 1)
    s = StokesSystem(KuhnMesh(n, V), 1.0, 1.0)
    ms = wl.Manufactured(seed=1)
    f = ms.body_force(s.mesh.p2_coords(), 1.0, 1.0)
    U, P = schur_cg_solve(s, s.load(f))
    a = l2_errors(s, s.expand_velocity(U), P, ms, q=5)
    b = l2_errors_chunked(s.mesh, s.expand_velocity(U), P, ms, q=5, chunk=101)
    assert np.allclose(a, b, rtol=1e-12), (a, b)
