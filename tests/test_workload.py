"""Seeded input generator checks (CPU only)."""

import numpy as np

import workload as wl


def test_splitmix64_reference_outputs():
    # first outputs of SplitMix64 seeded with 0 (Steele, Lea & Flood 2014)
    ref = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    got = [int(x) for x in wl.counter_u64(0, 0, np.arange(4))]
    assert got == ref


def test_jitter_bounds_and_boundary():
    n = 6
    X0 = wl.kuhn_vertices(n, 0.0, 3)
    X = wl.kuhn_vertices(n, 0.2, 3)
    d = np.abs(X - X0)
    assert d.max() <= 0.2 / n + 1e-15 and d.max() > 0.1 / n
    on_bnd = np.any((X0 == 0) | (X0 == 1), axis=1)
    assert np.all(d[on_bnd] == 0)
    assert np.array_equal(X, wl.kuhn_vertices(n, 0.2, 3))          # deterministic
    assert not np.array_equal(X, wl.kuhn_vertices(n, 0.2, 4))


def test_manufactured_field_properties():
    ms = wl.Manufactured(seed=5)
    rng = np.random.default_rng(0)
    X = rng.uniform(0.1, 0.9, size=(40, 3))
    h = 1e-4

    def fd(fun, X, a):
        e = np.zeros(3)
        e[a] = h
        return (fun(X + e) - fun(X - e)) / (2 * h)

    div = sum(fd(lambda Y: ms.velocity(Y)[:, a], X, a) for a in range(3))
    assert np.abs(div).max() < 1e-6 * np.abs(ms.velocity(X)).max() + 1e-7
    lap_fd = np.zeros((40, 3))
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        lap_fd += (ms.velocity(X + e) - 2 * ms.velocity(X) + ms.velocity(X - e)) / h ** 2
    assert np.allclose(lap_fd, ms.velocity_laplacian(X), rtol=1e-4, atol=1e-4 * np.abs(lap_fd).max())
    gp = np.stack([fd(ms.pressure, X, a) for a in range(3)], axis=1)
    assert np.allclose(gp, ms.pressure_gradient(X), rtol=1e-6, atol=1e-8)
    # zero velocity on every face of the unit cube
    B = rng.uniform(0, 1, size=(30, 3))
    for a in range(3):
        for v in (0.0, 1.0):
            Y = B.copy()
            Y[:, a] = v
            assert np.abs(ms.velocity(Y)).max() < 1e-12
    # zero-mean pressure (midpoint rule on a fine grid)
    g = (np.arange(40) + 0.5) / 40
    G = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    assert abs(ms.pressure(G).mean()) < 1e-12


def test_dof_counts():
    assert wl.num_dofs(8) == 15468
    assert wl.num_dofs(48) == 2738019 + 117649
    assert wl.num_dofs(96) == 21567171 + 912673
