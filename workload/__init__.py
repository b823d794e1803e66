"""Seeded synthetic inputs for the generalized Stokes solver.

This module is shared by the CPU oracle, the GPU tests and the benchmark. It
produces problem *data* only: vertex coordinates of a jittered Kuhn mesh of the
unit cube, nodal body-force fields and pressure loads. It contains none of the
discretisation or solver arithmetic (no basis functions, no element integrals,
no matrices, no Krylov steps); each side implements those on its own.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014). Its k-th output (k >= 1) for
the seed S is mix(S + k * GOLDEN); here S = seed XOR (stream * STREAM_MUL) and
the word for ``index`` is output k = index + 1. No state is carried between
calls, so any entry can be regenerated on its own.

Conventions shared with the C-ABI (plain data layouts, not arithmetic):

* vertices: ``(n+1)**3`` rows, lexicographic with x fastest:
  ``v = i + (n+1)*(j + (n+1)*k)``; coordinates in [0,1]^3 before jitter.
* P2 nodes: the ``(2n+1)**3`` half-grid, lexicographic with x fastest; the node
  with half-grid coordinates ``q`` sits at the midpoint of vertices
  ``floor(q/2)`` and ``ceil(q/2)`` (a vertex when all coordinates are even).
* vector fields at P2 nodes are node-interleaved: ``[(2n+1)**3][3]``.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
STREAM_MUL = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_JITTER = 1
STREAM_FORCE = 2
STREAM_MANUFACTURED = 3
STREAM_PRESSURE_LOAD = 4
STREAM_BATCH = 5


def splitmix64_mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied elementwise to uint64 values."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def counter_u64(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    """Counter-based 64-bit random words for (seed, stream, index)."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        S = np.uint64(seed) ^ (np.uint64(stream) * STREAM_MUL)
        key = S + (idx + np.uint64(1)) * GOLDEN
    return splitmix64_mix(key)


def uniform01(seed: int, stream: int, index: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0,1) from the top 53 bits of the counter hash."""
    w = counter_u64(seed, stream, index)
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal01(seed: int, stream: int, count: int) -> np.ndarray:
    """Standard normal samples by Box-Muller on pairs of counter uniforms."""
    m = (count + 1) // 2
    k = np.arange(m, dtype=np.uint64)
    u1 = uniform01(seed, stream, 2 * k)
    u2 = uniform01(seed, stream, 2 * k + np.uint64(1))
    r = np.sqrt(-2.0 * np.log1p(-u1))  # 1-u1 in (0,1]
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    return z[:count]


# ---------------------------------------------------------------------------
# Mesh data
# ---------------------------------------------------------------------------

def kuhn_vertices(n: int, jitter: float = 0.0, seed: int = 0) -> np.ndarray:
    """Vertex coordinates of the n^3-cube grid of [0,1]^3, shape ((n+1)^3, 3).

    Interior vertices are moved by an independent uniform offset in
    [-jitter*h, jitter*h) per coordinate, h = 1/n, keyed by (seed, vertex, axis).
    Boundary vertices stay on the boundary planes (their coordinates along the
    boundary normal are not moved; tangential coordinates are not moved either).
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    h = 1.0 / n
    g = np.arange(n + 1, dtype=np.float64) * h
    k, j, i = np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n + 1), indexing="ij")
    X = np.stack([g[i.ravel()], g[j.ravel()], g[k.ravel()]], axis=1)
    if jitter != 0.0:
        interior = ((i > 0) & (i < n) & (j > 0) & (j < n) & (k > 0) & (k < n)).ravel()
        vid = np.nonzero(interior)[0].astype(np.uint64)
        for a in range(3):
            u = uniform01(seed, STREAM_JITTER, vid * np.uint64(3) + np.uint64(a))
            X[interior, a] += (2.0 * u - 1.0) * jitter * h
    return X


def p2_node_coords(vertices: np.ndarray, n: int) -> np.ndarray:
    """Coordinates of the (2n+1)^3 half-grid nodes (midpoint rule of the layout)."""
    N = 2 * n + 1
    q = np.arange(N)
    K, J, I = np.meshgrid(q, q, q, indexing="ij")
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    nv = n + 1

    def vid(a, b, c):
        return a + nv * (b + nv * c)

    lo = vid(I // 2, J // 2, K // 2)
    hi = vid((I + 1) // 2, (J + 1) // 2, (K + 1) // 2)
    return 0.5 * (vertices[lo] + vertices[hi])


def num_dofs(n: int) -> int:
    """Total DOF count used by the throughput metric: 3(2n+1)^3 + (n+1)^3."""
    return 3 * (2 * n + 1) ** 3 + (n + 1) ** 3


# ---------------------------------------------------------------------------
# Manufactured solution: u = curl(psi), psi_a = c_a s_a(x) s_a(y) s_a(z),
# s_a(t) = sin^2(m_a pi t); p = d cos(pi x) cos(pi y) cos(pi z).
# u vanishes on the boundary of the unit cube, div u = 0, mean(p) = 0.
# ---------------------------------------------------------------------------

def _sdiff(m: int, k: int, t: np.ndarray) -> np.ndarray:
    """k-th derivative of s(t) = sin^2(m pi t) = (1 - cos(2 m pi t)) / 2."""
    w = 2.0 * m * math.pi
    if k == 0:
        return 0.5 * (1.0 - np.cos(w * t))
    # d^k/dt^k of -cos(w t)/2
    phase = [np.cos, lambda x: -np.sin(x), lambda x: -np.cos(x), np.sin]
    return -0.5 * (w ** k) * phase[k % 4](w * t)


@dataclass
class Manufactured:
    """Seeded smooth divergence-free velocity and zero-mean pressure."""

    seed: int = 1
    c: np.ndarray = field(init=False)
    m: np.ndarray = field(init=False)
    d: float = field(init=False)

    def __post_init__(self):
        z = normal01(self.seed, STREAM_MANUFACTURED, 4)
        u = uniform01(self.seed, STREAM_MANUFACTURED, np.arange(100, 103, dtype=np.uint64))
        self.c = z[:3].copy()
        self.m = np.where(u < 0.5, 1, 2).astype(int)
        self.d = float(z[3])

    # psi_a derivative: d^(ex) d^(ey) d^(ez) of c_a s(x) s(y) s(z)
    def _psi(self, a: int, X: np.ndarray, ex: int, ey: int, ez: int) -> np.ndarray:
        m = int(self.m[a])
        return (self.c[a] * _sdiff(m, ex, X[:, 0]) * _sdiff(m, ey, X[:, 1])
                * _sdiff(m, ez, X[:, 2]))

    def _u_component(self, comp: int, X: np.ndarray, extra=(0, 0, 0)) -> np.ndarray:
        # u = curl psi: u_x = d_y psi_z - d_z psi_y, etc.
        a1, d1, a2, d2 = {0: (2, 1, 1, 2), 1: (0, 2, 2, 0), 2: (1, 0, 0, 1)}[comp]
        e1 = list(extra)
        e1[d1] += 1
        e2 = list(extra)
        e2[d2] += 1
        return self._psi(a1, X, *e1) - self._psi(a2, X, *e2)

    def velocity(self, X: np.ndarray) -> np.ndarray:
        return np.stack([self._u_component(c, X) for c in range(3)], axis=1)

    def velocity_laplacian(self, X: np.ndarray) -> np.ndarray:
        out = []
        for c in range(3):
            out.append(sum(self._u_component(c, X, extra=tuple(2 if q == r else 0 for q in range(3)))
                           for r in range(3)))
        return np.stack(out, axis=1)

    def pressure(self, X: np.ndarray) -> np.ndarray:
        pi = math.pi
        return self.d * np.cos(pi * X[:, 0]) * np.cos(pi * X[:, 1]) * np.cos(pi * X[:, 2])

    def pressure_gradient(self, X: np.ndarray) -> np.ndarray:
        pi = math.pi
        cx, cy, cz = (np.cos(pi * X[:, a]) for a in range(3))
        sx, sy, sz = (np.sin(pi * X[:, a]) for a in range(3))
        return -self.d * pi * np.stack([sx * cy * cz, cx * sy * cz, cx * cy * sz], axis=1)

    def body_force(self, X: np.ndarray, mu: float, dt: float) -> np.ndarray:
        """f = u/dt - mu*Lap(u) + grad(p)  (the strong form of a(u,v) - b(v,p) = (f,v)
        for a divergence-free u, where -div(2 mu eps(u)) = -mu Lap(u))."""
        return (self.velocity(X) / dt - mu * self.velocity_laplacian(X)
                + self.pressure_gradient(X))


def manufactured_force(n: int, vertices: np.ndarray, mu: float, dt: float, seed: int) -> np.ndarray:
    """Nodal body force f at all P2 nodes, shape ((2n+1)^3, 3)."""
    ms = Manufactured(seed)
    return ms.body_force(p2_node_coords(vertices, n), mu, dt)


def random_force(n: int, seed: int) -> np.ndarray:
    """N(0,1) body force per nodal component at all P2 nodes, ((2n+1)^3, 3)."""
    N = (2 * n + 1) ** 3
    return normal01(seed, STREAM_FORCE, 3 * N).reshape(N, 3)


def random_pressure_load(n: int, seed: int) -> np.ndarray:
    """A P1 load vector g with sum(g) = 0 (compatible with B u = g)."""
    Np = (n + 1) ** 3
    g = normal01(seed, STREAM_PRESSURE_LOAD, Np)
    return g - g.mean()


@dataclass
class Instance:
    """One seeded generalized Stokes problem on a jittered Kuhn mesh."""

    n: int
    mu: float
    dt: float
    gamma: float = 0.0
    jitter: float = 0.0
    seed: int = 1
    rhs: str = "manufactured"  # or "random"

    def vertices(self) -> np.ndarray:
        return kuhn_vertices(self.n, self.jitter, self.seed)

    def force(self, vertices: np.ndarray | None = None) -> np.ndarray:
        if vertices is None:
            vertices = self.vertices()
        if self.rhs == "manufactured":
            return manufactured_force(self.n, vertices, self.mu, self.dt, self.seed)
        if self.rhs == "random":
            return random_force(self.n, self.seed)
        raise ValueError(self.rhs)

    @property
    def dofs(self) -> int:
        return num_dofs(self.n)


def batched_instances(count: int = 32, seed: int = 4, n_lo: int = 12, n_hi: int = 40,
                      jitter: float = 0.2) -> list[Instance]:
    """Uneven batch: n uniform in [n_lo, n_hi], mu log-U[1e-4,1], dt log-U[1e-4,1e-2]."""
    u = uniform01(seed, STREAM_BATCH, np.arange(3 * count, dtype=np.uint64)).reshape(count, 3)
    out = []
    for b in range(count):
        n = n_lo + int(u[b, 0] * (n_hi - n_lo + 1))
        mu = 10.0 ** (-4.0 + 4.0 * u[b, 1])
        dt = 10.0 ** (-4.0 + 2.0 * u[b, 2])
        out.append(Instance(n=n, mu=mu, dt=dt, jitter=jitter, seed=seed * 1000 + b, rhs="random"))
    return out
