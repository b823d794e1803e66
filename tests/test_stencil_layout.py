"""CPU check of the stencil-structured product the GPU uses for A~_3 (no GPU,
no library code): rows are grouped by the parity class of their half-grid
coordinates, every class has one list of neighbour offsets d with linear
offsets lin(d) = dx + m dy + m^2 dz, entries whose neighbour lies outside the
interior are stored as 0, and every row runs the same loop over its class
list reading x at clamp(row + lin(d), 0, m^3 - 1). Built here from the
oracle's assembled matrix, that product must equal A~_3 x, which pins the
two facts the kernel relies on: the class lists cover every matrix entry,
and a clamped or wrapped read always meets a zero weight."""

import numpy as np

import workload as wl
from oracle.assemble import StokesSystem
from oracle.mesh import KuhnMesh


def test_branch_free_stencil_product_equals_matrix():
    for n in (2, 3, 4):
        V = wl.kuhn_vertices(n, 0.2, 21)
        A = StokesSystem(KuhnMesh(n, V), 0.3, 0.02).A3s.tocsr()
        m = 2 * n - 1
        idx = np.arange(m ** 3)
        q = np.stack([idx % m, (idx // m) % m, idx // (m * m)], 1) + 1
        cls = (q[:, 0] % 2) + 2 * (q[:, 1] % 2) + 4 * (q[:, 2] % 2)
        offsets = {c: set() for c in range(8)}
        for i in range(A.shape[0]):
            for j in A.indices[A.indptr[i]:A.indptr[i + 1]]:
                offsets[cls[i]].add(tuple(q[j] - q[i]))
        assert all(max(abs(v) for d in offs for v in d) <= 2 for offs in offsets.values() if offs)
        x = np.random.default_rng(n).standard_normal(m ** 3)
        y = np.zeros(m ** 3)
        for i in range(m ** 3):
            row = dict(zip(A.indices[A.indptr[i]:A.indptr[i + 1]], A.data[A.indptr[i]:A.indptr[i + 1]]))
            for d in sorted(offsets[cls[i]]):
                nb = q[i] + np.array(d)
                inside = np.all((nb >= 1) & (nb <= m))
                j = int((nb[0] - 1) + m * (nb[1] - 1) + m * m * (nb[2] - 1)) if inside else -1
                w = row.get(j, 0.0) if inside else 0.0
                lin = d[0] + m * d[1] + m * m * d[2]
                k = min(max(i + lin, 0), m ** 3 - 1)
                if w != 0.0:
                    assert k == j                       # an inside read is never clamped
                y[i] += w * x[k]
        ref = A @ x
        assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()


def _split(i, m, n):
    """Parity-split numbering of a natural interior P2 index (even x-index t
    of a line first at t // 2, odd t at n + t // 2)."""
    t = i % m
    return i - t + np.where(t % 2 == 1, n + t // 2, t // 2)


def test_split_numbering_offsets_are_constant_per_class():
    """The parity-split finest level keeps one linear offset per (class,
    neighbour offset): for every row of a class, split(j) - split(i) equals
    (p' - p) n + floor((p + dx) / 2) + m (dy + m dz), p the parity of the row's
    x-index t = qx - 1 and p' that of t + dx; and the split map is a
    permutation. Checked by brute force over all rows and offsets."""
    for n in (2, 3, 5, 8):
        m = 2 * n - 1
        idx = np.arange(m ** 3)
        s = _split(idx, m, n)
        assert np.array_equal(np.sort(s), idx)
        q = np.stack([idx % m, (idx // m) % m, idx // (m * m)], 1) + 1
        for c in range(8):
            rows = idx[((q[:, 0] % 2) + 2 * (q[:, 1] % 2) + 4 * (q[:, 2] % 2)) == c]
            p = (q[rows[0], 0] - 1) % 2
            for dx in range(-2, 3):
                for dy in range(-2, 3):
                    for dz in range(-2, 3):
                        nb = q[rows] + np.array([dx, dy, dz])
                        ok = np.all((nb >= 1) & (nb <= m), axis=1)
                        j = (nb[ok, 0] - 1) + m * (nb[ok, 1] - 1) + m * m * (nb[ok, 2] - 1)
                        if j.size == 0:
                            continue
                        pn = (p + dx) % 2
                        lin = (pn - p) * n + (p + dx) // 2 + m * (dy + m * dz)
                        assert np.all(_split(j, m, n) - s[rows[ok]] == lin), (n, c, dx, dy, dz)
