"""CPU check of the symmetric stencil product the GPU uses for the strain-form
A (no GPU, no library code). Rows of the interior P2 nodes are grouped by the
parity class of their half-grid coordinates; a row stores its diagonal 3x3
block and the blocks of its neighbours at lexicographically positive offsets
(z, then y, then x), laid out [entry][9][row-in-class]; the block of a
neighbour j = i + o at a negative offset is read, transposed, from row j's
storage: class(j) = class(i) XOR parity(o), entry -o, row-in-class position
shifted by (q0(i) + o - q0(j)) / 2 per axis. Blocks walk the half-grid
z-planes in order (odd plane k, even plane k, ...), within a plane the four
classes that have rows there, 128 / G rows per block of 128 threads (G
threads share a row).

Rebuilt here from the oracle's assembled A, the scheme must cover every row
exactly once, read only inside the stored values and the vector, and give
A x; this pins the layout, the transposed read and the launch order that
the kernel relies on."""

import numpy as np

import workload as wl
from oracle.assemble import StokesSystem
from oracle.mesh import KuhnMesh


def lex(d):
    return d[2] if d[2] else (d[1] if d[1] else d[0])


def test_symmetric_stencil_product_equals_matrix():
    for n in (2, 3, 4, 5):
        V = wl.kuhn_vertices(n, 0.2, 31)
        A = StokesSystem(KuhnMesh(n, V), 0.3, 0.02).A.tocsr()      # node-interleaved 3x3 blocks
        m = 2 * n - 1
        nn = m ** 3
        idx = np.arange(nn)
        q = np.stack([idx % m, (idx // m) % m, idx // (m * m)], 1) + 1
        cls = (q[:, 0] % 2) + 2 * (q[:, 1] % 2) + 4 * (q[:, 2] % 2)
        offs = {c: set() for c in range(8)}
        Ab = {}
        for i in range(nn):
            for k in range(A.indptr[3 * i], A.indptr[3 * i + 1]):
                j = A.indices[k] // 3
                offs[cls[i]].add(tuple(int(t) for t in q[j] - q[i]))
        for r in range(3 * nn):
            for k in range(A.indptr[r], A.indptr[r + 1]):
                Ab.setdefault((r // 3, A.indices[k] // 3), np.zeros((3, 3)))[r % 3, A.indices[k] % 3] = A.data[k]
        q0 = {c: [1 if (c >> k) & 1 else 2 for k in range(3)] for c in range(8)}
        ext = {c: [n if (c >> k) & 1 else n - 1 for k in range(3)] for c in range(8)}
        prows = {c: ext[c][0] * ext[c][1] * ext[c][2] for c in range(8)}
        up = {c: [(0, 0, 0)] + sorted((d for d in offs[c] if lex(d) > 0), key=lambda d: (d[2], d[1], d[0]))
              for c in range(8)}
        low = {c: [d for d in offs[c] if lex(d) < 0] for c in range(8)}
        voff, off = {}, 0
        for c in range(8):
            voff[c] = off
            off += 9 * len(up[c]) * prows[c]
        vals = np.full(off, np.nan)
        pos_of = {}
        for i in range(nn):
            c = cls[i]
            ix, iy, iz = [(q[i][k] - q0[c][k]) // 2 for k in range(3)]
            pr = ix + ext[c][0] * (iy + ext[c][1] * iz)
            pos_of[i] = (c, ix, iy, iz, pr)
        # fill (k_sym3_fill)
        for c in range(8):
            for pr in range(prows[c]):
                ix, iy, iz = pr % ext[c][0], (pr // ext[c][0]) % ext[c][1], pr // (ext[c][0] * ext[c][1])
                qi = np.array([q0[c][0] + 2 * ix, q0[c][1] + 2 * iy, q0[c][2] + 2 * iz])
                i = int((qi[0] - 1) + m * (qi[1] - 1) + m * m * (qi[2] - 1))
                for e, d in enumerate(up[c]):
                    qj = qi + np.array(d)
                    inside = np.all((qj >= 1) & (qj <= m))
                    j = int((qj[0] - 1) + m * (qj[1] - 1) + m * m * (qj[2] - 1)) if inside else -1
                    blk = Ab.get((i, j), np.zeros((3, 3))) if inside else np.zeros((3, 3))
                    for k in range(9):
                        vals[voff[c] + (9 * e + k) * prows[c] + pr] = blk[k // 3, k % 3]
        assert not np.isnan(vals).any()
        # launch order (sym3_locate): every row exactly once
        nb = {c: -(-ext[c][0] * ext[c][1] // 128) for c in range(8)}
        bo, be = sum(nb[c] for c in (4, 5, 6, 7)), sum(nb[c] for c in (0, 1, 2, 3))
        grid = n * bo + (n - 1) * be
        seen = np.zeros(nn, int)
        x = np.random.default_rng(n).standard_normal(3 * nn)      # node-interleaved
        xc = x.reshape(nn, 3).T.ravel()                             # component-major, as on the GPU
        y = np.zeros(3 * nn)
        for b in range(grid):
            pair, rem = divmod(b, bo + be)
            odd = rem < bo
            if not odd:
                rem -= bo
            c = 4 if odd else 0
            for _ in range(3):
                if rem >= nb[c]:
                    rem -= nb[c]
                    c += 1
            plane = ext[c][0] * ext[c][1]
            for t in range(rem * 128, rem * 128 + 128):
                if t >= plane:
                    continue
                ix, iy, iz = t % ext[c][0], t // ext[c][0], pair
                pr = iz * plane + t
                qi = np.array([q0[c][0] + 2 * ix, q0[c][1] + 2 * iy, q0[c][2] + 2 * iz])
                assert np.all((qi >= 1) & (qi <= m))
                row = int((qi[0] - 1) + m * (qi[1] - 1) + m * m * (qi[2] - 1))
                assert cls[row] == c
                seen[row] += 1
                acc = np.zeros(3)
                for e, d in enumerate(up[c]):
                    lin = d[0] + m * d[1] + m * m * d[2]
                    cc = min(max(row + lin, 0), nn - 1)
                    w = np.array([vals[voff[c] + (9 * e + k) * prows[c] + pr] for k in range(9)]).reshape(3, 3)
                    acc += w @ xc.reshape(3, nn)[:, cc]
                for o in low[c]:
                    qj = qi + np.array(o)
                    inside = bool(np.all((qj >= 1) & (qj <= m)))
                    cs = c ^ ((o[0] & 1) | ((o[1] & 1) << 1) | ((o[2] & 1) << 2))
                    es = up[cs].index(tuple(-t_ for t_ in o))
                    dl = [(q0[c][k] + o[k] - q0[cs][k]) // 2 for k in range(3)]
                    assert all((q0[c][k] + o[k] - q0[cs][k]) % 2 == 0 for k in range(3))
                    jx, jy, jz = ix + dl[0], iy + dl[1], iz + dl[2]
                    rj = jx + ext[cs][0] * (jy + ext[cs][1] * jz) if inside else 0
                    assert 0 <= rj < prows[cs]
                    base = voff[cs] + 9 * es * prows[cs] + rj
                    w = np.array([vals[base + k * prows[cs]] for k in range(9)]).reshape(3, 3)
                    if not inside:
                        w[:] = 0.0
                    else:
                        j = int((qj[0] - 1) + m * (qj[1] - 1) + m * m * (qj[2] - 1))
                        assert pos_of[j][4] == rj and pos_of[j][0] == cs
                    lin = o[0] + m * o[1] + m * m * o[2]
                    cc = min(max(row + lin, 0), nn - 1)
                    acc += w.T @ xc.reshape(3, nn)[:, cc]
                y[3 * row:3 * row + 3] = acc
        assert np.all(seen == 1)
        # with G threads per row a block covers 128 / G rows: every row exactly once
        for G in (2, 4, 8):
            rpb = 128 // G
            nbg = {c: -(-ext[c][0] * ext[c][1] // rpb) for c in range(8)}
            bog, beg = sum(nbg[c] for c in (4, 5, 6, 7)), sum(nbg[c] for c in (0, 1, 2, 3))
            cover = np.zeros(nn, int)
            for b in range(n * bog + (n - 1) * beg):
                pair, rem = divmod(b, bog + beg)
                odd = rem < bog
                if not odd:
                    rem -= bog
                c = 4 if odd else 0
                for _ in range(3):
                    if rem >= nbg[c]:
                        rem -= nbg[c]
                        c += 1
                plane = ext[c][0] * ext[c][1]
                for t in range(rem * rpb, rem * rpb + rpb):
                    if t < plane:
                        qi = [q0[c][0] + 2 * (t % ext[c][0]), q0[c][1] + 2 * (t // ext[c][0]), q0[c][2] + 2 * pair]
                        cover[(qi[0] - 1) + m * (qi[1] - 1) + m * m * (qi[2] - 1)] += 1
            assert np.all(cover == 1), G
        ref = A @ x
        assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max(), n
        # against the full stencil storage of every block: the upper half plus the diagonal
        full = sum((len(up[c]) + len(low[c])) * prows[c] for c in range(8))
        assert off // 9 == (full + nn) // 2
