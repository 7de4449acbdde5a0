"""A CPU model of the scatter kernel's index arithmetic, checked against the
oracle's sparse-grid index on every chunk of small schemes and on sampled
chunks of the 4-d level-14 scheme.  It restates, in Python integers, what a
CTA of the kernel computes: the subspace ranking table, the chunk's parts of
dimensions >= 2 per plane and budget, its parts of dimensions >= 1 per row
and value of max(j_0, 1), the 32-bit reciprocal divisions, and each point's
position; and it checks every table index and table size the kernel relies
on.  CPU only (the GPU tests check the kernel itself bit for bit)."""
import numpy as np
import pytest

CHUNK = 2048


def fdiv(t, S):                      # 64-bit reciprocal division, as on the device
    return t if S == 1 else (t * (((1 << 64) - 1) // S + 1)) >> 64


def magic_u32(dv):
    return 0 if dv == 1 else (0xFFFFFFFF // dv) + 1


def umulhi(a, b):
    return (a * b) >> 32


def omega(j):
    return 2 if j == 0 else 1 << (j - 1)


def build_rank(d, n):
    """R[k][jj][b]: points of the blocks that agree with j before dimension k
    and have a smaller j_k, per unit weight of the earlier dimensions."""
    T = n + d - 1
    C = [[0] * (T + 1) for _ in range(d + 1)]
    C[d] = [1] * (T + 1)
    R = [[[0] * (T + 1) for _ in range(n + 1)] for _ in range(d)]
    for k in range(d - 1, -1, -1):
        for b in range(T + 1):
            acc = 0
            for jj in range(n + 1):
                R[k][jj][b] = acc
                r = b - max(jj, 1)
                if r >= 0:
                    acc += omega(jj) * C[k + 1][r]
            C[k][b] = acc
    return R


def level_pos(l, i):
    if i == 0 or i == (1 << l):
        return 0, int(i != 0)
    tz = (i & -i).bit_length() - 1
    return l - tz, i >> (tz + 1)


def div_row(t, n0, mag):
    return int(t >= n0) if n0 > CHUNK else umulhi(t, mag)


def chunk_positions(l, d, n, R, f0):
    """Positions of the points of the chunk starting at f0, as the kernel
    computes them, with its table bounds asserted."""
    T = n + d - 1
    S = [1]
    for v in l[:-1]:
        S.append(S[-1] * ((1 << v) + 1))
    N = S[-1] * ((1 << l[-1]) + 1)
    n0 = (1 << l[0]) + 1
    n1 = (1 << l[1]) + 1 if d > 1 else 1
    t0, row0, npts = f0 % n0, f0 // n0, min(CHUNK, N - f0)
    rows = (f0 + npts - 1) // n0 - row0 + 1
    plane0 = row0 // n1
    planes = (row0 + rows - 1) // n1 - plane0 + 1
    nbud = max(l[0], 1)
    nb2 = nbud + max(l[1], 1) - 1 if d > 2 else 0
    nent, nent2 = rows * nbud, planes * nb2 if d > 2 else 0
    assert rows <= (CHUNK - 1) // n0 + 2
    mag0, magb, magb2 = magic_u32(min(n0, 1 << 30)), magic_u32(nbud), magic_u32(nb2) if nb2 else 0
    out2 = []
    for e in range(nent2):
        pp = umulhi(e, magb2) if magb2 else e
        assert pp == e // nb2
        s = e - pp * nb2 + 2
        fp = (plane0 + pp) * S[2]
        assert fp < N
        o, W, b, q = 0, 1, T - s, plane0 + pp
        for k in range(2, d):
            q1 = fdiv(fp, S[k + 1]) if k + 1 < d else 0
            i = q - q1 * ((1 << l[k]) + 1)
            assert 0 <= i <= 1 << l[k]
            j, p = level_pos(l[k], i)
            assert 0 <= b <= T and j <= n
            o += W * (R[k][j][b] + p)
            W <<= 1 if j == 0 else j - 1
            b -= max(j, 1)
            q = q1
        out2.append(o)
    out = []
    for e in range(nent):
        rr = umulhi(e, magb) if magb else e
        assert rr == e // nbud
        m = e - rr * nbud + 1
        o = 0
        if d > 1:
            row = row0 + rr
            plane = fdiv(row * n0, S[2]) if d > 2 else 0
            j1, p1 = level_pos(l[1], row - plane * n1)
            o = R[1][j1][T - m] + p1
            if d > 2:
                ei = (plane - plane0) * nb2 + m + max(j1, 1) - 2
                assert 0 <= ei < nent2
                o += out2[ei] << (1 if j1 == 0 else j1 - 1)
        out.append(o)
    pos = []
    for oo in range(npts):
        t = t0 + oo
        rr = div_row(t, n0, mag0)
        assert rr == t // n0
        j0, p0 = level_pos(l[0], t - rr * n0)
        ei = rr * nbud + max(j0, 1) - 1
        assert 0 <= ei < nent
        pos.append(R[0][j0][T] + p0 + (out[ei] << (1 if j0 == 0 else j0 - 1)))
    return pos


@pytest.mark.parametrize("d,n,sample", [(1, 6, None), (2, 5, None), (3, 4, None), (4, 4, None),
                                        (5, 3, None), (8, 2, None), (2, 9, None), (4, 14, 12)])
def test_scatter_index_model_matches_oracle(orc, d, n, sample):
    lv, _ = orc.scheme(d, n)
    R = build_rank(d, n)
    chunks = [(g, f0) for g, l in enumerate(lv) for f0 in range(0, orc.num_points(l), CHUNK)]
    if sample is not None:
        rng = np.random.default_rng(5)
        picks = set(int(v) for v in rng.integers(0, len(chunks), sample)) | {0, len(chunks) - 1}
        chunks = [chunks[i] for i in sorted(picks)]
    refs = {}
    M = orc.sparse_num_points(d, n)
    for g, f0 in chunks:
        l = [int(v) for v in lv[g]]
        if g not in refs:
            refs[g] = orc.sparse_index_of_grid(d, n, l)
        pos = chunk_positions(l, d, n, R, f0)
        assert max(pos) < M
        assert np.array_equal(np.array(pos), refs[g][f0:f0 + len(pos)])
