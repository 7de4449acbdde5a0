"""CPU model of the plain path's pair kernel (two consecutive dimensions per
pass): the host's tile choice, and the kernel's copy, pole and store index
maps replayed in numpy for every CTA of small shapes.  Checks that every
access stays inside the shared tile and the grid, that each grid element is
loaded and stored exactly once per pass, that the 16-byte pieces are aligned
on both sides, that each pole the kernel forms is a pole of the grid, and
that sweeping the modelled poles with the oracle's 1-D transforms gives the
oracle's d-dimensional result."""
import numpy as np
import pytest

import oracle
from paper_1309_0392_gb300 import inputs

THREADS = 256
PAIR_BYTES = 104 * 1024


def max_level(es):
    return 6 if es == 4 else 5


def pair_tile(levels, k, es, batch=1):
    """Planes per CTA (k = 0) or bundle width (k >= 1); 0 = no pair."""
    d = len(levels)
    if k + 1 >= d:
        return 0
    la, lb = levels[k], levels[k + 1]
    if la < 1 or lb < 1 or la > max_level(es) or lb > max_level(es):
        return 0
    M = (2 ** la + 1) * (2 ** lb + 1)
    cap = PAIR_BYTES // es
    if k == 0:
        Q = (cap - 16 // es) // M
        return min(Q, 256) if Q >= 1 else 0
    Sa = int(np.prod([2 ** l + 1 for l in levels[:k]]))
    B = 128
    while B > 8 and (B * M > cap or B > Sa):
        B >>= 1
    return B if (B * M <= cap and B <= Sa) else 0


def square_run(es, L):
    """Positions per CTA of the square kernel: runs of at least 64 bytes, and
    for short poles as many positions as keep the CTA near 256 threads."""
    n = 2 ** L + 1
    by_threads = 4
    for b in (64, 32, 16, 8):
        if 256 // n >= b:
            by_threads = b
            break
    return max(64 // es, by_threads)


def square_fits(levels, k, es):
    """The square kernel's test: outer pair of equal levels in [1, 5] with at
    least one run of positions below it."""
    if not (k >= 1 and k + 1 < len(levels) and levels[k] == levels[k + 1] and 1 <= levels[k] <= 5):
        return False
    Sa = int(np.prod([2 ** l + 1 for l in levels[:k]]))
    return Sa >= square_run(es, levels[k])


def passes(levels, es):
    """The plain path's passes: ('square', k), ('pair', k, Q) or ('single', k)."""
    out, k = [], 0
    while k < len(levels):
        if levels[k] == 0:
            k += 1
            continue
        if square_fits(levels, k, es):
            out.append(("square", k))
            k += 2
            continue
        Q = pair_tile(levels, k, es)
        if Q:
            out.append(("pair", k, Q))
            k += 2
        else:
            out.append(("single", k))
            k += 1
    return out


def ctas_rows(levels, Q, es, batch, misalign):
    """Per CTA of a plane pass: the copies (shared index, grid index, width
    in elements, as arrays), the poles of dimensions 0 and 1 (shared indices,
    one row per pole) and the tile's size; misalign = the grid pointer's
    offset from a 16-byte boundary, in elements."""
    na, nb = 2 ** levels[0] + 1, 2 ** levels[1] + 1
    M = na * nb
    total = batch * int(np.prod([2 ** l + 1 for l in levels]))
    planes = total // M
    VEC = 16 // es
    for b in range((planes + Q - 1) // Q):
        p0 = b * Q
        Qc = min(Q, planes - p0)
        cnt = Qc * M
        g0 = p0 * M
        mis = (misalign + g0) % VEC
        head = min(cnt, (VEC - mis) % VEC)
        body = (cnt - head) // VEC
        tail = head + body * VEC
        e = np.concatenate([np.arange(head), head + VEC * np.arange(body), np.arange(tail, cnt)])
        w = np.concatenate([np.ones(head, np.int64), np.full(body, VEC), np.ones(cnt - tail, np.int64)])
        q = np.arange(Qc * nb)
        poles_a = mis + q[:, None] * na + np.arange(na)[None, :]
        q = np.arange(Qc * na)
        poles_b = mis + (q // na)[:, None] * M + (q % na)[:, None] + na * np.arange(nb)[None, :]
        yield (mis + e, g0 + e, w), poles_a, poles_b, Q * M + VEC


def ctas_bundles(levels, k, B, es, batch):
    """Per CTA of a bundle pass over dimensions (k, k+1): as ctas_rows."""
    na, nb = 2 ** levels[k] + 1, 2 ** levels[k + 1] + 1
    M = na * nb
    Sa = int(np.prod([2 ** l + 1 for l in levels[:k]]))
    total = batch * int(np.prod([2 ** l + 1 for l in levels]))
    outer = total // (Sa * M)
    bpo = (Sa + B - 1) // B
    lgB = B.bit_length() - 1
    assert THREADS % B == 0
    w_all = np.arange(B * M)
    for blk in range(outer * bpo):
        o, jb = divmod(blk, bpo)
        j0 = jb * B
        Bc = min(B, Sa - j0)
        g = o * Sa * M + j0
        # thread tid copies w = tid, tid + THREADS, ... with r = w >> lgB
        # (its jj = tid & (B - 1) is fixed because B divides THREADS)
        jj, r = w_all & (B - 1), w_all >> lgB
        keep = jj < Bc
        sidx = w_all[keep]
        gidx = g + jj[keep] + Sa * r[keep]
        qa = np.arange(B * nb)
        qa = qa[(qa & (B - 1)) < Bc]
        poles_a = ((qa >> lgB) * na * B + (qa & (B - 1)))[:, None] + B * np.arange(na)[None, :]
        qb = np.arange(B * na)
        qb = qb[(qb & (B - 1)) < Bc]
        poles_b = ((qb >> lgB) * B + (qb & (B - 1)))[:, None] + na * B * np.arange(nb)[None, :]
        yield (sidx, gidx, np.ones(sidx.size, np.int64)), poles_a, poles_b, B * M


SHAPES = [(6, 6), (3, 4), (5, 5, 5, 5), (1, 1, 1, 1, 1, 1), (2, 6, 6), (4, 2, 6, 5, 1), (7, 3, 3),
          (0, 5, 5), (5, 0, 5), (2, 3, 2, 3, 2, 3), (1, 1, 4, 4, 4, 4)]


def test_pass_plan_matches_gpu_test_table():
    """The pair counts the GPU launch test expects follow from this model."""
    import test_gpu_pair as tg
    for levels, p32, p64 in tg.SHAPES:
        assert sum(p[0] != "single" for p in passes(levels, 4)) == p32, levels
        assert sum(p[0] != "single" for p in passes(levels, 8)) == p64, levels


def test_headline_fp32_plan():
    """(6,6,5,5,5) in fp32: planes of 65 x 65 (six per CTA), the square
    kernel for dimensions (2, 3), dimension 4 alone: three passes."""
    assert passes((6, 6, 5, 5, 5), 4) == [("pair", 0, 6), ("square", 2), ("single", 4)]


@pytest.mark.parametrize("levels", SHAPES + [(6, 6, 5, 5, 5)[:2] + (2, 2)])
@pytest.mark.parametrize("es", [4, 8])
@pytest.mark.parametrize("batch,misalign", [(1, 0), (2, 1), (3, 3)])
def test_index_maps(levels, es, batch, misalign):
    if es == 8:
        misalign %= 2
    N = int(np.prod([2 ** l + 1 for l in levels]))
    total = batch * N
    shape = (batch,) + tuple(2 ** l + 1 for l in reversed(levels))
    for p in passes(levels, es):
        if p[0] == "square":
            check_square_maps(levels, p[1], es, batch, shape, total)
            continue
        if p[0] != "pair":
            continue
        _, k, Q = p
        # flat global index of every element, as the grid's coordinates
        cover = np.zeros(total, dtype=np.int64)
        it = ctas_rows(levels, Q, es, batch, misalign) if k == 0 else ctas_bundles(levels, k, Q, es, batch)
        for (S, G, W), pa, pb, smem_elems in it:
            assert (S >= 0).all() and (S + W <= smem_elems).all()
            assert (G >= 0).all() and (G + W <= total).all()
            vec = W > 1
            assert ((S[vec] * es) % 16 == 0).all() and (((misalign + G[vec]) * es) % 16 == 0).all()
            # expand the pieces into single elements
            rep = np.repeat(np.arange(S.size), W)
            off = np.arange(rep.size) - np.repeat(np.cumsum(W) - W, W)
            se, ge = S[rep] + off, G[rep] + off
            np.add.at(cover, ge, 1)
            s2g = np.full(smem_elems, -1, dtype=np.int64)
            s2g[se] = ge
            # each pole lies in the tile and is a whole pole of the grid
            # along dimension k (pa) or k + 1 (pb)
            for poles, dim in ((pa, k), (pb, k + 1)):
                if poles.size == 0:
                    continue
                gs = s2g[poles]
                assert (gs >= 0).all()
                co = np.stack(np.unravel_index(gs, shape))        # (axes, poles, points)
                axis = len(levels) - dim                           # numpy axis of dimension dim
                step = np.diff(co, axis=2)
                want = np.zeros(len(shape), dtype=np.int64)
                want[axis] = 1
                assert (step == want[:, None, None]).all()
                assert (co[axis, :, 0] == 0).all() and gs.shape[1] == shape[axis]
        assert (cover == 1).all()


def ctas_square(levels, k, es, batch):
    """Per CTA of the square kernel: for phase a the (grid index, shared
    index) of every thread's pole, one row per thread, and for phase b the
    (shared index, grid index) rows."""
    n = 2 ** levels[k] + 1
    B = square_run(es, levels[k])
    Sa = int(np.prod([2 ** l + 1 for l in levels[:k]]))
    total = batch * int(np.prod([2 ** l + 1 for l in levels]))
    bpo = (Sa + B - 1) // B
    blocks = total // (Sa * n * n) * bpo
    tid = np.arange(B * n)
    jj, q = tid & (B - 1), tid // B
    i = np.arange(n)[None, :]
    for blk in range(blocks):
        o, jb = divmod(blk, bpo)
        j0 = jb * B
        act = j0 + jj < Sa
        g = o * Sa * n * n + j0 + jj[act][:, None]
        qa, ja = q[act][:, None], jj[act][:, None]
        a_glob = g + Sa * n * qa + Sa * i
        a_sm = (qa * n + i) * B + ja
        b_sm = (i * n + qa) * B + ja
        b_glob = g + Sa * qa + Sa * n * i
        yield (a_glob, a_sm), (b_sm, b_glob), B * n * n


def check_square_maps(levels, k, es, batch, shape, total):
    rd = np.zeros(total, dtype=np.int64)
    wr = np.zeros(total, dtype=np.int64)
    for (a_glob, a_sm), (b_sm, b_glob), smem in ctas_square(levels, k, es, batch):
        assert (a_glob >= 0).all() and (a_glob < total).all() and (b_glob >= 0).all() and (b_glob < total).all()
        assert (a_sm >= 0).all() and (a_sm < smem).all() and (b_sm >= 0).all() and (b_sm < smem).all()
        np.add.at(rd, a_glob.ravel(), 1)
        np.add.at(wr, b_glob.ravel(), 1)
        # phase b reads every shared slot phase a wrote, for the same grid point
        s2g = np.full(smem, -1, dtype=np.int64)
        s2g[a_sm.ravel()] = a_glob.ravel()
        assert (s2g[b_sm] == b_glob).all()
        for rows, dim in ((a_glob, k), (b_glob, k + 1)):
            co = np.stack(np.unravel_index(rows, shape))
            axis = len(levels) - dim
            want = np.zeros(len(shape), dtype=np.int64)
            want[axis] = 1
            assert (np.diff(co, axis=2) == want[:, None, None]).all()
            assert (co[axis, :, 0] == 0).all() and rows.shape[1] == shape[axis]
    assert (rd == 1).all() and (wr == 1).all()


def apply_square_model(u, levels, k, es, op1d):
    out = u.copy()
    for (a_glob, a_sm), (b_sm, b_glob), smem in ctas_square(levels, k, es, 1):
        sm = np.full(smem, np.nan)
        for gr, sr in zip(a_glob, a_sm):
            sm[sr] = op1d(out[gr].copy(), levels[k])
        for sr, gr in zip(b_sm, b_glob):
            out[gr] = op1d(sm[sr].copy(), levels[k + 1])
    return out


def apply_pass_model(u, levels, k, Q, es, op1d):
    """One pair pass replayed through the modelled maps: each CTA's tile
    gathered, its poles swept with the 1-D transform, the tile stored."""
    out = u.copy()
    it = ctas_rows(levels, Q, es, 1, 0) if k == 0 else ctas_bundles(levels, k, Q, es, 1)
    for (S, G, W), pa, pb, smem_elems in it:
        sm = np.full(smem_elems, np.nan)
        rep = np.repeat(np.arange(S.size), W)
        off = np.arange(rep.size) - np.repeat(np.cumsum(W) - W, W)
        se, ge = S[rep] + off, G[rep] + off
        sm[se] = out[ge]
        for poles, dim in ((pa, k), (pb, k + 1)):
            for pole in poles:
                sm[pole] = op1d(sm[pole].copy(), levels[dim])
        out[ge] = sm[se]
    return out


@pytest.mark.parametrize("levels", [(3, 4), (2, 2, 3, 1), (4, 2, 3, 2, 1), (1, 3, 3, 2), (2, 1, 3, 3), (3, 2, 2, 2, 2)])
@pytest.mark.parametrize("op", ["h", "d"])
def test_pass_model_reproduces_oracle(levels, op):
    op1d = {"h": lambda v, l: oracle.hierarchize(v, (l,)), "d": lambda v, l: oracle.dehierarchize(v, (l,))}[op]
    ref = {"h": oracle.hierarchize, "d": oracle.dehierarchize}[op]
    u = inputs.uniform(levels, 77)
    out = u.copy()
    N = u.size
    shape = tuple(2 ** l + 1 for l in reversed(levels))
    for p in passes(levels, 8):
        if p[0] == "square":
            out = apply_square_model(out, levels, p[1], 8, op1d)
        elif p[0] == "pair":
            out = apply_pass_model(out, levels, p[1], p[2], 8, op1d)
        else:
            k = p[1]
            a = out.reshape(shape)
            a = np.apply_along_axis(lambda v: op1d(v.copy(), levels[k]), len(levels) - 1 - k, a)
            out = a.reshape(N)
    np.testing.assert_allclose(out, ref(u, levels), rtol=0, atol=1e-13)
