"""The dyadic split that the GPU uses for one long pole, checked on the CPU
with the oracle as the 1-D transform: hierarchizing every block of level m
(end points shared, read only) and then the coarse pole of the multiples of
2^m gives the oracle's transform of the whole pole bit for bit, and the
inverse runs the two parts in the opposite order.  Block level as on the
GPU: m = max(13, L - 14).  CPU only."""
import numpy as np
import pytest


def split_transform(orc, u, L, op):
    m = max(13, L - 14)
    bm, nblk = 1 << m, 1 << (L - m)
    one = orc.hierarchize if op == "h" else orc.dehierarchize
    v = u.copy()

    def blocks():
        for a in range(nblk):
            seg = one(v[a * bm:(a + 1) * bm + 1].copy(), (m,))
            assert seg[0] == v[a * bm] and seg[-1] == v[(a + 1) * bm]   # end points untouched
            v[a * bm + 1:(a + 1) * bm] = seg[1:-1]

    def coarse():
        v[::bm] = one(v[::bm].copy(), (L - m,))

    if op == "h":
        blocks()
        coarse()
    else:
        coarse()
        blocks()
    return v


@pytest.mark.parametrize("L", [15, 17, 20])
@pytest.mark.parametrize("op", ["h", "d"])
def test_long_pole_split_equals_whole_transform(orc, L, op):
    u = np.random.default_rng(L).uniform(-1, 1, (1 << L) + 1)
    whole = (orc.hierarchize if op == "h" else orc.dehierarchize)(u, (L,))
    assert np.array_equal(split_transform(orc, u, L, op), whole)
