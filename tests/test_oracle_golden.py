"""The oracle reproduces the committed golden fixtures bit for bit, and the
closed-form fixture is the closed form (CPU only)."""
import numpy as np

from golden_io import load
from paper_1309_0392_gb300 import inputs


def test_cfg1a_golden(orc):
    levels, u = inputs.cfg1a()
    assert np.array_equal(orc.hierarchize(u, levels), load("cfg1a_hierarchize.txt"))
    assert np.array_equal(orc.dehierarchize(u, levels), load("cfg1a_dehierarchize.txt"))
    assert np.array_equal(orc.hierarchize_adjoint(u, levels), load("cfg1a_adjoint.txt"))
    assert np.array_equal(orc.dehierarchize_adjoint(u, levels), load("cfg1a_dehier_adjoint.txt"))


def test_scheme_gather_and_scatter_golden(orc):
    d, n = 2, 4
    lv, c = orc.scheme(d, n)
    alphas = [orc.hierarchize(inputs.scheme_grid(l, 1000 + g), l) for g, l in enumerate(lv)]
    sparse = orc.gather(d, n, lv, c, alphas)
    assert np.array_equal(sparse, load("scheme_2_4_gather.txt"))
    back = np.concatenate(orc.scatter(d, n, lv, c, sparse))
    assert np.array_equal(back, load("scheme_2_4_scatter.txt"))


def test_cfg1b_golden_is_closed_form(orc):
    levels, u = inputs.cfg1b()
    g = load("cfg1b_hierarchize.txt").reshape(33, 33)      # [y, x]
    expect = np.zeros((33, 33))
    for ix in range(1, 32):
        j = 5 - ((ix & -ix).bit_length() - 1)
        expect[0, ix] = expect[32, ix] = -(4.0 ** -j)
    expect[0, 0], expect[0, 32], expect[32, 0], expect[32, 32] = 0.0, 1.0, 0.0, 4.0
    assert np.array_equal(g, expect)
    assert np.array_equal(orc.hierarchize(u, levels), g.reshape(-1))
