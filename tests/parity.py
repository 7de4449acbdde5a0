"""Error measures shared by the GPU parity tests.

The tolerances are relative to max|u|, u the nodal vector of the transform
(the reading of "relative to max|u|" for every operation):

- hierarchization and its transpose: u is the input;
- dehierarchization: u is its output, the nodal side (the reference output
  of the oracle);
- transpose of the dehierarchization: its output, the side that accumulates
  (every point collects half of each descendant's value, so a coarse point's
  output is a sum of up to 2^l terms, as every nodal value of the
  dehierarchization is a sum over its predecessors).

Bounds for composite steps (the gather of a combination scheme, a round of
the iterated combination technique) are derived from these per-point
tolerances and the combination coefficients, point by point; no test pads a
tolerance by a constant factor.
"""
import numpy as np

import oracle

TOL64 = 1e-13
TOL32 = 1e-5
EPS64 = 2.0 ** -53


def nodal_scale(u_in, ref, op):
    """max|u| of the nodal vector of op ('h', 'a': the input; 'd', 't': the
    reference output)."""
    side = ref if op in ("d", "t") else u_in
    return max(float(np.abs(np.asarray(side, dtype=np.float64)).max()) if np.size(side) else 0.0, 1e-300)


def rel_err(got, ref, u_in, op):
    """max|got - ref| / max|u| with u the nodal vector of op."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if got.size == 0:
        return 0.0
    return float(np.abs(got - ref).max()) / nodal_scale(u_in, ref, op)


def gather_weights(d, n, lv, c):
    """Per sparse point p: W(p) = sum over the grids holding p of |c_g| and
    K(p) = the number of those grids (both from the oracle's gather of
    constant grids, exact in fp64: small integers)."""
    ones = [np.ones(oracle.num_points(l)) for l in lv]
    W = oracle.gather(d, n, lv, np.abs(np.asarray(c, dtype=np.float64)), ones)
    K = oracle.gather(d, n, lv, np.ones(len(lv)), ones)
    return W, K


def gather_bound(d, n, lv, c, alphas, grid_err):
    """Pointwise bound on |gather(alpha + e) - gather(alpha)| when every
    surplus of grid g is off by at most grid_err[g]: the coefficients carry
    each error over, sum_g |c_g| grid_err[g], and the two fused
    multiply-add chains round differently by at most one unit in the last
    place of every partial sum (half a unit each), K(p) 2^-52 times a bound
    on the partial sums, sum_g |c_g alpha_g(p)| plus the carried error."""
    c = np.asarray(c, dtype=np.float64)
    per_grid = [np.full(oracle.num_points(l), float(e)) for l, e in zip(lv, grid_err)]
    carried = oracle.gather(d, n, lv, np.abs(c), per_grid)
    S = oracle.gather(d, n, lv, np.abs(c), [np.abs(a) for a in alphas])
    _, K = gather_weights(d, n, lv, c)
    return carried + K * 2.0 * EPS64 * (S + carried) + 1e-300
