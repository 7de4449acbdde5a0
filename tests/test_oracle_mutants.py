"""Planted mistakes in the oracle: each mutant of gbh_oracle.c (a flipped sign,
a shifted index, a wrong loop bound or order, a wrong stride) is compiled on
the CPU and must fail at least one of the independent pins (hat-basis brute
force against Phi, Phi^-1 and their transposes; for the sparse grid, the coordinate
dictionary and the transpose identity).  Shows that the pins can catch a
plausible error anywhere in the sweeps, the gather and the scatter.  CPU only."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from test_oracle_pins import _coord_key, _sparse_layout, hat_matrix

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "gbh_oracle.c")

MUTANTS = {
    "hier_sign": ("u[i * S] = u[i * S] - 0.5 * (u[(i - s) * S] + u[(i + s) * S]);",
                  "u[i * S] = u[i * S] + 0.5 * (u[(i - s) * S] + u[(i + s) * S]);"),
    "hier_dropped_right": ("u[i * S] = u[i * S] - 0.5 * (u[(i - s) * S] + u[(i + s) * S]);",
                           "u[i * S] = u[i * S] - 0.5 * (u[(i - s) * S] + u[(i - s) * S]);"),
    "hier_paper_bound": ("    for (int lev = l; lev >= 1; --lev) {\n        const int64_t s = (int64_t)1 << (l - lev);\n        for (int64_t i = s; i < last; i += 2 * s)\n            u[i * S] = u[i * S] - 0.5",
                         "    for (int lev = l; lev >= 2; --lev) {\n        const int64_t s = (int64_t)1 << (l - lev);\n        for (int64_t i = s; i < last; i += 2 * s)\n            u[i * S] = u[i * S] - 0.5"),
    "hier_wrong_order": ("    for (int lev = l; lev >= 1; --lev) {\n        const int64_t s = (int64_t)1 << (l - lev);\n        for (int64_t i = s; i < last; i += 2 * s)\n            u[i * S] = u[i * S] - 0.5",
                         "    for (int lev = 1; lev <= l; ++lev) {\n        const int64_t s = (int64_t)1 << (l - lev);\n        for (int64_t i = s; i < last; i += 2 * s)\n            u[i * S] = u[i * S] - 0.5"),
    "dehier_wrong_order": ("    for (int lev = 1; lev <= l; ++lev) {\n        const int64_t s = (int64_t)1 << (l - lev);\n        for (int64_t i = s; i < last; i += 2 * s)\n            u[i * S] = u[i * S] + 0.5",
                           "    for (int lev = l; lev >= 1; --lev) {\n        const int64_t s = (int64_t)1 << (l - lev);\n        for (int64_t i = s; i < last; i += 2 * s)\n            u[i * S] = u[i * S] + 0.5"),
    "adjoint_wrong_order": ("    for (int lev = 1; lev <= l; ++lev) {\n        const int64_t s = (int64_t)1 << (l - lev);\n        for (int64_t i = s; i < last; i += 2 * s) {\n            y[(i - s) * S]",
                            "    for (int lev = l; lev >= 1; --lev) {\n        const int64_t s = (int64_t)1 << (l - lev);\n        for (int64_t i = s; i < last; i += 2 * s) {\n            y[(i - s) * S]"),
    "adjoint_one_parent": ("            y[(i + s) * S] = y[(i + s) * S] - 0.5 * y[i * S];",
                           "            y[(i - s) * S] = y[(i - s) * S] - 0.5 * y[i * S];"),
    "stride_off_by_one": ("for (int m = 0; m < k && m < d; ++m)", "for (int m = 0; m <= k && m < d; ++m)"),
    "dehier_adjoint_wrong_order": ("    for (int lev = l; lev >= 1; --lev) {\n        const int64_t s = (int64_t)1 << (l - lev);\n        for (int64_t i = s; i < last; i += 2 * s) {\n            y[(i - s) * S] = y[(i - s) * S] + 0.5",
                                   "    for (int lev = 1; lev <= l; ++lev) {\n        const int64_t s = (int64_t)1 << (l - lev);\n        for (int64_t i = s; i < last; i += 2 * s) {\n            y[(i - s) * S] = y[(i - s) * S] + 0.5"),
    "dehier_adjoint_sign": ("            y[(i + s) * S] = y[(i + s) * S] + 0.5 * y[i * S];",
                            "            y[(i + s) * S] = y[(i + s) * S] - 0.5 * y[i * S];"),
}

# mistakes in the sparse-grid index, the gather and the scatter (every mutant
# keeps its indexes inside the arrays)
SPARSE_MUTANTS = {
    "boundary_positions_swapped": ("if (i == 0) { *j = 0; *p = 0; return; }",
                                   "if (i == 0) { *j = 0; *p = 1; return; }"),
    "position_dims_reversed": ("        for (int k = 0; k < d; ++k) {\n            pos += p[k] * mul;",
                               "        for (int k = d - 1; k >= 0; --k) {\n            pos += p[k] * mul;"),
    "gather_drops_coefficient": ("sparse[idx[f]] = fma(coeffs[g], grids[g][f], sparse[idx[f]]);",
                                 "sparse[idx[f]] = grids[g][f] + sparse[idx[f]];"),
    "scatter_ignores_scale": ("grids[g][f] = scaled ? coeffs[g] * sparse[idx[f]] : sparse[idx[f]];",
                              "grids[g][f] = sparse[idx[f]];"),
}

LEVELS = [(3,), (2, 3), (2, 1, 2)]


def _compile(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           str(path), "-o", str(so), "-lm"])
    lib = ctypes.CDLL(str(so))
    for fn in ("orc_hierarchize", "orc_dehierarchize", "orc_hierarchize_adjoint", "orc_dehierarchize_adjoint"):
        getattr(lib, fn).argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_int)]
    return lib


def _run(lib, fn, u, levels):
    out = np.array(u, dtype=np.float64, copy=True)
    lv = np.array(levels, dtype=np.int32)
    getattr(lib, fn)(out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(levels),
                     lv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return out


def _pins_hold(lib):
    rng = np.random.default_rng(0)
    for levels in LEVELS:
        phi = hat_matrix(list(levels))
        u = rng.uniform(-1, 1, phi.shape[0])
        if np.abs(_run(lib, "orc_hierarchize", u, levels) - np.linalg.solve(phi, u)).max() > 1e-12:
            return False
        if np.abs(_run(lib, "orc_dehierarchize", u, levels) - phi @ u).max() > 1e-12:
            return False
        if np.abs(_run(lib, "orc_hierarchize_adjoint", u, levels) - np.linalg.solve(phi.T, u)).max() > 1e-12:
            return False
        if np.abs(_run(lib, "orc_dehierarchize_adjoint", u, levels) - phi.T @ u).max() > 1e-12 * np.abs(phi.T @ u).max():
            return False
    return True


_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)


def _sparse_pins_hold(lib):
    """Gather and scatter of the schemes (2, 3) and (3, 3) against the
    coordinate dictionary, and the scaled scatter against the transpose of
    the gather."""
    lib.orc_scheme_count.restype = ctypes.c_int
    lib.orc_sparse_num_points.restype = ctypes.c_int64
    lib.orc_num_points.restype = ctypes.c_int64
    for d, n in [(2, 3), (3, 3)]:
        G = lib.orc_scheme_count(d, n)
        lv = np.zeros((G, d), dtype=np.int32)
        c = np.zeros(G)
        lib.orc_scheme_levels(d, n, lv.ctypes.data_as(_IP), c.ctypes.data_as(_DP))
        M = int(lib.orc_sparse_num_points(d, n))
        layout = _sparse_layout(d, n)
        where = {x: q for q, (_, _, x) in enumerate(layout)}
        rng = np.random.default_rng(21)
        alphas = [rng.integers(-8, 9, int(np.prod([2 ** v + 1 for v in l]))).astype(np.float64) for l in lv]
        s = rng.integers(-8, 9, M).astype(np.float64)
        # gather against a dictionary keyed by exact coordinates
        sparse = np.zeros(M)
        ptrs = (_DP * G)(*[a.ctypes.data_as(_DP) for a in alphas])
        lib.orc_gather(d, n, G, lv.ctypes.data_as(_IP), c.ctypes.data_as(_DP), ptrs, sparse.ctypes.data_as(_DP))
        acc = {}
        for l, cg, a in zip(lv, c, alphas):
            for f in range(a.size):
                acc[_coord_key(l, f)] = acc.get(_coord_key(l, f), 0.0) + cg * a[f]
        if any(sparse[q] != acc[x] for x, q in where.items()):
            return False
        for scaled in (0, 1):
            outs = [np.zeros(a.size) for a in alphas]
            optrs = (_DP * G)(*[o.ctypes.data_as(_DP) for o in outs])
            lib.orc_scatter(d, n, G, lv.ctypes.data_as(_IP), c.ctypes.data_as(_DP), scaled,
                            s.ctypes.data_as(_DP), optrs)
            for l, cg, o in zip(lv, c, outs):
                for f in range(o.size):
                    v = s[where[_coord_key(l, f)]]
                    if o[f] != (cg * v if scaled else v):
                        return False
            if scaled and np.dot(sparse, s) != sum(np.dot(a, o) for a, o in zip(alphas, outs)):
                return False
    return True


def test_unmutated_source_passes(tmp_path):
    lib = _compile(tmp_path, "clean", "/* grid geometry", "/* grid geometry")
    assert _pins_hold(lib)
    assert _sparse_pins_hold(lib)


@pytest.mark.parametrize("name", sorted(SPARSE_MUTANTS))
def test_sparse_mutant_is_caught(tmp_path, name):
    old, new = SPARSE_MUTANTS[name]
    lib = _compile(tmp_path, name, old, new)
    assert not _sparse_pins_hold(lib), f"planted mistake {name} escaped the pins"


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    lib = _compile(tmp_path, name, old, new)
    assert not _pins_hold(lib), f"planted mistake {name} escaped the pins"
