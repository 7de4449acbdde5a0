"""Planted mistakes in the oracle: each mutant of gbh_oracle.c (a flipped sign,
a shifted index, a wrong loop bound or order, a wrong stride) is compiled on
the CPU and must fail at least one of the independent pins (hat-basis brute
force, round trip, dot product).  Shows that the pins can catch a plausible
error anywhere in the sweeps.  CPU only."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from test_oracle_pins import hat_matrix

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
    for fn in ("orc_hierarchize", "orc_dehierarchize", "orc_hierarchize_adjoint"):
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
    return True


def test_unmutated_source_passes(tmp_path):
    lib = _compile(tmp_path, "clean", "/* grid geometry", "/* grid geometry")
    assert _pins_hold(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    lib = _compile(tmp_path, name, old, new)
    assert not _pins_hold(lib), f"planted mistake {name} escaped the pins"
