"""Writes the golden fixtures of this folder.  Calls only the CPU oracle and
the seeded input generators; no value here comes from the GPU library.

    python tests/golden/make_golden.py

Fixtures (one float.hex value per line, flat order, dimension 0 fastest):
  cfg1a_{hierarchize,dehierarchize,adjoint}.txt
      2-D grid of level (5,5), u = uniform[-1,1] from PCG64 seed 0; the boundary
      form of Alg. 1 (Sec. 3), its inverse and its transpose.
  cfg1a_dehier_adjoint.txt
      the same grid: the transpose of the dehierarchization.
  cfg1b_hierarchize.txt
      the same grid, u = x^2 + 3xy; every value is dyadic, so this file is also
      the closed form (-4^{-j_x} on the y-boundary rows, 0 elsewhere, corners
      0, 1, 0, 4) and must be met bit for bit.
  scheme_2_4_gather.txt / scheme_2_4_scatter.txt
      the combination scheme d = 2, n = 4 (Sec. 2): every grid uniform[-1,1]
      from seed 1000 + grid index, hierarchized, gathered into the sparse grid
      (subspace-major layout); then that sparse grid scattered back onto the
      grids (grids concatenated in scheme order).
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1309_0392_gb300 import inputs  # noqa: E402


def write(name, values, header):
    with open(os.path.join(HERE, name), "w") as f:
        for line in header:
            f.write(f"# {line}\n")
        for v in values:
            f.write(float(v).hex() + "\n")


def main():
    levels, u = inputs.cfg1a()
    src = "level (5,5), uniform[-1,1] seed 0 (PCG64), flat order, dim 0 fastest"
    write("cfg1a_hierarchize.txt", oracle.hierarchize(u, levels),
          ["hierarchize: Alg. 1 (Sec. 3), boundary form", src])
    write("cfg1a_dehierarchize.txt", oracle.dehierarchize(u, levels),
          ["dehierarchize: inverse of Alg. 1 (Sec. 2, iterated combination technique)", src])
    write("cfg1a_adjoint.txt", oracle.hierarchize_adjoint(u, levels),
          ["hierarchize adjoint: transpose of Alg. 1", src])
    write("cfg1a_dehier_adjoint.txt", oracle.dehierarchize_adjoint(u, levels),
          ["dehierarchize adjoint: transpose of the inverse of Alg. 1", src])
    levels, u = inputs.cfg1b()
    write("cfg1b_hierarchize.txt", oracle.hierarchize(u, levels),
          ["hierarchize of x^2 + 3xy on level (5,5): closed form, dyadic, bit-exact"])
    d, n = 2, 4
    lv, c = oracle.scheme(d, n)
    alphas = [oracle.hierarchize(inputs.scheme_grid(l, 1000 + g), l) for g, l in enumerate(lv)]
    sparse = oracle.gather(d, n, lv, c, alphas)
    src = "scheme d=2 n=4 (Sec. 2), grids uniform[-1,1] seed 1000 + grid index, hierarchized"
    write("scheme_2_4_gather.txt", sparse, ["gather into the sparse grid, subspace-major", src])
    back = oracle.scatter(d, n, lv, c, sparse)
    write("scheme_2_4_scatter.txt", [v for b in back for v in b],
          ["scatter of that sparse grid onto the grids, concatenated in scheme order", src])


if __name__ == "__main__":
    main()
