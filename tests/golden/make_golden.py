"""Writes the stored expected values in this folder from the CPU oracle.

Only `oracle/` computes them (the input generator `meshgen` supplies the
seeded inputs); nothing here touches the CUDA library. Run from the
repository root:

    python tests/golden/make_golden.py

Files (plain text, one node per line, %.17e so that doubles round-trip):
  rhs_kuhn8_lex.txt  the assembled RHS [N=729 lines] x (u, v, w, p) rows of the
                     8x8x8-hex unit cube (6 Kuhn tets per hex, 3072 tets),
                     interior nodes jittered by U(-0.1 h, 0.1 h) (seed 1),
                     lexicographic node order, Taylor-Green velocity plus
                     N(0, 1e-2) noise and p ~ U(-1, 1) (seed 2), rho 1,
                     mu 1e-2, no Vreman model; the stabilised P1 weak form of
                     the explicit momentum step (Sec. II, V-A, V-B) with the
                     4-point rule.
  vjp_kuhn8_lex.txt  (d RHS / d up)^T w on the same mesh and state for the
                     cotangent w ~ N(0, 1) (seed 4), from the oracle's
                     complex-step element Jacobians.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import meshgen as mg  # noqa: E402
import oracle  # noqa: E402


def write(path, header, a):
    with open(path, "w") as f:
        for line in header.strip().splitlines():
            f.write("# " + line + "\n")
        for row in a.T:
            f.write(" ".join("%.17e" % x for x in row) + "\n")


def main():
    w = mg.tiny()
    rhs = oracle.assemble(w.coords, w.conn, w.up, w.rho, w.mu)
    write(os.path.join(HERE, "rhs_kuhn8_lex.txt"),
          "RHS of the 8^3-hex Kuhn mesh (see make_golden.py); columns u v w p; "
          "written by the oracle", rhs)
    cot = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
    g = oracle.vjp(w.coords, w.conn, w.up, cot, w.rho, w.mu)
    write(os.path.join(HERE, "vjp_kuhn8_lex.txt"),
          "(dRHS/dup)^T w on the 8^3-hex Kuhn mesh, w ~ N(0,1) seed 4 (see make_golden.py); "
          "columns u v w p; written by the oracle", g)


if __name__ == "__main__":
    main()
