"""Writes the stored expected values under tests/golden/ by calling only the oracle.

  mesh10.json   the 10-node, 18-edge triangle mesh of Fig. 3 (unit weights): two-hop
                sets, eps, mu, b and the first 4 generalized eigenpairs of (A, B).
  ring9.json    the odd ring C_9 (Fig. 2(b) generalised to 9 nodes): eps, mu and all
                generalized eigenvalues, which the closed form of Sec. 4 also fixes.

Run from the repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import manifold_graphs as mg          # noqa: E402
from oracle import graph_ops as go    # noqa: E402
from oracle import eigen as ge        # noqa: E402


def dump(name, g, K):
    ops = go.from_graph(g)
    res = ge.dense_geneig(ops.A, ops.b, K)
    out = {
        "graph": g.name, "n": g.n,
        "row_ptr": g.row_ptr.tolist(), "col": g.col.tolist(), "w": g.w.tolist(),
        "two_hop": [ops.t_col[ops.t_ptr[i]:ops.t_ptr[i + 1]].tolist() for i in range(g.n)],
        "eps": ops.eps, "mu": ops.mu, "b": ops.b.tolist(),
        "a_ptr": ops.a_ptr.tolist(), "a_col": ops.a_col.tolist(), "a_val": ops.a_val.tolist(),
        "lam": res.lam.tolist(), "V": res.V.tolist(),
    }
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    dump("mesh10.json", mg.triangle_mesh(), 4)
    dump("ring9.json", mg.ring(9), 9)
