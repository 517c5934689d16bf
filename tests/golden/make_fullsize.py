"""Reference results for the benchmark workloads at full size, computed by the oracle only.

  swiss_roll_200k.json   200,000 swiss-roll points (seed 2), symmetric 10-NN, Gaussian
                         weights: eps = lambda_2(Q) (Sec. 4.2), mu (Eq. 9), ||A||_G,
                         max b_i, and the first K + 2 = 10 generalized eigenvalues of
                         (A, B) (Eq. 10-11), all in FP64.
  sphere_2m.json         2,000,000 points uniform on the unit sphere (seed 3), 10-NN: the
                         same quantities, first K + 2 = 18 eigenvalues.
  oracle/_cache/<key>.npz   the matching eigenvectors (n x 10 or n x 18 FP64: too large to
                         commit, so cached under a git-ignored folder keyed by the
                         workload and recomputed when missing).

Every value comes from oracle/: the operator build of Sec. 4 (graph_ops), eps by
shift-invert Lanczos on Q (graph_ops.fiedler_value_sparse) and the eigenpairs by
shift-invert Lanczos on B^{-1/2} A B^{-1/2} (eigen.sparse_geneig) -- both library
eigensolvers at machine precision, so the references carry no iteration tolerance of
their own.  About two minutes of CPU time for the 200k workload.

Run from the repository root:  python tests/golden/make_fullsize.py [name ...]
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import manifold_graphs as mg          # noqa: E402
from oracle import eigen as ge        # noqa: E402
from oracle import graph_ops as go    # noqa: E402

CACHE = os.path.join(ROOT, "oracle", "_cache")

# name -> (shape, n, k, seed, number of eigenpairs kept)
WORKLOADS = {
    "swiss_roll_200k": ("swiss_roll", 200_000, 10, 2, 10),
    "sphere_2m": ("sphere", 2_000_000, 10, 3, 18),
}


def key(name):
    shape, n, k, seed, K = WORKLOADS[name]
    h = hashlib.sha1(f"{shape}:{n}:{k}:{seed}:{K}:laplacian".encode()).hexdigest()[:12]
    return f"{name}_{h}"


def compute(name):
    """The oracle's FP64 reference for one workload: (summary dict, V[n, K])."""
    shape, n, k, seed, K = WORKLOADS[name]
    t0 = time.time()
    g = mg.manifold_graph(shape, n, k, seed)
    t_ptr, t_col, T = go.two_hop_sets(g.n, g.row_ptr, g.col)
    Q = go.q_matrix(g.n, t_ptr, t_col)
    ncomp = go.two_hop_components(g.n, t_ptr, t_col)
    eps, eps_res = go.fiedler_value_sparse(Q, ncomp)
    ops = go.build_graph_ops(g.n, g.row_ptr, g.col, g.w, eps_override=eps)
    res = ge.sparse_geneig(ops.A, ops.b, K)
    eta = ge.backward_errors(ops.A, ops.b, res.lam, res.V)
    summary = {
        "workload": name, "shape": shape, "n": n, "k": k, "seed": seed,
        "two_hop_components": ncomp, "eps": eps, "eps_residual": eps_res, "mu": ops.mu,
        "norm_a": ge.gershgorin_norm(ops.A), "bmax": float(np.max(ops.b)),
        "nnz_a": int(ops.a_col.shape[0]),
        "lam": res.lam.tolist(), "eta": eta.tolist(),
        "seconds": round(time.time() - t0, 1),
    }
    return summary, res.V


def load_or_compute(name, write_golden=False):
    """(summary, V) from the cache when present, else computed (and cached)."""
    path = os.path.join(CACHE, key(name) + ".npz")
    if os.path.exists(path):
        z = np.load(path)
        summary = json.loads(str(z["summary"]))
        V = z["V"]
    else:
        summary, V = compute(name)
        os.makedirs(CACHE, exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp.npz"
        np.savez(tmp, V=V, summary=json.dumps(summary))
        os.replace(tmp, path)
    if write_golden:
        with open(os.path.join(HERE, name + ".json"), "w") as f:
            json.dump(summary, f, indent=1)
    return summary, V


if __name__ == "__main__":
    for nm in (sys.argv[1:] or list(WORKLOADS)):
        s, _ = load_or_compute(nm, write_golden=True)
        print(nm, "eps", s["eps"], "lam", s["lam"][:4], "...", f"{s['seconds']} s")
