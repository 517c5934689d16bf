"""The benchmark workload at full size (200,000 swiss-roll points, 10-NN, K = 8, FP32 and
BF16 forms, relative residual 1e-5), checked against the oracle at that size:
  * the whole A / Q structure and the two-hop counts, bit-exact (oracle sparse build);
  * eps against the oracle's value by shift-invert Lanczos on Q (machine precision, its
    residual asserted), 2e-5 relative: the FP32 eps solve's tolerance;
  * ||A||_G and max b_i of the GPU build against the oracle's (same eps), 1e-12 relative;
  * the eigenvalues against the oracle's first K generalized eigenvalues of (A, B) by
    shift-invert Lanczos (Eq. 10-11), 1e-4 relative -- the reduced-precision tolerance;
  * each eigenvector against the oracle's (largest principal angle per eigenvalue cluster,
    relative gap < 1e-6), 1e-3 radians;
  * the returned pairs' backward errors, recomputed in FP64 by the oracle with its own A, B;
  * B-orthonormality V^T B V = I and the ascending order.
The oracle's reference comes from tests/golden/make_fullsize.py: its eigenvalues are
committed in tests/golden/swiss_roll_200k.json, its eigenvectors cached under the
git-ignored oracle/_cache/ and recomputed by the oracle (about two minutes) when absent.
"""
import importlib.util
import json
import os

import numpy as np
import pytest

import manifold_graphs as mg
from oracle import eigen as oe
from oracle import graph_ops as og

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _reference(name):
    spec = importlib.util.spec_from_file_location("make_fullsize", os.path.join(GOLDEN, "make_fullsize.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    summary, V = mod.load_or_compute(name)
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        committed = json.load(f)
    # the cache must hold the committed reference, not a stale one
    np.testing.assert_allclose(summary["lam"], committed["lam"], rtol=1e-12)
    return committed, V


def clusters(lam, rel=1e-6):
    out, cur = [], [0]
    for j in range(1, len(lam)):
        if abs(lam[j] - lam[j - 1]) <= rel * abs(lam[j]):
            cur.append(j)
        else:
            out.append(cur)
            cur = [j]
    out.append(cur)
    return out


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_config_swiss_roll_200k(gpu_lib, prec):
    K = 8
    ref_s, ref_V = _reference("swiss_roll_200k")
    assert ref_s["eps_residual"] < 1e-12          # the eps reference converged
    assert max(ref_s["eta"]) < 1e-12              # and so did its eigenpairs
    g = mg.manifold_graph("swiss_roll", 200_000, 10, 2)
    with gpu_lib.Context(0) as ctx:
        ops = ctx.build(g, precision=prec)
        info = ops.info()
        ex = ops.export()
        lam, V, ei, s = ctx.embed(ops, K, 1e-5, precision=prec)
        ops.close()
    assert s == 0
    assert np.all(np.asarray(ei.resid[:K]) <= 1e-5)     # the solver's own relative residual
    t_ptr, t_col, T = og.two_hop_sets(g.n, g.row_ptr, g.col)
    assert np.array_equal(ex["T"], T)
    a_ptr, a_col = og.a_structure(g.n, g.row_ptr, g.col, t_ptr, t_col)
    assert np.array_equal(ex["a_ptr"], a_ptr) and np.array_equal(ex["a_col"], a_col)
    # eps against the oracle's machine-precision value
    print("eps rel err", abs(info.eps - ref_s["eps"]) / ref_s["eps"])
    assert info.eps == pytest.approx(ref_s["eps"], rel=2e-5)
    assert info.mu == pytest.approx(ref_s["mu"], rel=2e-5)
    # the oracle's operators built with the GPU's eps: values, norms, residuals
    ref = og.build_graph_ops(g.n, g.row_ptr, g.col, g.w, eps_override=info.eps)
    np.testing.assert_allclose(ex["a_val"], ref.a_val, rtol=1e-12, atol=1e-16)
    assert info.norm_a == pytest.approx(oe.gershgorin_norm(ref.A), rel=1e-12)
    assert info.bmax == pytest.approx(float(np.max(ref.b)), rel=1e-12)
    eta = oe.backward_errors(ref.A, ref.b, lam, V)
    assert np.all(eta <= 2e-5), eta
    assert np.all(np.diff(lam) > 0)
    VBV = V.T @ (ref.b[:, None] * V)
    assert np.max(np.abs(VBV - np.eye(K))) < 1e-4
    # eigenpairs against the oracle's (computed with its own eps)
    ref_lam = np.array(ref_s["lam"][:K])
    rel = np.abs(lam - ref_lam) / ref_lam
    print("lambda rel err", rel)
    assert np.max(rel) <= 1e-4, rel
    angles = []
    for c in clusters(ref_s["lam"][:K + 1])[:]:
        c = [j for j in c if j < K]
        if not c:
            continue
        angles.append(oe.subspace_angle(V[:, c], ref_V[:, c]))
    print("angles", angles)
    assert max(angles) <= 1e-3, angles
