"""Autotuning of the Chebyshev step (mge_ctx_set_autotune): a new shape is timed in every
configuration and the fastest is kept, in the context and in its JSON cache file; a cache
file forces a configuration; every configuration gives the same pairs (they compute the same
values in the same order; the Grams' cross-cluster FP64 atomics leave run-to-run differences
at rounding level).
"""
import json

import numpy as np
import pytest

import manifold_graphs as mg

pytestmark = pytest.mark.gpu

BUDGETS = {32768, 49152, 65536, 98304}


@pytest.fixture(scope="module")
def graph():
    return mg.manifold_graph("swiss_roll", 20000, 10, 41)


def embed(gpu_lib, g, mode, path=None, K=8):
    from paper_2112_07862_gb300 import mge
    c = gpu_lib.Context(0)
    try:
        mge.mge_ctx_set_autotune(c.h, mode, path)
        ops = c.build(g, precision="fp32")
        lam, V, info, s = c.embed(ops, K, 1e-5, precision="fp32")
        ops.close()
        st = c.stats()
        return lam, V, info, s, st.tune_entries
    finally:
        c.close()


def test_new_shapes_are_tuned_and_cached(gpu_lib, graph, tmp_path):
    path = str(tmp_path / "tune.json")
    lam, V, info, s, n_entries = embed(gpu_lib, graph, 1, path)
    assert s == 0
    d = json.load(open(path))
    # the embedding (m = 16) and the eps solve (m = 8) each tuned their shape
    assert n_entries == len(d) >= 2
    keys = sorted(d)
    assert any(k.startswith("cheb/m16/f32/n2^14/") for k in keys), keys
    assert any(k.startswith("cheb/m8/f32/n2^14/") for k in keys), keys
    for k, e in d.items():
        assert e["budget"] in BUDGETS and e["prefetch"] in (0, 1) and e["us"] > 0, (k, e)
    # a second context reading the cache tunes nothing new for the same graph
    lam2, V2, info2, s2, n2 = embed(gpu_lib, graph, 1, path)
    assert s2 == 0 and n2 == len(d) and json.load(open(path)) == d


@pytest.mark.parametrize("budget,prefetch", [(32768, 1), (98304, 0), (49152, 1)])
def test_every_configuration_gives_the_same_pairs(gpu_lib, graph, tmp_path, budget, prefetch):
    lam0, V0, info0, s0, _ = embed(gpu_lib, graph, 0)
    assert s0 == 0
    # learn the keys of this graph, then force one configuration for all of them
    learn = str(tmp_path / "learn.json")
    embed(gpu_lib, graph, 1, learn)
    forced = {k: {"budget": budget, "prefetch": prefetch, "us": 1.0} for k in json.load(open(learn))}
    path = str(tmp_path / "forced.json")
    json.dump(forced, open(path, "w"))
    lam, V, info, s, n_entries = embed(gpu_lib, graph, 2, path)
    assert s == 0 and n_entries == len(forced)
    assert json.load(open(path)) == forced          # mode 2 adds nothing
    assert abs(info.iters - info0.iters) <= 1
    np.testing.assert_allclose(lam, lam0, rtol=1e-7)
    for k in range(V.shape[1]):
        assert abs(abs(float(V[:, k] @ V0[:, k])) / (np.linalg.norm(V[:, k]) * np.linalg.norm(V0[:, k])) - 1) < 1e-6


def test_bad_arguments(gpu_lib, tmp_path):
    from paper_2112_07862_gb300 import mge
    c = gpu_lib.Context(0)
    try:
        with pytest.raises(mge.MgeError) as e:
            mge.mge_ctx_set_autotune(c.h, 3)
        assert e.value.status == mge.MGE_EINVAL
        bad = tmp_path / "bad.json"
        bad.write_text('{"cheb/m16/f32/n2^14/slots15": {"budget": 65536}}')
        with pytest.raises(mge.MgeError) as e:
            mge.mge_ctx_set_autotune(c.h, 2, str(bad))
        assert e.value.status == mge.MGE_EINVAL
        mge.mge_ctx_set_autotune(c.h, 2, str(tmp_path / "absent.json"))      # no file yet: fine
    finally:
        c.close()
