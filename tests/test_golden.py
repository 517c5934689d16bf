"""The stored fixtures under tests/golden/ against the closed form and the current oracle."""
import json
import math
import os

import numpy as np
import pytest

import manifold_graphs as mg
from oracle import graph_ops as go

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def test_ring9_fixture_matches_closed_form():
    d = load("ring9.json")
    n = 9
    eps = 2 - 2 * math.cos(2 * math.pi / n)
    assert d["eps"] == pytest.approx(eps, rel=1e-14)
    assert d["mu"] == pytest.approx(eps / 4, rel=1e-14)
    t = 2 * np.pi * np.arange(n) / n
    lam = np.sort((2 - 2 * np.cos(t)) - d["mu"] * (2 - 2 * np.cos(2 * t)) + d["eps"])
    assert np.max(np.abs(np.array(d["lam"]) - lam)) < 1e-13


def test_mesh10_fixture_is_reproduced_by_oracle():
    d = load("mesh10.json")
    g = mg.triangle_mesh()
    assert d["row_ptr"] == g.row_ptr.tolist() and d["col"] == g.col.tolist()
    ops = go.from_graph(g)
    assert d["a_ptr"] == ops.a_ptr.tolist() and d["a_col"] == ops.a_col.tolist()
    assert np.allclose(d["a_val"], ops.a_val, rtol=1e-14, atol=1e-15)
    assert d["eps"] == pytest.approx(ops.eps, rel=1e-13)
