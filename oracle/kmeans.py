"""Oracle for k-means clustering of the embedding (Sec. 5.2, Table 3: the embeddings are
clustered by kmeans).  Test infrastructure only: nothing in the product path imports it.

Lloyd's algorithm from given initial centres, in FP64.  The paper names the method only;
the readings used:
  * the input is the N x K embedding (one row per node), the C initial centres are given
    (random choices are the caller's, passed in), and at most T iterations run;
  * assignment: each point goes to the centre of least squared distance, the squared
    distance summed over the coordinates in order with each product and sum rounded to
    FP64 (no fused multiply-add); equal distances go to the lower centre index;
  * update: each centre becomes the mean of its points -- their sum rounded once (exactly
    rounded, math.fsum), divided by their count; a centre without points keeps its place;
  * iteration t assigns every point; when t > 0 and no assignment changed, it stops (the
    centres are then a fixed point); otherwise the centres are updated.
Returns the last assignment, the centres and the number of assignment steps taken.
"""
from __future__ import annotations

import math

import numpy as np


def assign(X: np.ndarray, centres: np.ndarray) -> np.ndarray:
    """Index of the nearest centre for every row of X (ties: lower index)."""
    X = np.asarray(X, dtype=np.float64)
    C = np.asarray(centres, dtype=np.float64)
    d2 = np.zeros((X.shape[0], C.shape[0]))
    for k in range(X.shape[1]):
        diff = X[:, k][:, None] - C[None, :, k]
        d2 = d2 + diff * diff
    return np.argmin(d2, axis=1).astype(np.int32)      # argmin returns the first minimum


def update(X: np.ndarray, a: np.ndarray, centres: np.ndarray) -> np.ndarray:
    """Means of the clusters (exactly rounded sums / counts); empty clusters unchanged."""
    X = np.asarray(X, dtype=np.float64)
    out = np.array(centres, dtype=np.float64, copy=True)
    for c in range(out.shape[0]):
        members = X[a == c]
        if members.shape[0] == 0:
            continue
        for k in range(X.shape[1]):
            out[c, k] = math.fsum(members[:, k].tolist()) / members.shape[0]
    return out


def kmeans(X: np.ndarray, centres0: np.ndarray, iters: int):
    """Lloyd's k-means: (assignment int32 [N], centres [C, K], assignment steps)."""
    centres = np.array(centres0, dtype=np.float64, copy=True)
    prev = None
    steps = 0
    a = None
    for t in range(iters):
        a = assign(X, centres)
        steps = t + 1
        if prev is not None and np.array_equal(a, prev):
            break
        centres = update(X, a, centres)
        prev = a
    return a, centres, steps


def inertia(X: np.ndarray, a: np.ndarray, centres: np.ndarray) -> float:
    """Sum of squared distances of the points to their centres."""
    d = np.asarray(X, dtype=np.float64) - np.asarray(centres)[a]
    return float(np.sum(d * d))
