"""CPU FP64 reference for the learned control variate (test infrastructure only).

The paper has no learned component; the workload adds one: a small MLP that
predicts, for every node, the relative Rao-Blackwell correction c_i / v_i of
the overlapping RBMC estimator (Algorithm 4: v_i = Sigma*_ii + c_i with
c_i = E[w_i^2]) from local features of Q, the time distance to the nearest
separator slab and theta.  A planner uses the prediction to choose the
overlap and the number of samples; the estimate itself stays plain RBMC, so
it is unbiased whatever the prediction.

Features of node (t, i) (14 values):
  0      log Q_ii
  1..8   log |Q_il| of the 8 largest off-diagonal entries of row (t, i),
         sorted descending (log of 1e-30 where the row has fewer)
  9      time distance from slab t to the nearest separator slab of its
         subdomain, capped at SEPARATOR_CAP (the cap also when there is none)
  10     graph distance from node i to the mesh boundary (boundary = nodes
         with fewer stiffness neighbours than the maximum), capped at
         BOUNDARY_CAP
Both distances are capped so that a network trained on small models sees
the same feature range as the large models it is applied to.
  11..13 theta = (log kappa, log tau, logit rho)
Network: 14 -> 64 -> 64 -> 1, GELU (erf form) on both hidden layers, inputs
standardised with fixed per-feature mean and scale; the output is
log(c_i / v_i).  Weights are rounded to bfloat16 before use (the device keeps
FP32 master weights and BF16 copies); accumulation in float64 here.
"""
from __future__ import annotations

import math
from collections import deque

import numpy as np
import scipy.sparse as sp

from . import qsel_oracle as o

N_FEATURES = 14
HIDDEN = 64
SEPARATOR_CAP = 16.0
BOUNDARY_CAP = 8.0


def boundary_distance(model: o.Model) -> np.ndarray:
    """Graph distance (stiffness graph) from each spatial node to the nearest
    boundary node, capped at BOUNDARY_CAP; boundary nodes have fewer
    neighbours than the maximum."""
    G = model.G.tocsr()
    deg = np.array([np.count_nonzero(G.indices[G.indptr[i]:G.indptr[i + 1]] != i) for i in range(model.n_s)])
    dist = np.full(model.n_s, -1, dtype=np.int64)
    q = deque()
    for i in np.flatnonzero(deg < deg.max()):
        dist[i] = 0
        q.append(i)
    if not q:
        return np.zeros(model.n_s)
    while q:
        i = q.popleft()
        for j in G.indices[G.indptr[i]:G.indptr[i + 1]]:
            if dist[j] < 0:
                dist[j] = dist[i] + 1
                q.append(j)
    return np.minimum(dist.astype(np.float64), BOUNDARY_CAP)


def separator_distance(n_t: int, slab_start, n_l: int) -> np.ndarray:
    """For every slab: distance to the nearest separator slab of the
    subdomain that owns it, capped at SEPARATOR_CAP (the cap when that
    subdomain has no separator)."""
    out = np.zeros(n_t)
    for part in o.partition(n_t, slab_start, n_l):
        s0, s1 = part.own
        for t in range(s0, s1):
            out[t] = min([abs(t - s) for s in part.sep] + [SEPARATOR_CAP])
    return out


def features(model: o.Model, theta, slab_start, n_l: int) -> np.ndarray:
    """(n, 14) feature matrix, node order t * n_s + i."""
    Q = o.precision(model, theta).tocsr()
    n = model.n
    F = np.zeros((n, N_FEATURES))
    sep = separator_distance(model.n_t, slab_start, n_l)
    bd = boundary_distance(model)
    for r in range(n):
        cols = Q.indices[Q.indptr[r]:Q.indptr[r + 1]]
        vals = Q.data[Q.indptr[r]:Q.indptr[r + 1]]
        diag = vals[cols == r][0]
        keep = (cols != r) & (vals != 0.0)
        off = np.sort(np.abs(vals[keep]))[::-1][:8]
        F[r, 0] = math.log(diag)
        top = np.full(8, 1e-30)
        top[:len(off)] = np.maximum(off, 1e-30)
        F[r, 1:9] = np.log(top)
        t, i = divmod(r, model.n_s)
        F[r, 9] = sep[t]
        F[r, 10] = bd[i]
    F[:, 11:14] = np.asarray(theta, dtype=np.float64)
    return F


def bf16_round(x) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even)."""
    a = np.asarray(x, dtype=np.float32)
    bits = a.view(np.uint32).astype(np.uint64)
    rounded = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + np.vectorize(math.erf)(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)


def forward(params: dict, X: np.ndarray, bf16: bool = True):
    """Returns (y, cache).  params: W1 (64,14), b1 (64), W2 (64,64), b2 (64),
    W3 (1,64), b3 (1), mu (14), scale (14)."""
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    Xn = (X - params["mu"]) / params["scale"]
    a1 = Xn @ r(params["W1"]).T + params["b1"]
    h1 = gelu(a1)
    a2 = h1 @ r(params["W2"]).T + params["b2"]
    h2 = gelu(a2)
    y = (h2 @ r(params["W3"]).T)[:, 0] + params["b3"][0]
    return y, (Xn, a1, h1, a2, h2)


def loss_and_grad(params: dict, X: np.ndarray, target: np.ndarray, bf16: bool = True):
    """Mean squared error (1/N) sum (y - target)^2 and its gradient with
    respect to W1, b1, W2, b2, W3, b3 (the weights as used, bf16 or not)."""
    r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    y, (Xn, a1, h1, a2, h2) = forward(params, X, bf16)
    N = X.shape[0]
    dy = 2.0 * (y - target) / N
    g = {"W3": dy[None, :] @ h2, "b3": np.array([dy.sum()])}
    dh2 = dy[:, None] * r(params["W3"])
    da2 = dh2 * gelu_grad(a2)
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(axis=0)
    dh1 = da2 @ r(params["W2"])
    da1 = dh1 * gelu_grad(a1)
    g["W1"] = da1.T @ Xn
    g["b1"] = da1.sum(axis=0)
    return float(np.mean((y - target) ** 2)), g
