"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module produces *inputs* only: the finite-element mesh matrices of a
regular planar grid (lumped mass C and stiffness G), the observation mask,
the five workload configurations and seeded Gaussian matrices used as
injected samples.  It holds none of the selected-inversion method's
arithmetic: the precision matrix Q, its derivatives, the sampler, the
factorisations and the estimators live separately in ``oracle/`` (CPU
reference) and in the CUDA library (product).

Mesh (Section 2.1, Eq. spde:2): nodes sit on an m x m grid with spacing
h = 1, node (i, j) at coordinates (i, j) with index i*m + j.  Every grid
cell [i, i+1] x [j, j+1] is split by the diagonal (i, j)-(i+1, j+1) into
two right triangles; G is the piecewise-linear stiffness matrix and C the
lumped (diagonal) mass matrix, whose entry for node i is one third of the
area of the triangles touching it.  Because every triangle is right
isosceles, the stiffness contribution across the diagonal edge vanishes and
G is the 5-point stencil with -1/2 on boundary edges.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = ["GridMesh", "grid_mesh", "obs_mask", "Workload", "workload", "WORKLOADS",
           "seeded_normal", "balanced_slab_start", "BatchModel", "uneven_batch"]


@dataclasses.dataclass(frozen=True)
class GridMesh:
    """P1 finite elements on an m x m grid: lumped mass and CSR stiffness."""
    m: int
    c_diag: np.ndarray      # (n_s,) float64, lumped mass
    g_rowptr: np.ndarray    # (n_s+1,) int32
    g_col: np.ndarray       # (nnz,) int32, sorted within each row
    g_val: np.ndarray       # (nnz,) float64

    @property
    def n_s(self) -> int:
        return self.m * self.m

    def g_dense(self) -> np.ndarray:
        g = np.zeros((self.n_s, self.n_s))
        for r in range(self.n_s):
            for p in range(self.g_rowptr[r], self.g_rowptr[r + 1]):
                g[r, self.g_col[p]] += self.g_val[p]
        return g


def grid_mesh(m: int) -> GridMesh:
    """Assemble P1 stiffness and lumped mass on the m x m unit-spacing grid."""
    if m < 2:
        raise ValueError("grid needs m >= 2")
    n_s = m * m
    c = np.zeros(n_s)
    entries: dict[tuple[int, int], float] = {}
    for i in range(m - 1):
        for j in range(m - 1):
            for tri in (((i, j), (i + 1, j), (i + 1, j + 1)),
                        ((i, j), (i + 1, j + 1), (i, j + 1))):
                xy = np.array(tri, dtype=np.float64)
                idx = [a * m + b for a, b in tri]
                # gradients of the barycentric basis functions
                mat = np.column_stack([np.ones(3), xy])
                area = 0.5 * abs(np.linalg.det(mat))
                grads = np.linalg.inv(mat)[1:, :]          # 2 x 3
                ke = area * grads.T @ grads
                for a in range(3):
                    c[idx[a]] += area / 3.0
                    for b in range(3):
                        key = (idx[a], idx[b])
                        entries[key] = entries.get(key, 0.0) + ke[a, b]
    rows: list[list[tuple[int, float]]] = [[] for _ in range(n_s)]
    for (r, col), v in entries.items():
        if abs(v) > 1e-14:
            rows[r].append((col, v))
    rowptr = np.zeros(n_s + 1, dtype=np.int32)
    cols, vals = [], []
    for r in range(n_s):
        rows[r].sort()
        rowptr[r + 1] = rowptr[r] + len(rows[r])
        cols.extend(cc for cc, _ in rows[r])
        vals.extend(vv for _, vv in rows[r])
    return GridMesh(m, c, rowptr, np.asarray(cols, dtype=np.int32), np.asarray(vals, dtype=np.float64))


def obs_mask(n: int, frac: float, seed: int) -> np.ndarray:
    """Exactly round(frac*n) observed nodes drawn without replacement (uint8 mask)."""
    n_obs = int(round(frac * n))
    rng = np.random.Generator(np.random.Philox(seed))
    mask = np.zeros(n, dtype=np.uint8)
    if n_obs:
        mask[rng.choice(n, size=n_obs, replace=False)] = 1
    return mask


def balanced_slab_start(n_t: int, n_p: int) -> np.ndarray:
    """Contiguous time partition: the first n_t mod n_p parts get one extra slab."""
    base, extra = divmod(n_t, n_p)
    sizes = [base + (1 if p < extra else 0) for p in range(n_p)]
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)


def seeded_normal(shape, seed: int) -> np.ndarray:
    """Seeded standard normal matrix (float64), e.g. injected samples x_S."""
    return np.random.Generator(np.random.Philox(seed)).standard_normal(shape)


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic space-time workload: mesh size, hyperparameters, partition."""
    name: str
    m: int            # spatial grid side, n_s = m*m
    n_t: int          # time slabs
    kappa: float
    tau: float
    rho: float
    obs_frac: float
    sigma: float
    n_parts: int
    overlap: int
    n_samples: int
    pcg_tol: float
    model_seed: int = 1

    @property
    def n_s(self) -> int:
        return self.m * self.m

    @property
    def n(self) -> int:
        return self.n_s * self.n_t

    @property
    def theta(self) -> tuple[float, float, float]:
        """(log kappa, log tau, logit rho)."""
        return (float(np.log(self.kappa)), float(np.log(self.tau)),
                float(np.log(self.rho / (1.0 - self.rho))))

    def mesh(self) -> GridMesh:
        return grid_mesh(self.m)

    def mask(self) -> np.ndarray:
        return obs_mask(self.n, self.obs_frac, self.model_seed)


WORKLOADS = {
    # 16x16 grid, n_t = 8 (n = 2048): plain FP64, 2 subdomains, overlap 1, 64 samples
    "grid16_nt8": Workload("grid16_nt8", 16, 8, 0.5, 1.0, 0.9, 0.30, 0.5, 2, 1, 64, 1e-10),
    # 64x64 grid, n_t = 64 (n = 262,144): plain FP64, 8 subdomains, overlap 2, 256 samples
    "grid64_nt64": Workload("grid64_nt64", 64, 64, 0.2, 1.0, 0.95, 0.25, 0.5, 8, 2, 256, 1e-10),
    # 64x64 grid, n_t = 16: same 4096-node blocks with fewer slabs (profiling captures)
    "grid64_nt16": Workload("grid64_nt16", 64, 16, 0.2, 1.0, 0.95, 0.25, 0.5, 2, 2, 256, 1e-10),
    # 96x96 grid, n_t = 256 (n = 2,359,296): mixed precision, 16 subdomains, overlap 2, 512 samples
    "grid96_nt256": Workload("grid96_nt256", 96, 256, 0.1, 1.0, 0.98, 0.10, 0.5, 16, 2, 512, 1e-10),
    # 96x96 grid, n_t = 8: same 9216-node blocks with few slabs (profiling captures)
    "grid96_nt8": Workload("grid96_nt8", 96, 8, 0.1, 1.0, 0.98, 0.10, 0.5, 2, 1, 256, 1e-10),
}


def workload(name: str) -> Workload:
    return WORKLOADS[name]


@dataclasses.dataclass(frozen=True)
class BatchModel:
    """One model of the uneven batch: grid side, slabs, parts, theta, seed."""
    m: int
    n_t: int
    n_parts: int
    theta: tuple
    seed: int
    overlap: int = 1
    obs_frac: float = 0.25
    sigma: float = 0.5

    @property
    def n_s(self) -> int:
        return self.m * self.m

    @property
    def n(self) -> int:
        return self.n_s * self.n_t

    def mask(self) -> np.ndarray:
        return obs_mask(self.n, self.obs_frac, self.seed)


def uneven_batch(n_models: int = 64, base_seed: int = 1000) -> list:
    """Independent models of uneven size: model i draws, from a generator
    seeded with base_seed + i, the grid side m uniformly from {16, 24, ..., 64},
    n_t uniformly from [8, 128], n_parts uniformly from
    [2, min(8, n_t // (2 overlap + 1))] with overlap 1, and theta with
    log kappa ~ U[-3, 0], log tau ~ U[-1, 1], rho ~ U[0.5, 0.99];
    25 % observed, sigma = 0.5."""
    out = []
    for i in range(n_models):
        rng = np.random.Generator(np.random.Philox(base_seed + i))
        m = int(rng.choice(np.arange(16, 65, 8)))
        n_t = int(rng.integers(8, 129))
        n_p = int(rng.integers(2, min(8, n_t // 3) + 1))
        lk = float(rng.uniform(-3.0, 0.0))
        lt = float(rng.uniform(-1.0, 1.0))
        rho = float(rng.uniform(0.5, 0.99))
        out.append(BatchModel(m, n_t, n_p, (lk, lt, float(np.log(rho / (1.0 - rho)))), base_seed + i))
    return out
