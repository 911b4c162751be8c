"""Plain CPU FP64 oracle for overlapping Rao-Blackwellized Monte Carlo (RBMC)
selected inversion of a space-time SPDE precision matrix.

TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA library: it is written directly from the paper (Zhumekenov, Krainski,
Rue, "Parallel selected inversion for space-time Gaussian Markov random
fields") in plain numpy/scipy, FP64, without blocking, fusion or reordering
beyond what the paper's definitions and algorithms state.

What it computes, each with the passage it follows:

* the model: spatial precision Q_s of the alpha = 2 Whittle-Matern SPDE with
  lumped mass (Section 2.1, Eq. spde:2 and the formula after it), separable
  space-time prior tau * Q_t (x) Q_s (Section 2.2), Gaussian likelihood
  Q = Q_x + A^T Q_y A (Section 2.3, Eq. lgm:2), and dQ/dtheta_j;
* the exact target: dense inverse, its diagonal, and the traces
  tr(Q^-1 dQ/dtheta_j) through the elementwise identity (Eq. lgm:4);
* the time-slab partition with overlap and separators (Section 3.2.3,
  Algorithms 3 and 4: extend each part by n_l neighbour layers, the
  separator is the next layer);
* the exact subdomain selected inverse: block Cholesky of the block
  tridiagonal Q_{Omega*Omega*} and the Takahashi recursion (Section 1,
  Erisman-Tinney; Section 3.2.3 "direct factorization");
* the Rao-Blackwell correction w = Q_{**}^-1 Q_{*S} x_S and the overlapping
  RBMC estimate of diag(Q^-1) (Algorithm 4) and of the traces (Section 3.4.2,
  Eq. hyperpar:4);
* exact samples x ~ N(0, Q^-1) by the perturbation construction
  Q x = L z + R w (Section 2.4 and Section 3.3, Papandreou-Yuille), with the
  Gaussian noise from the Philox4x32-10 counter-based generator (Salmon,
  Moraes, Dror, Shaw, SC'11) and the Box-Muller transform;
* log|Q| from the block Cholesky factor (for finite-difference checks of the
  traces, Section 1: d log|Q| / dtheta = tr(Q^-1 dQ/dtheta)).

Readings where the paper is silent (all listed in the design notes):
theta = (log kappa, log tau, logit rho); tau multiplies the Kronecker
product; Q_t is the unit-marginal-variance AR(1) precision; the correction is
squared as in Algorithm 4 (Eq. intro:4 drops the square); the trace uses the
uncentred sample second moment (1/k) sum_s w_i w_l for the off-diagonal
selected entries.

Parity pins for every function live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# ----------------------------------------------------------------------------
# Model (Sections 2.1-2.3)
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class Model:
    """Space-time model inputs: mesh, observation mask, noise level."""
    n_s: int
    n_t: int
    c_diag: np.ndarray            # lumped mass C (n_s,)
    G: sp.csr_matrix              # stiffness (n_s x n_s)
    obs_mask: np.ndarray          # (n_s*n_t,) 0/1, space-fastest ordering
    sigma: float

    @property
    def n(self) -> int:
        return self.n_s * self.n_t


def model_from_csr(n_s, n_t, c_diag, g_rowptr, g_col, g_val, obs_mask, sigma) -> Model:
    G = sp.csr_matrix((np.asarray(g_val, float), np.asarray(g_col), np.asarray(g_rowptr)),
                      shape=(n_s, n_s))
    return Model(n_s, n_t, np.asarray(c_diag, float), G,
                 np.asarray(obs_mask).astype(np.uint8), float(sigma))


def theta_to_natural(theta):
    """theta = (log kappa, log tau, logit rho) -> (kappa, tau, rho)."""
    kappa = math.exp(theta[0])
    tau = math.exp(theta[1])
    rho = 1.0 / (1.0 + math.exp(-theta[2]))
    return kappa, tau, rho


def spatial_K(model: Model, kappa: float) -> sp.csr_matrix:
    """K = kappa^2 C + G, the discretised (kappa^2 - Laplacian) of Eq. spde:2."""
    return (kappa ** 2 * sp.diags(model.c_diag) + model.G).tocsr()


def spatial_precision(model: Model, kappa: float) -> sp.csr_matrix:
    """Q_s = (kappa^2 C + G) C^-1 (kappa^2 C + G) for alpha = 2 (Section 2.1)."""
    K = spatial_K(model, kappa)
    return (K @ sp.diags(1.0 / model.c_diag) @ K).tocsr()


def spatial_precision_dlogkappa(model: Model, kappa: float) -> sp.csr_matrix:
    """d Q_s / d log kappa.  With K' = dK/dlog kappa = 2 kappa^2 C, the product
    rule on K C^-1 K gives K' C^-1 K + K C^-1 K' = 2 kappa^2 (K + K) = 4 kappa^2 K."""
    return (4.0 * kappa ** 2 * spatial_K(model, kappa)).tocsr()


def ar1_R(rho: float, n_t: int) -> np.ndarray:
    """R = B^T B for the AR(1) innovation matrix B (B_00 = sqrt(1-rho^2),
    B_tt = 1, B_{t,t-1} = -rho): diagonal (1, 1+rho^2, ..., 1+rho^2, 1),
    off-diagonals -rho."""
    R = np.zeros((n_t, n_t))
    for t in range(n_t):
        R[t, t] = 1.0 + rho ** 2
        if t + 1 < n_t:
            R[t, t + 1] = R[t + 1, t] = -rho
    R[0, 0] = 1.0
    R[n_t - 1, n_t - 1] = 1.0
    if n_t == 1:
        R[0, 0] = 1.0 - rho ** 2
    return R


def ar1_B(rho: float, n_t: int) -> np.ndarray:
    """AR(1) innovation matrix: (B x)_0 = sqrt(1-rho^2) x_0, (B x)_t = x_t - rho x_{t-1}."""
    B = np.eye(n_t)
    B[0, 0] = math.sqrt(1.0 - rho ** 2)
    for t in range(1, n_t):
        B[t, t - 1] = -rho
    return B


def temporal_precision(rho: float, n_t: int) -> np.ndarray:
    """Unit-marginal-variance stationary AR(1) precision Q_t = R / (1 - rho^2)."""
    return ar1_R(rho, n_t) / (1.0 - rho ** 2)


def temporal_precision_drho(rho: float, n_t: int) -> np.ndarray:
    """d Q_t / d rho = R' / (1-rho^2) + R * 2 rho / (1-rho^2)^2, where R' has
    diagonal (0, 2 rho, ..., 2 rho, 0) and off-diagonals -1."""
    R = ar1_R(rho, n_t)
    dR = np.zeros((n_t, n_t))
    for t in range(n_t):
        dR[t, t] = 2.0 * rho
        if t + 1 < n_t:
            dR[t, t + 1] = dR[t + 1, t] = -1.0
    dR[0, 0] = 0.0
    dR[n_t - 1, n_t - 1] = 0.0
    if n_t == 1:
        dR[0, 0] = -2.0 * rho
    return dR / (1.0 - rho ** 2) + R * (2.0 * rho / (1.0 - rho ** 2) ** 2)


def obs_precision(model: Model) -> sp.csr_matrix:
    """A^T Q_y A with A selecting the observed nodes and Q_y = I / sigma^2 (Eq. lgm:2)."""
    return sp.diags(model.obs_mask.astype(float) / model.sigma ** 2).tocsr()


def precision(model: Model, theta) -> sp.csr_matrix:
    """Posterior precision Q = tau Q_t (x) Q_s + A^T A / sigma^2 (Sections 2.2, 2.3)."""
    kappa, tau, rho = theta_to_natural(theta)
    Qs = spatial_precision(model, kappa)
    Qt = sp.csr_matrix(temporal_precision(rho, model.n_t))
    return (tau * sp.kron(Qt, Qs) + obs_precision(model)).tocsr()


def precision_derivatives(model: Model, theta) -> list:
    """[dQ/dlog kappa, dQ/dlog tau, dQ/dlogit rho]; the likelihood term does not
    depend on theta."""
    kappa, tau, rho = theta_to_natural(theta)
    Qs = spatial_precision(model, kappa)
    dQs = spatial_precision_dlogkappa(model, kappa)
    Qt = sp.csr_matrix(temporal_precision(rho, model.n_t))
    dQt = sp.csr_matrix(temporal_precision_drho(rho, model.n_t) * rho * (1.0 - rho))
    return [(tau * sp.kron(Qt, dQs)).tocsr(),
            (tau * sp.kron(Qt, Qs)).tocsr(),
            (tau * sp.kron(dQt, Qs)).tocsr()]


# ----------------------------------------------------------------------------
# Exact target (Eq. lgm:4), dense -- small problems only
# ----------------------------------------------------------------------------


def exact_selinv(Q, dQs):
    """Dense Sigma = Q^-1; returns (diag Sigma, [tr(Sigma dQ_j)]) with the trace as
    the elementwise sum of Sigma and dQ_j (Eq. lgm:4)."""
    Qd = Q.toarray() if sp.issparse(Q) else np.asarray(Q)
    Sigma = np.linalg.inv(Qd)
    Sigma = 0.5 * (Sigma + Sigma.T)
    traces = []
    for d in dQs:
        dd = d.toarray() if sp.issparse(d) else np.asarray(d)
        traces.append(float(np.sum(Sigma * dd)))
    return np.diag(Sigma).copy(), traces


# ----------------------------------------------------------------------------
# Partition (Section 3.2.3, Algorithms 3 and 4)
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class Part:
    own: tuple            # [s0, s1): slabs of Omega_p
    ext: tuple            # [e0, e1): slabs of Omega_p^* (own extended by n_l, clipped)
    sep: list             # separator slabs S_p (the next slab outside ext, if any)


def partition(n_t: int, slab_start, n_l) -> list:
    """Omega_p are contiguous slab ranges [slab_start[p], slab_start[p+1]).  Because
    Q is block tridiagonal in time and every spatial node couples to itself in
    the neighbouring slab, the graph neighbours of a slab range are the two
    adjacent slabs; extending n_l times adds n_l slabs on each side (clipped to
    the time axis) and the separator is the slab just beyond (Algorithm 3).
    n_l is one overlap for every part or a sequence with one per part
    (Algorithm 3 extends each subdomain on its own)."""
    parts = []
    for p in range(len(slab_start) - 1):
        nl = int(n_l[p]) if np.ndim(n_l) else int(n_l)
        s0, s1 = int(slab_start[p]), int(slab_start[p + 1])
        e0, e1 = max(0, s0 - nl), min(n_t, s1 + nl)
        sep = []
        if e0 - 1 >= 0:
            sep.append(e0 - 1)
        if e1 < n_t:
            sep.append(e1)
        parts.append(Part((s0, s1), (e0, e1), sep))
    return parts


def balanced_slab_start(n_t: int, n_p: int) -> np.ndarray:
    base, extra = divmod(n_t, n_p)
    sizes = [base + (1 if p < extra else 0) for p in range(n_p)]
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


# ----------------------------------------------------------------------------
# Block tridiagonal Cholesky and Takahashi (exact subdomain selected inverse)
# ----------------------------------------------------------------------------


def block(Q, n_s: int, t: int, u: int) -> np.ndarray:
    """Dense n_s x n_s block (t, u) of Q (space-fastest ordering)."""
    return Q[t * n_s:(t + 1) * n_s, u * n_s:(u + 1) * n_s].toarray()


def block_cholesky(diag_blocks, sub_blocks):
    """Q = L L^T for block tridiagonal Q with diagonal blocks A_tt and
    sub-diagonal blocks A_{t+1,t}:  L_00 = chol(A_00),
    L_{t+1,t} = A_{t+1,t} L_tt^-T,  L_{t+1,t+1} = chol(A_{t+1,t+1} - L_{t+1,t} L_{t+1,t}^T)."""
    T = len(diag_blocks)
    L_diag, L_sub = [], []
    S = diag_blocks[0]
    for t in range(T):
        Ltt = np.linalg.cholesky(S)
        L_diag.append(Ltt)
        if t + 1 < T:
            # X L_tt^T = A_{t+1,t}  <=>  L_tt X^T = A_{t+1,t}^T
            Lsub = sla.solve_triangular(Ltt, sub_blocks[t].T, lower=True).T
            L_sub.append(Lsub)
            S = diag_blocks[t + 1] - Lsub @ Lsub.T
    return L_diag, L_sub


def block_takahashi(L_diag, L_sub, t_stop: int = 0):
    """Takahashi / Erisman-Tinney recursion from Sigma L = L^-T for a block lower
    bidiagonal L:  Sigma_TT = L_TT^-T L_TT^-1;  for t = T-2 .. t_stop:
    W = L_{t+1,t} L_tt^-1,  Sigma_{t+1,t} = -Sigma_{t+1,t+1} W,
    Sigma_tt = L_tt^-T L_tt^-1 - W^T Sigma_{t+1,t}.
    Returns (Sigma_diag, Sigma_sub) with Sigma_sub[t] = Sigma_{t+1,t}; entries below
    t_stop are None."""
    T = len(L_diag)
    n = L_diag[0].shape[0]
    eye = np.eye(n)
    Linv = [None] * T
    Sd = [None] * T
    Ss = [None] * (T - 1)
    Linv[T - 1] = sla.solve_triangular(L_diag[T - 1], eye, lower=True)
    Sd[T - 1] = Linv[T - 1].T @ Linv[T - 1]
    for t in range(T - 2, t_stop - 1, -1):
        Linv[t] = sla.solve_triangular(L_diag[t], eye, lower=True)
        W = L_sub[t] @ Linv[t]
        Ss[t] = -Sd[t + 1] @ W
        Sd[t] = Linv[t].T @ Linv[t] - W.T @ Ss[t]
    return Sd, Ss


def block_solve(L_diag, L_sub, b_blocks):
    """Solve (L L^T) w = b blockwise: forward y_t = L_tt^-1 (b_t - L_{t,t-1} y_{t-1}),
    backward w_t = L_tt^-T (y_t - L_{t+1,t}^T w_{t+1})."""
    T = len(L_diag)
    y = [None] * T
    for t in range(T):
        rhs = b_blocks[t] if t == 0 else b_blocks[t] - L_sub[t - 1] @ y[t - 1]
        y[t] = sla.solve_triangular(L_diag[t], rhs, lower=True)
    w = [None] * T
    for t in range(T - 1, -1, -1):
        rhs = y[t] if t == T - 1 else y[t] - L_sub[t].T @ w[t + 1]
        w[t] = sla.solve_triangular(L_diag[t], rhs, lower=True, trans='T')
    return w


def logdet(Q, n_s: int, n_t: int) -> float:
    """log|Q| = 2 sum log diag(L) from the block Cholesky factor."""
    diag_b = [block(Q, n_s, t, t) for t in range(n_t)]
    sub_b = [block(Q, n_s, t + 1, t) for t in range(n_t - 1)]
    L_diag, _ = block_cholesky(diag_b, sub_b)
    return float(2.0 * sum(np.sum(np.log(np.diag(L))) for L in L_diag))


# ----------------------------------------------------------------------------
# Overlapping RBMC (Algorithm 4) and the trace estimator (Eq. hyperpar:4)
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class SubdomainResult:
    part: Part
    sigma_star_diag: np.ndarray     # diag(Q_{**}^-1) for rows of Omega_p
    corr_diag: np.ndarray           # (1/k) sum_s w_i^2 for rows of Omega_p
    corr4_diag: np.ndarray          # (1/k) sum_s w_i^4 for rows of Omega_p
    traces: np.ndarray              # partial traces over rows of Omega_p (3,)


def subdomain_estimate(Q, dQs, n_s: int, part: Part, X_sep: dict, k: int):
    """One subdomain of Algorithm 4 plus its rows of Eq. hyperpar:4.

    X_sep maps each separator slab to its samples (n_s x k).  The correction is
    w = Q_{**}^-1 Q_{*S} x_S (Eq. var:2 with Omega* in place of Omega); the
    variance estimate on Omega_p is diag(Sigma*) + (1/k) sum_s w_i^2 and the
    selected entries for the trace are Sigma*_il + (1/k) sum_s w_i w_l."""
    e0, e1 = part.ext
    s0, s1 = part.own
    T = e1 - e0
    diag_b = [block(Q, n_s, e0 + t, e0 + t) for t in range(T)]
    sub_b = [block(Q, n_s, e0 + t + 1, e0 + t) for t in range(T - 1)]
    L_diag, L_sub = block_cholesky(diag_b, sub_b)
    t_stop = max(0, s0 - e0 - 1)
    Sd, Ss = block_takahashi(L_diag, L_sub, t_stop)

    # b = Q_{*S} x_S is non-zero only in the slabs adjacent to a separator
    b = [np.zeros((n_s, k)) for _ in range(T)]
    for s in part.sep:
        for t in range(T):
            if abs((e0 + t) - s) == 1:
                b[t] += block(Q, n_s, e0 + t, s) @ X_sep[s]
    if part.sep:
        w = block_solve(L_diag, L_sub, b)
    else:
        w = [np.zeros((n_s, k)) for _ in range(T)]

    own_rows = range(s0 - e0, s1 - e0)
    sig_diag = np.concatenate([np.diag(Sd[t]) for t in own_rows])
    corr = np.concatenate([np.sum(w[t] ** 2, axis=1) / k for t in own_rows])
    corr4 = np.concatenate([np.sum(w[t] ** 4, axis=1) / k for t in own_rows])

    traces = np.zeros(len(dQs))
    for j, dQ in enumerate(dQs):
        acc = 0.0
        for t in own_rows:
            for u in (t - 1, t, t + 1):
                if u < 0 or u >= T:
                    continue
                if u == t:
                    sig = Sd[t]
                elif u == t + 1:
                    sig = Ss[t].T            # Sigma_{t,t+1} = Sigma_{t+1,t}^T
                else:
                    sig = Ss[u]              # Sigma_{t,t-1}
                sel = sig + (w[t] @ w[u].T) / k
                acc += float(np.sum(sel * block(dQ, n_s, e0 + t, e0 + u)))
        traces[j] = acc
    return SubdomainResult(part, sig_diag, corr, corr4, traces)


def rbmc(model: Model, theta, slab_start, n_l: int, X: np.ndarray):
    """Overlapping RBMC (Algorithm 4) for diag(Q^-1) and the trace estimator of
    Eq. hyperpar:4, given global samples X (n x k, columns x^(s) ~ N(0, Q^-1)).

    Returns (v_hat (n,), t_hat (3,), list of SubdomainResult)."""
    Q = precision(model, theta)
    dQs = precision_derivatives(model, theta)
    n_s, n_t = model.n_s, model.n_t
    k = X.shape[1]
    parts = partition(n_t, slab_start, n_l)
    v = np.zeros(model.n)
    t_hat = np.zeros(3)
    results = []
    for part in parts:
        X_sep = {s: X[s * n_s:(s + 1) * n_s, :] for s in part.sep}
        res = subdomain_estimate(Q, dQs, n_s, part, X_sep, k)
        s0, s1 = part.own
        v[s0 * n_s:s1 * n_s] = res.sigma_star_diag + res.corr_diag
        t_hat += res.traces
        results.append(res)
    return v, t_hat, results


def error_estimate(v: np.ndarray, results, k: int):
    """Sample-based standard error of the RBMC estimate (Algorithm 4): the
    correction of node i is the mean of k values w_i^2, whose variance is
    estimated by (m4_i - m2_i^2) / (k - 1) with m2, m4 the sample means of
    w_i^2 and w_i^4.  Returns (per part, global) root mean square over rows of
    the standard error relative to v_i."""
    per_part, tot, rows = [], 0.0, 0
    for res in results:
        s0, s1 = res.part.own
        n_s = res.corr_diag.size // (s1 - s0)
        vv = v[s0 * n_s:s1 * n_s]
        var = np.maximum(res.corr4_diag - res.corr_diag ** 2, 0.0) / (k - 1)
        q = var / vv ** 2
        per_part.append(math.sqrt(q.mean()))
        tot += q.sum()
        rows += q.size
    return np.array(per_part), math.sqrt(tot / rows)


# ----------------------------------------------------------------------------
# Sampling (Sections 2.4 and 3.3): Philox4x32-10 noise, perturbation RHS,
# direct solve
# ----------------------------------------------------------------------------

_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint32(0x9E3779B9)
_PHILOX_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds (Salmon et al., SC'11).  ctr: (4, N) uint32,
    key: (2,) uint32.  Each round multiplies words 0 and 2 by the two Philox
    constants, swaps the high/low halves across the lanes and xors in the key;
    the key is bumped by the Weyl constants between rounds."""
    c = [np.asarray(ctr[i], dtype=np.uint32).copy() for i in range(4)]
    k0 = np.uint32(key[0])
    k1 = np.uint32(key[1])
    with np.errstate(over="ignore"):
        for r in range(10):
            if r > 0:
                k0 = np.uint32((int(k0) + int(_PHILOX_W0)) & 0xFFFFFFFF)
                k1 = np.uint32((int(k1) + int(_PHILOX_W1)) & 0xFFFFFFFF)
            p0 = _PHILOX_M0 * c[0].astype(np.uint64)
            p1 = _PHILOX_M1 * c[2].astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK32).astype(np.uint32)
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c)


def philox_normals(seed: int, stream: int, n_rows: int, k: int) -> np.ndarray:
    """Standard normals z[i, s] for i < n_rows, s < k.  The pair of columns
    (2q, 2q+1) of row i comes from one Philox call with counter
    (i, q, stream, 0) and key (seed mod 2^32, seed div 2^32): words 0,1 give
    u1 = (53-bit integer + 1) 2^-53 in (0, 1], words 2,3 give u2 = 53-bit
    integer 2^-53 in [0, 1); Box-Muller returns sqrt(-2 ln u1) cos(2 pi u2)
    and sqrt(-2 ln u1) sin(2 pi u2)."""
    n_pairs = (k + 1) // 2
    ii, qq = np.meshgrid(np.arange(n_rows, dtype=np.uint64), np.arange(n_pairs, dtype=np.uint64),
                         indexing="ij")
    ctr = np.stack([ii.ravel().astype(np.uint32), qq.ravel().astype(np.uint32),
                    np.full(ii.size, stream, dtype=np.uint32), np.zeros(ii.size, dtype=np.uint32)])
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    out = philox4x32_10(ctr, key).astype(np.uint64)
    a = ((out[0] << np.uint64(32)) | out[1]) >> np.uint64(11)
    b = ((out[2] << np.uint64(32)) | out[3]) >> np.uint64(11)
    u1 = (a.astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = b.astype(np.float64) * 2.0 ** -53
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty((ii.size, 2))
    z[:, 0] = r * np.cos(2.0 * np.pi * u2)
    z[:, 1] = r * np.sin(2.0 * np.pi * u2)
    return z.reshape(n_rows, 2 * n_pairs)[:, :k].copy()


def noise(model: Model, seed: int, k: int):
    """z1 ~ N(0, I_n) (stream 0) and z2 ~ N(0, I_{n_obs}) (stream 1), the observed
    nodes taken in increasing global index."""
    n_obs = int(model.obs_mask.sum())
    return philox_normals(seed, 0, model.n, k), philox_normals(seed, 1, n_obs, k)


def perturbation_rhs(model: Model, theta, z1: np.ndarray, z2: np.ndarray) -> np.ndarray:
    """r = F^T z1 + A^T z2 / sigma with F = sqrt(tau/(1-rho^2)) (B (x) C^-1/2 K), so
    that F^T F + A^T A / sigma^2 = tau Q_t (x) Q_s + A^T A / sigma^2 = Q and
    Q^-1 r ~ N(0, Q^-1) (perturbation sampling, Sections 2.4 and 3.3)."""
    kappa, tau, rho = theta_to_natural(theta)
    K = spatial_K(model, kappa)
    M = (K @ sp.diags(1.0 / np.sqrt(model.c_diag))).tocsr()          # K C^-1/2
    B = sp.csr_matrix(ar1_B(rho, model.n_t))
    FT = math.sqrt(tau / (1.0 - rho ** 2)) * sp.kron(B.T, M)
    obs_idx = np.flatnonzero(model.obs_mask)
    AT = sp.csr_matrix((np.ones(obs_idx.size), (obs_idx, np.arange(obs_idx.size))),
                       shape=(model.n, obs_idx.size))
    return FT @ z1 + (AT @ z2) / model.sigma


def rhs(model: Model, theta, seed: int, k: int) -> np.ndarray:
    z1, z2 = noise(model, seed, k)
    return perturbation_rhs(model, theta, z1, z2)


def solve_direct(model: Model, theta, R: np.ndarray) -> np.ndarray:
    """X = Q^-1 R through the block Cholesky factor of the full Q."""
    Q = precision(model, theta)
    n_s, n_t = model.n_s, model.n_t
    diag_b = [block(Q, n_s, t, t) for t in range(n_t)]
    sub_b = [block(Q, n_s, t + 1, t) for t in range(n_t - 1)]
    L_diag, L_sub = block_cholesky(diag_b, sub_b)
    b = [R[t * n_s:(t + 1) * n_s, :] for t in range(n_t)]
    return np.concatenate(block_solve(L_diag, L_sub, b), axis=0)


def samples(model: Model, theta, seed: int, k: int) -> np.ndarray:
    """Exact samples x^(s) = Q^-1 r^(s), s < k."""
    return solve_direct(model, theta, rhs(model, theta, seed, k))


# ----------------------------------------------------------------------------
# Sampled rows at sizes where the block algorithms are too slow on the CPU
# ----------------------------------------------------------------------------


def subdomain_rows_sparse(model: Model, theta, part: Part, X_sep: dict, k: int, rows):
    """For selected global rows i of Omega_p: Sigma*_ii = e_i^T Q_{**}^-1 e_i and
    (1/k) sum_s w_i^2 with w = Q_{**}^-1 Q_{*S} x_S, using a sparse direct solve
    of Q_{**} (the plain definitions, for full-size spot checks)."""
    Q = precision(model, theta)
    n_s = model.n_s
    e0, e1 = part.ext
    sl = slice(e0 * n_s, e1 * n_s)
    Qss = Q[sl, sl].tocsc()
    lu = spla.splu(Qss)
    loc = np.asarray(rows) - e0 * n_s
    E = np.zeros((Qss.shape[0], len(loc)))
    E[loc, np.arange(len(loc))] = 1.0
    sig = np.einsum("ij,ij->j", E, lu.solve(E))
    if part.sep:
        b = np.zeros((Qss.shape[0], k))
        for s in part.sep:
            b += Q[sl, s * n_s:(s + 1) * n_s] @ X_sep[s]
        w = lu.solve(b)
        corr = np.sum(w[loc, :] ** 2, axis=1) / k
    else:
        corr = np.zeros(len(loc))
    return sig, corr
