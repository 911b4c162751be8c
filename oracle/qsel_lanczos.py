"""CPU FP64 reference of the preconditioned Krylov sampler (test infrastructure
only: imported by tests/ and by nothing in the product path).

Section 3.3 (Lanczos quadrature for matrix functions, Eqs. sampling:2 and
sampling:6-8, and the preconditioned Krylov sampler, Algorithm 5.1): a sample
x ~ N(0, Q^-1) is drawn without factoring Q as

    x = L^-T x~,   x~ = Q~^-1/2 z ~= V f(T) (eta e1),   f(t) = t^-1/2,

with a symmetric split preconditioner L L^T ~= Q, the preconditioned operator
Q~ = L^-1 Q L^-T, z ~ N(0, I), eta = ||z||, and V, T the Lanczos vectors and
tridiagonal matrix of the Krylov subspace K_m(Q~, z); f(T) is evaluated
through the eigendecomposition of T (the Gauss quadrature nodes and weights).

Preconditioner (the paper names IC(0) or block Jacobi): block Jacobi over
contiguous blocks of b global rows, L = blockdiag(chol(Q_bb)) (the last block
may be shorter).  Noise: Philox stream 0 of the seed (the rows of z1 of the
perturbation sampler).  Lanczos without reorthogonalisation; a column whose
beta_j vanishes stops at step j.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import qsel_oracle as o


def block_factors(Q, b: int):
    """[(r0, L_b, L_b^-1)] for the diagonal blocks of b rows, L_b = chol(Q_bb)."""
    Qd = Q.tocsr()
    n = Qd.shape[0]
    out = []
    for r0 in range(0, n, b):
        r1 = min(n, r0 + b)
        Qbb = Qd[r0:r1, r0:r1].toarray()
        L = np.linalg.cholesky(Qbb)
        Linv = sla.solve_triangular(L, np.eye(r1 - r0), lower=True)
        out.append((r0, L, Linv))
    return out


def apply_Linv(factors, x):
    y = np.empty_like(x)
    for r0, _, Linv in factors:
        y[r0:r0 + Linv.shape[0]] = Linv @ x[r0:r0 + Linv.shape[0]]
    return y


def apply_LinvT(factors, x):
    y = np.empty_like(x)
    for r0, _, Linv in factors:
        y[r0:r0 + Linv.shape[0]] = Linv.T @ x[r0:r0 + Linv.shape[0]]
    return y


def lanczos(op, z, m: int):
    """m Lanczos steps on op from z (one column).  Returns (alpha, beta, V):
    alpha (m_eff,), beta (m_eff,) with beta[j] = ||w_j|| after step j, and the
    orthonormal basis V (n, m_eff)."""
    eta = np.linalg.norm(z)
    v = z / eta
    v_prev = np.zeros_like(z)
    b_prev = 0.0
    alpha, beta, V = [], [], []
    for _ in range(m):
        V.append(v)
        w = op(v) - b_prev * v_prev
        a = float(v @ w)
        w = w - a * v
        bj = float(np.linalg.norm(w))
        alpha.append(a)
        beta.append(bj)
        if bj == 0.0:
            break
        v_prev, v, b_prev = v, w / bj, bj
    return np.array(alpha), np.array(beta), np.array(V).T


def f_T_e1(alpha, beta, eta):
    """eta f(T) e1 with f(t) = t^-1/2, T = tridiag(beta, alpha, beta), through
    the eigendecomposition T = U diag(lambda) U^T: sum_j lambda_j^-1/2
    U_1j U_:j eta (Eq. sampling:5)."""
    lam, U = sla.eigh_tridiagonal(alpha, beta[:len(alpha) - 1])
    return eta * (U @ (lam ** -0.5 * U[0, :]))


def sample(model: o.Model, theta, seed: int, k: int, m: int, b: int = 64):
    """Algorithm 5.1 for k columns.  Returns (X (n, k), alphas, betas) with
    alphas[s], betas[s] the Lanczos coefficients of column s."""
    return sample_q(o.precision(model, theta), seed, k, m, b)


def sample_q(Q, seed: int, k: int, m: int, b: int = 64):
    """Algorithm 5.1 on a given precision Q (n x n sparse), as sample()."""
    Q = Q.tocsr()
    n = Q.shape[0]
    fac = block_factors(Q, b)
    Z = o.philox_normals(seed, 0, n, k)

    def op(v):
        return apply_Linv(fac, Q @ apply_LinvT(fac, v))

    X = np.zeros((n, k))
    alphas, betas = [], []
    for s in range(k):
        z = Z[:, s]
        a, bt, V = lanczos(op, z, m)
        xt = V @ f_T_e1(a, bt, np.linalg.norm(z))
        X[:, s] = apply_LinvT(fac, xt)
        alphas.append(a)
        betas.append(bt)
    return X, alphas, betas
