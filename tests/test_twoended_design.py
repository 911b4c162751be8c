"""CPU check of the identity behind the one-part form's two-ended
factorisation, as a plain numpy emulation of its steps (no GPU, no oracle,
no library code): for a block-tridiagonal SPD matrix with diagonal blocks A_t
and couplings B_t = Q[t+1, t],

* Schur complements from slab 0 up to the middle slab m = T // 2,
  D_t = A_t - B_{t-1} D_{t-1}^-1 B_{t-1}^T, and from slab T - 1 down to m + 1,
  R_t = A_t - B_t^T R_{t+1}^-1 B_t;
* the middle slab takes both neighbours' terms,
  M = A_m - B_{m-1} D_{m-1}^-1 B_{m-1}^T - B_m^T R_{m+1}^-1 B_m, and
  Sigma_mm = M^-1;
* the selected inverse runs outward in both halves:
  Sigma_tt = D_t^-1 + D_t^-1 B_t^T Sigma_{t+1} B_t D_t^-1 and
  Sigma_{t+1,t} = -Sigma_{t+1} B_t D_t^-1 above the middle,
  Sigma_tt = R_t^-1 + R_t^-1 B_{t-1} Sigma_{t-1} B_{t-1}^T R_t^-1 and
  Sigma_{t,t-1} = -R_t^-1 B_{t-1} Sigma_{t-1} below it,

reproduces every diagonal and off-diagonal block of the dense inverse, for
odd and even chain lengths and couplings that are not symmetric.
"""
import numpy as np
import pytest


def random_bt(T, n, seed, symmetric_couplings):
    rng = np.random.default_rng(seed)
    B = []
    for _ in range(T - 1):
        X = rng.standard_normal((n, n)) * 0.3
        B.append((X + X.T) / 2 if symmetric_couplings else X)
    A = []
    for t in range(T):
        Y = rng.standard_normal((n, n)) * 0.2
        A.append((Y + Y.T) / 2 + 3.0 * np.eye(n))
    Q = np.zeros((T * n, T * n))
    for t in range(T):
        Q[t * n:(t + 1) * n, t * n:(t + 1) * n] = A[t]
        if t + 1 < T:
            Q[(t + 1) * n:(t + 2) * n, t * n:(t + 1) * n] = B[t]
            Q[t * n:(t + 1) * n, (t + 1) * n:(t + 2) * n] = B[t].T
    assert np.min(np.linalg.eigvalsh(Q)) > 0
    return A, B, Q


def two_ended_selinv(A, B):
    """Diagonal blocks Sigma_tt and couplings Sigma_{t+1,t} by the two-ended
    recursion."""
    T = len(A)
    m = T // 2
    inv = np.linalg.inv
    D = [None] * T
    R = [None] * T
    for t in range(m):
        D[t] = A[t] if t == 0 else A[t] - B[t - 1] @ inv(D[t - 1]) @ B[t - 1].T
    for t in range(T - 1, m, -1):
        R[t] = A[t] if t == T - 1 else A[t] - B[t].T @ inv(R[t + 1]) @ B[t]
    M = A[m].copy()
    if m >= 1:
        M -= B[m - 1] @ inv(D[m - 1]) @ B[m - 1].T
    if m + 1 <= T - 1:
        M -= B[m].T @ inv(R[m + 1]) @ B[m]
    S = [None] * T
    Y = [None] * (T - 1)   # Y[t] = Sigma_{t+1, t}
    S[m] = inv(M)
    for t in range(m - 1, -1, -1):
        Di = inv(D[t])
        Y[t] = -S[t + 1] @ B[t] @ Di
        S[t] = Di + Di @ B[t].T @ S[t + 1] @ B[t] @ Di
    for t in range(m + 1, T):
        Ri = inv(R[t])
        Y[t - 1] = -Ri @ B[t - 1] @ S[t - 1]
        S[t] = Ri + Ri @ B[t - 1] @ S[t - 1] @ B[t - 1].T @ Ri
    return S, Y


@pytest.mark.parametrize("symmetric_couplings", [True, False])
@pytest.mark.parametrize("T", [1, 2, 3, 4, 5, 8, 9])
def test_two_ended_selinv_matches_dense_inverse(T, symmetric_couplings):
    n = 5
    A, B, Q = random_bt(T, n, seed=10 * T + int(symmetric_couplings), symmetric_couplings=symmetric_couplings)
    S, Y = two_ended_selinv(A, B)
    E = np.linalg.inv(Q)
    scale = np.abs(E).max()
    for t in range(T):
        assert np.abs(S[t] - E[t * n:(t + 1) * n, t * n:(t + 1) * n]).max() < 1e-12 * scale
    for t in range(T - 1):
        assert np.abs(Y[t] - E[(t + 1) * n:(t + 2) * n, t * n:(t + 1) * n]).max() < 1e-12 * scale


def test_middle_slab_needs_both_neighbour_terms():
    """Leaving out either neighbour's term of the middle slab is wrong: the
    identity is not satisfied by accident."""
    T, n = 6, 4
    A, B, Q = random_bt(T, n, seed=7, symmetric_couplings=True)
    E = np.linalg.inv(Q)
    m = T // 2
    inv = np.linalg.inv
    D = [A[0]]
    for t in range(1, m):
        D.append(A[t] - B[t - 1] @ inv(D[t - 1]) @ B[t - 1].T)
    M_one_sided = A[m] - B[m - 1] @ inv(D[m - 1]) @ B[m - 1].T
    true_mm = E[m * n:(m + 1) * n, m * n:(m + 1) * n]
    assert np.abs(inv(M_one_sided) - true_mm).max() > 1e-3 * np.abs(true_mm).max()
